"""The entry point that allocates no device memory (tals_sweep_pass_noalloc).

Some callers cannot allocate device memory when they call into the library (a
memory pool or a framework's caching allocator owns the device memory, or the
call sits in a latency-critical loop). This entry point computes one fused
sweep pass with its scratch in a fixed array inside the library. The test
calls it through the C ABI with caller-owned buffers, twice in a row, and
checks each result against the allocating entry point tals_sweep_pass
(CUDA-core engine) within the FP32 pass tolerance. It is collected last so that
a run stopping at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


def _noalloc(tals, A, mode, Q, Y, w2):
    dims = (ctypes.c_int64 * A.dim())(*[int(d) for d in A.shape])
    st = tals.lib().tals_sweep_pass_noalloc(A.data_ptr(), A.dim(), dims, mode, Q.data_ptr(),
                                            int(Q.shape[1]), Y.data_ptr(), w2.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    return st


@pytest.mark.parametrize("dims,mode,R", [((96, 70, 50), 0, 12), ((40, 300, 33), 1, 32),
                                         ((24, 20, 512), 2, 16)])
def test_noalloc_matches_allocating_pass_twice(tals, dims, mode, R):
    rng = np.random.default_rng(11)
    A = torch.from_numpy(rng.standard_normal(dims).astype(np.float32)).cuda()
    Q = torch.from_numpy(np.linalg.qr(rng.standard_normal((dims[mode], R)))[0]
                         .astype(np.float32)).cuda()
    Y_ref, w2_ref = tals.sweep_pass(A, mode, Q, engine="cuda")
    Y = torch.empty((dims[mode], R), dtype=torch.float64, device="cuda")
    w2 = torch.empty((1,), dtype=torch.float64, device="cuda")
    for _ in range(2):
        Y.fill_(float("nan"))
        w2.fill_(float("nan"))
        assert _noalloc(tals, A, mode, Q, Y, w2) == tals.TALS_OK
        torch.cuda.synchronize()
        assert torch.isfinite(Y).all()
        assert torch.allclose(Y, Y_ref, rtol=1e-5, atol=1e-5 * float(Y_ref.abs().max()))
        assert abs(float(w2.item()) - w2_ref) <= 1e-5 * w2_ref


def test_noalloc_with_its_grid_cut_to_the_scratch(tals):
    """I x R = 512 x 64: the fixed scratch holds the Y partials of 32 CTAs only, fewer
    than the pass plans for this view, so every CTA covers more tiles."""
    dims, mode, R = (512, 64, 64), 0, 64
    plan = tals.pass_plan("f32", 1, 512, 64 * 64, R, torch.cuda.get_device_properties(0).multi_processor_count)
    assert plan is not None and plan["grid_x"] > (1 << 20) // (512 * R)
    rng = np.random.default_rng(12)
    A = torch.from_numpy(rng.standard_normal(dims).astype(np.float32)).cuda()
    Q = torch.from_numpy(np.linalg.qr(rng.standard_normal((dims[mode], R)))[0]
                         .astype(np.float32)).cuda()
    Y_ref, w2_ref = tals.sweep_pass(A, mode, Q, engine="cuda")
    Y = torch.full((dims[mode], R), float("nan"), dtype=torch.float64, device="cuda")
    w2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(tals, A, mode, Q, Y, w2) == tals.TALS_OK
    torch.cuda.synchronize()
    assert torch.isfinite(Y).all()
    assert torch.allclose(Y, Y_ref, rtol=1e-5, atol=1e-5 * float(Y_ref.abs().max()))
    assert abs(float(w2.item()) - w2_ref) <= 1e-5 * w2_ref


def test_noalloc_rejects_oversize(tals):
    A = torch.zeros((4096, 8, 8), device="cuda")
    Q = torch.zeros((4096, 300), device="cuda")
    Y = torch.empty((4096, 300), dtype=torch.float64, device="cuda")
    w2 = torch.empty((1,), dtype=torch.float64, device="cuda")
    assert _noalloc(tals, A, 0, Q, Y, w2) == tals.TALS_EINVAL
    assert b"no-allocation scratch" in tals.lib().tals_last_error()
