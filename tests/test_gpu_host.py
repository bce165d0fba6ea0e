"""Host-buffer entry points: st_hosvd_host (upload, decomposition, download) and
st_hosvd_host_many (the same, pipelined over two device buffers so that the
upload of tensor t+1 overlaps the decomposition of tensor t). Both must give
exactly the results of the device-resident call on the same tensors: the same
kernels run in the same order with deterministic reductions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


def _inputs(dims, ranks, count):
    return [W.planted(W.SEED_BASE + 40 + t, dims, ranks, "inv_k", 1e-2, dtype=np.float32).A
            for t in range(count)]


def _device_results(tals, arrays, ranks, precision):
    out = []
    for a in arrays:
        ctx = tals.Context(torch.from_numpy(a).cuda(), ranks, eta=1e-6, seed=1, precision=precision,
                           use_graph=True)
        G, Us, st = ctx.st_hosvd()
        out.append((G.cpu().numpy(), [u.cpu().numpy() for u in Us], st))
        ctx.close()
    return out


@pytest.mark.parametrize("dims,ranks,precision", [
    ((48, 40, 36), (6, 5, 4), "native"),
    ((256, 128, 128), (16, 12, 8), "mixed_bf16"),
])
def test_host_entry_points_match_device(tals, dims, ranks, precision):
    arrays = _inputs(dims, ranks, 3)
    ref = _device_results(tals, arrays, ranks, precision)
    hctx = tals.HostContext(dims, ranks, "f32", eta=1e-6, seed=1, precision=precision)
    A_h = [torch.from_numpy(a).pin_memory() for a in arrays]
    # one call per tensor
    for t, a in enumerate(A_h):
        G_h = torch.empty(ranks).pin_memory()
        U_h = [torch.empty((d, r)).pin_memory() for d, r in zip(dims, ranks)]
        st = hctx.st_hosvd(a, G_h, U_h)
        assert np.array_equal(G_h.numpy(), ref[t][0])
        for n in range(3):
            assert np.array_equal(U_h[n].numpy(), ref[t][1][n])
        assert st["sweeps"] == ref[t][2]["sweeps"] and st["rel_err"] == ref[t][2]["rel_err"]
    # pipelined over all three (both device buffers, one reused), twice
    for _ in range(2):
        G_hs = [torch.empty(ranks).pin_memory() for _ in arrays]
        U_hs = [[torch.empty((d, r)).pin_memory() for d, r in zip(dims, ranks)] for _ in arrays]
        sts = hctx.st_hosvd_many(A_h, G_hs, U_hs)
        for t in range(3):
            assert np.array_equal(G_hs[t].numpy(), ref[t][0])
            for n in range(3):
                assert np.array_equal(U_hs[t][n].numpy(), ref[t][1][n])
            assert sts[t]["sweeps"] == ref[t][2]["sweeps"]
            assert sts[t]["rel_err"] == ref[t][2]["rel_err"]
    hctx.close()


def test_host_many_rejects_mismatched_lists(tals):
    dims, ranks = (24, 20, 16), (4, 3, 2)
    hctx = tals.HostContext(dims, ranks, "f32", eta=1e-6, seed=1)
    a = torch.zeros(dims).pin_memory()
    with pytest.raises(ValueError):
        hctx.st_hosvd_many([a, a], [torch.empty(ranks)])
    hctx.close()
