"""GPU tests of the split-precision (3xTF32) tensor-core sweep (tcgen05 kind::tf32).

One sweep of products, Alg. 3 R- and L-updates fused as in Eq. 2.2: Y = B B^T Q for
the mode-n unfolding B, compared element by element with the FP64 product of the
same FP32 data. The split keeps each product within a few units of 2^-22 of
|a||b|; the tensor cores' FP32 accumulation rounds toward zero, which over the
K = I_n sum of the W product leaves a relative bias of about 1e-6 to 1e-5 (measured
and printed below). A single TF32 product (2^-11 ~ 5e-4) or a wrong tile fails
every bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tucker_oracle as O


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


def _case(dims, mode, R, seed, positive=False):
    rng = np.random.default_rng(seed)
    if positive:
        a = rng.uniform(0.5, 1.5, dims).astype(np.float32)
        q = rng.uniform(0.5, 1.5, (dims[mode], R)).astype(np.float32)
    else:
        a = rng.standard_normal(dims).astype(np.float32)
        q = np.linalg.qr(rng.standard_normal((dims[mode], R)))[0].astype(np.float32)
    return a, q


# (dims, mode, R): mode sizes with ragged 32-row and 128-row tails, Q from 32 up,
# P > 1 (32-column boxes from several p), every padded rank class (16, 32, 48, 64)
CASES = [
    ((512, 64, 96), 0, 32),
    ((96, 256, 64), 1, 16),
    ((300, 160), 0, 24),
    ((300, 160), 0, 48),
    ((130, 40, 96), 0, 7),
    ((16, 1024, 64), 1, 64),
    ((70, 200, 32), 1, 33),
]


@pytest.mark.parametrize("dims,mode,R", CASES)
def test_tf32_sweep_matches_fp64(tals, dims, mode, R):
    a, q = _case(dims, mode, R, seed=11 + R)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    m = O.unfold(a.astype(np.float64), mode)
    q64 = q.astype(np.float64)
    w_ref = m.T @ q64
    y_ref = m @ w_ref
    yabs = np.abs(m) @ (np.abs(m).T @ np.abs(q64))
    Y, w2 = tals.sweep_pass(A, mode, Qt, engine="tf32")
    Y = Y.cpu().numpy()
    rel = {}
    for eng in ("tf32_w", "tf32_y"):   # each tensor-core pass beside the CUDA-core one
        Yd, w2d = tals.sweep_pass(A, mode, Qt, engine=eng)
        Yd = Yd.cpu().numpy()
        rel[eng] = np.linalg.norm(Yd - y_ref) / np.linalg.norm(y_ref)
        print(f"{dims} {mode} {R} {eng}: Y {rel[eng]:.3e} "
              f"w2 {(w2d - O.frob2(w_ref)) / O.frob2(w_ref):.3e}")
    assert max(rel.values()) <= 1e-5, rel
    print(f"{dims} {mode} {R} tf32: Y {np.linalg.norm(Y - y_ref) / np.linalg.norm(y_ref):.3e} "
          f"w2 {(w2 - O.frob2(w_ref)) / O.frob2(w_ref):.3e}")
    err = np.abs(Y - y_ref)
    # element-wise: split products and FP32 accumulation, far below one TF32 rounding
    assert np.all(err <= 5e-5 * yabs + 1e-30), float((err / yabs).max())
    assert np.linalg.norm(Y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
    assert abs(w2 - O.frob2(w_ref)) <= 2e-5 * O.frob2(w_ref)


def test_tf32_sweep_vs_cuda_core_pass(tals):
    """The two engines agree to FP32 accuracy on a benchmark-shaped view."""
    dims, mode, R = (512, 128, 256), 0, 32
    a, q = _case(dims, mode, R, seed=5)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    Yt, w2t = tals.sweep_pass(A, mode, Qt, engine="tf32")
    Yc, w2c = tals.sweep_pass(A, mode, Qt, engine="cuda")
    d = (Yt - Yc).norm().item() / Yc.norm().item()
    assert d <= 1e-5, d
    assert abs(w2t - w2c) <= 2e-5 * w2c


def test_tf32_accumulation_bias(tals):
    """All-positive data: the accumulator's rounding toward zero biases every sum low
    by a fraction of an FP32 unit per accumulation step (measured about 1.6e-5 for
    ||W||^2 at K = 1024); the bound is five times that, far below one TF32 rounding."""
    dims, mode, R = (1024, 64, 128), 0, 32
    a, q = _case(dims, mode, R, seed=9, positive=True)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    m = O.unfold(a.astype(np.float64), mode)
    w_ref = m.T @ q.astype(np.float64)
    y_ref = m @ w_ref
    Y, w2 = tals.sweep_pass(A, mode, Qt, engine="tf32")
    rel_w2 = (w2 - O.frob2(w_ref)) / O.frob2(w_ref)
    rel_y = (Y.cpu().numpy().sum() - y_ref.sum()) / y_ref.sum()
    print(f"split-TF32 bias on positive data: ||W||^2 {rel_w2:.3e}, sum(Y) {rel_y:.3e}")
    assert abs(rel_w2) <= 8e-5 and abs(rel_y) <= 8e-5


# ---------------------------------------------------------------------------
# Whole decompositions with the FP32 products on the split-precision passes
# (fp32_engine="tensor": every mode whose view qualifies), against the FP64 oracle
# on the same seeded input, at the FP32 tolerances of the CUDA-core path:
# relative error of the returned (G, U) within 1e-6 of the oracle's, the GPU's own
# estimate within 1e-5, e_n^2 within 2e-7 ||A||^2, angles below 1e-4, and at fixed
# sweep counts factors within 1e-3 and the core within 1e-3 max|G|.
# ---------------------------------------------------------------------------
import workloads as W


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cmp32(res_gpu, ref, a64, fixed=True):
    G, Us, st = res_gpu
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, G.double().cpu().numpy(), [u.double().cpu().numpy() for u in Us])
    assert abs(rel_own - rel_ref) <= 1e-6, (rel_own, rel_ref)
    assert abs(st["rel_err"] - rel_ref) <= 1e-5, (st["rel_err"], rel_ref)
    norm_a2 = O.frob2(a64)
    for n in range(a64.ndim):
        u = Us[n].double().cpu().numpy()
        assert O.principal_angles(u, ref.U[n]).max() <= 1e-4
        assert abs(st["err_per_mode"][n] ** 2 - ref.err_per_mode[n] ** 2) <= 2e-7 * norm_a2, n
        if fixed:
            assert st["sweeps"][n] == ref.sweeps[n]
            assert np.abs(u - ref.U[n]).max() <= 1e-3
    if fixed:
        g = G.double().cpu().numpy()
        assert np.abs(g - ref.G).max() <= 1e-3 * np.abs(ref.G).max()


# mode views: (96 | Q = 128) first, then (256 | Q = 1536); the last (Q = 1) on CUDA cores
DEC = ((256, 96, 128), (16, 12, 20))


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("driver", ["st", "t"])
def test_tensor_engine_fixed_sweeps(tals, driver, use_graph):
    dims, ranks = DEC
    p = W.planted(W.SEED_BASE + 31, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    ref = f(a64, ranks, eta=-1.0, seed=5, max_sweeps=3)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    res = g(_gpu(p.A), ranks, eta=-1.0, seed=5, max_sweeps=3, fp32_engine="tensor",
            use_graph=use_graph)
    _cmp32(res, ref, a64, fixed=True)


def test_tensor_engine_tolerance_run(tals):
    dims, ranks = (128, 160, 96), (24, 16, 32)
    p = W.planted(W.SEED_BASE + 32, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=1)
    G, Us, st = tals.st_hosvd(_gpu(p.A), ranks, eta=1e-6, seed=1, fp32_engine="tensor")
    for n in range(3):
        assert abs(st["sweeps"][n] - ref.sweeps[n]) <= 1
    _cmp32((G, Us, st), ref, a64, fixed=False)


def test_tensor_engine_mixed_precision(tals):
    """BF16 bulk sweeps, then split-precision finishing sweeps (mode 0 first: the
    BF16 pass covers its view)."""
    dims, ranks = (512, 96, 128), (32, 16, 24)
    p = W.planted(W.SEED_BASE + 21, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=3, order=[0, 1, 2])
    for use_graph in (True, False):
        G, Us, st = tals.st_hosvd(_gpu(p.A), ranks, eta=1e-6, seed=3, precision="mixed_bf16",
                                  use_graph=use_graph, order=[0, 1, 2], fp32_engine="tensor")
        assert st["bulk_sweeps"][0] >= 1
        _cmp32((G, Us, st), ref, a64, fixed=False)


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
def test_rank64_mode_1024(tals, engine):
    """The ranks of the 1024 x 1024 x 512 workload on 1024-long modes: mode 2
    (R = 32, Q = 1) first, then mode 0 (I = 1024, R = 64) and mode 1 (I = 256,
    R = 64), compared with the oracle at fixed sweep counts. A Gaussian core keeps
    the weakest of the 64 directions well separated for the FP32 angle check."""
    dims, ranks = (1024, 256, 64), (64, 64, 32)
    p = W.planted(W.SEED_BASE + 33, dims, ranks, "gauss", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    ref = O.st_hosvd_als(a64, ranks, eta=-1.0, seed=7, max_sweeps=3)
    res = tals.st_hosvd(_gpu(p.A), ranks, eta=-1.0, seed=7, max_sweeps=3, fp32_engine=engine)
    _cmp32(res, ref, a64, fixed=True)


def test_tensor_engine_user_driven_sweeps(tals):
    """als_mode_sweep / als_mode_finish on the split-precision passes: the mode's
    error after the stop rule fires is the explicit residual of the returned pair."""
    dims, ranks = DEC
    p = W.planted(W.SEED_BASE + 34, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    ctx = tals.Context(_gpu(p.A), ranks, eta=-1.0, seed=2, max_sweeps=3, fp32_engine="tensor")
    try:
        e1, conv = ctx.mode_sweep(1, 10)
        U1 = ctx.mode_finish(1, truncate=True).double().cpu().numpy()
    finally:
        ctx.close()
    m = O.unfold(a64, 1)
    resid = m - U1 @ (U1.T @ m)
    assert abs(e1 ** 2 - O.frob2(resid)) <= 2e-7 * O.frob2(a64)
