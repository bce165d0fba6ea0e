"""GPU tests of the two-product sweep (fp32_engine="products"): W = B^T Q by the
register-tiled mode product, then Y = B W split over column ranges (adjoint.cu),
both in exact FP32 arithmetic on CUDA cores.

One sweep of products (Alg. 3 R- and L-updates, Eq. 2.2): Y = B B^T Q for the
mode-n unfolding B, compared element by element with the FP64 product of the same
FP32 data. Every product is exact FP32 (rounding to nearest): each entry of W is
an FP32 dot product of length I_n and each Y partial one of length J / S, the
partials summed in FP64, so the element-wise error stays within a few units of
2^-24 times sqrt(length) |B|(|B|^T |Q|) -- the bound below is 2e-5 of that
absolute product, which a dropped column tile (1/J_tiles of an entry) or a wrong
rank index fails by orders of magnitude. Then whole decompositions on this form
against the FP64 oracle at the FP32 path's tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tucker_oracle as O
import workloads as W


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


# (dims, mode, R): row tiles of 256 with ragged tails (300, 520), P > 1 with
# Q = 32 and Q = 48, a last column range shorter than the others (J = 2000 in three
# ranges of 672, 672, 656), one split only (J < 1024), both rank
# classes (<= 32, <= 64) with padded ranks (24, 36), R = 1..64; R not a multiple of
# 4 only where I_n <= 64 (the mode product keeps such a basis resident).
CASES = [
    ((300, 16, 48), 0, 24),
    ((520, 125, 16), 0, 32),
    ((40, 16, 48), 1, 16),
    ((64, 48, 32), 1, 36),
    ((48, 64, 80), 0, 7),
    ((64, 256, 96), 1, 64),
    ((20, 16, 32), 1, 1),
    ((8, 40, 48), 1, 12),
]


@pytest.mark.parametrize("dims,mode,R", CASES)
def test_products_sweep_matches_fp64(tals, dims, mode, R):
    a, q = _case(dims, mode, R, seed=41 + R)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    m = O.unfold(a.astype(np.float64), mode)
    q64 = q.astype(np.float64)
    w_ref = m.T @ q64
    y_ref = m @ w_ref
    yabs = np.abs(m) @ (np.abs(m).T @ np.abs(q64))
    Y, w2 = tals.sweep_pass(A, mode, Qt, engine="products")
    Y = Y.cpu().numpy()
    err = np.abs(Y - y_ref)
    print(f"{dims} {mode} {R}: max |dY| / |B|(|B|^T|Q|) {float((err / yabs).max()):.3e}, "
          f"||W||^2 {(w2 - O.frob2(w_ref)) / O.frob2(w_ref):.3e}")
    assert np.all(err <= 2e-5 * yabs + 1e-30), float((err / yabs).max())
    assert np.linalg.norm(Y - y_ref) <= 2e-6 * np.linalg.norm(y_ref)
    assert abs(w2 - O.frob2(w_ref)) <= 2e-6 * O.frob2(w_ref)


def test_products_positive_data_unbiased(tals):
    """All-positive data, the sums long (J = 65536 over the splits): round-to-nearest
    FP32 leaves no drift -- the relative error of sum(Y) and ||W||^2 stays near
    2^-24 sqrt(length), far below the 1e-5 a truncating accumulator shows here."""
    dims, mode, R = (512, 256, 256), 0, 32
    a, q = _case(dims, mode, R, seed=9, positive=True)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    m = O.unfold(a.astype(np.float64), mode)
    w_ref = m.T @ q.astype(np.float64)
    y_ref = m @ w_ref
    Y, w2 = tals.sweep_pass(A, mode, Qt, engine="products")
    rel_w2 = (w2 - O.frob2(w_ref)) / O.frob2(w_ref)
    rel_y = (Y.cpu().numpy().sum() - y_ref.sum()) / y_ref.sum()
    print(f"two-product form on positive data: ||W||^2 {rel_w2:.3e}, sum(Y) {rel_y:.3e}")
    assert abs(rel_w2) <= 1e-6 and abs(rel_y) <= 1e-6


def test_products_agree_with_fused_pass(tals):
    """The two FP32 engines on a benchmark-shaped view agree to FP32 accuracy."""
    dims, mode, R = (512, 128, 256), 0, 32
    a, q = _case(dims, mode, R, seed=5)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    Yp, w2p = tals.sweep_pass(A, mode, Qt, engine="products")
    Yc, w2c = tals.sweep_pass(A, mode, Qt, engine="cuda")
    d = (Yp - Yc).norm().item() / Yc.norm().item()
    assert d <= 2e-6, d
    assert abs(w2p - w2c) <= 2e-6 * w2c


def test_products_limits(tals):
    """Views outside the form's limits are refused, not approximated: Q % 16 != 0,
    and R not a multiple of 4 with I_n > 64."""
    for dims, mode, R in (((64, 10, 12), 0, 8), ((300, 16, 48), 0, 7)):
        a, q = _case(dims, mode, R, seed=3)
        with pytest.raises(tals.TalsError):
            tals.sweep_pass(torch.from_numpy(a).cuda(), mode, torch.from_numpy(q).cuda(), engine="products")


# ---------------------------------------------------------------------------
# Whole decompositions on the two-product form against the FP64 oracle on the same
# seeded input: relative error of (G, U) within 1e-6 of the oracle's, the GPU's
# estimate within 1e-5, e_n^2 within 2e-7 ||A||^2, angles below 1e-4, and at fixed
# sweep counts factors within 1e-3 and the core within 1e-3 max|G|. The tensor has
# more than 2^24 elements, so the full-size modes take e_k from ||B||^2 - ||W||^2
# (the form's own statistic) rather than from an explicit residual.
# ---------------------------------------------------------------------------
DEC = ((512, 192, 176), (32, 16, 24))


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


@pytest.fixture(scope="module")
def planted():
    dims, ranks = DEC
    p = W.planted(W.SEED_BASE + 51, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    return p, p.A.astype(np.float64)


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("driver", ["st", "t"])
def test_products_engine_fixed_sweeps(tals, planted, driver, use_graph):
    p, a64 = planted
    dims, ranks = DEC
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    kw = {"order": [0, 1, 2]} if driver == "st" else {}
    ref = f(a64, ranks, eta=-1.0, seed=5, max_sweeps=3, **kw)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    res = g(_gpu(p.A), ranks, eta=-1.0, seed=5, max_sweeps=3, fp32_engine="products", use_graph=use_graph,
            **kw)
    st = res[2]
    assert st["two_product"][0]
    if driver == "t":
        assert st["two_product"][1] and not st["two_product"][2]   # mode 2: Q = 1
    _cmp32(res, ref, a64, fixed=True)


@pytest.mark.parametrize("use_graph", [True, False])
def test_products_engine_tolerance_run(tals, planted, use_graph):
    """eta = 1e-6: the stop rule on the form's ||W||^2, with split sweeps (W alone,
    the test, then Y only if the mode goes on); sweep counts within one of the
    oracle's."""
    p, a64 = planted
    dims, ranks = DEC
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=1, order=[0, 1, 2])
    G, Us, st = tals.st_hosvd(_gpu(p.A), ranks, eta=1e-6, seed=1, order=[0, 1, 2], fp32_engine="products",
                              use_graph=use_graph)
    assert st["two_product"][0] and st["split_capable"][0]
    for n in range(3):
        assert abs(st["sweeps"][n] - ref.sweeps[n]) <= 1
    _cmp32((G, Us, st), ref, a64, fixed=False)


def test_products_engine_mixed_precision(tals, planted):
    """BF16 bulk sweeps, then FP32 finishing sweeps on the two-product form."""
    p, a64 = planted
    dims, ranks = DEC
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=3, order=[0, 1, 2])
    G, Us, st = tals.st_hosvd(_gpu(p.A), ranks, eta=1e-6, seed=3, precision="mixed_bf16", order=[0, 1, 2],
                              fp32_engine="products")
    assert st["bulk_sweeps"][0] >= 1 and st["two_product"][0]
    _cmp32((G, Us, st), ref, a64, fixed=False)
