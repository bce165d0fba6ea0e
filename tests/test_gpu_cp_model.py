"""GPU parity on long modes: the CP-model workload of Sec. 6.1.1 (I x I x 100 I,
truncation 0.2 I, lambda in [5, 10], absolute noise 1e-4) and a Tucker-model shape
with a long first mode (Sec. 6.1.2's I x 100 x 100 x 100, reduced). Their long
modes (K = 100 I; I_1 = 2500) are beyond the fused pass's shared-memory tile and
run the two-pass sweep (tiled W = B^T Q, then Y = B W). Compared with the FP64
oracle on the same inputs: fixed sweep counts elementwise (FP64 factors 1e-8,
core 1e-8 max|G|; FP32 factors 1e-3), converged runs by relative error (1e-10 /
1e-6), principal angles (1e-8 / 1e-4) and sweep counts; HOOI and the singular
vectors on a two-pass mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import tucker_oracle as O


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.double().cpu().numpy()


def _uses_twopass(tals, dt, dims, ranks):
    """The last mode's view is outside the fused pass (so the two-pass form runs)."""
    P = int(np.prod(dims[:-1]))
    assert tals.pass_plan(dt, P, dims[-1], 1, ranks[-1]) is None


@pytest.mark.parametrize("driver", ["st", "t"])
def test_cp_model_fixed_sweeps_f64(tals, driver):
    c = W.cp_model(W.CP_SEED, 20, dtype=np.float64)
    ranks = (4, 4, 4)
    _uses_twopass(tals, "f64", c.A.shape, ranks)
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    ref = f(c.A, ranks, eta=-1.0, seed=3, max_sweeps=4)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    G, Us, st = g(_gpu(c.A), ranks, eta=-1.0, seed=3, max_sweeps=4, use_graph=(driver == "st"))
    for n in range(3):
        assert st["sweeps"][n] == ref.sweeps[n]
        assert np.abs(_np(Us[n]) - ref.U[n]).max() <= 1e-8
    assert np.abs(_np(G) - ref.G).max() <= 1e-8 * np.abs(ref.G).max()
    assert abs(st["rel_err"] - O.rel_error(c.A, ref.G, ref.U)) <= 1e-10


@pytest.mark.parametrize("I,dt", [(20, np.float64), (40, np.float32)])
@pytest.mark.parametrize("driver", ["st", "t"])
def test_cp_model_converged(tals, I, dt, driver):
    c = W.cp_model(W.CP_SEED, I, dtype=dt)
    R = int(round(0.2 * I))
    ranks = (R, R, R)
    a64 = c.A.astype(np.float64)
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    ref = f(a64, ranks, eta=1e-6, seed=1)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    G, Us, st = g(_gpu(c.A), ranks, eta=1e-6, seed=1)
    f64 = dt == np.float64
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= (1e-10 if f64 else 1e-6) * max(1.0, rel_ref)
    for n in range(3):
        assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= (1e-8 if f64 else 1e-4)
        if f64:
            assert st["sweeps"][n] == ref.sweeps[n]
        else:
            assert abs(st["sweeps"][n] - ref.sweeps[n]) <= 1
    # the paper's measure, against the noiseless CP tensor
    base = W.cp_model(W.CP_SEED, I, delta=0.0, dtype=np.float64).A
    b = O.reconstruct(_np(G), [_np(u) for u in Us])
    bref = O.reconstruct(ref.G, ref.U)
    e_own = np.linalg.norm(b - base) / np.linalg.norm(base)
    e_ref = np.linalg.norm(bref - base) / np.linalg.norm(base)
    assert abs(e_own - e_ref) <= (1e-10 if f64 else 1e-5)


def test_long_first_mode_fixed_sweeps_f32(tals):
    """A Tucker-model shape with I_1 = 2500 (uniform [5, 10] core, Sec. 6.1.2's
    recipe at reduced trailing sizes): mode 1 runs the two-pass form in FP32."""
    dims, ranks = (2500, 24, 20, 16), (25, 4, 4, 3)
    p = W.planted(W.SEED_BASE + 21, dims, ranks, "uniform510", 1e-4, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    for driver in ("st", "t"):
        f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
        ref = f(a64, ranks, eta=-1.0, seed=2, max_sweeps=3)
        g = tals.st_hosvd if driver == "st" else tals.t_hosvd
        G, Us, st = g(_gpu(p.A), ranks, eta=-1.0, seed=2, max_sweeps=3)
        rel_ref = O.rel_error(a64, ref.G, ref.U)
        rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
        assert abs(rel_own - rel_ref) <= 1e-6, (driver, rel_own, rel_ref)
        for n in range(4):
            assert st["sweeps"][n] == ref.sweeps[n]
            assert np.abs(_np(Us[n]) - ref.U[n]).max() <= 1e-3, (driver, n)


def test_hooi_and_singular_vectors_on_a_long_mode(tals):
    c = W.cp_model(W.CP_SEED + 1, 20, dtype=np.float64)
    ranks = (4, 4, 4)
    ctx = tals.Context(_gpu(c.A), ranks, eta=1e-3, max_sweeps=2, use_graph=False)
    _, Us, _ = ctx.t_hosvd()
    us0 = [_np(u) for u in Us]
    # singular vectors of the long mode from its t-HOSVD-ALS basis
    U2, s2 = ctx.singular_vectors(2, Us[2])
    uo, so = O.singular_vectors(c.A, 2, us0[2])
    assert np.allclose(s2, so, rtol=1e-10)
    sgn = np.sign(np.sum(_np(U2) * uo, axis=0))
    assert np.abs(_np(U2) - uo * sgn).max() <= 1e-8
    # HOOI: its inner ALS on A x_1 U1^T x_2 U2^T (a 4 x 4 x 2000 tensor) keeps the long mode
    G, Us, info = ctx.hooi(Us, tol=1e-13, max_iters=30, inner_eta=1e-15, inner_sweeps=30)
    ref = O.hooi(c.A, us0, tol=1e-13, max_iters=30)
    assert abs(info["resid"][-1] - ref.resid[-1]) <= 1e-11
    assert abs(info["iters"] - ref.iters) <= 1
    for n in range(3):
        assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= 1e-7
    ctx.close()


def test_long_mode_with_many_columns_t_hosvd(tals):
    """The long mode's Y = B_(n) W sums 60000 columns: held to the FP32 gates, so
    the column splits' FP32 sums must stay short (they are added in FP64).

    Sweep counts: at noise 1e-3, e_n^2 / ||B||^2 ~ 1e-6, and e_n comes from
    ||B||^2 - ||W||^2 with W from FP32 products (~1e-8 relative in ||W||^2 once the
    dominant direction of this all-positive core is summed over its 60000 columns):
    e_n is known to ~0.5% of itself, ~5e-6 ||A||, above eta ||A|| = 1e-6 ||A||. The
    stop decision is then taken at FP32 noise level and any change of summation
    order moves it by a sweep or two; the sweep counts are held to [-1, +2] of the
    oracle's, the results to the FP32 gates."""
    dims, ranks = (2400, 50, 40, 30), (24, 5, 5, 5)
    p = W.planted(W.SEED_BASE + 22, dims, ranks, "uniform510", 1e-3, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    assert tals.pass_plan("f32", 1, 2400, 60000, 24) is None
    ref = O.t_hosvd_als(a64, ranks, eta=1e-6, seed=6)
    G, Us, st = tals.t_hosvd(_gpu(p.A), ranks, eta=1e-6, seed=6)
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= 1e-6 * max(1.0, rel_ref), (rel_own, rel_ref)
    for n in range(4):
        assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= 1e-4, n
        assert -1 <= st["sweeps"][n] - ref.sweeps[n] <= 2, (n, st["sweeps"], ref.sweeps)
