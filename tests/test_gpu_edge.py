"""Degenerate and extreme shapes against the FP64 oracle (fixed sweep counts, so
the iterates are compared one for one): matrices (N = 2, where st-HOSVD-ALS is
the rank-R ALS approximation of a matrix and converges to the truncated SVD),
fifth and eighth order (the largest order the boundary accepts), a mode of size
one, rank-one truncations in every mode, and a 2 x 2 x 2 tensor."""
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


def _np(t):
    return t.double().cpu().numpy()


CASES = [
    ((300, 200), (8, 8)),
    ((6, 7, 5, 8, 4), (2, 3, 2, 3, 2)),
    ((3, 3, 3, 3, 3, 3, 3, 3), (2, 2, 2, 2, 2, 2, 2, 2)),
    ((1, 30, 40), (1, 5, 5)),
    ((20, 18, 16), (1, 1, 1)),
    ((2, 2, 2), (1, 2, 2)),
]


@pytest.mark.parametrize("dims,ranks", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("driver", ["st", "t"])
def test_edge_shapes_fixed_sweeps(tals, dims, ranks, dtype, driver):
    # Gaussian cores: with a rank-one mode the 1/k core spectrum turns into 1/k^2 on
    # the other modes, and three fixed sweeps of such a spectrum move by ~5e-5 in
    # angle under a relative input perturbation of FP32 rounding size (6e-8) alone;
    # with Gaussian cores every case here stays below 1e-6
    p = W.planted(W.SEED_BASE + 60, dims, ranks, "gauss", 1e-2, dtype=dtype)
    a64 = p.A.astype(np.float64)
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    ref = f(a64, ranks, eta=-1.0, seed=7, max_sweeps=3)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    G, Us, st = g(torch.from_numpy(np.ascontiguousarray(p.A)).cuda(), ranks, eta=-1.0, seed=7, max_sweeps=3)
    tol_rel = 1e-10 if dtype == np.float64 else 1e-6
    tol_ang = 1e-8 if dtype == np.float64 else 1e-4
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= tol_rel, (rel_own, rel_ref)
    for n in range(len(dims)):
        u = _np(Us[n])
        assert u.shape == ref.U[n].shape
        assert O.principal_angles(u, ref.U[n]).max() <= tol_ang
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= (1e-12 if dtype == np.float64 else 1e-5)
        assert st["sweeps"][n] == ref.sweeps[n]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_matrix_case_reaches_truncated_svd(tals, dtype):
    # N = 2: the ALS subspaces converge to the leading singular subspaces (Thm. 2)
    rng = np.random.default_rng(3)
    m, n, r = 240, 160, 6
    u0 = np.linalg.qr(rng.standard_normal((m, r)))[0]
    v0 = np.linalg.qr(rng.standard_normal((n, r)))[0]
    s = np.array([10.0, 8.0, 6.5, 5.0, 4.0, 3.0])
    a = (u0 * s) @ v0.T + 1e-3 * rng.standard_normal((m, n))
    a = a.astype(dtype)
    G, Us, st = tals.st_hosvd(torch.from_numpy(a).cuda(), (r, r), eta=1e-12 if dtype == np.float64 else 1e-7,
                              seed=1, max_sweeps=50)
    uu, ss, vvt = np.linalg.svd(a.astype(np.float64), full_matrices=False)
    tol = 1e-8 if dtype == np.float64 else 1e-4
    assert O.principal_angles(_np(Us[0]), uu[:, :r]).max() <= tol
    assert O.principal_angles(_np(Us[1]), vvt[:r].T).max() <= tol
    # the error of the rank-r truncation (Eckart-Young)
    best = np.sqrt(np.sum(ss[r:] ** 2)) / np.linalg.norm(a.astype(np.float64))
    own = O.rel_error(a.astype(np.float64), _np(G), [_np(u) for u in Us])
    assert abs(own - best) <= (1e-10 if dtype == np.float64 else 1e-6)
