"""GPU parity: HOOI refinement (Sec. 6.3) and singular-vector recovery (Sec. 5,
after Alg. 4) through the C ABI against the FP64 oracle on the same seeded
inputs.

HOOI: the GPU's inner solver is the paper's ALS warm-started from the current
factor, the oracle's the SVD. Both follow the same iteration when the inner ALS
converges, so in FP64 the residual histories agree to 1e-11, the cycle counts
to within one, the factors' subspaces to 1e-7 rad and the reconstructions
G x U elementwise to 1e-9 max|A| (bases differ, so U and G are not compared
entrywise); the GPU's result is also checked to be a stationary point on its
own. FP32: final residuals within 2e-5 relative, angles below 1e-3.

Singular vectors: the GPU forms the R x R Gram and diagonalises it by Jacobi,
the oracle takes the SVD of Qhat^T A_(n). FP64: singular values within 1e-10
relative, vectors elementwise within 1e-8; FP32: 1e-5 and 2e-3 (the eigenvector
error grows like eps * lambda_1 / gap)."""
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


def _host(t):
    return t.double().cpu().numpy()


def _stationary(a64, us, tol):
    """Every U_n spans the dominant invariant subspace of Y_(n) Y_(n)^T."""
    N = a64.ndim
    for n in range(N):
        y = a64
        for m in range(N):
            if m != n:
                y = O.mode_product(y, us[m].T, m)
        yn = O.unfold(y, n)
        m_ = yn @ yn.T
        u = us[n]
        off = m_ @ u - u @ (u.T @ (m_ @ u))
        assert np.linalg.norm(off) <= tol * np.linalg.norm(m_), n
        top = np.sort(np.linalg.eigvalsh(m_))[::-1][:u.shape[1]]
        mine = np.sort(np.linalg.eigvalsh(u.T @ m_ @ u))[::-1]
        assert np.allclose(mine, top, rtol=max(tol, 1e-12) * 10, atol=0), n


HOOI_CASES = [
    # dims, ranks, core, noise, init eta (a loose start leaves HOOI some work)
    ((24, 20, 16), (4, 3, 3), "inv_k", 2e-2, 1e-2),
    ((12, 10, 9, 8), (3, 3, 2, 2), "gauss", 5e-2, 1e-2),
    ((40, 33, 28), (5, 6, 4), "ratio", 1e-2, 1e-2),
]


@pytest.mark.parametrize("dims,ranks,core,noise,eta0", HOOI_CASES)
@pytest.mark.parametrize("init", ["st", "t"])
def test_hooi_fp64_matches_oracle(tals, dims, ranks, core, noise, eta0, init):
    p = W.planted(501, dims, ranks, core, noise, dtype=np.float64)
    a = _gpu(p.A)
    ctx = tals.Context(a, ranks, eta=eta0, max_sweeps=3, use_graph=False)
    G0, Us, _ = ctx.st_hosvd() if init == "st" else ctx.t_hosvd()
    us0 = [_host(u) for u in Us]
    G, Us, info = ctx.hooi(Us, tol=1e-13, max_iters=40, inner_eta=1e-15, inner_sweeps=30)
    ref = O.hooi(p.A, us0, tol=1e-13, max_iters=40)
    # r_0 of the same initial guess, then the same trajectory
    assert abs(info["resid"][0] - ref.resid[0]) <= 1e-12
    assert abs(info["iters"] - ref.iters) <= 1
    k = min(info["iters"], ref.iters)
    assert np.allclose(info["resid"][:k + 1], ref.resid[:k + 1], rtol=0, atol=1e-11)
    assert abs(info["resid"][-1] - ref.resid[-1]) <= 1e-11
    assert info["converged"]
    us = [_host(u) for u in Us]
    for n in range(len(dims)):
        assert np.allclose(us[n].T @ us[n], np.eye(ranks[n]), atol=1e-12)
        assert O.principal_angles(us[n], ref.U[n]).max() <= 1e-7
    b = O.reconstruct(_host(G), us)
    bref = O.reconstruct(ref.G, ref.U)
    assert np.abs(b - bref).max() <= 1e-9 * np.abs(p.A).max()
    # G is the projection of A on the returned factors
    assert np.allclose(_host(G), O.project(p.A, us), atol=1e-11 * np.abs(p.A).max())
    _stationary(p.A, us, 1e-8)
    # the residual never rose
    assert np.all(np.diff(info["resid"]) <= 1e-14)
    ctx.close()


def test_hooi_fp32_matches_oracle(tals):
    dims, ranks = (96, 80, 64), (8, 6, 5)
    p = W.planted(502, dims, ranks, "inv_k", 3e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    ctx = tals.Context(_gpu(p.A), ranks, eta=1e-2, max_sweeps=2, use_graph=False)
    _, Us, _ = ctx.st_hosvd()
    us0 = [_host(u) for u in Us]
    G, Us, info = ctx.hooi(Us, tol=1e-7, max_iters=20, inner_eta=1e-9, inner_sweeps=10)
    ref = O.hooi(a64, us0, tol=1e-7, max_iters=20)
    us = [_host(u) for u in Us]
    # the residual of the returned (G, U), evaluated exactly on the host
    own = O.rel_error(a64, _host(G), us)
    assert abs(own - ref.resid[-1]) <= 2e-5 * ref.resid[-1]
    assert abs(info["resid"][-1] - ref.resid[-1]) <= 2e-5 * ref.resid[-1] + 1e-6
    for n in range(3):
        assert O.principal_angles(us[n], ref.U[n]).max() <= 1e-3
    assert info["resid"][-1] <= info["resid"][0] + 1e-6
    ctx.close()


def test_hooi_limits_and_edges(tals):
    p = W.planted(503, (20, 16, 12), (3, 3, 2), "gauss", 1e-2, dtype=np.float64)
    ctx = tals.Context(_gpu(p.A), (3, 3, 2), eta=1e-2, max_sweeps=2, use_graph=False)
    _, Us, _ = ctx.st_hosvd()
    us0 = [_host(u) for u in Us]
    # one cycle exactly, and a huge tolerance that stops after the first cycle
    G1, U1, info1 = ctx.hooi([u.clone() for u in Us], tol=0.0, max_iters=1)
    assert info1["iters"] == 1 and not info1["converged"] and len(info1["resid"]) == 2
    _, _, info2 = ctx.hooi([u.clone() for u in Us], tol=1.0, max_iters=10)
    assert info2["iters"] == 1 and info2["converged"]
    ref = O.hooi(p.A, us0, tol=0.0, max_iters=1)
    assert abs(info1["resid"][1] - ref.resid[1]) <= 1e-11
    # an exact low-rank tensor from a poor start: the residual falls to rounding level
    q = W.planted(504, (18, 14, 10), (2, 3, 2), "gauss", 0.0, dtype=np.float64)
    c2 = tals.Context(_gpu(q.A), (2, 3, 2), eta=1e-1, max_sweeps=1, use_graph=False)
    _, V, _ = c2.t_hosvd()
    _, V, info3 = c2.hooi(V, tol=1e-15, max_iters=30)
    assert info3["resid"][-1] < 1e-7
    for n in range(3):
        assert O.principal_angles(_host(V[n]), q.factors[n]).max() < 1e-7
    with pytest.raises(ValueError):
        ctx.hooi(Us, max_iters=0)
    with pytest.raises(ValueError):
        ctx.hooi(Us[:2])
    ctx.close()
    c2.close()


# ---------------------------------------------------------------- singular vectors
def _check_svec(u_gpu, s_gpu, u_ref, s_ref, stol, utol):
    assert np.allclose(s_gpu, s_ref, rtol=stol, atol=0)
    # the sign rule on the GPU's own output
    idx = np.argmax(np.abs(u_gpu), axis=0)
    assert np.all(u_gpu[idx, np.arange(u_gpu.shape[1])] > 0)
    # against the oracle (same sign rule; align anyway so that a near-tie in the
    # largest entry cannot flip a column on one side only)
    sgn = np.sign(np.sum(u_gpu * u_ref, axis=0))
    assert np.abs(u_gpu - u_ref * sgn).max() <= utol


SVEC_CASES = [
    ((30, 24, 20), (5, 4, 4), np.float64, 1e-10, 1e-8),
    ((33, 17, 21), (1, 5, 5), np.float64, 1e-10, 1e-8),      # R = 1
    ((33, 17, 21), (3, 5, 7), np.float64, 1e-10, 1e-8),      # odd ranks
    ((128, 96, 64), (8, 8, 6), np.float32, 1e-5, 2e-3),
]


@pytest.mark.parametrize("dims,ranks,dt,stol,utol", SVEC_CASES)
def test_singular_vectors_match_oracle(tals, dims, ranks, dt, stol, utol):
    p = W.planted(510, dims, ranks, "inv_k", 1e-2, dtype=dt)
    a64 = p.A.astype(np.float64)
    ctx = tals.Context(_gpu(p.A), ranks, eta=1e-8 if dt == np.float64 else 1e-6,
                       use_graph=False)
    _, Us, _ = ctx.t_hosvd()
    for n in range(len(dims)):
        U, sig = ctx.singular_vectors(n, Us[n])
        uo, so = O.singular_vectors(a64, n, _host(Us[n]))
        _check_svec(_host(U), np.array(sig), uo, so, stol, utol)
        # U^(n) spans the same subspace as the basis it came from
        assert O.principal_angles(_host(U), _host(Us[n])).max() <= (1e-10 if dt == np.float64 else 1e-4)
    ctx.close()


def test_singular_vectors_from_an_exact_basis(tals):
    """Qhat a rotated exact leading basis of A_(n): the result is the leading
    singular triplet of A_(n) itself (numpy's SVD of the unfolding)."""
    p = W.planted(511, (48, 40, 36), (8, 6, 5), "inv_k", 1e-2, dtype=np.float64)
    ctx = tals.Context(_gpu(p.A), (8, 6, 5), use_graph=False)
    rng = np.random.default_rng(3)
    for n, r in enumerate((8, 6, 5)):
        m = O.unfold(p.A, n)
        u, s, _ = np.linalg.svd(m, full_matrices=False)
        rot = np.linalg.qr(rng.standard_normal((r, r)))[0]
        U, sig = ctx.singular_vectors(n, _gpu(u[:, :r] @ rot))
        _check_svec(_host(U), np.array(sig), O.sign_fix(u[:, :r]), s[:r], 1e-10, 1e-8)
    ctx.close()


def test_singular_vectors_rank64(tals):
    """The largest supported rank: a 64 x 64 Gram through the Jacobi kernel."""
    dims, ranks = (128, 80, 72), (64, 16, 16)
    p = W.planted(512, dims, ranks, "ratio", 1e-3, dtype=np.float64, ratio=0.95)
    ctx = tals.Context(_gpu(p.A), ranks, eta=1e-10, use_graph=False)
    _, Us, _ = ctx.t_hosvd()
    U, sig = ctx.singular_vectors(0, Us[0])
    uo, so = O.singular_vectors(p.A, 0, _host(Us[0]))
    _check_svec(_host(U), np.array(sig), uo, so, 1e-9, 1e-6)
    with pytest.raises(ValueError):
        ctx.singular_vectors(3, Us[0])
    with pytest.raises(ValueError):
        ctx.singular_vectors(0, Us[0], U=Us[0])
    ctx.close()
