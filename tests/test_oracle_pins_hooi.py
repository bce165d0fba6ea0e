"""Pins for the oracle's HOOI (Sec. 6.3), its singular-vector recovery (Sec. 5,
after Alg. 4) and the CP-model workload generator (Sec. 6.1.1). Each check ties
the function to something other than itself: the truncated SVD of a matrix
(Eckart-Young), the stationarity of a HOOI fixed point, monotonicity, planted
exact subspaces, and brute force. Three tests plant a mistake in the oracle and
check that a pin fails. CPU only."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
import workloads as W


def _rand_orth(rng, m, r):
    q, _ = np.linalg.qr(rng.standard_normal((m, r)))
    return q


def _spectrum_matrix(rng, m, n, sv):
    u = _rand_orth(rng, m, len(sv))
    v = _rand_orth(rng, n, len(sv))
    return (u * np.asarray(sv)) @ v.T


def _angles(u, v):
    qu = np.linalg.qr(u)[0]
    qv = np.linalg.qr(v)[0]
    res = qv - qu @ (qu.T @ qv)
    return np.linalg.svd(res, compute_uv=False)


def _y_modes_3(a, us):
    """Y_n = A x_{m != n} U_m^T written out with einsum (3-way), as I_n x rest."""
    u0, u1, u2 = us
    y0 = np.einsum("ijk,jb,kc->ibc", a, u1, u2).reshape(a.shape[0], -1)
    y1 = np.einsum("ijk,ia,kc->jac", a, u0, u2).reshape(a.shape[1], -1)
    y2 = np.einsum("ijk,ia,jb->kab", a, u0, u1).reshape(a.shape[2], -1)
    return [y0, y1, y2]


# ---------------------------------------------------------------- HOOI
def _matrix_case():
    rng = np.random.default_rng(31)
    sv = [10.0, 8.0, 6.5, 5.0, 1.0, 0.7, 0.5, 0.3, 0.2, 0.1]
    a = _spectrum_matrix(rng, 30, 25, sv)
    r = (4, 4)
    us0 = [_rand_orth(rng, 30, 4), _rand_orth(rng, 25, 4)]
    return a, r, us0, sv


def test_hooi_on_a_matrix_reaches_the_truncated_svd():
    """N = 2: HOOI is an alternating subspace iteration whose fixed point is the
    rank-4 truncated SVD; its residual is Eckart-Young's sqrt(sum_{i>4} s_i^2)."""
    a, r, us0, sv = _matrix_case()
    h = O.hooi(a, us0, tol=1e-16, max_iters=400)
    s = np.linalg.svd(a, compute_uv=False)
    want = np.sqrt(np.sum(s[4:] ** 2)) / np.linalg.norm(a)
    assert abs(h.resid[-1] - want) <= 1e-12 * want
    u, _, vt = np.linalg.svd(a)
    assert np.max(_angles(h.U[0], u[:, :4])) < 1e-7
    assert np.max(_angles(h.U[1], vt[:4].T)) < 1e-7


def test_hooi_residual_is_monotone_and_never_above_the_start():
    p = W.planted(41, (14, 12, 10), (3, 4, 2), "gauss", 5e-2, dtype=np.float64)
    rng = np.random.default_rng(5)
    us0 = [_rand_orth(rng, d, r) for d, r in zip((14, 12, 10), (3, 4, 2))]
    h = O.hooi(p.A, us0, tol=1e-15, max_iters=60)
    rs = np.array(h.resid)
    assert np.all(np.diff(rs) <= 1e-14)
    assert rs[-1] <= rs[0]
    assert h.converged and h.iters >= 2
    # the initial residual is that of the initial guess, by explicit reconstruction
    g0 = np.einsum("ijk,ia,jb,kc->abc", p.A, *us0)
    b0 = np.einsum("abc,ia,jb,kc->ijk", g0, *us0)
    assert abs(rs[0] - np.linalg.norm(p.A - b0) / np.linalg.norm(p.A)) < 1e-14


def test_hooi_fixed_point_is_stationary():
    """At convergence every U_n spans the dominant invariant subspace of
    Y_(n) Y_(n)^T, with Y_n built from the other (converged) factors."""
    p = W.planted(42, (16, 13, 11), (4, 3, 3), "inv_k", 2e-2, dtype=np.float64)
    r0 = O.st_hosvd_als(p.A, (4, 3, 3), eta=1e-3, max_sweeps=3)
    h = O.hooi(p.A, r0.U, tol=1e-15, max_iters=100)
    ys = _y_modes_3(p.A, h.U)
    for n in range(3):
        m = ys[n] @ ys[n].T
        u = h.U[n]
        off = m @ u - u @ (u.T @ (m @ u))
        assert np.linalg.norm(off) <= 1e-9 * np.linalg.norm(m)
        top = np.sort(np.linalg.eigvalsh(m))[::-1][:u.shape[1]]
        mine = np.sort(np.linalg.eigvalsh(u.T @ m @ u))[::-1]
        assert np.allclose(mine, top, rtol=1e-10, atol=0)
    # the core is the projection on the converged factors
    g = np.einsum("ijk,ia,jb,kc->abc", p.A, *h.U)
    assert np.allclose(h.G, g, atol=1e-12 * np.abs(g).max())


def test_hooi_recovers_an_exact_low_rank_tensor():
    p = W.planted(43, (12, 11, 9), (3, 2, 3), "gauss", 0.0, dtype=np.float64)
    rng = np.random.default_rng(9)
    us0 = [_rand_orth(rng, d, r) for d, r in zip((12, 11, 9), (3, 2, 3))]
    h = O.hooi(p.A, us0, tol=1e-16, max_iters=200)
    assert h.resid[-1] < 1e-12
    for n in range(3):
        assert np.max(_angles(h.U[n], p.factors[n])) < 1e-8


def test_pins_catch_an_off_by_one_singular_vector(monkeypatch):
    """Plant a mistake (the subspace update keeps singular vectors 2..R+1) and
    check that the stationarity pin fails."""
    real = O._leading_left

    def shifted(m, r):
        u, s, vt = real(m, r + 1)
        return u[:, 1:r + 1], s, vt
    p = W.planted(42, (16, 13, 11), (4, 3, 3), "inv_k", 2e-2, dtype=np.float64)
    r0 = O.st_hosvd_als(p.A, (4, 3, 3), eta=1e-3, max_sweeps=3)
    monkeypatch.setattr(O, "_leading_left", shifted)
    h = O.hooi(p.A, r0.U, tol=1e-15, max_iters=30)
    monkeypatch.undo()
    ys = _y_modes_3(p.A, h.U)
    m = ys[0] @ ys[0].T
    top = np.sort(np.linalg.eigvalsh(m))[::-1][:4]
    mine = np.sort(np.linalg.eigvalsh(h.U[0].T @ m @ h.U[0]))[::-1]
    assert not np.allclose(mine, top, rtol=1e-6, atol=0)


# ---------------------------------------------------------------- singular vectors
def test_sign_fix_by_brute_force():
    u = np.array([[0.1, -0.9, 0.5],
                  [-0.8, 0.2, -0.5],
                  [0.3, 0.4, 0.1]])
    f = O.sign_fix(u)
    # column 0: largest |.| is -0.8 -> flip; column 1: -0.9 -> flip; column 2: a tie
    # of 0.5 and -0.5, the first (0.5) wins -> keep
    assert np.array_equal(f, u * np.array([-1.0, -1.0, 1.0]))


def test_singular_vectors_from_an_exact_basis_match_the_unfolding_svd():
    """With Qhat an arbitrary orthonormal basis of the leading R-dim left subspace
    of A_(n), Qhat U equals the leading left singular vectors of A_(n) and S its
    leading singular values, noise or not."""
    p = W.planted(44, (15, 12, 10), (4, 3, 3), "inv_k", 1e-2, dtype=np.float64)
    rng = np.random.default_rng(12)
    for n, r in enumerate((4, 3, 3)):
        m = np.moveaxis(p.A, n, 0).reshape(p.A.shape[n], -1)
        u, s, _ = np.linalg.svd(m, full_matrices=False)
        rot = _rand_orth(rng, r, r)
        q = u[:, :r] @ rot
        un, sn = O.singular_vectors(p.A, n, q)
        assert np.allclose(sn, s[:r], rtol=1e-12)
        # same singular vectors up to sign; the oracle's sign is the fixed one
        ref = u[:, :r] * np.sign(np.sum(u[:, :r] * un, axis=0))
        assert np.max(np.abs(un - ref)) < 1e-10
        idx = np.argmax(np.abs(un), axis=0)
        assert np.all(un[idx, np.arange(r)] > 0)


def test_singular_values_do_not_depend_on_the_basis():
    p = W.planted(45, (10, 9, 8), (3, 3, 2), "gauss", 5e-2, dtype=np.float64)
    rng = np.random.default_rng(13)
    q = _rand_orth(rng, 10, 3)
    u1, s1 = O.singular_vectors(p.A, 0, q)
    u2, s2 = O.singular_vectors(p.A, 0, q @ _rand_orth(rng, 3, 3))
    assert np.allclose(s1, s2, rtol=1e-12)
    assert np.allclose(u1, u2, atol=1e-10)
    # U^(n) lies in range(Qhat) and has orthonormal columns
    assert np.allclose(u1.T @ u1, np.eye(3), atol=1e-13)
    assert np.linalg.norm(u1 - q @ (q.T @ u1)) < 1e-13


def test_pins_catch_ascending_singular_values(monkeypatch):
    real = np.linalg.svd

    def ascending(x, full_matrices=True, compute_uv=True, **kw):
        if not compute_uv:
            return real(x, full_matrices=full_matrices, compute_uv=False)[::-1]
        u, s, vt = real(x, full_matrices=full_matrices)
        return u[:, ::-1], s[::-1], vt[::-1]
    p = W.planted(44, (15, 12, 10), (4, 3, 3), "inv_k", 1e-2, dtype=np.float64)
    m = np.moveaxis(p.A, 0, 0).reshape(15, -1)
    u, s, _ = real(m, full_matrices=False)
    monkeypatch.setattr(O.np.linalg, "svd", ascending)
    _, sn = O.singular_vectors(p.A, 0, u[:, :4])
    monkeypatch.undo()
    assert not np.allclose(sn, s[:4], rtol=1e-6)


# ---------------------------------------------------------------- CP workload
def test_cp_model_recipe():
    c0 = W.cp_model(7, 10, delta=0.0, dtype=np.float64)
    assert c0.A.shape == (10, 10, 1000) and len(c0.lam) == 2
    assert np.all((c0.lam >= 5) & (c0.lam <= 10))
    for f in c0.factors:
        assert np.allclose(np.linalg.norm(f, axis=0), 1.0, atol=1e-14)
    a, b, c = c0.factors
    brute = np.zeros((10, 10, 1000))
    for r in range(2):
        brute += c0.lam[r] * a[:, r][:, None, None] * b[:, r][None, :, None] * c[:, r][None, None, :]
    assert np.allclose(c0.A, brute, atol=1e-13)
    for n in range(3):                       # multilinear rank (R, R, R)
        sv = np.linalg.svd(np.moveaxis(c0.A, n, 0).reshape(c0.A.shape[n], -1),
                           compute_uv=False)
        assert sv[2] < 1e-12 * sv[0]
    c1 = W.cp_model(7, 10, delta=1e-4, dtype=np.float64)
    e = (c1.A - c0.A) / 1e-4                 # same seed: same factors, then the noise
    assert abs(np.std(e) - 1.0) < 0.02 and abs(np.mean(e)) < 0.02
    assert W.cp_model(7, 20).A.shape == (20, 20, 2000)
    assert len(W.cp_model(7, 20).lam) == 4


def test_tucker_model_device_recipe():
    """Sec. 6.1.2's Tucker model drawn with torch (here on the CPU): planted
    multilinear rank, the projection on the leading subspaces keeps the base's
    spectrum, absolute noise 1e-4, seeded."""
    torch = pytest.importorskip("torch")
    dims, ranks = (30, 9, 8, 7), (3, 2, 3, 2)
    a = W.tucker_model_device(11, dims, ranks, device="cpu").double().numpy()
    b = W.tucker_model_device(11, dims, ranks, device="cpu", base_only=True).double().numpy()
    e = (a - b) / 1e-4
    assert abs(np.std(e) - 1.0) < 0.05 and abs(np.mean(e)) < 0.05
    for n in range(4):
        sv = np.linalg.svd(O.unfold(b, n), compute_uv=False)
        assert sv[ranks[n]] < 1e-5 * sv[0]
    # the leading subspaces span the base's unfoldings
    us = [np.linalg.svd(O.unfold(b, n), full_matrices=False)[0][:, :ranks[n]] for n in range(4)]
    g = O.project(b, us)
    assert np.allclose(np.sort(np.abs(np.linalg.svd(O.unfold(g, 0), compute_uv=False))),
                       np.sort(np.linalg.svd(O.unfold(b, 0), compute_uv=False)[:3]), rtol=1e-5)
    again = W.tucker_model_device(11, dims, ranks, device="cpu").double().numpy()
    assert np.array_equal(a, again)
