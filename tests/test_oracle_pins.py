"""Pins for the FP64 oracle: each check ties an oracle function to something
other than itself -- published test vectors, textbook SVD results, closed
forms from the paper's appendix, invariants, brute force on tiny inputs, and
finite differences. CPU only."""
import itertools
import os

import numpy as np
import pytest

from oracle import tucker_oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator
def _golden_splitmix():
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            seed, count = int(parts[0]), int(parts[1])
            vals = [int(x, 0) for x in parts[2:2 + count]]
            rows.append((seed, vals))
    return rows


def test_splitmix64_published_vectors():
    for seed, vals in _golden_splitmix():
        got = [int(x) for x in O.splitmix64_stream(seed, len(vals))]
        assert got == vals


def test_splitmix64_random_access_matches_stream():
    full = O.splitmix64_stream(99, 40)
    part = O.splitmix64_stream(99, 10, start=30)
    assert np.array_equal(full[30:], part)


def test_init_sketch_mapping_and_uniformity():
    s = O.init_sketch(0, 0, 4, 1)
    # entry (0,0) is output 0 of the seed-0 stream, top 24 bits / 2^24
    assert s[0, 0] == (0xE220A8397B1DCDAF >> 40) / float(1 << 24)
    s = O.init_sketch(7, 2, 4000, 8)
    assert s.min() >= 0.0 and s.max() < 1.0
    assert np.all(s * (1 << 24) == np.floor(s * (1 << 24)))       # 24-bit grid
    assert abs(s.mean() - 0.5) < 0.01 and abs(s.var() - 1.0 / 12) < 0.005
    # mode enters the state: different modes give different matrices
    assert not np.array_equal(O.init_sketch(7, 0, 10, 3), O.init_sketch(7, 1, 10, 3))
    assert np.linalg.matrix_rank(s) == 8                              # dense, full rank


# ---------------------------------------------------------------- Sec. 2 notation
def _brute_unfold(x, n):
    shape = x.shape
    N = len(shape)
    J = int(np.prod([shape[m] for m in range(N) if m != n]))
    out = np.zeros((shape[n], J))
    for idx in itertools.product(*[range(s) for s in shape]):
        j = 0
        for m in range(N):                       # row-major over remaining modes
            if m == n:
                continue
            j = j * shape[m] + idx[m]
        out[idx[n], j] = x[idx]
    return out


def test_unfold_fold_bruteforce():
    x = np.arange(3 * 4 * 5 * 2, dtype=np.float64).reshape(3, 4, 5, 2) * 0.5 - 7
    for n in range(4):
        m = O.unfold(x, n)
        assert np.array_equal(m, _brute_unfold(x, n))
        assert np.array_equal(O.fold(m, n, x.shape), x)


def test_mode_product_bruteforce():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5))
    u = rng.standard_normal((2, 4))
    y = O.mode_product(x, u, 1)
    ref = np.zeros((3, 2, 5))
    for a in range(3):
        for j in range(2):
            for c in range(5):
                ref[a, j, c] = sum(x[a, i, c] * u[j, i] for i in range(4))
    assert np.allclose(y, ref, rtol=0, atol=1e-13)
    # unfolding identity: (X x_n U)_(n) = U X_(n)
    assert np.allclose(O.unfold(y, 1), u @ O.unfold(x, 1), atol=1e-13)


def test_frob2_bruteforce():
    x = np.arange(24, dtype=np.float32).reshape(2, 3, 4)
    assert O.frob2(x) == float(sum(v * v for v in range(24)))


def test_qr_pos_properties():
    rng = np.random.default_rng(2)
    y = rng.standard_normal((30, 6))
    q, r = O.qr_pos(y)
    assert np.allclose(q @ r, y, atol=1e-13)
    assert np.allclose(q.T @ q, np.eye(6), atol=1e-14)
    assert np.allclose(np.tril(r, -1), 0)
    assert np.all(np.diag(r) > 0)
    # the positive-diagonal QR factor is the classical Gram-Schmidt basis
    gs = np.zeros_like(y)
    for k in range(6):
        v = y[:, k] - gs[:, :k] @ (gs[:, :k].T @ y[:, k])
        v = v - gs[:, :k] @ (gs[:, :k].T @ v)
        gs[:, k] = v / np.linalg.norm(v)
    assert np.allclose(gs, q, atol=1e-12)


def test_principal_angles_known():
    e = np.eye(5)
    for th in [1e-9, 1e-4, 0.3, 1.2]:
        v = np.cos(th) * e[:, :1] + np.sin(th) * e[:, 1:2]
        a = O.principal_angles(e[:, :1], v)
        assert abs(a[0] - th) < 1e-12 * max(1, th) + 1e-15
    u = e[:, :2]
    v = np.c_[e[:, 1], np.cos(0.5) * e[:, 0] + np.sin(0.5) * e[:, 3]]
    assert np.allclose(O.principal_angles(u, v), [0.0, 0.5], atol=1e-12)


# ---------------------------------------------------------------- Alg. 3
def _spectral_matrix(m, n, s, seed):
    rng = np.random.default_rng(seed)
    u = np.linalg.qr(rng.standard_normal((m, len(s))))[0]
    v = np.linalg.qr(rng.standard_normal((n, len(s))))[0]
    return u * s @ v.T, u, v


def test_als_matrix_reduces_to_truncated_svd():
    # N = 2: ALS converges to the dominant subspace (Thm. 2) and the
    # Eckart-Young error sqrt(sum_{k>r} s_k^2).
    s = np.array([10, 8, 6, 5, 4, 1.0, 0.5, 0.3, 0.2, 0.1])
    m, u, _ = _spectral_matrix(40, 60, s, 3)
    r = 5
    # the stop rule sees the error, which is second order in the angle: pin the
    # subspace with a fixed sweep count and the error with the tolerance run
    fixed = O.als(m, r, eta=-1, norm_a=np.linalg.norm(m), seed=11, max_sweeps=60)
    res = O.als(m, r, eta=1e-15, norm_a=np.linalg.norm(m), seed=11, max_sweeps=200)
    assert res.converged
    ang = O.principal_angles(fixed.L, u[:, :r])
    assert ang.max() < 1e-10
    ey = np.sqrt(np.sum(s[r:] ** 2))
    assert abs(res.err - ey) <= 1e-12 * np.linalg.norm(m)


def test_als_error_nonincreasing_and_ls_optimal():
    rng = np.random.default_rng(4)
    m = rng.standard_normal((25, 70)) + 3 * np.outer(rng.standard_normal(25), rng.standard_normal(70))
    res = O.als(m, 4, eta=-1, norm_a=np.linalg.norm(m), seed=5, max_sweeps=12)
    e = np.array(res.errs)
    assert len(e) == 12 and not res.converged
    assert np.all(np.diff(e) <= 1e-12 * e[0])
    # R_k solves the LS problem min_R ||L R^T - A|| (Remark 2 / lstsq)
    rt = np.linalg.lstsq(res.L, m, rcond=None)[0]
    assert np.allclose(rt.T, res.R, atol=1e-10)
    # e_k agrees with the projection identity ||A||^2 - ||P_L A||^2
    q = np.linalg.qr(res.L)[0]
    e_id = np.sqrt(np.sum(m ** 2) - np.sum((q.T @ m) ** 2))
    assert abs(e_id - res.err) < 1e-9 * np.linalg.norm(m)


def test_als_one_step_matches_closed_form_E22():
    # Appendix A, Eq. (2.2): L_{k+1} = A A^T L_k (L_k^T A A^T L_k)^{-1} (L_k^T L_k).
    rng = np.random.default_rng(6)
    m = rng.standard_normal((20, 50))
    l0 = rng.standard_normal((20, 3))           # deliberately non-orthonormal
    r2 = O.als(m, 3, eta=-1, norm_a=1.0, max_sweeps=2, l0=l0)
    aat = m @ m.T
    l1 = aat @ l0 @ np.linalg.inv(l0.T @ aat @ l0) @ (l0.T @ l0)
    assert np.allclose(r2.L, l1, rtol=1e-10, atol=1e-12)


def test_stop_rule_fires_at_the_first_qualifying_sweep():
    # Eq. 5.01: the loop ends at the first k >= 1 with |e_{k-1} - e_k| <= eta ||A||_F.
    # The error sequence comes from a run that never stops (eta < 0); the stop
    # index is found in it directly, and the stopped run must end exactly there
    # with the same errors
    s = np.array([10.0, 9.0, 8.0, 4.0, 2.0, 1.0, 0.5])
    m, _, _ = _spectral_matrix(30, 60, s, 12)
    na = np.linalg.norm(m)
    free = O.als(m, 3, eta=-1.0, norm_a=na, seed=4, max_sweeps=40)
    assert free.sweeps == 40 and not free.converged
    d = np.abs(np.diff(np.array(free.errs)))
    for eta in (1e-3, 1e-6, 1e-9):
        hits = np.nonzero(d <= eta * na)[0]
        assert hits.size > 0
        k_stop = int(hits[0]) + 1                  # d[k-1] = |e_k - e_{k-1}|
        res = O.als(m, 3, eta=eta, norm_a=na, seed=4, max_sweeps=40)
        assert res.converged and res.sweeps == k_stop + 1
        assert res.errs == free.errs[:k_stop + 1]
    # max_sweeps bounds the loop when the rule never fires
    res = O.als(m, 3, eta=0.0, norm_a=na, seed=4, max_sweeps=5)
    assert res.sweeps == 5 and not res.converged


def test_als_literal_iteration_is_stationary_at_convergence():
    s = np.array([9.0, 7, 5, 0.01, 0.005])
    m, _, _ = _spectral_matrix(15, 30, s, 7)
    a = O.als(m, 3, eta=-1, norm_a=1.0, seed=1, max_sweeps=30)
    b = O.als(m, 3, eta=-1, norm_a=1.0, seed=1, max_sweeps=31)
    assert np.allclose(a.L, b.L, atol=1e-12)


def test_als_reorth_invariance():
    rng = np.random.default_rng(8)
    m = rng.standard_normal((18, 40))
    a = O.als(m, 4, eta=-1, norm_a=1.0, seed=2, max_sweeps=10)
    b = O.als(m, 4, eta=-1, norm_a=1.0, seed=2, max_sweeps=10, reorth=True)
    assert np.allclose(a.errs, b.errs, rtol=1e-11)
    assert O.principal_angles(a.L, b.L).max() < 1e-9


def test_als_convergence_rate_theorem2():
    # q-linear rate ~ sigma_{r+1}^2 / sigma_r^2 of the subspace distance (Thm. 2)
    s = np.array([10.0, 9.0, 8.0, 4.0, 2.0, 1.0, 0.5])
    m, u, _ = _spectral_matrix(30, 45, s, 9)
    r = 3
    ang = []
    for k in range(1, 9):
        res = O.als(m, r, eta=-1, norm_a=1.0, seed=3, max_sweeps=k)
        ang.append(O.principal_angles(res.L, u[:, :r]).max())
    ratios = np.array(ang[3:]) / np.array(ang[2:-1])
    expect = (s[r] / s[r - 1]) ** 2
    assert np.all(np.abs(ratios - expect) < 0.1 * expect)


def test_als_exact_recovery_and_full_rank_edge():
    m, _, _ = _spectral_matrix(12, 30, np.array([5.0, 3, 2]), 10)
    res = O.als(m, 3, eta=1e-12, norm_a=np.linalg.norm(m), seed=4)
    assert res.errs[0] <= 1e-12 * np.linalg.norm(m)      # L0 already spans R(A)
    assert res.converged and res.sweeps == 2
    # r = min(m, n): ALS reproduces the matrix exactly (reading R9)
    rng = np.random.default_rng(11)
    sq = rng.standard_normal((6, 9))
    res = O.als(sq, 6, eta=1e-12, norm_a=np.linalg.norm(sq), seed=1)
    assert res.err < 1e-12 * np.linalg.norm(sq) and res.converged


# ---------------------------------------------------------------- Prop. 1
def test_order_prop1_bruteforce():
    dims = [40, 40, 40, 40]
    for ranks in [(3, 9, 5, 7), (8, 2, 2, 6), (4, 4, 4, 4)]:
        costs = {o: O.st_cost(dims, ranks, o) for o in itertools.permutations(range(4))}
        best = min(costs.values())
        assert costs[tuple(O.default_order(ranks))] == best


def test_st_cost_hand_value():
    # dims (10, 20), ranks (2, 3), order (0, 1):  2*10*20 + 2*3*20 = 520
    assert O.st_cost([10, 20], [2, 3], [0, 1]) == 520
    assert O.default_order([5, 2, 5, 1]) == [3, 1, 0, 2]


# ---------------------------------------------------------------- Alg. 1/2/4/5
def _planted(dims, ranks, noise, seed=123, core="gauss"):
    return W.planted(seed, dims, ranks, core, noise, dtype=np.float64).A


def test_hosvd_svd_order2_is_truncated_svd():
    s = np.array([6.0, 4, 3, 1, 0.5, 0.2])
    m, u, v = _spectral_matrix(14, 11, s, 12)
    for res in (O.t_hosvd_svd(m, [3, 3]), O.st_hosvd_svd(m, [3, 3])):
        assert abs(O.rel_error(m, res.G, res.U) * np.linalg.norm(m) -
                   np.sqrt(np.sum(s[3:] ** 2))) < 1e-12
        assert O.principal_angles(res.U[0], u[:, :3]).max() < 1e-10


@pytest.mark.parametrize("driver", ["st", "t"])
def test_hosvd_als_matches_svd_at_tight_tolerance(driver):
    a = _planted((9, 8, 7), (3, 4, 2), 0.05)
    ranks = [3, 4, 2]
    if driver == "st":
        ref = O.st_hosvd_svd(a, ranks)
        got = O.st_hosvd_als(a, ranks, eta=-1, seed=5, max_sweeps=300)
    else:
        ref = O.t_hosvd_svd(a, ranks)
        got = O.t_hosvd_als(a, ranks, eta=-1, seed=5, max_sweeps=300)
    for n in range(3):
        assert O.principal_angles(got.U[n], ref.U[n]).max() < 1e-8
        assert abs(got.err_per_mode[n] - ref.err_per_mode[n]) < 1e-12 * got.norm_a
    ea = O.rel_error(a, got.G, got.U)
    eb = O.rel_error(a, ref.G, ref.U)
    assert abs(ea - eb) < 1e-12


@pytest.mark.parametrize("driver", ["st", "t"])
def test_hosvd_als_invariants(driver):
    a = _planted((10, 9, 8, 6), (3, 2, 4, 2), 0.1, seed=7)
    ranks = [3, 2, 4, 2]
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    res = f(a, ranks, eta=1e-6, seed=3)
    for n, u in enumerate(res.U):
        assert u.shape == (a.shape[n], ranks[n])
        assert np.allclose(u.T @ u, np.eye(ranks[n]), atol=1e-14)
    err2 = O.frob2(a - O.reconstruct(res.G, res.U))
    assert abs(err2 - (O.frob2(a) - O.frob2(res.G))) < 1e-11 * O.frob2(a)
    if driver == "st":
        # Lemma 2 setting: st-HOSVD squared error = sum of mode-wise errors
        assert abs(err2 - sum(e * e for e in res.err_per_mode)) < 1e-11 * O.frob2(a)


def test_hosvd_als_exact_recovery():
    a = _planted((12, 10, 9), (3, 2, 4), 0.0, seed=8)
    for f in (O.st_hosvd_als, O.t_hosvd_als):
        res = f(a, [3, 2, 4], eta=1e-12, seed=1)
        assert O.rel_error(a, res.G, res.U) < 1e-12
        assert all(res.converged)
        assert all(s == 2 for s in res.sweeps)


def test_error_bounds_lemma2_thm4():
    a = _planted((11, 10, 9), (3, 3, 3), 0.2, seed=9)
    ranks = [3, 3, 3]
    norm2 = O.frob2(a)
    gam = []
    for n in range(3):
        sv = np.linalg.svd(O.unfold(a, n), compute_uv=False)
        gam.append(float(np.sum(sv[ranks[n]:] ** 2)))
    t_svd = O.t_hosvd_svd(a, ranks)
    assert O.frob2(a - O.reconstruct(t_svd.G, t_svd.U)) <= sum(gam) * (1 + 1e-12)
    for eta in (1e-2, 1e-4):
        for f in (O.st_hosvd_als, O.t_hosvd_als):
            res = f(a, ranks, eta=eta, seed=2)
            rel = O.rel_error(a, res.G, res.U)
            bound = np.sqrt(sum(eta ** 2 + g / norm2 for g in gam))   # Eq. 5.62
            assert rel <= bound * (1 + 1e-12)


def test_st_order_changes_only_through_order():
    a = _planted((9, 8, 7), (2, 3, 4), 0.05, seed=10)
    r1 = O.st_hosvd_als(a, [2, 3, 4], eta=-1, seed=1, order=[0, 1, 2], max_sweeps=300)
    r2 = O.st_hosvd_svd(a, [2, 3, 4], order=[0, 1, 2])
    assert abs(O.rel_error(a, r1.G, r1.U) - O.rel_error(a, r2.G, r2.U)) < 1e-12


# ---------------------------------------------------------------- differentiation
def _fd_check(fun, x, grad, h=1e-6, rtol=1e-6):
    num = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        num[i] = (fun(xp) - fun(xm)) / (2 * h)
    assert np.linalg.norm(num - grad) <= rtol * max(np.linalg.norm(grad), 1e-30)


def test_recon_loss_grad_finite_differences():
    rng = np.random.default_rng(13)
    a = rng.standard_normal((6, 5, 4))
    us = [np.linalg.qr(rng.standard_normal((d, r)))[0] for d, r in zip(a.shape, (3, 2, 2))]
    us[1] = us[1] * 1.3          # non-orthonormal: exercises every adjoint term
    ga, gu = O.recon_loss_grad(a, us)
    _fd_check(lambda x: O.recon_loss(x, us), a, ga)
    for n in range(3):
        def f(x, n=n):
            v = list(us); v[n] = x
            return O.recon_loss(a, v)
        _fd_check(f, us[n], gu[n])


def test_project_and_reconstruct_vjp_inner_products():
    rng = np.random.default_rng(14)
    a = rng.standard_normal((5, 4, 6))
    us = [rng.standard_normal((d, r)) for d, r in zip(a.shape, (2, 3, 2))]
    g = rng.standard_normal((2, 3, 2))
    gbar = rng.standard_normal((2, 3, 2))
    bbar = rng.standard_normal(a.shape)
    # <dG, Gbar> for a perturbation of A equals <dA, Abar> (linearity in A)
    dA = rng.standard_normal(a.shape)
    abar, ubar = O.project_vjp(a, us, gbar)
    assert abs(np.sum(O.project(dA, us) * gbar) - np.sum(dA * abar)) < 1e-11
    # FD in each U for both maps
    for n in range(3):
        def fp(x, n=n):
            v = list(us); v[n] = x
            return float(np.sum(O.project(a, v) * gbar))
        _fd_check(fp, us[n], ubar[n])
    gb, ub = O.reconstruct_vjp(g, us, bbar)
    _fd_check(lambda x: float(np.sum(O.reconstruct(x, us) * bbar)), g, gb)
    for n in range(3):
        def fr(x, n=n):
            v = list(us); v[n] = x
            return float(np.sum(O.reconstruct(g, v) * bbar))
        _fd_check(fr, us[n], ub[n])


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_dropped_inverse(monkeypatch):
    """Plant a mistake in the oracle (drop (R^T R)^{-1} in the L-update) and
    check that the closed-form pin fails."""
    rng = np.random.default_rng(6)
    m = rng.standard_normal((20, 50))
    l0 = rng.standard_normal((20, 3))
    real_solve = np.linalg.solve
    calls = {"n": 0}

    def broken(a, b):
        calls["n"] += 1
        if calls["n"] % 2 == 0:              # every L-update
            return b
        return real_solve(a, b)
    monkeypatch.setattr(O.np.linalg, "solve", broken)
    r2 = O.als(m, 3, eta=-1, norm_a=1.0, max_sweeps=2, l0=l0)
    monkeypatch.undo()
    aat = m @ m.T
    l1 = aat @ l0 @ np.linalg.inv(l0.T @ aat @ l0) @ (l0.T @ l0)
    assert not np.allclose(r2.L, l1, rtol=1e-6)


def test_pins_catch_a_transposed_operand(monkeypatch):
    """Plant a transposed factor in the mode product (contract X's mode with U's
    first index instead of its second) and check that the brute-force pin fails."""
    def transposed(x, u, n):
        return np.moveaxis(np.tensordot(u, x, axes=([0], [n])), 0, n)
    rng = np.random.default_rng(21)
    x = rng.standard_normal((3, 4, 5))
    u = rng.standard_normal((4, 4))                # square, so the shapes still agree
    monkeypatch.setattr(O, "mode_product", transposed)
    y = O.mode_product(x, u, 1)
    monkeypatch.undo()
    ref = np.zeros((3, 4, 5))
    for a in range(3):
        for j in range(4):
            for c in range(5):
                ref[a, j, c] = sum(x[a, i, c] * u[j, i] for i in range(4))
    assert not np.allclose(y, ref, atol=1e-6)


def test_pins_catch_a_sign_error_in_an_adjoint(monkeypatch):
    """Plant a wrong sign in one factor's term of the reconstruction adjoint and
    check that the finite-difference pin fails."""
    real = O.reconstruct_vjp

    def broken(g, us, b_bar):
        gb, ub = real(g, us, b_bar)
        return gb, [ub[0], -ub[1], ub[2]]
    rng = np.random.default_rng(22)
    g = rng.standard_normal((2, 3, 2))
    us = [rng.standard_normal((d, r)) for d, r in zip((5, 4, 6), (2, 3, 2))]
    bbar = rng.standard_normal((5, 4, 6))
    monkeypatch.setattr(O, "reconstruct_vjp", broken)
    _, ub = O.reconstruct_vjp(g, us, bbar)
    monkeypatch.undo()

    def fr(x):
        v = list(us); v[1] = x
        return float(np.sum(O.reconstruct(g, v) * bbar))
    with pytest.raises(AssertionError):
        _fd_check(fr, us[1], ub[1])


def test_workload_generator_recipe():
    p = W.planted(5, (10, 9, 8), (3, 2, 4), "inv_k", 1e-2, dtype=np.float64)
    for u in p.factors:
        assert np.allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-14)
    e = p.A - p.A0
    assert abs(np.linalg.norm(e) / np.linalg.norm(p.A0) - 1e-2) < 1e-12
    for n in range(3):                       # A0 has the planted multilinear rank
        sv = np.linalg.svd(O.unfold(p.A0, n), compute_uv=False)
        assert sv[p.core.shape[n]] < 1e-12 * sv[0]
    again = W.planted(5, (10, 9, 8), (3, 2, 4), "inv_k", 1e-2, dtype=np.float64)
    assert np.array_equal(again.A, p.A)


def test_batched_workload_recipe():
    # 4096 uneven third-order tensors: sizes ~ U{16..96}, ranks ~ U{4..16}, every
    # sequential truncation feasible (R_n <= I_n and R_n <= the product of the others)
    shapes = W.batched_shapes(W.SEED_BASE + 3, 4096)
    assert len(shapes) == 4096 and shapes == W.batched_shapes(W.SEED_BASE + 3, 4096)
    dims = np.array([d for d, _ in shapes])
    ranks = np.array([r for _, r in shapes])
    assert dims.min() == 16 and dims.max() == 96 and ranks.min() == 4 and ranks.max() == 16
    assert np.all(ranks <= dims)
    for n in range(3):
        other = np.prod(np.delete(ranks, n, axis=1), axis=1)
        assert np.all(ranks[:, n] <= other)
    # the sizes spread over the whole range (not a few repeated shapes)
    assert len({d for d, _ in shapes}) > 3000

