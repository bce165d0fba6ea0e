"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (one Context, CUDA graph, default options of each precision).

Where the FP64 oracle finishes in seconds on the host (512^3, 128^4, the small
batched tensors) the GPU result is compared with it directly; on the 2 GiB
differentiation workload the checks are properties that hold at any size
(orthonormal factors, the core equal to the projection of A at sampled
entries, the reported error against ||A||^2 - ||G||^2), with every reference value
computed in FP64 on the host; its gradients are compared with the FP64 oracle's
in full (relative Frobenius 1e-4) and with FP64 central differences along four
seeded directions. A rank-64 decomposition on 1024-long modes is compared with
the oracle directly."""
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


def _orthonormality(Us):
    return max(float(np.abs(_np(u).T @ _np(u) - np.eye(u.shape[1])).max()) for u in Us)


def _sampled_core(a64, Us, G, rng, n=6):
    """max |G - A x U^T| / max |G| over n sampled core entries (FP64 on the host)."""
    us = [_np(u) for u in Us]
    g = _np(G)
    worst = 0.0
    a_idx = rng.choice(g.shape[0], size=min(n, g.shape[0]), replace=False)
    t1 = np.tensordot(us[0][:, a_idx].T, a64, axes=(1, 0))   # (n, I2, I3, ...)
    for m, a in enumerate(a_idx):
        idx = tuple(int(rng.integers(0, s)) for s in g.shape[1:])
        x = t1[m]
        for k, b in enumerate(idx):
            x = np.tensordot(us[k + 1][:, b], x, axes=(0, 0))
        worst = max(worst, abs(float(x) - g[(a,) + idx]))
    return worst / float(np.abs(g).max())


@pytest.mark.parametrize("precision", ["native", "mixed_bf16"])
def test_c2_512cube_vs_oracle(tals, precision):
    cfg = W.CONFIGS["c512_f32"]
    p = W.make(cfg)
    a64 = p.A.astype(np.float64)
    A = torch.from_numpy(p.A).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision=precision, use_graph=True)
    G, Us, st = ctx.st_hosvd()
    ctx.close()
    ref = O.st_hosvd_als(a64, cfg.ranks, eta=cfg.eta, seed=1)
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= 1e-6
    assert abs(st["rel_err"] - rel_own) <= 1e-6
    for n in range(3):
        assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= 1e-4
    assert _orthonormality(Us) <= 1e-5
    assert _sampled_core(a64, Us, G, np.random.default_rng(11)) <= 1e-4
    assert all(st["converged"])
    if precision == "mixed_bf16":
        assert st["bulk_sweeps"][st["order"][0]] >= 1


def test_c3_128quartic_mixed_vs_oracle(tals):
    cfg = W.CONFIGS["q128_f32"]
    p = W.make(cfg)
    a64 = p.A.astype(np.float64)
    A = torch.from_numpy(p.A).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="mixed_bf16", use_graph=True)
    G, Us, st = ctx.st_hosvd()
    ctx.close()
    ref = O.st_hosvd_als(a64, cfg.ranks, eta=cfg.eta, seed=1)
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= 1e-6
    for n in range(4):
        assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= 1e-4
    assert _orthonormality(Us) <= 1e-5
    assert st["bulk_sweeps"][st["order"][0]] >= 1


def test_c4_batched_4096_vs_oracle(tals):
    count, eta = 4096, 1e-6
    items = W.batched(W.SEED_BASE + 3, count)
    As = [torch.from_numpy(a).cuda() for a, _, _ in items]
    ranks = [r for _, _, r in items]
    runner = tals.BatchedRunner(As, ranks, eta=eta, seed=1)
    runner.run()
    sts = runner.stats()
    assert all(s["status"] == 0 for s in sts)
    worst_orth = 0.0
    for t in range(0, count, 97):
        worst_orth = max(worst_orth, _orthonormality(runner.Us[t]))
    assert worst_orth <= 1e-5
    rng = np.random.default_rng(5)
    for t in rng.choice(count, size=24, replace=False):
        a, dims, rk = items[int(t)]
        a64 = a.astype(np.float64)
        ref = O.st_hosvd_als(a64, rk, eta=eta, seed=1)
        own = O.rel_error(a64, _np(runner.Gs[t]), [_np(u) for u in runner.Us[t]])
        assert abs(own - O.rel_error(a64, ref.G, ref.U)) <= 1e-6
        for n in range(3):
            assert O.principal_angles(_np(runner.Us[t][n]), ref.U[n]).max() <= 1e-4


@pytest.fixture(scope="module")
def c5_input():
    return W.make(W.CONFIGS["d1024_f32"]).A


def test_c5_2gib_forward_properties(tals, c5_input):
    cfg = W.CONFIGS["d1024_f32"]
    a32 = c5_input
    A = torch.from_numpy(a32).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="native", use_graph=True)
    G, Us, st = ctx.st_hosvd()
    ctx.close()
    assert _orthonormality(Us) <= 1e-5
    a64 = a32.astype(np.float64)
    us = [_np(u) for u in Us]
    # the core is the projection of A: all core entries from one FP64 contraction chain
    g_ref = O.project(a64, us)
    g = _np(G)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    # reported error against ||A||^2 - ||G||^2 (orthonormal factors)
    na2 = O.frob2(a64)
    rel_id = np.sqrt(max(na2 - O.frob2(g_ref), 0.0) / na2)
    assert abs(st["rel_err"] - rel_id) <= 1e-6


def _perturbed(Us, seed, scale=0.05):
    """The factors moved by a seeded relative step (no longer orthonormal), as FP32:
    a general point of f(A, U), where both terms of every gradient are active."""
    rng = np.random.default_rng(seed)
    out = []
    for u in Us:
        h = _np(u)
        e = rng.standard_normal(h.shape)
        out.append((h + scale * np.linalg.norm(h) * e / np.linalg.norm(e)).astype(np.float32))
    return out


def _gradient_parity(tals, a32, us32, seed):
    """GPU FP32 gradients of f(A, U) = ||A - (A x U^T) x U||^2 against the FP64 oracle
    (relative Frobenius <= 1e-4), and four seeded directional central differences of
    f evaluated in FP64 on the host (two along A, h = 1e-3: f is quadratic in A; two
    along the factors, h = 1e-5), which must match the oracle's directional
    derivative to 1e-6 and the GPU's to 1e-4."""
    a64 = a32.astype(np.float64)
    us64 = [u.astype(np.float64) for u in us32]
    Ar = torch.from_numpy(a32).cuda().requires_grad_(True)
    Ur = [torch.from_numpy(u).cuda().requires_grad_(True) for u in us32]
    B = tals.tucker_reconstruct(tals.tucker_project(Ar, Ur), Ur)
    loss = ((Ar - B) ** 2).sum()
    loss.backward()
    ab, ub = O.recon_loss_grad(a64, us64)
    ga = Ar.grad.double()
    ab_d = torch.from_numpy(ab).cuda()
    rel_a = float(torch.linalg.vector_norm(ga - ab_d) / torch.linalg.vector_norm(ab_d))
    assert rel_a <= 1e-4, rel_a
    for n, (u, g) in enumerate(zip(Ur, ub)):
        rel_u = np.linalg.norm(_np(u.grad) - g) / np.linalg.norm(g)
        assert rel_u <= 1e-4, (n, rel_u)
    f64 = O.recon_loss(a64, us64)
    assert abs(float(loss.detach()) - f64) <= 1e-5 * f64
    rng = np.random.default_rng(seed)
    for k in range(4):
        if k < 2:
            va = rng.standard_normal(a64.shape)
            va *= np.linalg.norm(a64) / np.linalg.norm(va)
            vu = [np.zeros_like(u) for u in us64]
            h = 1e-3
        else:
            va = None
            vu = [rng.standard_normal(u.shape) for u in us64]
            vu = [v * np.linalg.norm(u) / np.linalg.norm(v) for u, v in zip(us64, vu)]
            h = 1e-5
        d_ref = sum(float(np.sum(g * v)) for g, v in zip(ub, vu))
        d_gpu = sum(float(np.sum(_np(u.grad) * v)) for u, v in zip(Ur, vu))
        if va is not None:
            va_d = torch.from_numpy(va).cuda()
            d_ref += float(torch.sum(ab_d * va_d))
            d_gpu += float(torch.sum(ga * va_d))
            del va_d
            fp = O.recon_loss(a64 + h * va, us64)
            fm = O.recon_loss(a64 - h * va, us64)
        else:
            fp = O.recon_loss(a64, [u + h * v for u, v in zip(us64, vu)])
            fm = O.recon_loss(a64, [u - h * v for u, v in zip(us64, vu)])
        fd = (fp - fm) / (2 * h)
        assert abs(fd - d_ref) <= 1e-6 * abs(d_ref), (k, fd, d_ref)
        assert abs(fd - d_gpu) <= 1e-4 * abs(fd), (k, fd, d_gpu)
        del va


def test_c5_2gib_gradients_vs_oracle(tals, c5_input):
    """The full 1024 x 1024 x 512 workload: gradients w.r.t. A and every U_n at the
    st-HOSVD factors moved to a general point, against the FP64 oracle and FP64
    central differences on the host."""
    cfg = W.CONFIGS["d1024_f32"]
    A = torch.from_numpy(c5_input).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="native", use_graph=True)
    _, Us, _ = ctx.st_hosvd()
    ctx.close()
    del A
    _gradient_parity(tals, c5_input, _perturbed(Us, 17), 23)


def test_rank64_decomposition_vs_oracle(tals):
    """Rank 64 (the context limit) on 1024-long modes in an oracle-compared
    decomposition: 1024 x 256 x 64 at (64, 64, 32), FP32, fixed sweeps (factors
    elementwise 1e-3, angles 1e-4, relative error 1e-6) and a tolerance run
    (sweeps within one)."""
    dims, ranks = (1024, 256, 64), (64, 64, 32)
    p = W.planted(W.SEED_BASE + 31, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    A = torch.from_numpy(p.A).cuda()
    for driver in ("st", "t"):
        f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
        g = tals.st_hosvd if driver == "st" else tals.t_hosvd
        ref = f(a64, ranks, eta=-1.0, seed=4, max_sweeps=3)
        G, Us, st = g(A, ranks, eta=-1.0, seed=4, max_sweeps=3)
        rel_ref = O.rel_error(a64, ref.G, ref.U)
        assert abs(O.rel_error(a64, _np(G), [_np(u) for u in Us]) - rel_ref) <= 1e-6
        for n in range(3):
            u = _np(Us[n])
            assert st["sweeps"][n] == ref.sweeps[n]
            assert np.abs(u - ref.U[n]).max() <= 1e-3, (driver, n)
            assert O.principal_angles(u, ref.U[n]).max() <= 1e-4
        ref = f(a64, ranks, eta=1e-6, seed=4)
        G, Us, st = g(A, ranks, eta=1e-6, seed=4)
        rel_ref = O.rel_error(a64, ref.G, ref.U)
        assert abs(O.rel_error(a64, _np(G), [_np(u) for u in Us]) - rel_ref) <= 1e-6
        for n in range(3):
            assert O.principal_angles(_np(Us[n]), ref.U[n]).max() <= 1e-4
            assert abs(st["sweeps"][n] - ref.sweeps[n]) <= 1


def test_gradients_vs_oracle_midsize(tals):
    """The same gradient checks on a 256 x 256 x 128 tensor at ranks (32, 32, 16)."""
    p = W.planted(W.SEED_BASE + 32, (256, 256, 128), (32, 32, 16), "inv_k", 1e-2, dtype=np.float32)
    A = torch.from_numpy(p.A).cuda()
    _, Us, _ = tals.st_hosvd(A, (32, 32, 16), eta=1e-6, seed=1)
    _gradient_parity(tals, p.A, _perturbed(Us, 18), 24)


def test_rank500_dense_test_fullsize(tals):
    """Sec. 6.4's dense test at its full size: 5000 x 5000 x 50 FP32 of multilinear
    rank (500, 500, 5) plus noise 1e-2, st-HOSVD-ALS at eta 1e-4 (the large-rank path
    for modes 1 and 2). Properties, every reference in FP64 on the device with torch
    (independent of the library's kernels): orthonormal factors; each factor within
    the noise-level angle of the planted one (sin <= 1e-2; ~4e-3 measured); the core
    equal to A x_n U_n^T; the reported error equal to ||A - G x U|| / ||A|| (1e-5)."""
    dims, ranks = W.RANK500_DIMS, W.RANK500_RANKS
    A, F = W.tucker_model_device(W.RANK500_SEED, dims, ranks,
                                 delta=W.tucker_delta(dims, ranks, W.RANK500_NOISE), return_factors=True)
    G, Us, st = tals.st_hosvd(A, ranks, eta=1e-4, seed=1)
    u = [x.double() for x in Us]
    for n in range(3):
        assert float((u[n].T @ u[n] - torch.eye(ranks[n], dtype=torch.float64, device="cuda")).abs().max()) <= 1e-6
        c = torch.linalg.svdvals((u[n].T @ F[n]).cpu())
        assert float(torch.sqrt(torch.clamp(1.0 - c.min() ** 2, min=0.0))) <= 1e-2, n
    # core = A x_1 U_1^T x_2 U_2^T x_3 U_3^T and ||A - G x U||, 500 rows of A at a time
    g = G.double()
    t = torch.einsum("abc,kc->abk", g, u[2])
    t = torch.einsum("abk,jb->ajk", t, u[1])                      # G x_2 U_2 x_3 U_3 (500 x 5000 x 50)
    proj = torch.zeros(ranks, dtype=torch.float64, device="cuda")
    res2, na2 = 0.0, 0.0
    for i0 in range(0, dims[0], 500):
        a = A[i0:i0 + 500].double()
        proj += torch.einsum("ijk,ia,jb,kc->abc", a, u[0][i0:i0 + 500], u[1], u[2])
        b = torch.einsum("ajk,ia->ijk", t, u[0][i0:i0 + 500])
        res2 += float(((a - b) ** 2).sum())
        na2 += float((a ** 2).sum())
    assert float((g - proj).abs().max()) <= 1e-4 * float(proj.abs().max())
    direct = (res2 / na2) ** 0.5
    assert abs(st["rel_err"] - direct) <= 1e-5, (st["rel_err"], direct)
    assert 0.009 <= direct <= 0.011
