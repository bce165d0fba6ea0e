"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (one Context, CUDA graph, default options of each precision).

Where the FP64 oracle finishes in seconds on the host (512^3, 128^4, the small
batched tensors) the GPU result is compared with it directly; on the 2 GiB
differentiation workload the checks are properties that hold at any size
(orthonormal factors, the core equal to the projection of A at sampled
entries, the reported error against ||A||^2 - ||G||^2, the loss gradient at
sampled entries), with every reference value computed in FP64 on the host."""
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


def test_c5_2gib_forward_and_gradient_properties(tals):
    cfg = W.CONFIGS["d1024_f32"]
    p = W.make(cfg)
    A = torch.from_numpy(p.A).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="native", use_graph=True)
    G, Us, st = ctx.st_hosvd()
    ctx.close()
    assert _orthonormality(Us) <= 1e-5
    a64 = p.A.astype(np.float64)
    us = [_np(u) for u in Us]
    # the core is the projection of A: all core entries from one FP64 contraction chain
    g_ref = O.project(a64, us)
    g = _np(G)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    # reported error against ||A||^2 - ||G||^2 (orthonormal factors)
    na2 = O.frob2(a64)
    rel_id = np.sqrt(max(na2 - O.frob2(g_ref), 0.0) / na2)
    assert abs(st["rel_err"] - rel_id) <= 1e-6
    # gradient of ||A - (A x U^T) x U||^2 w.r.t. A at sampled entries: 2 (A - B)
    # minus the (vanishing for orthonormal U) adjoint of the projection
    Ar = A.detach().requires_grad_(True)
    Ur = [u.detach() for u in Us]
    B = tals.tucker_reconstruct(tals.tucker_project(Ar, Ur), Ur)
    loss = ((Ar - B) ** 2).sum()
    loss.backward()
    grad = Ar.grad
    rng = np.random.default_rng(13)
    worst = 0.0
    scale = 0.0
    for _ in range(16):
        i, j, k = (int(rng.integers(0, s)) for s in cfg.dims)
        b = float(np.einsum("abc,a,b,c->", g_ref, us[0][i], us[1][j], us[2][k]))
        r = 2.0 * (a64[i, j, k] - b)
        worst = max(worst, abs(float(grad[i, j, k]) - r))
        scale = max(scale, abs(r))
    assert worst <= 1e-3 * max(scale, 1e-30)
