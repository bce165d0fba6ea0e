"""GPU parity of the Tucker operators and their adjoints (core projection,
reconstruction, hand-written backward kernels) against the FP64 oracle, plus
finite differences through the autograd.Functions."""
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


def _case(dims, ranks, dtype, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(dims).astype(dtype)
    us = [np.linalg.qr(rng.standard_normal((d, r)))[0].astype(dtype) for d, r in zip(dims, ranks)]
    g = rng.standard_normal(ranks).astype(dtype)
    return a, us, g


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [((23, 17, 40), (5, 4, 7)), ((12, 9, 8, 10), (3, 2, 4, 5)), ((64, 33, 70), (16, 8, 9)),
         ((130, 20, 6), (40, 5, 6)),
         # pipelined mode products: staged contractions (B_in > 64) in both views,
         # ragged a/p/q tails, resident expansions to a Q == 1 view with 100 columns
         ((70, 36, 100), (12, 20, 8)),
         # more tiles than CTAs: the persistent loop wraps (mode-1 view: 512 q-tiles)
         ((100, 64, 1024), (12, 16, 8))]


@pytest.mark.parametrize("dims,ranks", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_project_and_reconstruct(tals, dims, ranks, dtype):
    a, us, g = _case(dims, ranks, dtype, 1)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    G = tals.project(_t(a), [_t(u) for u in us]).double().cpu().numpy()
    ref = O.project(a.astype(np.float64), [u.astype(np.float64) for u in us])
    assert np.abs(G - ref).max() <= tol * np.abs(ref).max()
    B = tals.reconstruct(_t(g), [_t(u) for u in us]).double().cpu().numpy()
    refb = O.reconstruct(g.astype(np.float64), [u.astype(np.float64) for u in us])
    assert np.abs(B - refb).max() <= tol * np.abs(refb).max()


@pytest.mark.parametrize("dims,ranks", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_backward_kernels(tals, dims, ranks, dtype):
    a, us, g = _case(dims, ranks, dtype, 2)
    rng = np.random.default_rng(3)
    bbar = rng.standard_normal(dims).astype(dtype)
    gbar = rng.standard_normal(ranks).astype(dtype)
    tol = 1e-11 if dtype == np.float64 else 1e-4
    u64 = [u.astype(np.float64) for u in us]
    # reconstruct adjoint
    Gb, Ub = tals.reconstruct_backward(_t(g), [_t(u) for u in us], _t(bbar))
    rg, ru = O.reconstruct_vjp(g.astype(np.float64), u64, bbar.astype(np.float64))
    assert np.linalg.norm(Gb.double().cpu().numpy() - rg) <= tol * np.linalg.norm(rg)
    for n in range(len(dims)):
        x = Ub[n].double().cpu().numpy()
        assert np.linalg.norm(x - ru[n]) <= tol * np.linalg.norm(ru[n])
    # project adjoint
    Ab, Ub = tals.project_backward(_t(a), [_t(u) for u in us], _t(gbar))
    ra, ru = O.project_vjp(a.astype(np.float64), u64, gbar.astype(np.float64))
    assert np.linalg.norm(Ab.double().cpu().numpy() - ra) <= tol * np.linalg.norm(ra)
    for n in range(len(dims)):
        x = Ub[n].double().cpu().numpy()
        assert np.linalg.norm(x - ru[n]) <= tol * np.linalg.norm(ru[n])


def test_autograd_gradcheck_f64(tals):
    # finite differences through the hand-written backward kernels (FP64)
    a, us, _ = _case((6, 5, 4), (3, 2, 2), np.float64, 4)
    A = _t(a).requires_grad_(True)
    Us = [_t(u).requires_grad_(True) for u in us]

    def f(A, *Us):
        B = tals.tucker_reconstruct(tals.tucker_project(A, Us), Us)
        return ((A - B) ** 2).sum()
    assert torch.autograd.gradcheck(f, (A, *Us), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_recon_loss_gradient_vs_oracle(tals, dtype, tol):
    # loss ||A - (A x U^T) x U||^2 on a planted low rank + noise tensor, at factors
    # away from the optimum (there the gradient is O(1); at the optimum it is the
    # difference of O(||A||^2) terms and FP32 cannot resolve it to 1e-4)
    p = W.planted(W.SEED_BASE + 5, (48, 40, 36), (6, 5, 4), "inv_k", 1e-2, dtype=np.float64)
    rng = np.random.default_rng(7)
    facs = [np.linalg.qr(f + 0.3 * rng.standard_normal(f.shape))[0] for f in p.factors]
    A = torch.from_numpy(p.A).to("cuda", dtype).requires_grad_(True)
    Us = [torch.from_numpy(f).to("cuda", dtype).requires_grad_(True) for f in facs]
    G = tals.tucker_project(A, Us)
    B = tals.tucker_reconstruct(G, Us)
    loss = ((A - B) ** 2).sum()
    loss.backward()
    ga, gu = O.recon_loss_grad(p.A, facs)
    assert np.linalg.norm(A.grad.double().cpu().numpy() - ga) <= tol * np.linalg.norm(ga)
    for n in range(3):
        x = Us[n].grad.double().cpu().numpy()
        assert np.linalg.norm(x - gu[n]) <= tol * max(np.linalg.norm(gu[n]), 1e-30)
