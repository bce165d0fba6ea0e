"""GPU checks of the tensor-core (tcgen05, BF16) sweep pass and of the mixed-
precision st-HOSVD-ALS against the FP64 oracle.

One tensor-core pass is compared elementwise with Y = B bf16(B^T Q) evaluated
in FP64 on the BF16-rounded tensor and basis, W rounded to BF16 between the two
products as the pass does (bound per entry: FP32 accumulation plus at most three
one-ulp rounding flips of W); ||W||^2 (FP32 accumulation of exact BF16 products)
to 1e-5. The mixed decomposition ends with FP32 sweeps, so its
result is held to the FP32 tolerances."""
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


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16).to(torch.float64).numpy()


# R = 30 takes the scalar store of the final Y (rows not 16-byte multiples);
# R = 20 the TMA store with a ragged box; (256, 128, 384) and (128, 512, 256)
# give every CTA several tiles; Q = 192 is a multiple of the 64-column tile but
# not of 128.
PASS_CASES = [((128, 64, 256), 0, 16), ((512, 16, 256), 0, 32), ((8, 256, 128), 1, 48),
              ((6, 384, 256), 1, 64), ((256, 128, 384), 0, 30), ((128, 512, 256), 1, 20),
              ((4, 128, 192), 1, 16)]


@pytest.mark.parametrize("dims,mode,R", PASS_CASES)
def test_tensor_core_pass_vs_oracle(tals, dims, mode, R):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(dims).astype(np.float32)
    q = np.linalg.qr(rng.standard_normal((dims[mode], R)))[0].astype(np.float32)
    A = torch.from_numpy(a).cuda()
    Qt = torch.from_numpy(q).cuda()
    m = O.unfold(_bf16(a), mode)
    qb = _bf16(q)
    w_ref = m.T @ qb
    Y, w2 = tals.sweep_pass(A, mode, Qt, engine="tc")
    Y = Y.cpu().numpy()
    # elementwise: the pass rounds its FP32 W to BF16 (round to nearest) before the
    # second product, so the reference does too; what remains is FP32 accumulation
    # (1e-5 of the sum of |products|) and W entries whose FP32 value rounds to the
    # other BF16 neighbour than the FP64 one (rare: within ~1e-7 of a rounding
    # boundary), each moving Y by one BF16 ulp of |w| times |b| -- at most three per
    # entry allowed. A wrong or missing tile moves entries by ~|Y|.
    wb = _bf16(w_ref.astype(np.float32))
    y_ref = m @ wb
    acc = np.abs(m) @ np.abs(wb)
    am = np.abs(m)
    flip = np.stack([np.max(am * np.abs(wb[:, r])[None, :], axis=1) for r in range(wb.shape[1])], axis=1)
    tol = 1e-5 * acc + 3 * 2.0 ** -7 * flip
    err = np.abs(Y - y_ref)
    assert np.all(err <= tol), (float((err / tol).max()), np.unravel_index(np.argmax(err / tol), err.shape))
    assert np.linalg.norm(Y - y_ref) <= 1e-4 * np.linalg.norm(y_ref)
    assert abs(w2 - O.frob2(w_ref)) <= 1e-5 * O.frob2(w_ref)
    # the CUDA-core pass on the FP32 data, against FP64
    m32 = O.unfold(a.astype(np.float64), mode)
    y32 = m32 @ (m32.T @ q.astype(np.float64))
    Yc, w2c = tals.sweep_pass(A, mode, Qt, engine="cuda")
    assert np.linalg.norm(Yc.cpu().numpy() - y32) <= 1e-5 * np.linalg.norm(y32)


def test_mixed_st_hosvd_matches_oracle(tals):
    dims, ranks = (512, 96, 128), (32, 16, 24)
    p = W.planted(W.SEED_BASE + 21, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    A = torch.from_numpy(p.A).cuda()
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=3)
    G, Us, st = tals.st_hosvd(A, ranks, eta=1e-6, seed=3, precision="mixed_bf16", use_graph=False)
    rel_own = O.rel_error(a64, G.double().cpu().numpy(), [u.double().cpu().numpy() for u in Us])
    assert abs(rel_own - O.rel_error(a64, ref.G, ref.U)) <= 1e-6
    for n in range(3):
        assert O.principal_angles(Us[n].double().cpu().numpy(), ref.U[n]).max() <= 1e-4
    assert st["converged"] == [True, True, True]
    # the first mode (order: ascending rank -> mode 1 first) is not tensor-core eligible
    # here; mode 0 (I = 512) reads the full tensor only if processed first, so run the
    # order that puts it first as well
    G2, Us2, st2 = tals.st_hosvd(A, ranks, eta=1e-6, seed=3, precision="mixed_bf16",
                                 use_graph=False, order=[0, 1, 2])
    ref2 = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=3, order=[0, 1, 2])
    rel2 = O.rel_error(a64, G2.double().cpu().numpy(), [u.double().cpu().numpy() for u in Us2])
    assert abs(rel2 - O.rel_error(a64, ref2.G, ref2.U)) <= 1e-6
    for n in range(3):
        assert O.principal_angles(Us2[n].double().cpu().numpy(), ref2.U[n]).max() <= 1e-4
    # the reported error rests on ||A||^2 taken during the BF16 conversion
    assert abs(st2["rel_err"] - rel2) <= 1e-6
    assert st2["bulk_sweeps"][0] >= 1
    assert st2["sweeps"][0] >= st2["bulk_sweeps"][0] + 2   # at least two FP32 sweeps finish


@pytest.mark.parametrize("kind", ["st", "t"])
def test_mixed_graph_matches_host_loop(tals, kind):
    # the graph (device-side bulk and FP32 WHILE loops) runs the same kernels in
    # the same order as the host-driven loop: identical results and sweep counts
    dims, ranks = (256, 96, 128), (16, 24, 20)
    p = W.planted(W.SEED_BASE + 22, dims, ranks, "inv_k", 1e-2, dtype=np.float32)
    A = torch.from_numpy(p.A).cuda()
    fn = tals.st_hosvd if kind == "st" else tals.t_hosvd
    kw = dict(eta=1e-6, seed=5, precision="mixed_bf16", order=[0, 1, 2]) if kind == "st" else \
        dict(eta=1e-6, seed=5, precision="mixed_bf16")
    Gh, Uh, sh = fn(A, ranks, use_graph=False, **kw)
    Gg, Ug, sg = fn(A, ranks, use_graph=True, **kw)
    assert sh["sweeps"] == sg["sweeps"] and sh["bulk_sweeps"] == sg["bulk_sweeps"]
    assert sg["bulk_sweeps"][0] >= 1
    assert torch.equal(Gh, Gg)
    for a, b in zip(Uh, Ug):
        assert torch.equal(a, b)
    assert sh["rel_err"] == sg["rel_err"]
    # and the result is the oracle's to the FP32 tolerances
    a64 = p.A.astype(np.float64)
    ref = O.st_hosvd_als(a64, ranks, eta=1e-6, seed=5, order=[0, 1, 2]) if kind == "st" else \
        O.t_hosvd_als(a64, ranks, eta=1e-6, seed=5)
    rel = O.rel_error(a64, Gg.double().cpu().numpy(), [u.double().cpu().numpy() for u in Ug])
    assert abs(rel - O.rel_error(a64, ref.G, ref.U)) <= 1e-6
    for n in range(3):
        assert O.principal_angles(Ug[n].double().cpu().numpy(), ref.U[n]).max() <= 1e-4
