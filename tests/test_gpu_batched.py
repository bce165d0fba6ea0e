"""GPU parity of the batched st-HOSVD-ALS (one persistent launch over many
uneven small tensors) against the FP64 oracle and against the single-tensor
path on the same seeded inputs."""
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


def test_batched_matches_oracle_and_single_path(tals):
    batch = W.batched(W.SEED_BASE + 3, 48)
    As = [torch.from_numpy(a).cuda() for a, _, _ in batch]
    ranks = [r for _, _, r in batch]
    Gs, Us, stats = tals.batched_st_hosvd(As, ranks, eta=-1.0, max_sweeps=3, seed=4)
    for t, (a, dims, rk) in enumerate(batch):
        a64 = a.astype(np.float64)
        ref = O.st_hosvd_als(a64, rk, eta=-1.0, seed=4, max_sweeps=3)
        rel_ref = O.rel_error(a64, ref.G, ref.U)
        g = Gs[t].double().cpu().numpy()
        us = [u.double().cpu().numpy() for u in Us[t]]
        assert abs(O.rel_error(a64, g, us) - rel_ref) <= 1e-6
        assert abs(stats[t]["rel_err"] - rel_ref) <= 1e-5
        assert stats[t]["sweeps"] == ref.sweeps
        for n in range(3):
            assert O.principal_angles(us[n], ref.U[n]).max() <= 1e-4
        # same arithmetic as the single-tensor path
        if t < 8:
            G1, U1, s1 = tals.st_hosvd(As[t], rk, eta=-1.0, max_sweeps=3, seed=4)
            assert torch.allclose(G1, Gs[t], rtol=1e-4, atol=1e-4 * float(G1.abs().max()))


def test_batched_tolerance_and_replay(tals):
    batch = W.batched(W.SEED_BASE + 4, 200)
    As = [torch.from_numpy(a).cuda() for a, _, _ in batch]
    ranks = [r for _, _, r in batch]
    Gs, Us, stats = tals.batched_st_hosvd(As, ranks, eta=1e-6, seed=1)
    Gs2, Us2, stats2 = tals.batched_st_hosvd(As, ranks, eta=1e-6, seed=1)   # graph replay
    for t in range(0, len(batch), 17):
        a, dims, rk = batch[t]
        a64 = a.astype(np.float64)
        ref = O.st_hosvd_als(a64, rk, eta=1e-6, seed=1)
        rel_own = O.rel_error(a64, Gs[t].double().cpu().numpy(),
                              [u.double().cpu().numpy() for u in Us[t]])
        assert abs(rel_own - O.rel_error(a64, ref.G, ref.U)) <= 1e-6
        for n in range(3):
            assert abs(stats[t]["sweeps"][n] - ref.sweeps[n]) <= 1
    for t in range(len(batch)):
        assert torch.equal(Gs[t], Gs2[t])
        assert stats[t]["rel_err"] == stats2[t]["rel_err"]


def test_batched_rejects_bad_input(tals):
    a = torch.randn((20, 10, 12), device="cuda")
    with pytest.raises(tals.TalsError):
        tals.batched_st_hosvd([a], [(11, 3, 3)])
    big = torch.randn((200, 10, 12), device="cuda")
    with pytest.raises(tals.TalsError):
        tals.batched_st_hosvd([big], [(4, 3, 3)])
