"""Mode sizes near the sweep pass's shared-memory limits, against the FP64
oracle (fixed sweep counts). A last mode above 1024 with Q = 1 and I % 4 == 0
has no transposed-tile configuration, so the untransposed tile (element-wise
column copies, one buffer, rank chunk 8, rows 8 per thread) takes the view."""
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


@pytest.mark.parametrize("driver", ["st", "t"])
def test_long_last_mode_f32(tals, driver):
    dims, ranks = (6, 5, 1100), (3, 3, 8)
    assert tals.pass_plan("f32", 30, 1100, 1, 8)["tr"] == 0
    assert tals.pass_plan("f32", 9, 1100, 1, 8)["tr"] == 0
    p = W.planted(W.SEED_BASE + 13, dims, ranks, "gauss", 1e-2, dtype=np.float32)
    a64 = p.A.astype(np.float64)
    f = O.st_hosvd_als if driver == "st" else O.t_hosvd_als
    ref = f(a64, ranks, eta=-1.0, seed=5, max_sweeps=3)
    g = tals.st_hosvd if driver == "st" else tals.t_hosvd
    G, Us, st = g(torch.from_numpy(np.ascontiguousarray(p.A)).cuda(), ranks, eta=-1.0, seed=5,
                  max_sweeps=3)
    rel_ref = O.rel_error(a64, ref.G, ref.U)
    rel_own = O.rel_error(a64, _np(G), [_np(u) for u in Us])
    assert abs(rel_own - rel_ref) <= 1e-6, (rel_own, rel_ref)
    for n in range(3):
        u = _np(Us[n])
        assert u.shape == ref.U[n].shape
        assert O.principal_angles(u, ref.U[n]).max() <= 1e-4
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-5
        assert st["sweeps"][n] == ref.sweeps[n]
