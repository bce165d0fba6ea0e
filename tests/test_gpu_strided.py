"""Strided input (tucker_als_init_strided, used by Context for non-contiguous
tensors): a permuted view and a sliced view decompose to exactly what their
contiguous copies decompose to -- the gather writes the same dense tensor, so the
results are bit-identical -- through both drivers and both loops. The contiguous
path itself is held to the oracle by the other parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


def _views():
    base = torch.from_numpy(W.uniform_tensor(W.SEED_BASE + 71, (40, 36, 52))).cuda()
    p = W.planted(W.SEED_BASE + 72, (30, 44, 24), (5, 6, 4), "inv_k", 1e-2, dtype=np.float64)
    b64 = torch.from_numpy(p.A).cuda()
    return [
        (base.permute(2, 0, 1), (6, 5, 7)),                 # 52 x 40 x 36, strides (1, 1872, 52)
        (base[:, ::2, 1:45], (5, 4, 6)),                   # sliced: 40 x 18 x 44
        (b64.transpose(0, 2), (4, 6, 5)),                  # FP64, 24 x 44 x 30
    ]


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("driver", ["st", "t"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_strided_view_matches_contiguous_copy(tals, k, driver, use_graph):
    view, ranks = _views()[k]
    assert not view.is_contiguous()
    dense = view.contiguous()
    f = tals.st_hosvd if driver == "st" else tals.t_hosvd
    Gv, Uv, sv = f(view, ranks, eta=1e-8, seed=3, use_graph=use_graph)
    Gd, Ud, sd = f(dense, ranks, eta=1e-8, seed=3, use_graph=use_graph)
    assert torch.equal(Gv, Gd)
    for a, b in zip(Uv, Ud):
        assert torch.equal(a, b)
    assert sv["rel_err"] == sd["rel_err"] and sv["sweeps"] == sd["sweeps"]


def test_strided_view_refused_when_aliasing(tals):
    """An expanded (broadcast) tensor has a zero stride: refused, not decomposed."""
    x = torch.randn((1, 30, 20), device="cuda").expand(25, 30, 20)
    with pytest.raises(tals.TalsError) as ex:
        tals.st_hosvd(x, (3, 3, 3))
    assert ex.value.status == tals.TALS_EINVAL
