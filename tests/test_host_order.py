"""Host logic of the Tucker operators, no GPU: the order of the mode products
that project / reconstruct apply is the exact minimum of the multiply-add count
over all orders. Checked against brute force over every permutation, with the
cost written out from its definition: a mode product costs min(I_n, R_n)
multiply-adds per element of its larger side (the input of a contraction, the
output of an expansion)."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2004_02583_gb300 import build
    build.build()
    import paper_2004_02583_gb300 as p
    p.lib()
    return p


def _cost(dims, ranks, order, expand):
    cur = list(ranks) if expand else list(dims)
    total = 0.0
    for m in order:
        before = float(np.prod(cur))
        cur[m] = dims[m] if expand else ranks[m]
        after = float(np.prod(cur))
        total += (after if expand else before) * min(dims[m], ranks[m])
    return total


@pytest.mark.parametrize("expand", [False, True])
def test_order_is_the_brute_force_minimum(pkg, expand):
    rng = np.random.default_rng(11)
    for _ in range(60):
        n = int(rng.integers(1, 6))
        dims = [int(x) for x in rng.integers(2, 300, n)]
        ranks = [int(rng.integers(1, d + 1)) for d in dims]
        order, madds = pkg.mode_product_order(dims, ranks, expand)
        assert sorted(order) == list(range(n))
        best = min(_cost(dims, ranks, p, expand) for p in itertools.permutations(range(n)))
        assert abs(madds - best) <= 1e-9 * best
        assert abs(_cost(dims, ranks, order, expand) - best) <= 1e-9 * best


def test_order_of_the_1024x1024x512_workload(pkg):
    # ranks (64, 64, 32): the projection contracts the rank-32 mode first
    # (19.46 G multiply-adds against 36.57 G in the natural order); the
    # reconstruction expands it last
    dims, ranks = (1024, 1024, 512), (64, 64, 32)
    order, madds = pkg.mode_product_order(dims, ranks, False)
    assert order[0] == 2 and abs(madds - 19461570560.0) < 1.0
    assert abs(_cost(dims, ranks, (0, 1, 2), False) - 36574330880.0) < 1.0
    order, madds = pkg.mode_product_order(dims, ranks, True)
    assert order[-1] == 2 and abs(madds - 19461570560.0) < 1.0


def test_order_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.TalsError):
        pkg.mode_product_order([4, 0, 3], [2, 1, 1])
    with pytest.raises(pkg.TalsError):
        pkg.mode_product_order([2] * 9, [1] * 9)
