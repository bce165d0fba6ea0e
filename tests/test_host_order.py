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


# The fused pass's configuration (host logic, no GPU): every mode size up to the
# limits the header states (1920 in FP32, 852 in FP64, R <= 64) has a
# configuration that fits in shared memory, in any view -- including Q = 1
# views above 1024, where no transposed-tile instantiation fits and the
# untransposed one takes over -- and the next size up has none.
@pytest.mark.parametrize("dtype,limit", [("f32", 1920), ("f64", 852)])
def test_pass_plan_covers_the_stated_limits(pkg, dtype, limit):
    for R in (1, 5, 8, 16, 17, 32, 33, 64):
        for Q in (1, 2, 3, 64):
            for I in sorted({max(R, 1), 100, 512, 1024, 1028, 1280, limit - 1, limit}):
                if I < R or I > limit:
                    continue
                plan = pkg.pass_plan(dtype, 7, I, Q, R)
                assert plan is not None, (dtype, I, Q, R)
                assert plan["smem"] <= 227 * 1024
                assert plan["rc"] * plan["grid_y"] >= R
                if plan["tr"]:
                    assert dtype == "f32" and Q == 1 and I % 4 == 0
            assert pkg.pass_plan(dtype, 7, limit + 1, Q, min(R, 8)) is None


def test_pass_plan_of_the_512cube_views(pkg):
    # the 512^3 st-HOSVD's first view (1 x 512 x 262144) and its last (1024 x 512 x 1)
    p = pkg.pass_plan("f32", 1, 512, 512 * 512, 32)
    assert (p["rc"], p["rpt"], p["rw"], p["nt"], p["jt"], p["nbuf"], p["tr"]) == (32, 4, 16, 256, 16, 2, 0)
    assert p["grid_x"] == 152 and p["grid_y"] == 1
    p = pkg.pass_plan("f32", 1024, 512, 1, 32)
    assert p["tr"] == 1 and p["rc"] == 32
    with pytest.raises(pkg.TalsError):
        pkg.pass_plan("f32", 0, 512, 1, 32)
