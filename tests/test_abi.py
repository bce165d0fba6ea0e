"""CPU checks of the C ABI library: it builds, loads and exports every symbol
that include/tals.h declares (no compute calls: no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([A-Za-z_]\w*)\s*\(", txt, flags=re.M):
            name = m.group(1)
            if name in ("if", "while", "for", "sizeof") or name.isupper():
                continue
            names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_02583_gb300 import build
    build.build()
    import paper_2004_02583_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["tucker_als_init", "als_mode_sweep", "st_hosvd", "t_hosvd", "reconstruct"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    import paper_2004_02583_gb300 as pkg
    assert set(_declared()) <= set(pkg.SIGNATURES)


def test_host_only_calls(lib):
    import paper_2004_02583_gb300 as pkg
    o = pkg.default_opts()
    assert o.eta == 1e-4 and o.max_sweeps == 50 and o.use_graph == 1
    assert b"sm_103a" in lib.tals_version()


def test_product_path_does_not_touch_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2004_02583_gb300")
    for dp, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.replace("the oracle", ""), f


def test_host_validation_without_a_gpu(lib):
    # tucker_als_init_owned validates on the host before any CUDA call
    import ctypes
    import paper_2004_02583_gb300 as pkg

    def init(dtype, dims, ranks):
        h = ctypes.c_void_p()
        d = (ctypes.c_int64 * len(dims))(*dims)
        r = (ctypes.c_int * len(ranks))(*ranks)
        o = pkg.default_opts()
        return lib.tucker_als_init_owned(ctypes.byref(h), dtype, len(dims), d, r, ctypes.byref(o), None)

    assert init(pkg.TALS_F32, (10, 9, 8), (11, 2, 2)) == pkg.TALS_EINVAL     # R > I
    assert init(pkg.TALS_F32, (10, 9, 8), (5, 2, 2)) == pkg.TALS_EINVAL      # R_0 > R_1 R_2
    assert init(pkg.TALS_F32, (10,), (2,)) == pkg.TALS_EINVAL                # ndim < 2
    assert init(7, (10, 9, 8), (2, 2, 2)) == pkg.TALS_EINVAL                 # dtype
    assert init(pkg.TALS_F32, (1100, 40, 40), (1030, 40, 40)) == pkg.TALS_ENOTSUP   # R > 1024
    assert b"largest supported rank 1024" in lib.tals_last_error()


def test_strided_init_validates_on_the_host(lib):
    """tucker_als_init_strided rejects strides that cannot describe a tensor before
    any device work: NULL pointers, a negative stride, a zero stride on an axis of
    size above 1, and strides under which two elements share an address."""
    import ctypes
    import paper_2004_02583_gb300 as pkg

    def init(dims, strides, A=ctypes.c_void_p(256), ranks=None):
        h = ctypes.c_void_p()
        d = (ctypes.c_int64 * len(dims))(*dims)
        s = None if strides is None else (ctypes.c_int64 * len(strides))(*strides)
        r = (ctypes.c_int * len(dims))(*(ranks or [2] * len(dims)))
        o = pkg.default_opts()
        return lib.tucker_als_init_strided(ctypes.byref(h), A, pkg.TALS_F32, len(dims), d, s, r,
                                           ctypes.byref(o), None)

    assert init((4, 5, 6), None) == pkg.TALS_EINVAL
    assert init((4, 5, 6), (30, 6, 1), A=None) == pkg.TALS_EINVAL
    assert init((4, 5, 6), (30, -6, 1)) == pkg.TALS_EINVAL
    assert init((4, 5, 6), (30, 0, 1)) == pkg.TALS_EINVAL      # broadcast axis
    assert init((4, 5, 6), (6, 5, 1)) == pkg.TALS_EINVAL       # axes 0 and 1 overlap
    assert init((4, 5, 6), (30, 6, 2)) == pkg.TALS_EINVAL      # axis 1 does not step over axis 2
    assert b"overlap" in lib.tals_last_error()
