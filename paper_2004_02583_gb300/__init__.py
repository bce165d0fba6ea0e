"""Python binding of libtals: ALS-based truncated HOSVD (t-/st-HOSVD-ALS) on GB300.

This module only marshals arguments to the C ABI declared in ``include/tals.h``
(same names): every step of the computation runs in the library's CUDA kernels.
There is no CPU fallback -- importing works anywhere, but every call raises if
``libtals.so`` has not been built or no CUDA device is present.

Tensors are torch CUDA tensors, contiguous, row-major, float32 or float64.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtals.so")
MAX_NDIM = 8

TALS_OK, TALS_EINVAL, TALS_ENOMEM, TALS_ECUDA, TALS_ESINGULAR, TALS_ETIMEOUT, TALS_ENOTSUP = range(7)
TALS_F64, TALS_F32 = 0, 1
PREC_NATIVE, PREC_MIXED_BF16 = 0, 1
_STATUS_NAMES = {0: "TALS_OK", 1: "TALS_EINVAL", 2: "TALS_ENOMEM", 3: "TALS_ECUDA",
                 4: "TALS_ESINGULAR", 5: "TALS_ETIMEOUT", 6: "TALS_ENOTSUP"}


class TalsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tals_opts(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("max_sweeps", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("has_order", ctypes.c_int),
                ("order", ctypes.c_int * MAX_NDIM), ("precision", ctypes.c_int),
                ("bulk_sweeps", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("fp32_engine", ctypes.c_int)]


class tals_stats(ctypes.Structure):
    _fields_ = [("rel_err", ctypes.c_double), ("norm_a", ctypes.c_double),
                ("err_per_mode", ctypes.c_double * MAX_NDIM),
                ("sweeps", ctypes.c_int * MAX_NDIM), ("bulk_sweeps", ctypes.c_int * MAX_NDIM),
                ("tc_sweeps", ctypes.c_int * MAX_NDIM),
                ("converged", ctypes.c_int * MAX_NDIM), ("order", ctypes.c_int * MAX_NDIM),
                ("status", ctypes.c_int), ("split_capable", ctypes.c_int * MAX_NDIM),
                ("split_sweeps", ctypes.c_int * MAX_NDIM),
                ("two_product", ctypes.c_int * MAX_NDIM)]

    def to_dict(self, ndim: int) -> dict:
        return {"rel_err": self.rel_err, "norm_a": self.norm_a,
                "err_per_mode": list(self.err_per_mode[:ndim]),
                "sweeps": list(self.sweeps[:ndim]),
                "bulk_sweeps": list(self.bulk_sweeps[:ndim]),
                "tc_sweeps": list(self.tc_sweeps[:ndim]),
                "converged": [bool(x) for x in self.converged[:ndim]],
                "order": list(self.order[:ndim]), "status": self.status,
                "split_capable": [bool(x) for x in self.split_capable[:ndim]],
                "split_sweeps": list(self.split_sweeps[:ndim]),
                "two_product": [bool(x) for x in self.two_product[:ndim]]}


class tals_hooi_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("resid0", ctypes.c_double), ("resid", ctypes.c_double),
                ("inner_sweeps", ctypes.c_int * MAX_NDIM)]


_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_IP = ctypes.POINTER(ctypes.c_int)
_VPP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/tals.h
SIGNATURES = {
    "tals_default_opts": (None, [ctypes.POINTER(tals_opts)]),
    "tucker_als_init": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, ctypes.c_int, ctypes.c_int,
                                       _I64P, _IP, ctypes.POINTER(tals_opts), _VP]),
    "tucker_als_init_owned": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int,
                                             _I64P, _IP, ctypes.POINTER(tals_opts), _VP]),
    "tucker_als_init_strided": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, ctypes.c_int, ctypes.c_int,
                                               _I64P, _I64P, _IP, ctypes.POINTER(tals_opts), _VP]),
    "tals_ctx_tensor": (_VP, [_VP]),
    "als_mode_sweep": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), _IP]),
    "als_mode_finish": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "st_hosvd": (ctypes.c_int, [_VP, _VP, _VPP, ctypes.POINTER(tals_stats)]),
    "t_hosvd": (ctypes.c_int, [_VP, _VP, _VPP, ctypes.POINTER(tals_stats)]),
    "st_hosvd_host": (ctypes.c_int, [_VP, _VP, _VP, _VPP, ctypes.POINTER(tals_stats)]),
    "tals_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_double, _VP]),
    "st_hosvd_host_many": (ctypes.c_int, [_VP, ctypes.c_int, _VPP, _VPP, _VPP,
                                          ctypes.POINTER(tals_stats)]),
    "reconstruct": (ctypes.c_int, [_VP, _VPP, ctypes.c_int, ctypes.c_int, _I64P, _IP, _VP, _VP]),
    "reconstruction_loss": (ctypes.c_int, [_VP, _VPP, _VP, ctypes.c_int, ctypes.c_int, _I64P, _IP, _VP,
                                           _VP, _VP]),
    "project": (ctypes.c_int, [_VP, _VPP, ctypes.c_int, ctypes.c_int, _I64P, _IP, _VP, _VP]),
    "reconstruct_backward": (ctypes.c_int, [_VP, _VPP, _VP, ctypes.c_int, ctypes.c_int, _I64P,
                                            _IP, _VP, _VPP, _VP]),
    "project_backward": (ctypes.c_int, [_VP, _VPP, _VP, ctypes.c_int, ctypes.c_int, _I64P, _IP,
                                        _VP, _VPP, _VP]),
    "tals_pass_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int, ctypes.c_int, _IP]),
    "tals_mode_product_order": (ctypes.c_int, [ctypes.c_int, _I64P, _IP, ctypes.c_int, _IP,
                                               ctypes.POINTER(ctypes.c_double)]),
    "tals_batched_st_hosvd": (ctypes.c_int, [ctypes.c_int, _VPP, _I64P, _IP,
                                             ctypes.POINTER(tals_opts), _VPP, _VPP,
                                             ctypes.POINTER(tals_stats), _VP]),
    "tals_time_pass": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "tals_time_sweep": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "tals_sweep_pass": (ctypes.c_int, [_VP, ctypes.c_int, _I64P, ctypes.c_int, _VP, ctypes.c_int,
                                       ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    "tals_sweep_pass_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, _I64P, ctypes.c_int, _VP,
                                               ctypes.c_int, _VP, _VP, _VP]),
    "tals_hooi": (ctypes.c_int, [_VP, _VPP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(tals_hooi_stats)]),
    "tals_singular_vectors": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP,
                                             ctypes.POINTER(ctypes.c_double)]),
    "tals_destroy": (None, [_VP]),
    "tals_last_error": (ctypes.c_char_p, []),
    "tals_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libtals.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                f"g.build()\"`. There is no CPU fallback.")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status: int):
    if status != TALS_OK:
        msg = lib().tals_last_error()
        raise TalsError(status, msg.decode() if msg else "")


def selftest_wait_timeout(seconds=0.01, stream=None) -> int:
    """Run the failure path of the bounded device waits once (a wait on a barrier
    nothing arrives at, giving up after `seconds`); returns the status code,
    TALS_ETIMEOUT when the failure path works."""
    return int(lib().tals_selftest_wait_timeout(float(seconds), _stream_ptr(stream)))


def mode_product_order(dims, ranks, expand=False):
    """Order (and multiply-add count) in which project (expand=False) or
    reconstruct (expand=True) apply their mode products: host only, no GPU."""
    n = len(dims)
    d = (ctypes.c_int64 * n)(*[int(x) for x in dims])
    r = (ctypes.c_int * n)(*[int(x) for x in ranks])
    out = (ctypes.c_int * n)()
    madds = ctypes.c_double()
    _check(lib().tals_mode_product_order(n, d, r, int(bool(expand)), out, ctypes.byref(madds)))
    return list(out), madds.value


def pass_plan(dtype, P, I, Q, R, num_sms=152):
    """Configuration of the fused sweep pass for a P x I x Q mode view at rank R
    (host only, no GPU): a dict, or None when no configuration fits."""
    code = TALS_F32 if dtype in ("f32", "float32", TALS_F32) else TALS_F64
    out = (ctypes.c_int * 10)()
    st = lib().tals_pass_plan(code, int(P), int(I), int(Q), int(R), int(num_sms), out)
    if st == TALS_ENOTSUP:
        return None
    _check(st)
    keys = ("rc", "rpt", "rw", "nt", "jt", "nbuf", "tr", "smem", "grid_x", "grid_y")
    return dict(zip(keys, list(out)))


def default_opts(**kw) -> tals_opts:
    o = tals_opts()
    lib().tals_default_opts(ctypes.byref(o))
    order = kw.pop("order", None)
    if order is not None:
        o.has_order = 1
        for i, n in enumerate(order):
            o.order[i] = int(n)
    eng = kw.pop("fp32_engine", None)
    if eng is not None:
        o.fp32_engine = {"auto": 0, "cuda": 1, "fused": 1, "tensor": 2, "products": 3}.get(eng, eng)
    prec = kw.pop("precision", None)
    if prec is not None:
        o.precision = {"native": PREC_NATIVE, "mixed_bf16": PREC_MIXED_BF16}.get(prec, prec)
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return TALS_F32
    if t.dtype == torch.float64:
        return TALS_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _require_cuda(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors (no CPU fallback)")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def _expect(t, shape, dtype, what):
    """ValueError unless tensor t has exactly `shape` and `dtype` (checked before any
    pointer reaches the library: a mismatch would read or write past a buffer)."""
    if t is None:
        return
    if [int(d) for d in t.shape] != [int(d) for d in shape]:
        raise ValueError(f"{what}: shape {tuple(t.shape)}, expected {tuple(int(d) for d in shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")


def _host_bytes(t, nbytes, what):
    if t.numel() * t.element_size() != nbytes or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous host buffer of {nbytes} bytes")


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptrs(ts) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Context:
    """A tals context over a CUDA tensor A (kept alive by this object)."""

    def __init__(self, A, ranks: Sequence[int], eta: float = 1e-4, max_sweeps: int = 50,
                 seed: int = 0, order: Optional[Sequence[int]] = None,
                 precision="native", bulk_sweeps: Optional[int] = None,
                 use_graph: bool = True, fp32_engine="auto", stream=None):
        # any strided CUDA tensor (a permuted or sliced view): a contiguous one is
        # read in place, another is gathered once into the context's own buffer
        if A is None or not A.is_cuda:
            raise ValueError("tensors must be CUDA tensors (no CPU fallback)")
        self.A = A
        self.ndim = A.dim()
        self.dims = [int(d) for d in A.shape]
        self.ranks = [int(r) for r in ranks]
        self.dtype = A.dtype
        self._code = _dtype_code(A)
        self._stream = stream
        o = default_opts(eta=float(eta), max_sweeps=int(max_sweeps), seed=int(seed),
                         order=order, precision=precision, bulk_sweeps=bulk_sweeps,
                         use_graph=int(bool(use_graph)), fp32_engine=fp32_engine)
        self._opts = o
        dims = (ctypes.c_int64 * self.ndim)(*self.dims)
        rk = (ctypes.c_int * self.ndim)(*self.ranks)
        h = ctypes.c_void_p()
        if A.is_contiguous():
            _check(lib().tucker_als_init(ctypes.byref(h), A.data_ptr(), self._code, self.ndim, dims,
                                         rk, ctypes.byref(o), _stream_ptr(stream)))
        else:
            strides = (ctypes.c_int64 * self.ndim)(*[int(x) for x in A.stride()])
            _check(lib().tucker_als_init_strided(ctypes.byref(h), A.data_ptr(), self._code, self.ndim, dims,
                                                 strides, rk, ctypes.byref(o), _stream_ptr(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tals_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outputs(self, G=None, Us=None):
        torch = _torch()
        if G is None:
            G = torch.empty(self.ranks, dtype=self.dtype, device=self.A.device)
        if Us is None:
            Us = [torch.empty((d, r), dtype=self.dtype, device=self.A.device)
                  for d, r in zip(self.dims, self.ranks)]
        if len(Us) != self.ndim:
            raise ValueError(f"{self.ndim} factor buffers expected, got {len(Us)}")
        _expect(G, self.ranks, self.dtype, "G")
        for n, u in enumerate(Us):
            _expect(u, (self.dims[n], self.ranks[n]), self.dtype, f"U[{n}]")
        _require_cuda(G, *Us)
        return G, Us

    def st_hosvd(self, G=None, Us=None):
        """st-HOSVD-ALS (Alg. 5). Returns (G, [U_n], stats)."""
        G, Us = self._outputs(G, Us)
        st = tals_stats()
        _check(lib().st_hosvd(self._h, G.data_ptr(), _ptrs(Us), ctypes.byref(st)))
        return G, Us, st.to_dict(self.ndim)

    def t_hosvd(self, G=None, Us=None):
        """t-HOSVD-ALS (Alg. 4). Returns (G, [U_n], stats)."""
        G, Us = self._outputs(G, Us)
        st = tals_stats()
        _check(lib().t_hosvd(self._h, G.data_ptr(), _ptrs(Us), ctypes.byref(st)))
        return G, Us, st.to_dict(self.ndim)

    def mode_sweep(self, mode: int, max_iters: int):
        err = ctypes.c_double()
        conv = ctypes.c_int()
        _check(lib().als_mode_sweep(self._h, int(mode), int(max_iters), ctypes.byref(err),
                                    ctypes.byref(conv)))
        return err.value, bool(conv.value)

    def mode_finish(self, mode: int, truncate: bool = True, U=None):
        torch = _torch()
        if not (0 <= int(mode) < self.ndim):
            raise ValueError(f"mode {mode} outside 0..{self.ndim - 1}")
        if U is None:
            U = torch.empty((self.dims[mode], self.ranks[mode]), dtype=self.dtype,
                            device=self.A.device)
        _expect(U, (self.dims[mode], self.ranks[mode]), self.dtype, "U")
        _require_cuda(U)
        _check(lib().als_mode_finish(self._h, int(mode), U.data_ptr(), int(bool(truncate))))
        return U


    def hooi(self, Us, G=None, tol: float = 1e-12, max_iters: int = 50,
             inner_eta: float = 1e-12, inner_sweeps: int = 20):
        """HOOI refinement (Sec. 6.3) started from the factors Us (overwritten with
        the refined ones). Returns (G, Us, info) with info = {"iters", "converged",
        "resid" (r_0 .. r_k), "inner_sweeps"}."""
        torch = _torch()
        if len(Us) != self.ndim:
            raise ValueError(f"{self.ndim} factor buffers expected, got {len(Us)}")
        if G is None:
            G = torch.empty(self.ranks, dtype=self.dtype, device=self.A.device)
        _expect(G, self.ranks, self.dtype, "G")
        for n, u in enumerate(Us):
            _expect(u, (self.dims[n], self.ranks[n]), self.dtype, f"U[{n}]")
        _require_cuda(G, *Us)
        if int(max_iters) < 1:
            raise ValueError("max_iters must be >= 1")
        hist = (ctypes.c_double * (int(max_iters) + 1))()
        st = tals_hooi_stats()
        _check(lib().tals_hooi(self._h, _ptrs(Us), G.data_ptr(), float(tol), int(max_iters),
                               float(inner_eta), int(inner_sweeps), hist, ctypes.byref(st)))
        info = {"iters": st.iters, "converged": bool(st.converged),
                "resid": list(hist[:st.iters + 1]),
                "inner_sweeps": list(st.inner_sweeps[:self.ndim])}
        return G, Us, info

    def singular_vectors(self, mode: int, Qhat, U=None):
        """Singular vectors of the mode-`mode` unfolding from the t-HOSVD-ALS basis
        Qhat (Sec. 5): returns (U, sigma) with U = Qhat V, sigma descending."""
        torch = _torch()
        if not (0 <= int(mode) < self.ndim):
            raise ValueError(f"mode {mode} outside 0..{self.ndim - 1}")
        shape = (self.dims[mode], self.ranks[mode])
        _expect(Qhat, shape, self.dtype, "Qhat")
        if U is None:
            U = torch.empty(shape, dtype=self.dtype, device=self.A.device)
        _expect(U, shape, self.dtype, "U")
        _require_cuda(Qhat, U)
        if U.data_ptr() == Qhat.data_ptr():
            raise ValueError("U must not alias Qhat")
        sig = (ctypes.c_double * self.ranks[mode])()
        _check(lib().tals_singular_vectors(self._h, int(mode), Qhat.data_ptr(), U.data_ptr(), sig))
        return U, list(sig)

    def time_sweep(self, mode: int = 0, engine: str = "tf32", iters: int = 10):
        """Per-pass mean durations (ms) and algorithmic bytes of one sweep's product
        passes, and the sweep's FP32-equivalent flops. engine: "cuda", "tc", "tf32"
        or "products" (the last two: two passes, W then Y)."""
        ms = (ctypes.c_double * 2)()
        by = (ctypes.c_double * 2)()
        fl = ctypes.c_double()
        code = {"cuda": 0, "tc": 1, "tf32": 2, "products": 3}[engine]
        _check(lib().tals_time_sweep(self._h, int(mode), code, int(iters), ms, by, ctypes.byref(fl)))
        return list(ms), list(by), fl.value

    def time_pass(self, mode: int = 0, iters: int = 10):
        """Mean duration (ms), algorithmic bytes and flops of one sweep pass."""
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().tals_time_pass(self._h, int(mode), int(iters), ctypes.byref(ms),
                                    ctypes.byref(by), ctypes.byref(fl)))
        return ms.value, by.value, fl.value


def st_hosvd(A, ranks, **kw):
    ctx = Context(A, ranks, **kw)
    try:
        return ctx.st_hosvd()
    finally:
        ctx.close()


def t_hosvd(A, ranks, **kw):
    ctx = Context(A, ranks, **kw)
    try:
        return ctx.t_hosvd()
    finally:
        ctx.close()


class HostContext:
    """Context owning its device tensor; st_hosvd() takes and returns host arrays
    (the end-to-end path: host->device copy, decomposition, device->host copies)."""

    def __init__(self, dims, ranks, dtype="f32", eta=1e-4, max_sweeps=50, seed=0,
                 precision="native", use_graph=True, fp32_engine="auto", stream=None):
        self.ndim = len(dims)
        self.dims = [int(d) for d in dims]
        self.ranks = [int(r) for r in ranks]
        self._code = TALS_F32 if dtype in ("f32", "float32") else TALS_F64
        o = default_opts(eta=float(eta), max_sweeps=int(max_sweeps), seed=int(seed),
                         precision=precision, use_graph=int(bool(use_graph)),
                         fp32_engine=fp32_engine)
        d = (ctypes.c_int64 * self.ndim)(*self.dims)
        rk = (ctypes.c_int * self.ndim)(*self.ranks)
        h = ctypes.c_void_p()
        _check(lib().tucker_als_init_owned(ctypes.byref(h), self._code, self.ndim, d, rk,
                                           ctypes.byref(o), _stream_ptr(stream)))
        self._h = h

    def _check_host(self, A_host, G_host, U_host):
        es = 4 if self._code == TALS_F32 else 8
        _host_bytes(A_host, math.prod(self.dims) * es, "A_host")
        _host_bytes(G_host, math.prod(self.ranks) * es, "G_host")
        if U_host is not None:
            if len(U_host) != self.ndim:
                raise ValueError(f"{self.ndim} factor buffers expected, got {len(U_host)}")
            for n, u in enumerate(U_host):
                if u is not None:
                    _host_bytes(u, self.dims[n] * self.ranks[n] * es, f"U_host[{n}]")

    def st_hosvd(self, A_host, G_host, U_host):
        """A_host, G_host, U_host: pinned (or pageable) host torch tensors."""
        self._check_host(A_host, G_host, U_host)
        st = tals_stats()
        _check(lib().st_hosvd_host(self._h, A_host.data_ptr(), G_host.data_ptr(),
                                   _ptrs(U_host), ctypes.byref(st)))
        return st.to_dict(self.ndim)

    def st_hosvd_many(self, A_hosts, G_hosts, U_hosts=None):
        """Pipelined st_hosvd over lists of host tensors: the upload of tensor t+1
        overlaps the decomposition of tensor t. U_hosts: None or one list of N
        factor tensors per input. Returns the per-tensor statistics."""
        n = len(A_hosts)
        if len(G_hosts) != n or (U_hosts is not None and len(U_hosts) != n):
            raise ValueError("one core (and factor list) per input tensor")
        for t in range(n):
            self._check_host(A_hosts[t], G_hosts[t], None if U_hosts is None else U_hosts[t])
        A = (ctypes.c_void_p * n)(*[a.data_ptr() for a in A_hosts])
        G = (ctypes.c_void_p * n)(*[g.data_ptr() for g in G_hosts])
        U = None
        if U_hosts is not None:
            U = (ctypes.c_void_p * (n * self.ndim))(*[u.data_ptr() for us in U_hosts for u in us])
        st = (tals_stats * n)()
        _check(lib().st_hosvd_host_many(self._h, n, A, G, U, st))
        return [st[i].to_dict(self.ndim) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tals_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _op_args(X, Us, x_is="dims"):
    """Sizes and ranks from the factors (U_n: I_n x R_n), after checking that X has
    the sizes (x_is="dims") or the ranks (x_is="ranks") and that every factor has
    X's dtype; ValueError before any pointer reaches the library."""
    Us = list(Us)
    if len(Us) != X.dim() or len(Us) < 1:
        raise ValueError(f"{X.dim()} factors expected, got {len(Us)}")
    _dtype_code(X)
    for n, u in enumerate(Us):
        if u.dim() != 2:
            raise ValueError(f"U[{n}] must be a matrix, got {u.dim()} dimensions")
        if u.dtype != X.dtype:
            raise ValueError(f"U[{n}]: dtype {u.dtype}, expected {X.dtype}")
    dl = [int(u.shape[0]) for u in Us]
    rl = [int(u.shape[1]) for u in Us]
    _expect(X, dl if x_is == "dims" else rl, X.dtype, "tensor")
    ndim = len(Us)
    dims = (ctypes.c_int64 * ndim)(*dl)
    ranks = (ctypes.c_int * ndim)(*rl)
    return ndim, dims, ranks


def project(A, Us, out=None, stream=None):
    """G = A x_1 U1^T ... x_N UN^T (the core projection of Alg. 1/4)."""
    torch = _torch()
    ndim, dims, ranks = _op_args(A, Us, "dims")
    _expect(out, list(ranks), A.dtype, "out")
    _require_cuda(A, out, *Us)
    G = out if out is not None else torch.empty([int(u.shape[1]) for u in Us], dtype=A.dtype,
                                                 device=A.device)
    _check(lib().project(A.data_ptr(), _ptrs(Us), _dtype_code(A), ndim, dims, ranks,
                         G.data_ptr(), _stream_ptr(stream)))
    return G


def reconstruct(G, Us, out=None, stream=None):
    """B = G x_1 U1 ... x_N UN (Tucker model)."""
    torch = _torch()
    ndim, dims, ranks = _op_args(G, Us, "ranks")
    _expect(out, list(dims), G.dtype, "out")
    _require_cuda(G, out, *Us)
    B = out if out is not None else torch.empty([int(u.shape[0]) for u in Us], dtype=G.dtype,
                                                 device=G.device)
    _check(lib().reconstruct(G.data_ptr(), _ptrs(Us), _dtype_code(G), ndim, dims, ranks,
                             B.data_ptr(), _stream_ptr(stream)))
    return B


def reconstruction_loss(A, G, Us, stream=None):
    """(f, D) with f = ||G x_1 U1 ... x_N UN - A||^2 (a 0-dim FP64 device tensor)
    and D = 2 (B - A), the gradient with respect to the reconstruction B, formed
    without writing B."""
    torch = _torch()
    ndim, dims, ranks = _op_args(G, Us, "ranks")
    _expect(A, list(dims), G.dtype, "A")
    _require_cuda(A, G, *Us)
    D = torch.empty_like(A)
    f = torch.empty((), dtype=torch.float64, device=A.device)
    _check(lib().reconstruction_loss(G.data_ptr(), _ptrs(Us), A.data_ptr(), _dtype_code(G), ndim, dims, ranks,
                                     D.data_ptr(), f.data_ptr(), _stream_ptr(stream)))
    return f, D


def reconstruct_backward(G, Us, B_bar, need_g=True, need_u=True, stream=None):
    """(G_bar, [U_bar_n]) of B = reconstruct(G, Us) for the output gradient B_bar."""
    torch = _torch()
    ndim, dims, ranks = _op_args(B_bar, Us, "dims")
    _expect(G, list(ranks), B_bar.dtype, "G")
    _require_cuda(B_bar, G, *Us)
    G_bar = torch.empty_like(G) if need_g else None
    U_bar = [torch.empty_like(u) for u in Us] if need_u else [None] * ndim
    _check(lib().reconstruct_backward(G.data_ptr(), _ptrs(Us), B_bar.data_ptr(), _dtype_code(G),
                                      ndim, dims, ranks, G_bar.data_ptr() if need_g else None,
                                      _ptrs(U_bar), _stream_ptr(stream)))
    return G_bar, U_bar


def project_backward(A, Us, G_bar, need_a=True, need_u=True, stream=None):
    """(A_bar, [U_bar_n]) of G = project(A, Us) for the output gradient G_bar."""
    torch = _torch()
    ndim, dims, ranks = _op_args(A, Us, "dims")
    _expect(G_bar, list(ranks), A.dtype, "G_bar")
    _require_cuda(A, G_bar, *Us)
    A_bar = torch.empty_like(A) if need_a else None
    U_bar = [torch.empty_like(u) for u in Us] if need_u else [None] * ndim
    _check(lib().project_backward(A.data_ptr(), _ptrs(Us), G_bar.data_ptr(), _dtype_code(A),
                                  ndim, dims, ranks, A_bar.data_ptr() if need_a else None,
                                  _ptrs(U_bar), _stream_ptr(stream)))
    return A_bar, U_bar


_AUTOGRAD = None


def _autograd():
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD


def _make_autograd():
    torch = _torch()

    class TalsProject(torch.autograd.Function):
        """G = A x_1 U1^T ... x_N UN^T with hand-written backward kernels."""

        @staticmethod
        def forward(ctx, A, *Us):
            A = A.contiguous()
            Us = [u.contiguous() for u in Us]
            ctx.save_for_backward(A, *Us)
            return project(A, Us)

        @staticmethod
        def backward(ctx, G_bar):
            A, *Us = ctx.saved_tensors
            need_a = ctx.needs_input_grad[0]
            need_u = any(ctx.needs_input_grad[1:])
            A_bar, U_bar = project_backward(A, Us, G_bar.contiguous(), need_a, need_u)
            return (A_bar, *U_bar)

    class TalsReconstruct(torch.autograd.Function):
        """B = G x_1 U1 ... x_N UN with hand-written backward kernels."""

        @staticmethod
        def forward(ctx, G, *Us):
            G = G.contiguous()
            Us = [u.contiguous() for u in Us]
            ctx.save_for_backward(G, *Us)
            return reconstruct(G, Us)

        @staticmethod
        def backward(ctx, B_bar):
            G, *Us = ctx.saved_tensors
            need_g = ctx.needs_input_grad[0]
            need_u = any(ctx.needs_input_grad[1:])
            G_bar, U_bar = reconstruct_backward(G, Us, B_bar.contiguous(), need_g, need_u)
            return (G_bar, *U_bar)

    class TalsReconstructionLoss(torch.autograd.Function):
        """f = ||G x_1 U1 ... x_N UN - A||^2 with the fused loss kernel forward and the
        reconstruction adjoint backward (B_bar = df/dB = 2 (B - A), kept from forward)."""

        @staticmethod
        def forward(ctx, A, G, *Us):
            A = A.contiguous()
            G = G.contiguous()
            Us = [u.contiguous() for u in Us]
            f, D = reconstruction_loss(A, G, Us)
            ctx.save_for_backward(G, D, *Us)
            return f

        @staticmethod
        def backward(ctx, f_bar):
            G, D, *Us = ctx.saved_tensors
            # df/dB = D; the adjoint is linear in its input, so the output gradient
            # scales the small results (no pass over D, no host synchronisation)
            c = f_bar.to(D.dtype)
            need_g = ctx.needs_input_grad[1]
            need_u = any(ctx.needs_input_grad[2:])
            G_bar, U_bar = None, [None] * len(Us)
            if need_g or need_u:
                G_bar, U_bar = reconstruct_backward(G, Us, D, need_g, need_u)
                G_bar = G_bar * c if G_bar is not None else None
                U_bar = [u * c if u is not None else None for u in U_bar]
            A_bar = -(D * c) if ctx.needs_input_grad[0] else None
            return (A_bar, G_bar, *U_bar)

    return TalsProject, TalsReconstruct, TalsReconstructionLoss


def tucker_project(A, Us):
    """Differentiable core projection (autograd.Function over the C ABI)."""
    return _autograd()[0].apply(A, *Us)


def tucker_reconstruct(G, Us):
    """Differentiable Tucker reconstruction (autograd.Function over the C ABI)."""
    return _autograd()[1].apply(G, *Us)


def tucker_reconstruction_loss(A, G, Us):
    """Differentiable ||G x_1 U1 ... x_N UN - A||^2 (0-dim FP64) with the fused loss
    kernel: the reconstruction is never written out."""
    return _autograd()[2].apply(A, G, *Us)


class BatchedRunner:
    """st-HOSVD-ALS of many small third-order FP32 CUDA tensors in one persistent,
    graph-captured launch, with the outputs and the argument arrays prepared once
    so that repeated runs cost one C-ABI call each. ranks: list of 3-tuples."""

    def __init__(self, As, ranks, eta=1e-4, max_sweeps=50, seed=0, stream=None):
        torch = _torch()
        count = len(As)
        if len(ranks) != count:
            raise ValueError("one rank triple per tensor")
        for a in As:
            _require_cuda(a)
            if a.dtype != torch.float32 or a.dim() != 3:
                raise ValueError("batched tensors are third-order float32")
        self.count = count
        self.As = list(As)
        self.Gs = [torch.empty(tuple(r), dtype=torch.float32, device=a.device) for a, r in zip(As, ranks)]
        self._Uflat = [torch.empty((int(a.shape[n]), int(r[n])), dtype=torch.float32, device=a.device)
                       for a, r in zip(As, ranks) for n in range(3)]
        self.Us = [self._Uflat[3 * t:3 * t + 3] for t in range(count)]
        self._a = _ptrs(self.As)
        self._g = _ptrs(self.Gs)
        self._u = _ptrs(self._Uflat)
        self._dims = (ctypes.c_int64 * (3 * count))(*[int(d) for a in As for d in a.shape])
        self._rk = (ctypes.c_int * (3 * count))(*[int(x) for r in ranks for x in r])
        self._o = default_opts(eta=float(eta), max_sweeps=int(max_sweeps), seed=int(seed))
        self._stats = (tals_stats * max(count, 1))()
        self._stream = stream

    def run(self):
        _check(lib().tals_batched_st_hosvd(self.count, self._a, self._dims, self._rk,
                                           ctypes.byref(self._o), self._g, self._u, self._stats,
                                           _stream_ptr(self._stream)))

    def stats(self):
        return [self._stats[t].to_dict(3) for t in range(self.count)]


def batched_st_hosvd(As, ranks, eta=1e-4, max_sweeps=50, seed=0, stream=None):
    """st-HOSVD-ALS of many small third-order FP32 CUDA tensors in one persistent,
    graph-captured launch. ranks: list of 3-tuples. Returns (Gs, Us, stats)."""
    r = BatchedRunner(As, ranks, eta, max_sweeps, seed, stream)
    r.run()
    return r.Gs, r.Us, r.stats()


def sweep_pass(A, mode, Q, engine="cuda", stream=None):
    """One sweep of products (diagnostics): returns (Y = B B^T Q in FP64, ||B^T Q||^2)
    for the mode-`mode` unfolding B of the FP32 tensor A. engine: "cuda" (fused pass,
    FP32 CUDA cores), "tc" (fused pass, tcgen05 BF16 on a BF16 copy) or "tf32" (two
    passes, tcgen05 split-precision 3xTF32 on the FP32 tensor); "tf32_w" / "tf32_y"
    replace the Y or the W pass of "tf32" by the CUDA-core pass (diagnostics);
    "products" (FP32 CUDA cores: the mode product W, then the split-K Y = B W)."""
    torch = _torch()
    if engine not in ("cuda", "tc", "tf32", "tf32_w", "tf32_y", "products"):
        raise ValueError(f"unknown engine {engine!r}")
    if A.dtype != torch.float32 or Q.dtype != torch.float32:
        raise ValueError("sweep_pass needs FP32 A and Q")
    if not (0 <= int(mode) < A.dim()):
        raise ValueError(f"mode {mode} outside 0..{A.dim() - 1}")
    if Q.dim() != 2 or int(Q.shape[0]) != int(A.shape[mode]) or int(Q.shape[1]) < 1:
        raise ValueError(f"Q must be I_mode x R = {int(A.shape[mode])} x R, got {tuple(Q.shape)}")
    _require_cuda(A, Q)
    ndim = A.dim()
    dims = (ctypes.c_int64 * ndim)(*[int(d) for d in A.shape])
    R = int(Q.shape[1])
    Y = torch.empty((int(A.shape[mode]), R), dtype=torch.float64, device=A.device)
    w2 = ctypes.c_double()
    _check(lib().tals_sweep_pass(A.data_ptr(), ndim, dims, int(mode), Q.data_ptr(), R,
                                 {"cuda": 0, "tc": 1, "tf32": 2, "tf32_w": 3, "tf32_y": 4,
                                  "products": 5}[engine],
                                 Y.data_ptr(), ctypes.byref(w2),
                                 _stream_ptr(stream)))
    return Y, w2.value


def version() -> str:
    return lib().tals_version().decode()
