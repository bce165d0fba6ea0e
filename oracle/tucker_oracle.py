"""Plain FP64 CPU oracle for ALS-based truncated HOSVD.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It follows Xiao, Yang and Li, "Efficient Alternating Least Squares Algorithms
for Low Multilinear Rank Approximation of Tensors" (arXiv 2004.02583) step by
step, in NumPy float64, sharing no code with the CUDA library. Every function
names the section, equation or algorithm it restates. Readings taken where the
paper is silent or ambiguous:

R1  Alg. 3 ends its loop after the L-update, and the stop rule (Eq. 5.01)
    compares the pairs (L_k, R_k) and (L_{k+1}, R_{k+1}). The test is taken
    right after each R-update and the consistent pair (L_k, R_k) is returned;
    ``sweeps`` counts R-updates; the first test is at k = 1. A negative eta
    never stops early (fixed sweep count).
R2  ``||A||_F`` in Eq. 5.01 is the norm of the ORIGINAL input tensor, for every
    mode of both drivers.
R3  The random S of the initial guess (Sec. 4, "uniform on [0,1]") is the
    splitmix64 stream seeded with ``seed XOR (mode << 56)``; entry (j, r) is
    output number ``j*R + r`` mapped to ``(z >> 40) * 2^-24`` (24-bit, exact in
    FP32 and FP64). The column index j is the row-major (C-order) linear
    index over the remaining modes in their logical order -- not the Fortran
    order of the unfolding definition in Sec. 2. In st-HOSVD the truncated
    modes keep their logical position.
R4  Reduced QR is made unique by ``diag(R) > 0`` (Alg. 4/5 QR step).
R5  L is not re-orthonormalised between sweeps (literal Alg. 3); ``reorth=True``
    is a variant that replaces L_{k+1} by the Q factor of its positive QR.
R6  Default st-HOSVD order: ascending R_n, ties by ascending n (Prop. 1).
R7  Noise is relative Frobenius noise (see ``workloads``).
R9  r = min(m, n) is allowed (Alg. 3 asks r < min(m, n)); ALS then reproduces
    the matrix exactly.
R10 HOOI (Sec. 6.3 refines the t-/st-HOSVD results with it; the paper takes the
    method from a toolbox and prints no steps): cycles over the modes in
    ascending order; mode n is replaced by the R_n leading left singular
    vectors of (A x_{m != n} U_m^T)_(n), using the factors already updated in
    the cycle. After cycle k the core is G = A x_1 U_1^T ... x_N U_N^T and the
    relative residual r_k = ||A - G x U|| / ||A||; r_0 is that of the initial
    guess. The loop stops after the first cycle with |r_{k-1} - r_k| < tol
    (the toolbox's change-of-fit test, fit = 1 - r), or after max_iters cycles.
R11 Singular vectors of a t-HOSVD-ALS basis (Sec. 5, after Alg. 4): the SVD of
    Qhat^T A_(n) = U S V^T gives U^(n) = Qhat U, in descending order of S. The
    sign of each singular vector is free; it is fixed so that the entry of
    largest magnitude of every column of U^(n) is positive (ties: the first).

Parity pins: every function here is checked by ``tests/test_oracle_pins.py``
against SVD-based definitions, closed forms, invariants, published test
vectors or brute force. No function is "parity unpinned".
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "frob2", "unfold", "fold", "mode_product", "tucker_to_tensor",
    "splitmix64_stream", "init_sketch", "qr_pos", "als", "ALSResult",
    "default_order", "st_cost", "st_hosvd_als", "t_hosvd_als",
    "t_hosvd_svd", "st_hosvd_svd", "HOSVDResult", "rel_error",
    "project", "reconstruct", "project_vjp", "reconstruct_vjp",
    "recon_loss", "recon_loss_grad", "principal_angles",
    "hooi", "HOOIResult", "singular_vectors", "sign_fix",
]

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------------------
# Sec. 2: notation
# ---------------------------------------------------------------------------

def frob2(x: np.ndarray) -> float:
    """Squared Frobenius norm (Sec. 2), accumulated in float64."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.dot(x.ravel(), x.ravel()))


def unfold(x: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization A_(n), I_n x prod(other sizes) (Sec. 2).

    Column index j runs row-major over the remaining modes in logical order
    (reading R3).
    """
    return np.moveaxis(np.asarray(x), n, 0).reshape(x.shape[n], -1)


def fold(m: np.ndarray, n: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of ``unfold`` for a tensor of the given shape."""
    shape = list(shape)
    rest = shape[:n] + shape[n + 1:]
    return np.moveaxis(np.asarray(m).reshape([shape[n]] + rest), 0, n)


def mode_product(x: np.ndarray, u: np.ndarray, n: int) -> np.ndarray:
    """Mode-n product  B = X x_n U,  B[.., j, ..] = sum_i X[.., i, ..] U[j, i]
    (Sec. 2, elementwise definition)."""
    y = np.tensordot(u, x, axes=([1], [n]))
    return np.moveaxis(y, 0, n)


def tucker_to_tensor(g: np.ndarray, us: Sequence[np.ndarray]) -> np.ndarray:
    """G x_1 U^(1) x_2 ... x_N U^(N) (Tucker model, Sec. 2)."""
    b = np.asarray(g, dtype=np.float64)
    for n, u in enumerate(us):
        b = mode_product(b, np.asarray(u, dtype=np.float64), n)
    return b


# ---------------------------------------------------------------------------
# Sec. 4: initial guess  (S uniform on [0,1], L0 = Q of QR(A_(n) S))
# ---------------------------------------------------------------------------

def splitmix64_stream(state: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of Vigna's splitmix64 generator.

    Published definition (Steele, Lea, Flood 2014; Vigna's splitmix64.c):
    ``state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; return z ^ (z >> 31)``.
    Output number c (0-based) is therefore mix(state + (c+1) * gamma).
    """
    c = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & MASK64) + (c + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def init_sketch(seed: int, mode: int, J: int, R: int) -> np.ndarray:
    """The J x R random matrix S of the initial guess (Sec. 4; reading R3)."""
    state = (int(seed) ^ (int(mode) << 56)) & MASK64
    z = splitmix64_stream(state, J * R)
    u = (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return u.reshape(J, R)


def qr_pos(y: np.ndarray):
    """Reduced QR with positive diagonal of R (reading R4)."""
    q, r = np.linalg.qr(np.asarray(y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s, r * s[:, None]


# ---------------------------------------------------------------------------
# Alg. 3: matrix ALS, with the Sec. 4 initial guess and the Eq. 5.01 stop rule
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ALSResult:
    L: np.ndarray          # L_k   (m x r)
    R: np.ndarray          # R_k   (n x r), the LS optimum for L_k
    err: float             # ||A - L_k R_k^T||_F
    errs: List[float]      # e_0 .. e_k
    sweeps: int            # number of R-updates performed (k + 1)
    converged: bool
    L0: np.ndarray


def _ls_err(m: np.ndarray, l: np.ndarray, rr: np.ndarray, chunk: int = 1 << 14) -> float:
    """||M - L R^T||_F from the plain definition, in column chunks."""
    tot = 0.0
    for j0 in range(0, m.shape[1], chunk):
        d = m[:, j0:j0 + chunk] - l @ rr[j0:j0 + chunk].T
        tot += float(np.dot(d.ravel(), d.ravel()))
    return float(np.sqrt(tot))


def als(m: np.ndarray, r: int, eta: float, norm_a: float, seed: int = 0, mode: int = 0,
        max_sweeps: int = 50, reorth: bool = False,
        l0: Optional[np.ndarray] = None) -> ALSResult:
    """Alg. 3 on the matrix ``m`` (I_n x J) with truncation ``r``.

    Steps, in the paper's order and notation:
      init (Sec. 4): S uniform, L_0 = Q of QR(A S);
      loop:  R_k = (A^T L_k)(L_k^T L_k)^{-1}              (Alg. 3, R-update)
             e_k = ||A - L_k R_k^T||_F;  stop if k >= 1 and
             |e_{k-1} - e_k| <= eta ||A||_F              (Eq. 5.01, R1, R2)
             L_{k+1} = (A R_k)(R_k^T R_k)^{-1}            (Alg. 3, L-update)
    """
    m = np.asarray(m, dtype=np.float64)
    I, J = m.shape
    if l0 is None:
        s = init_sketch(seed, mode, J, r)
        l0 = qr_pos(m @ s)[0]
    lk = np.array(l0, dtype=np.float64)
    errs: List[float] = []
    rk = None
    converged = False
    sweeps = 0
    for k in range(max_sweeps):
        gl = lk.T @ lk
        rk = np.linalg.solve(gl, (m.T @ lk).T).T          # (A^T L)(L^T L)^{-1}
        e = _ls_err(m, lk, rk)
        errs.append(e)
        sweeps = k + 1
        if k >= 1 and abs(errs[-2] - e) <= eta * norm_a:
            converged = True
            break
        if k == max_sweeps - 1:
            break
        gr = rk.T @ rk
        lk = np.linalg.solve(gr, (m @ rk).T).T            # (A R)(R^T R)^{-1}
        if reorth:
            lk = qr_pos(lk)[0]
    return ALSResult(L=lk, R=rk, err=errs[-1], errs=errs, sweeps=sweeps,
                     converged=converged, L0=np.array(l0))


# ---------------------------------------------------------------------------
# Prop. 1: processing order of st-HOSVD
# ---------------------------------------------------------------------------

def default_order(ranks: Sequence[int]) -> List[int]:
    """Ascending R_n, ties by ascending n (Prop. 1; reading R6)."""
    return sorted(range(len(ranks)), key=lambda n: (ranks[n], n))


def st_cost(dims: Sequence[int], ranks: Sequence[int], order: Sequence[int]) -> int:
    """The leading cost term of Eq. 2.2 (proof of Prop. 1) for a given order:
    sum over steps t of (R_{i_1} ... R_{i_t}) * (I_{i_t} ... I_{i_N})."""
    tot = 0
    for t in range(len(order)):
        rp = int(np.prod([ranks[order[s]] for s in range(t + 1)]))
        ip = int(np.prod([dims[order[s]] for s in range(t, len(order))]))
        tot += rp * ip
    return tot


# ---------------------------------------------------------------------------
# Alg. 4 / Alg. 5: the drivers
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class HOSVDResult:
    G: np.ndarray
    U: List[np.ndarray]
    err_per_mode: List[float]     # e_n of the ALS (or SVD) step of each mode
    sweeps: List[int]
    converged: List[bool]
    order: List[int]
    norm_a: float
    als: List[Optional[ALSResult]]

    @property
    def rel_err_identity(self) -> float:
        """sqrt(||A||^2 - ||G||^2) / ||A|| (orthogonal projection identity)."""
        return float(np.sqrt(max(self.norm_a ** 2 - frob2(self.G), 0.0)) / self.norm_a)


def st_hosvd_als(a: np.ndarray, ranks: Sequence[int], eta: float = 1e-4, seed: int = 0,
                 order: Optional[Sequence[int]] = None, max_sweeps: int = 50,
                 reorth: bool = False) -> HOSVDResult:
    """Alg. 5 (st-HOSVD-ALS).

    For n in the order: B_(n) <- B; [L, R] = ALS(B_(n), R_n); Q^, R^ = QR(L);
    U^(n) = Q^; B_(n) <- R^ R^T; B <- tensor. Finally G <- B.
    """
    a = np.asarray(a, dtype=np.float64)
    N = a.ndim
    order = list(default_order(ranks) if order is None else order)
    norm_a = float(np.sqrt(frob2(a)))
    b = a
    shape = list(a.shape)
    us: List[Optional[np.ndarray]] = [None] * N
    errs = [0.0] * N
    sweeps = [0] * N
    conv = [False] * N
    runs: List[Optional[ALSResult]] = [None] * N
    for n in order:
        mn = unfold(b, n)
        res = als(mn, ranks[n], eta, norm_a, seed=seed, mode=n,
                  max_sweeps=max_sweeps, reorth=reorth)
        qh, rh = qr_pos(res.L)
        us[n] = qh
        bn = rh @ res.R.T                     # Alg. 5: B_(n) <- R^ R^T
        shape[n] = ranks[n]
        b = fold(bn, n, shape)
        errs[n], sweeps[n], conv[n], runs[n] = res.err, res.sweeps, res.converged, res
    return HOSVDResult(G=np.array(b), U=us, err_per_mode=errs, sweeps=sweeps,
                       converged=conv, order=order, norm_a=norm_a, als=runs)


def project(a: np.ndarray, us: Sequence[np.ndarray]) -> np.ndarray:
    """G = A x_1 U^(1)T ... x_N U^(N)T (Alg. 1/4 core step)."""
    g = np.asarray(a, dtype=np.float64)
    for n, u in enumerate(us):
        g = mode_product(g, np.asarray(u, dtype=np.float64).T, n)
    return g


def reconstruct(g: np.ndarray, us: Sequence[np.ndarray]) -> np.ndarray:
    """B = G x_1 U^(1) ... x_N U^(N) (Tucker model, Sec. 2)."""
    return tucker_to_tensor(g, us)


def t_hosvd_als(a: np.ndarray, ranks: Sequence[int], eta: float = 1e-4, seed: int = 0,
                max_sweeps: int = 50, reorth: bool = False) -> HOSVDResult:
    """Alg. 4 (t-HOSVD-ALS): ALS on every A_(n), U^(n) = Q of QR(L),
    then G = A x_1 U^(1)T ... x_N U^(N)T."""
    a = np.asarray(a, dtype=np.float64)
    N = a.ndim
    norm_a = float(np.sqrt(frob2(a)))
    us, errs, sweeps, conv, runs = [], [], [], [], []
    for n in range(N):
        res = als(unfold(a, n), ranks[n], eta, norm_a, seed=seed, mode=n,
                  max_sweeps=max_sweeps, reorth=reorth)
        us.append(qr_pos(res.L)[0])
        errs.append(res.err)
        sweeps.append(res.sweeps)
        conv.append(res.converged)
        runs.append(res)
    g = project(a, us)
    return HOSVDResult(G=g, U=us, err_per_mode=errs, sweeps=sweeps, converged=conv,
                       order=list(range(N)), norm_a=norm_a, als=runs)


def _leading_left(m: np.ndarray, r: int):
    u, s, vt = np.linalg.svd(m, full_matrices=False)
    return u[:, :r], s, vt


def t_hosvd_svd(a: np.ndarray, ranks: Sequence[int]) -> HOSVDResult:
    """Alg. 1 (t-HOSVD): U^(n) = leading left singular vectors of A_(n)."""
    a = np.asarray(a, dtype=np.float64)
    us, errs = [], []
    for n in range(a.ndim):
        u, s, _ = _leading_left(unfold(a, n), ranks[n])
        us.append(u)
        errs.append(float(np.sqrt(np.sum(s[ranks[n]:] ** 2))))
    return HOSVDResult(G=project(a, us), U=us, err_per_mode=errs,
                       sweeps=[0] * a.ndim, converged=[True] * a.ndim,
                       order=list(range(a.ndim)), norm_a=float(np.sqrt(frob2(a))),
                       als=[None] * a.ndim)


def st_hosvd_svd(a: np.ndarray, ranks: Sequence[int],
                 order: Optional[Sequence[int]] = None) -> HOSVDResult:
    """Alg. 2 (st-HOSVD): U^(n) from the SVD of B_(n), B <- Sigma V^T."""
    a = np.asarray(a, dtype=np.float64)
    order = list(default_order(ranks) if order is None else order)
    b = a
    shape = list(a.shape)
    us: List[Optional[np.ndarray]] = [None] * a.ndim
    errs = [0.0] * a.ndim
    for n in order:
        u, s, vt = _leading_left(unfold(b, n), ranks[n])
        us[n] = u
        errs[n] = float(np.sqrt(np.sum(s[ranks[n]:] ** 2)))
        shape[n] = ranks[n]
        b = fold(s[:ranks[n], None] * vt[:ranks[n]], n, shape)
    return HOSVDResult(G=np.array(b), U=us, err_per_mode=errs, sweeps=[0] * a.ndim,
                       converged=[True] * a.ndim, order=order,
                       norm_a=float(np.sqrt(frob2(a))), als=[None] * a.ndim)


# ---------------------------------------------------------------------------
# Sec. 6.3: HOOI from the t-/st-HOSVD initial guess (reading R10)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class HOOIResult:
    G: np.ndarray
    U: List[np.ndarray]
    resid: List[float]     # r_0 (the initial guess), r_1 .. r_k
    iters: int             # cycles performed (k)
    converged: bool        # the change test fired before max_iters


def hooi(a: np.ndarray, us0: Sequence[np.ndarray], tol: float = 1e-12,
         max_iters: int = 50) -> HOOIResult:
    """Higher-order orthogonal iteration from the initial factors ``us0``.

    Cycle k, for n = 0 .. N-1:  Y = A x_{m != n} U_m^T  (current factors);
    U_n = the R_n leading left singular vectors of Y_(n). Then G = Y x_n U_n^T
    for the last n, r_k = ||A - G x U|| / ||A||, and the loop stops once
    |r_{k-1} - r_k| < tol (reading R10).
    """
    a = np.asarray(a, dtype=np.float64)
    N = a.ndim
    us = [np.array(u, dtype=np.float64) for u in us0]
    ranks = [u.shape[1] for u in us]
    resid = [rel_error(a, project(a, us), us)]
    g = None
    converged = False
    k = 0
    for k in range(1, max_iters + 1):
        for n in range(N):
            y = _partial(a, us, n, transpose=True)
            us[n] = _leading_left(unfold(y, n), ranks[n])[0]
        g = mode_product(y, us[N - 1].T, N - 1)
        resid.append(rel_error(a, g, us))
        if abs(resid[-2] - resid[-1]) < tol:
            converged = True
            break
    if g is None:
        g = project(a, us)
    return HOOIResult(G=g, U=us, resid=resid, iters=k, converged=converged)


# ---------------------------------------------------------------------------
# Sec. 5: singular vectors from the t-HOSVD-ALS basis (reading R11)
# ---------------------------------------------------------------------------

def sign_fix(u: np.ndarray) -> np.ndarray:
    """Flip each column so that its entry of largest magnitude is positive
    (first such entry on ties; reading R11)."""
    u = np.array(u, dtype=np.float64)
    idx = np.argmax(np.abs(u), axis=0)
    s = np.sign(u[idx, np.arange(u.shape[1])])
    s[s == 0] = 1.0
    return u * s


def singular_vectors(a: np.ndarray, n: int, qhat: np.ndarray):
    """U^(n) = Qhat U and the singular values S, where Qhat^T A_(n) = U S V^T
    (Sec. 5, after Alg. 4), signs fixed by ``sign_fix``."""
    m = unfold(np.asarray(a, dtype=np.float64), n)
    q = np.asarray(qhat, dtype=np.float64)
    u, s, _ = np.linalg.svd(q.T @ m, full_matrices=False)
    return sign_fix(q @ u), s


def rel_error(a: np.ndarray, g: np.ndarray, us: Sequence[np.ndarray]) -> float:
    """||A - G x U||_F / ||A||_F by explicit reconstruction (Sec. 6.1 measure)."""
    a = np.asarray(a, dtype=np.float64)
    d = a - reconstruct(g, us)
    return float(np.sqrt(frob2(d) / frob2(a)))


def principal_angles(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Principal angles between range(u) and range(v) (radians)."""
    qu = np.linalg.qr(np.asarray(u, dtype=np.float64))[0]
    qv = np.linalg.qr(np.asarray(v, dtype=np.float64))[0]
    s = np.linalg.svd(qu.T @ qv, compute_uv=False)
    s = np.clip(s, -1.0, 1.0)
    # arccos loses accuracy near 0: use arcsin of the residual norm instead
    res = qv - qu @ (qu.T @ qv)
    sin = np.linalg.svd(res, compute_uv=False)
    return np.sort(np.arcsin(np.clip(sin, 0.0, 1.0)))


# ---------------------------------------------------------------------------
# Differentiation: adjoints of the core projection and of the reconstruction
# (Tucker model, Sec. 2; partial contractions are recomputed, never stored)
# ---------------------------------------------------------------------------

def _partial(x: np.ndarray, us: Sequence[np.ndarray], skip: int, transpose: bool) -> np.ndarray:
    """X x_{m != skip} U_m^T (transpose=True) or X x_{m != skip} U_m."""
    y = np.asarray(x, dtype=np.float64)
    for m, u in enumerate(us):
        if m == skip:
            continue
        u = np.asarray(u, dtype=np.float64)
        y = mode_product(y, u.T if transpose else u, m)
    return y


def project_vjp(a: np.ndarray, us: Sequence[np.ndarray], g_bar: np.ndarray):
    """Adjoint of G = A x_1 U1^T ... x_N UN^T.

    A_bar = G_bar x_1 U1 ... x_N UN;
    U_n_bar = (A x_{m!=n} U_m^T)_(n) (G_bar)_(n)^T   (I_n x R_n).
    """
    a_bar = reconstruct(g_bar, us)
    u_bar = []
    for n in range(len(us)):
        p = _partial(a, us, n, transpose=True)
        u_bar.append(unfold(p, n) @ unfold(g_bar, n).T)
    return a_bar, u_bar


def reconstruct_vjp(g: np.ndarray, us: Sequence[np.ndarray], b_bar: np.ndarray):
    """Adjoint of B = G x_1 U1 ... x_N UN.

    G_bar = B_bar x_1 U1^T ... x_N UN^T;
    U_n_bar = (B_bar x_{m!=n} U_m^T)_(n) G_(n)^T   (I_n x R_n).
    """
    g_bar = project(b_bar, us)
    u_bar = []
    for n in range(len(us)):
        p = _partial(b_bar, us, n, transpose=True)
        u_bar.append(unfold(p, n) @ unfold(g, n).T)
    return g_bar, u_bar


def recon_loss(a: np.ndarray, us: Sequence[np.ndarray]) -> float:
    """f(A, U) = ||A - (A x U^T) x U||_F^2 (reconstruction loss)."""
    g = project(a, us)
    return frob2(np.asarray(a, dtype=np.float64) - reconstruct(g, us))


def recon_loss_grad(a: np.ndarray, us: Sequence[np.ndarray]):
    """Gradient of ``recon_loss`` w.r.t. A and every U_n, chaining the two
    adjoints above: B_bar = -2 (A - B), then reconstruct_vjp, then project_vjp,
    plus the direct term 2 (A - B) for A."""
    a = np.asarray(a, dtype=np.float64)
    g = project(a, us)
    b = reconstruct(g, us)
    d = a - b
    b_bar = -2.0 * d
    g_bar, ub_rec = reconstruct_vjp(g, us, b_bar)
    a_bar_proj, ub_proj = project_vjp(a, us, g_bar)
    a_bar = 2.0 * d + a_bar_proj
    u_bar = [x + y for x, y in zip(ub_rec, ub_proj)]
    return a_bar, u_bar


def all_orders(N: int):
    return list(itertools.permutations(range(N)))
