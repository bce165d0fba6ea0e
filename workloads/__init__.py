"""Seeded synthetic workloads: planted low-multilinear-rank tensors plus noise.

This module only *draws inputs*. It holds none of the ALS method's arithmetic
and is shared, read-only, by the FP64 oracle tests, the GPU parity tests and
the benchmark, so that both sides of every comparison see identical values.

Recipe (stands in for the paper's synthetic experiments, Sec. 6.1, and for
the workloads the benchmark times):

* factors ``U_n`` (``I_n x R_n``): Haar-random orthonormal columns -- the Q
  factor of a Gaussian matrix with column signs fixed so that ``diag(R) > 0``
  (Mezzadri 2007, "How to generate random matrices from the classical compact
  groups");
* core ``C`` (``R_1 x ... x R_N``), one of
    - ``"gauss"``: i.i.d. N(0, 1);
    - ``"inv_k"``: Gaussian ``Z`` scaled by ``1/k`` along every mode
      (``Z x_n diag(1, 1/2, ..., 1/R_n)``), a ``1/k`` mode spectrum;
    - ``"ratio"``: Gaussian ``Z`` scaled by ``rho^(k-1)`` along every mode;
    - ``"uniform510"``: i.i.d. U[5, 10], the core of the paper's Tucker-model
      experiment (Sec. 6.1.2);
* base ``A0 = C x_1 U_1 x_2 ... x_N U_N`` (the Tucker model, Sec. 2);
* noise ``E`` i.i.d. N(0, 1), rescaled so that ``||E||_F = nu * ||A0||_F``
  (relative Frobenius noise);
* ``A = A0 + E``, cast to the requested dtype. Consumers that need FP64 read
  ``float64(A)`` so that every side sees the same numbers.

The CP-model workload (``cp_model``) follows Sec. 6.1.1 instead: ``A0 =
sum_r lambda_r a_r o b_r o c_r`` with unit-norm Gaussian vectors ``a_r``
(``I``), ``b_r`` (``J = I``), ``c_r`` (``K = 100 I``), ``lambda_r ~ U[5, 10]``,
``R = 0.2 I`` terms, and ABSOLUTE noise ``A = A0 + delta E``, ``E`` i.i.d.
N(0, 1), ``delta = 1e-4`` (Sec. 6.1's noise model).

Seeds follow ``2004025830 + cfg`` for the named configurations.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

SEED_BASE = 2004025830


def _haar(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def _apply_along(x: np.ndarray, mat: np.ndarray, axis: int) -> np.ndarray:
    # y[..., a, ...] = sum_b mat[a, b] x[..., b, ...]; generator-only helper.
    y = np.tensordot(mat, x, axes=([1], [axis]))
    return np.moveaxis(y, 0, axis)


def _core(rng: np.random.Generator, ranks: Sequence[int], kind: str,
          ratio: float) -> np.ndarray:
    if kind == "uniform510":
        return rng.uniform(5.0, 10.0, size=tuple(ranks))
    z = rng.standard_normal(tuple(ranks))
    if kind == "gauss":
        return z
    for n, r in enumerate(ranks):
        k = np.arange(1, r + 1, dtype=np.float64)
        if kind == "inv_k":
            d = 1.0 / k
        elif kind == "ratio":
            d = ratio ** (k - 1.0)
        else:
            raise ValueError(f"unknown core kind {kind!r}")
        shape = [1] * len(ranks)
        shape[n] = r
        z = z * d.reshape(shape)
    return z


@dataclasses.dataclass
class Planted:
    A: np.ndarray            # the input tensor, in the requested dtype
    A0: np.ndarray           # noiseless base (float64 or float32 for big ones)
    core: np.ndarray
    factors: List[np.ndarray]
    noise_rel: float
    seed: int


def planted(seed: int, dims: Sequence[int], ranks: Sequence[int],
            core: str = "gauss", noise_rel: float = 1e-2,
            dtype=np.float32, ratio: float = 0.8,
            work_dtype=None) -> Planted:
    """Planted rank-(R_1..R_N) tensor plus relative Gaussian noise.

    ``work_dtype`` is the precision the base tensor and the noise are built in
    (float64 by default; float32 keeps memory down for the multi-GB shapes).
    """
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    if len(dims) != len(ranks):
        raise ValueError("dims and ranks differ in length")
    if work_dtype is None:
        work_dtype = np.float64 if int(np.prod(dims)) <= (1 << 26) else np.float32
    rng = np.random.Generator(np.random.PCG64(seed))
    factors = [_haar(rng, d, r) for d, r in zip(dims, ranks)]
    c = _core(rng, ranks, core, ratio)
    a0 = c.astype(work_dtype)
    for n, u in enumerate(factors):
        a0 = _apply_along(a0, u.astype(work_dtype), n)
    a0 = np.ascontiguousarray(a0, dtype=work_dtype)
    if noise_rel > 0:
        e = rng.standard_normal(a0.shape, dtype=np.float32 if work_dtype == np.float32
                                else np.float64)
        scale = noise_rel * np.sqrt(np.sum(a0.astype(np.float64) ** 2)) / \
            np.sqrt(np.sum(e.astype(np.float64) ** 2))
        e *= scale
        a = a0 + e.astype(work_dtype)
        del e
    else:
        a = a0.copy()
    return Planted(A=np.ascontiguousarray(a, dtype=dtype), A0=a0, core=c,
                   factors=factors, noise_rel=noise_rel, seed=seed)


@dataclasses.dataclass
class CPModel:
    A: np.ndarray            # the input tensor, in the requested dtype
    lam: np.ndarray          # the R weights lambda_r
    factors: List[np.ndarray]   # a (I x R), b (J x R), c (K x R), unit-norm columns
    delta: float
    seed: int


def cp_model(seed: int, I: int, R: int = None, delta: float = 1e-4, dtype=np.float32,
             k_ratio: int = 100, work_dtype=None) -> CPModel:
    """Sec. 6.1.1's random low CP-rank tensor plus absolute Gaussian noise.

    Shape ``I x I x k_ratio*I`` (the paper: ``k_ratio = 100``), ``R = round(0.2 I)``
    terms unless given; the truncation the paper applies is ``(R, R, R)``.
    """
    I = int(I)
    J, K = I, int(k_ratio) * I
    R = max(1, int(round(0.2 * I))) if R is None else int(R)
    n = I * J * K
    if work_dtype is None:
        work_dtype = np.float64 if n <= (1 << 26) else np.float32
    rng = np.random.Generator(np.random.PCG64(seed))
    fac = []
    for d in (I, J, K):
        x = rng.standard_normal((d, R))
        fac.append(x / np.linalg.norm(x, axis=0))
    lam = rng.uniform(5.0, 10.0, size=R)
    # entry (i, j, k) = sum_r lam_r a[i, r] b[j, r] c[k, r]: the (i, j) pairs as rows
    ab = ((fac[0] * lam)[:, None, :] * fac[1][None, :, :]).reshape(I * J, R)
    a0 = (ab.astype(work_dtype) @ fac[2].T.astype(work_dtype)).reshape(I, J, K)
    if delta > 0:
        e = rng.standard_normal(a0.shape, dtype=np.float32 if work_dtype == np.float32
                                else np.float64)
        a0 += (delta * e).astype(work_dtype)
        del e
    return CPModel(A=np.ascontiguousarray(a0, dtype=dtype), lam=lam, factors=fac,
                   delta=float(delta), seed=seed)


def tucker_model_device(seed: int, dims: Sequence[int], ranks: Sequence[int], delta: float = 1e-4,
                        device="cuda", base_only: bool = False, return_factors: bool = False):
    """Sec. 6.1.2's Tucker model at sizes too large to draw on the host, built on a
    torch device (FP32 result): Haar factors (QR of Gaussian, sign-fixed; the QR on
    the host), core
    i.i.d. U[5, 10], A0 = core x_1 U_1 ... x_N U_N, and A = A0 + delta E with E
    i.i.d. N(0, 1) (absolute noise, as the paper's Sec. 6.1). The expansions run
    in FP64 except the last (the first mode, the largest), which writes FP32; the
    noise is added in row blocks. Seeded through torch's generator on the device:
    the same seed gives the same tensor on one torch version. base_only: A0.
    return_factors: (A, [U_n]) with the planted FP64 factors."""
    import torch
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    factors = []
    for d, r in zip(dims, ranks):
        # the Gaussian draw on the device, its QR on the host (FP64)
        x = torch.randn((d, r), generator=g, device=device, dtype=torch.float64).cpu()
        q, rr = torch.linalg.qr(x)
        sg = torch.sign(torch.diagonal(rr))
        sg[sg == 0] = 1.0
        factors.append((q * sg).to(device))
    core = torch.rand(tuple(ranks), generator=g, device=device, dtype=torch.float64) * 5.0 + 5.0
    a = core
    for n in range(len(dims) - 1, 0, -1):
        a = torch.movedim(torch.tensordot(factors[n], a, dims=([1], [n])), 0, n)
    rest = a.reshape(ranks[0], -1).float()
    out = (factors[0].float() @ rest).reshape(dims)
    del a, rest
    if delta > 0 and not base_only:
        flat = out.view(dims[0], -1)
        step = max(1, (1 << 28) // flat.shape[1])
        for i0 in range(0, dims[0], step):
            blk = flat[i0:i0 + step]
            blk.add_(torch.randn(blk.shape, generator=g, device=device, dtype=torch.float32), alpha=delta)
    return (out, factors) if return_factors else out


def tucker_delta(dims: Sequence[int], ranks: Sequence[int], rel: float) -> float:
    """The absolute noise level delta of tucker_model_device that makes the noise
    about `rel` of the base tensor in norm: ||A0||^2 = ||core||^2 (orthonormal
    factors), E c^2 = 175/3 for c ~ U[5, 10], E ||E||^2 = prod(dims)."""
    return float(rel * np.sqrt(np.prod([float(r) for r in ranks]) * (175.0 / 3.0) /
                               np.prod([float(d) for d in dims])))


def uniform_tensor(seed: int, dims: Sequence[int], dtype=np.float32) -> np.ndarray:
    """Plain U[-1, 1) tensor (gradient and projection tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=tuple(dims)).astype(dtype)


def orthonormal(seed: int, rows: int, cols: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return _haar(rng, rows, cols).astype(dtype)


# ---------------------------------------------------------------------------
# Named configurations (the five workloads of the benchmark/parity suite)
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    dims: tuple
    ranks: tuple
    core: str
    noise_rel: float
    eta: float
    dtype: str        # "f64" or "f32"
    seed: int


CONFIGS = {
    # 64^3 FP64, multilinear rank (8,8,8), Gaussian core, 1e-3 noise, eta 1e-8
    "st64_f64": Config("st64_f64", (64, 64, 64), (8, 8, 8), "gauss", 1e-3, 1e-8,
                       "f64", SEED_BASE + 0),
    # 512^3 FP32, rank (32,32,32), 1/k core spectrum, 1e-2 noise, eta 1e-6
    "c512_f32": Config("c512_f32", (512, 512, 512), (32, 32, 32), "inv_k", 1e-2,
                       1e-6, "f32", SEED_BASE + 1),
    # 128^4 FP32, rank (16,16,16,16), 0.8^k spectrum, 1e-3 noise
    "q128_f32": Config("q128_f32", (128, 128, 128, 128), (16, 16, 16, 16), "ratio",
                       1e-3, 1e-6, "f32", SEED_BASE + 2),
    # 1024x1024x512 FP32, rank (64,64,32), 1/k spectrum, 1e-2 noise
    "d1024_f32": Config("d1024_f32", (1024, 1024, 512), (64, 64, 32), "inv_k", 1e-2,
                        1e-6, "f32", SEED_BASE + 4),
}


# Sec. 6.1.2's Tucker-model sizes: I x 100 x 100 x 100, I = 1000 .. 5000 (step 1000),
# truncation (I / 100, 10, 10, 10), core U[5, 10], delta = 1e-4
TUCKER_SIZES = (1000, 2000, 3000, 4000, 5000)
TUCKER_SEED = SEED_BASE + 7
# Sec. 6.4's dense test: a 5000 x 5000 x 50 Tucker tensor of multilinear rank
# (500, 500, 5) (the paper draws it with the Tensor Toolbox's ttensor), here the
# device-built Tucker model with noise 1e-2 of the base tensor in norm (so that
# e_k, and with it the stop rule, is well above FP32 rounding)
RANK500_DIMS = (5000, 5000, 50)
RANK500_RANKS = (500, 500, 5)
RANK500_SEED = SEED_BASE + 8
RANK500_NOISE = 1e-2

# Sec. 6.1.1's CP-model sizes: I = 20 .. 100 (step 20), shape I x I x 100 I,
# truncation (0.2 I, 0.2 I, 0.2 I), delta = 1e-4; the largest is 100 x 100 x 10000
CP_SIZES = (20, 40, 60, 80, 100)
CP_SEED = SEED_BASE + 6


def make(cfg: Config, **kw) -> Planted:
    dt = np.float64 if cfg.dtype == "f64" else np.float32
    return planted(cfg.seed, cfg.dims, cfg.ranks, cfg.core, cfg.noise_rel, dtype=dt, **kw)


def batched_shapes(seed: int, count: int, lo: int = 16, hi: int = 96,
                   rlo: int = 4, rhi: int = 16):
    """Uneven third-order shapes and ranks for the batched workload.

    Mode sizes ~ U{lo..hi}, ranks ~ U{rlo..rhi} clipped to the mode size and to
    the product of the other ranks (so every sequential truncation is feasible).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        dims = [int(x) for x in rng.integers(lo, hi + 1, size=3)]
        ranks = [int(min(x, d)) for x, d in zip(rng.integers(rlo, rhi + 1, size=3), dims)]
        for n in range(3):
            other = int(np.prod([ranks[m] for m in range(3) if m != n]))
            ranks[n] = min(ranks[n], other)
        out.append((tuple(dims), tuple(ranks)))
    return out


def batched(seed: int, count: int, noise_rel: float = 1e-2, **kw):
    """List of (A float32, dims, ranks) for the batched workload."""
    shapes = batched_shapes(seed, count, **kw)
    res = []
    for t, (dims, ranks) in enumerate(shapes):
        p = planted(seed * 7919 + t, dims, ranks, "gauss", noise_rel, dtype=np.float32)
        res.append((p.A, dims, ranks))
    return res
