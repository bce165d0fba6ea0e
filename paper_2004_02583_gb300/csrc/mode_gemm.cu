// One mode product of the Tucker model (Sec. 2) as a register-tiled FP32 GEMM:
//   out[p, a, q] = sum_b M[a, b] X[p, b, q]
// with X viewed as P x Bin x Q and out as P x Aout x Q. M is addressed through
// strides (element (a, b) at M[a*sa + b*sb]): M = U_n (sa = R, sb = 1) expands
// mode n from R_n to I_n (the Tucker reconstruction), M = U_n^T (sa = 1,
// sb = R) contracts it (the core projection). The contraction length Bin is a
// rank or a mode size; the products are short-K, so each CTA streams its X and
// output tiles once and keeps a 4 x 8 block of outputs per thread in registers
// (paired FMAs along the contiguous output index).
//
// Two layouts cover the views that occur: Q >= 64 (tiles of 64 a x 128 q per
// p, q contiguous) and Q == 1 (the last mode: tiles of 128 p x 64 a, a
// contiguous). Other views keep the sweep kernel's PROJECT pass.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tals {

namespace {

constexpr int kGK = 32;        // K chunk
constexpr int kGThreads = 256;

// Q >= 64: block (q-tile of 128, a-tile of 64, p). Thread (ty, tx) in 16 x 16
// owns a = 4 ty .. 4 ty + 3 and q = 8 tx .. 8 tx + 7.
__global__ void __launch_bounds__(kGThreads, 2)
    mode_gemm_cols(const float* __restrict__ X, long long Bin, long long Q, const float* __restrict__ M,
                   long long sa, long long sb, long long Aout, float* __restrict__ out, int vec) {
  __shared__ __align__(16) float Ms[kGK][64 + 4];    // [k][a]
  __shared__ __align__(16) float Xs[kGK][128 + 4];   // [k][q]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long q0 = (long long)blockIdx.x * 128, a0 = (long long)blockIdx.y * 64;
  const long long p = blockIdx.z;
  const float* Xp = X + p * Bin * Q;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long k0 = 0; k0 < Bin; k0 += kGK) {
    // M tile: 64 a x 32 k -> Ms[k][a]
    for (int e = tid; e < 64 * kGK; e += kGThreads) {
      const int a = sa == 1 ? e % 64 : e / kGK, k = sa == 1 ? e / 64 : e % kGK;
      const long long ga = a0 + a, gk = k0 + k;
      Ms[k][a] = (ga < Aout && gk < Bin) ? M[ga * sa + gk * sb] : 0.f;
    }
    // X tile: 32 k x 128 q (q contiguous)
    for (int e = tid; e < kGK * 128; e += kGThreads) {
      const int k = e >> 7, q = e & 127;
      const long long gk = k0 + k, gq = q0 + q;
      Xs[k][q] = (gk < Bin && gq < Q) ? Xp[gk * Q + gq] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGK; ++k) {
      const float4 m4 = *reinterpret_cast<const float4*>(&Ms[k][ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[k][tx * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[k][tx * 8 + 4]);
      const float2 xv[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y),
                            make_float2(x1.z, x1.w)};
      const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 m2 = make_float2(mv[i], mv[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __ffma2_rn(m2, xv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  float* op = out + p * Aout * Q;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long ga = a0 + ty * 4 + i;
    if (ga >= Aout) continue;
    const long long gq = q0 + tx * 8;
    float* row = op + ga * Q + gq;
    if (vec && gq + 8 <= Q && (Q & 3) == 0) {
      *reinterpret_cast<float4*>(row) = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
      *reinterpret_cast<float4*>(row + 4) = make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
    } else {
      const float v[8] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y,
                          acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y};
      for (int j = 0; j < 8; ++j)
        if (gq + j < Q) row[j] = v[j];
    }
  }
}

// Q == 1: out[p, a] = sum_b X[p, b] M[a, b]. Block (a-tile of 64, p-tile of
// 128). Thread (ty, tx) in 16 x 16 owns p = 8 ty .. 8 ty + 7, a = 4 tx .. 4 tx + 3.
__global__ void __launch_bounds__(kGThreads, 2)
    mode_gemm_rows(const float* __restrict__ X, long long P, long long Bin, const float* __restrict__ M,
                   long long sa, long long sb, long long Aout, float* __restrict__ out, int vec) {
  __shared__ __align__(16) float Xs[kGK][128 + 4];   // [k][p]
  __shared__ __align__(16) float Ms[kGK][64 + 4];    // [k][a]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long a0 = (long long)blockIdx.x * 64, p0 = (long long)blockIdx.y * 128;
  float2 acc[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  for (long long k0 = 0; k0 < Bin; k0 += kGK) {
    // X tile: 128 p x 32 k (k contiguous in memory) -> Xs[k][p]
    for (int e = tid; e < 128 * kGK; e += kGThreads) {
      const int pp = e / kGK, k = e % kGK;
      const long long gp = p0 + pp, gk = k0 + k;
      Xs[k][pp] = (gp < P && gk < Bin) ? X[gp * Bin + gk] : 0.f;
    }
    for (int e = tid; e < 64 * kGK; e += kGThreads) {
      const int a = sa == 1 ? e % 64 : e / kGK, k = sa == 1 ? e / 64 : e % kGK;
      const long long ga = a0 + a, gk = k0 + k;
      Ms[k][a] = (ga < Aout && gk < Bin) ? M[ga * sa + gk * sb] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGK; ++k) {
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[k][ty * 8 + 4]);
      const float4 m4 = *reinterpret_cast<const float4*>(&Ms[k][tx * 4]);
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float2 m01 = make_float2(m4.x, m4.y), m23 = make_float2(m4.z, m4.w);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 x2 = make_float2(xv[i], xv[i]);
        acc[i][0] = __ffma2_rn(x2, m01, acc[i][0]);
        acc[i][1] = __ffma2_rn(x2, m23, acc[i][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long gp = p0 + ty * 8 + i;
    if (gp >= P) continue;
    const long long ga = a0 + tx * 4;
    float* row = out + gp * Aout + ga;
    if (vec && ga + 4 <= Aout && (Aout & 3) == 0) {
      *reinterpret_cast<float4*>(row) = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
    } else {
      const float v[4] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y};
      for (int j = 0; j < 4; ++j)
        if (ga + j < Aout) row[j] = v[j];
    }
  }
}

// Residual form of mode_gemm_cols: instead of storing out = M X it accumulates
// sum (B - M X)^2 over the tile (exact squares in compensated FP32 per thread,
// FP64 per block) -- ||B_(n) - Q W^T||^2 with M = Q (I x R) and X = W (P x R x Q).
__global__ void __launch_bounds__(kGThreads, 2)
    mode_resid_cols(const float* __restrict__ X, long long Bin, long long Q, const float* __restrict__ M,
                    long long sa, long long sb, long long Aout, const float* __restrict__ B,
                    double* __restrict__ part) {
  __shared__ __align__(16) float Ms[kGK][64 + 4];
  __shared__ __align__(16) float Xs[kGK][128 + 4];
  __shared__ double red[32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long q0 = (long long)blockIdx.x * 128, a0 = (long long)blockIdx.y * 64;
  const long long p = blockIdx.z;
  const float* Xp = X + p * Bin * Q;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long k0 = 0; k0 < Bin; k0 += kGK) {
    for (int e = tid; e < 64 * kGK; e += kGThreads) {
      const int a = sa == 1 ? e % 64 : e / kGK, k = sa == 1 ? e / 64 : e % kGK;
      const long long ga = a0 + a, gk = k0 + k;
      Ms[k][a] = (ga < Aout && gk < Bin) ? M[ga * sa + gk * sb] : 0.f;
    }
    for (int e = tid; e < kGK * 128; e += kGThreads) {
      const int k = e >> 7, q = e & 127;
      const long long gk = k0 + k, gq = q0 + q;
      Xs[k][q] = (gk < Bin && gq < Q) ? Xp[gk * Q + gq] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGK; ++k) {
      const float4 m4 = *reinterpret_cast<const float4*>(&Ms[k][ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[k][tx * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[k][tx * 8 + 4]);
      const float2 xv[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y),
                            make_float2(x1.z, x1.w)};
      const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 m2 = make_float2(mv[i], mv[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __ffma2_rn(m2, xv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  const float* bp = B + p * Aout * Q;
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long ga = a0 + ty * 4 + i;
    if (ga >= Aout) continue;
    const float v[8] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y,
                        acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long gq = q0 + tx * 8 + j;
      if (gq >= Q) continue;
      const float d = bp[ga * Q + gq] - v[j];
      const float pq = d * d, pe = fmaf(d, d, -pq);
      const float tq = hi + pq;
      lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
      hi = tq;
    }
  }
  const double tot = block_sum((double)hi + (double)lo, red);
  if (tid == 0) part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot;
}

}  // namespace

// Number of partial sums launch_mode_resid_gemm writes (0: view not covered).
long long mode_resid_gemm_parts(long long P, long long Aout, long long Q) {
  if (Q < 64 || P > 65535 || (Aout + 63) / 64 > 65535) return 0;
  return ((Q + 127) / 128) * ((Aout + 63) / 64) * P;
}

cudaError_t launch_mode_resid_gemm(const float* X, long long P, long long Bin, long long Q,
                                   const float* M, long long sa, long long sb, long long Aout,
                                   const float* B, double* part, cudaStream_t s) {
  if (mode_resid_gemm_parts(P, Aout, Q) == 0) return cudaErrorNotSupported;
  const long long gx = (Q + 127) / 128, gy = (Aout + 63) / 64;
  mode_resid_cols<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)P), kGThreads, 0, s>>>(X, Bin, Q, M, sa, sb,
                                                                                   Aout, B, part);
  return cudaGetLastError();
}

cudaError_t launch_mode_gemm(const float* X, long long P, long long Bin, long long Q, const float* M,
                             long long sa, long long sb, long long Aout, float* out, cudaStream_t s) {
  if (P < 1 || Bin < 1 || Q < 1 || Aout < 1) return cudaErrorInvalidValue;
  const int vec = ((uintptr_t)out & 15) == 0;   // 16-byte stores only from an aligned base
  if (Q >= 64) {
    const long long gx = (Q + 127) / 128, gy = (Aout + 63) / 64;
    if (gy > 65535 || P > 65535) return cudaErrorNotSupported;
    mode_gemm_cols<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)P), kGThreads, 0, s>>>(X, Bin, Q, M, sa, sb,
                                                                                    Aout, out, vec);
    return cudaGetLastError();
  }
  if (Q == 1) {
    const long long gx = (Aout + 63) / 64, gy = (P + 127) / 128;
    if (gy > 65535) return cudaErrorNotSupported;
    mode_gemm_rows<<<dim3((unsigned)gx, (unsigned)gy), kGThreads, 0, s>>>(X, P, Bin, M, sa, sb, Aout, out, vec);
    return cudaGetLastError();
  }
  return cudaErrorNotSupported;
}

}  // namespace tals
