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
// Two layouts cover the views that occur: Q > 1 (tiles of a x flattened
// columns p*Q + q, q contiguous) and Q == 1 (the last mode: tiles of p x a,
// a contiguous). Views the kernels below do not take keep the sweep kernel's
// PROJECT pass or the any-view kernels at the end of this file.
//
// The main kernels (mg_pipe) are persistent: every CTA owns one a-tile for its
// whole life (the grid is a multiple of the number of a-tiles), walks its
// share of the column tiles and streams each tile's K chunks through a
// four-stage cp.async ring, so the HBM stream of X never waits on the FMAs.
// When the contraction is short (B_in <= 64, every expansion and the residual)
// the CTA's 64 x B_in slice of M stays in shared memory for the whole launch;
// longer contractions stage M with X. The first kernels below are the
// fallback for views the pipelined form does not take (unaligned bases, rows
// not a multiple of four floats).
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "internal.h"
#include "pass_impl.cuh"

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

// ---------------------------------------------------------------------------
// Persistent pipelined mode product.
constexpr int kMgThreads = 128;
constexpr int kMgBK = 16;        // K chunk per stage
constexpr int kMgResK = 64;      // longest contraction kept resident
constexpr int kRowsXS = kMgBK + 4;   // row stride of the rows kernel's X stage (odd count of 16 B)

struct MgArgs {
  const float* X;       // P x Bin x Q (Q == 1: P x Bin)
  long long P, Bin, Q;
  const float* M;       // M[a, b] at M[a * sa + b * sb]
  long long sa, sb, Aout;
  float* out;           // P x Aout x Q
  const float* B;       // residual form: P x Aout x Q
  double* part;         // residual form: one FP64 partial per CTA
  long long na;         // a-tiles (the grid is a multiple of na)
  long long nt;         // tiles per a-tile: cols ceil(P Q / TN), rows ceil(P / TN)
  int nk;               // K chunks
  int vec;              // 16-byte output stores
  const ModeState* gate;   // when set: run only while the mode's sweep is split and not done
  int every;               // with gate: run on every sweep until the mode is done
  const float* tgt;        // loss form (set: out = 2 (M X - tgt), part = per-CTA sums of (M X - tgt)^2)
};

// Tile geometry: TA a (outputs' rank side) x TN (cols: q, rows: p) = 8192
// outputs per CTA, 8 x 8 per thread.
template <bool ROWS, int TA>
struct MgShape {
  static constexpr int TN = 8192 / TA;
  static constexpr int STAGES = (ROWS && TA == 32) ? 3 : 4;
  static constexpr int XS = ROWS ? TN * kRowsXS : kMgBK * TN;   // floats per X stage
  static constexpr int NTX = ROWS ? TA / 8 : TN / 8;             // threads along the contiguous output index
};

template <bool ROWS, bool MRES, int TA>
constexpr size_t mg_smem_floats() {
  using S = MgShape<ROWS, TA>;
  const size_t ms = MRES ? 0 : (size_t)kMgBK * TA;
  return (size_t)S::STAGES * (S::XS + ms) + (MRES ? (size_t)kMgResK * TA : 0) + 64;  // + reduction
}

// out[p, a, q] (cols) / out[p, a] (rows): ROWS selects the view, MRES the
// resident M slice, RESID accumulates sum (B - M X)^2 instead of storing.
template <bool ROWS, bool MRES, bool RESID, int TA>
__global__ void __launch_bounds__(kMgThreads, 3) mg_pipe(MgArgs a) {
  if (a.gate != nullptr && ((!a.every && !a.gate->split) || a.gate->done)) return;   // uniform, before any barrier
  using S = MgShape<ROWS, TA>;
  constexpr int TN = S::TN, XS = S::XS, ST = S::STAGES;
  constexpr int MS = MRES ? 0 : kMgBK * TA;
  extern __shared__ __align__(16) float sm[];
  float* const ring = sm;
  float* const Mres = sm + ST * (XS + MS);
  const int tid = threadIdx.x;
  // cols: ty = a-group (a = ty*8 + u), tx = column group (flattened columns j = p*Q + q:
  //       tx*4 + {0..3} and TN/2 + tx*4 + {0..3} of the tile; Q % 4 == 0 keeps a group in one p)
  // rows: ty = p-group (p = ty + NP*u), tx = a-group (a = tx*4 + {0..3}, TA/2 + tx*4 + {0..3})
  constexpr int NP = TN / 8;   // rows: p-groups
  const int tx = tid % S::NTX, ty = tid / S::NTX;
  const long long at = blockIdx.x % a.na;
  const long long a0 = at * TA;
  const long long tb = blockIdx.x / a.na, ts = gridDim.x / a.na;
  const long long ntile = tb < a.nt ? (a.nt - tb + ts - 1) / ts : 0;
  const long long F = ntile * a.nk;

  if constexpr (MRES) {
    // the CTA's M slice, as [k][a] (zero beyond Bin and Aout)
    for (int e = tid; e < kMgResK * TA; e += kMgThreads) {
      int k, c;
      if (a.sb == 1) { c = e / kMgResK; k = e % kMgResK; } else { k = e / TA; c = e % TA; }
      const long long ga = a0 + c;
      Mres[k * TA + c] = (ga < a.Aout && k < a.Bin) ? a.M[ga * a.sa + k * a.sb] : 0.f;
    }
  }

  auto issue = [&](long long f) {
    if (f < F) {
      const long long i = f / a.nk;
      const int kc = (int)(f - i * a.nk);
      const long long t = tb + i * ts;
      const long long k0 = (long long)kc * kMgBK;
      float* xs = ring + (int)(f % ST) * (XS + MS);
      if constexpr (ROWS) {
        const long long p0 = t * TN;
#pragma unroll
        for (int j = 0; j < (TN * kMgBK / 4) / kMgThreads; ++j) {
          const int c = tid + j * kMgThreads;
          const int r = c >> 2, kq = (c & 3) * 4;
          const long long gp = p0 + r, gk = k0 + kq;
          const bool ok = gp < a.P && gk < a.Bin;
          cp_async16(xs + r * kRowsXS + kq, ok ? a.X + gp * a.Bin + gk : a.X, ok ? 16 : 0);
        }
      } else {
        // every chunk of this thread has the same column group (kMgThreads % (TN / 4) == 0)
        const int qc = (tid % (TN / 4)) * 4;
        const long long jc = t * TN + qc;
        const long long p = jc / a.Q, q = jc - p * a.Q;
        const bool jok = jc < a.P * a.Q;
        const float* Xp = a.X + p * a.Bin * a.Q + q;
#pragma unroll
        for (int j = 0; j < (kMgBK * TN / 4) / kMgThreads; ++j) {
          const int k = (tid + j * kMgThreads) / (TN / 4);
          const long long gk = k0 + k;
          const bool ok = jok && gk < a.Bin;
          cp_async16(xs + k * TN + qc, ok ? Xp + gk * a.Q : a.X, ok ? 16 : 0);
        }
      }
      if constexpr (!MRES) {
        float* ms = xs + XS;
#pragma unroll
        for (int j = 0; j < (kMgBK * TA / 4 + kMgThreads - 1) / kMgThreads; ++j) {
          const int c = tid + j * kMgThreads;
          if (c < kMgBK * TA / 4) {
            const int k = c / (TA / 4), ac = (c % (TA / 4)) * 4;
            const long long gk = k0 + k, ga = a0 + ac;
            const long long left = a.Aout - ga;
            const int nv = gk < a.Bin && left > 0 ? (left < 4 ? (int)left : 4) : 0;
            cp_async16(ms + k * TA + ac, nv > 0 ? a.M + gk * a.sb + ga : a.M, nv * 4);
          }
        }
      }
    }
    cp_async_commit();
  };

  float2 acc[8][4];
  float hi = 0.f, lo = 0.f;   // residual form: compensated sum of squares
#pragma unroll
  for (int s = 0; s < ST - 1; ++s) issue(s);
  for (long long f = 0; f < F; ++f) {
    issue(f + ST - 1);
    cp_async_wait<ST - 1>();
    __syncthreads();
    const long long i = f / a.nk;
    const int kc = (int)(f - i * a.nk);
    if (kc == 0) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = make_float2(0.f, 0.f);
    }
    const float* xs = ring + (int)(f % ST) * (XS + MS);
    const float* ms = MRES ? Mres + kc * kMgBK * TA : xs + XS;
    if constexpr (ROWS) {
#pragma unroll
      for (int kq = 0; kq < kMgBK; kq += 4) {
        float4 xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = *reinterpret_cast<const float4*>(xs + (ty + NP * u) * kRowsXS + kq);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const float4 m0 = *reinterpret_cast<const float4*>(ms + (kq + kk) * TA + tx * 4);
          const float4 m1 = *reinterpret_cast<const float4*>(ms + (kq + kk) * TA + TA / 2 + tx * 4);
          const float2 mp[4] = {make_float2(m0.x, m0.y), make_float2(m0.z, m0.w), make_float2(m1.x, m1.y),
                                make_float2(m1.z, m1.w)};
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float x = kk == 0 ? xv[u].x : kk == 1 ? xv[u].y : kk == 2 ? xv[u].z : xv[u].w;
            const float2 x2 = make_float2(x, x);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = __ffma2_rn(x2, mp[v], acc[u][v]);
          }
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMgBK; ++k) {
        const float4 m0 = *reinterpret_cast<const float4*>(ms + k * TA + ty * 8);
        const float4 m1 = *reinterpret_cast<const float4*>(ms + k * TA + ty * 8 + 4);
        const float4 x0 = *reinterpret_cast<const float4*>(xs + k * TN + tx * 4);
        const float4 x1 = *reinterpret_cast<const float4*>(xs + k * TN + TN / 2 + tx * 4);
        const float2 xp[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y),
                              make_float2(x1.z, x1.w)};
        const float mv[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float2 m2 = make_float2(mv[u], mv[u]);
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = __ffma2_rn(m2, xp[v], acc[u][v]);
        }
      }
    }
    if (kc == a.nk - 1) {
      const long long t = tb + i * ts;
      if constexpr (ROWS) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long gp = t * TN + ty + NP * u;
          if (gp >= a.P) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const long long ga = a0 + h * (TA / 2) + tx * 4;
            const float v4[4] = {acc[u][2 * h].x, acc[u][2 * h].y, acc[u][2 * h + 1].x, acc[u][2 * h + 1].y};
            float* row = a.out + gp * a.Aout + ga;
            if (a.tgt != nullptr) {
              // loss form: the gradient 2 (B - tgt) of ||B - tgt||^2, and its sum
              const float* trow = a.tgt + gp * a.Aout + ga;
              for (int e = 0; e < 4; ++e)
                if (ga + e < a.Aout) {
                  const float d = v4[e] - trow[e];
                  row[e] = 2.f * d;
                  const float pq = d * d, pe = fmaf(d, d, -pq), tq = hi + pq;
                  lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
                  hi = tq;
                }
            } else if (a.vec && ga + 4 <= a.Aout) {
              *reinterpret_cast<float4*>(row) = make_float4(v4[0], v4[1], v4[2], v4[3]);
            } else {
              for (int e = 0; e < 4; ++e)
                if (ga + e < a.Aout) row[e] = v4[e];
            }
          }
        }
      } else {
        long long base[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long jc = t * TN + h * (TN / 2) + tx * 4;
          const long long p = jc / a.Q, q = jc - p * a.Q;
          base[h] = jc < a.P * a.Q ? p * a.Aout * a.Q + q : -1;   // Q % 4 == 0: whole chunk or none
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long ga = a0 + ty * 8 + u;
          if (ga >= a.Aout) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (base[h] < 0) continue;
            const float v4[4] = {acc[u][2 * h].x, acc[u][2 * h].y, acc[u][2 * h + 1].x, acc[u][2 * h + 1].y};
            const long long off = base[h] + ga * a.Q;
            if constexpr (RESID) {
              const float4 b4 = *reinterpret_cast<const float4*>(a.B + off);
              const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float d = bv[e] - v4[e];
                const float pq = d * d, pe = fmaf(d, d, -pq), tq = hi + pq;
                lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
                hi = tq;
              }
            } else if (a.tgt != nullptr) {
              // loss form: the gradient 2 (B - tgt) of ||B - tgt||^2, and its sum
              const float4 t4 = *reinterpret_cast<const float4*>(a.tgt + off);
              const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
              float dv[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float d = v4[e] - tv[e];
                dv[e] = 2.f * d;
                const float pq = d * d, pe = fmaf(d, d, -pq), tq = hi + pq;
                lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
                hi = tq;
              }
              *reinterpret_cast<float4*>(a.out + off) = make_float4(dv[0], dv[1], dv[2], dv[3]);
            } else {
              *reinterpret_cast<float4*>(a.out + off) = make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  if (RESID || a.tgt != nullptr) {   // uniform across the CTA
    double* red = reinterpret_cast<double*>(Mres + (MRES ? kMgResK * TA : 0));
    const double tot = block_sum((double)hi + (double)lo, red);
    if (tid == 0) a.part[blockIdx.x] = tot;
  }
}

// Resident CTAs per SM of one instantiation, computed once per process (the
// attribute and the occupancy query are idempotent, so two threads racing on
// the first call both store the same value).
template <bool ROWS, bool MRES, bool RESID, int TA>
int mg_blocks_per_sm() {
  static std::atomic<int> occ{-1};
  int v = occ.load(std::memory_order_relaxed);
  if (v < 0) {
    const size_t smem = mg_smem_floats<ROWS, MRES, TA>() * sizeof(float);
    cudaFuncSetAttribute(mg_pipe<ROWS, MRES, RESID, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mg_pipe<ROWS, MRES, RESID, TA>, kMgThreads, smem) !=
            cudaSuccess ||
        n < 1)
      n = 1;
    occ.store(n, std::memory_order_relaxed);
    v = n;
  }
  return v;
}

template <bool ROWS, bool MRES, bool RESID, int TA>
void mg_run(const MgArgs& a, unsigned grid, cudaStream_t s) {
  mg_pipe<ROWS, MRES, RESID, TA><<<grid, kMgThreads, mg_smem_floats<ROWS, MRES, TA>() * sizeof(float), s>>>(a);
}

int mg_sms() {
  static std::atomic<int> sms[64];   // zero-initialised (static storage)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = sms[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    sms[dev].store(n, std::memory_order_relaxed);
    v = n;
  }
  return v;
}

// The pipelined form's launch for a view; ok = false where it does not apply
// (then the first kernels above run).
struct MgPlan {
  bool ok = false;
  bool rows = false, mres = false;
  int ta = 64;
  MgArgs a{};
  long long grid = 0;
};

template <bool ROWS, bool MRES, bool RESID>
int mg_occ(int ta) {
  return ta == 32 ? mg_blocks_per_sm<ROWS, MRES, RESID, 32>() : mg_blocks_per_sm<ROWS, MRES, RESID, 64>();
}

template <bool RESID>
MgPlan mg_plan(const float* X, long long P, long long Bin, long long Q, const float* M, long long sa,
               long long sb, long long Aout, float* out, const float* B = nullptr) {
  MgPlan pl;
  if (P < 1 || Bin < 1 || Q < 1 || Aout < 1) return pl;
  if (RESID && ((uintptr_t)B & 15) != 0) return pl;
  const bool rows = Q == 1;
  if (((uintptr_t)X & 15) != 0) return pl;
  if (rows ? (Bin & 3) != 0 : (Q & 3) != 0) return pl;
  const bool mres = Bin <= kMgResK;
  if (!mres && !(sa == 1 && (sb & 3) == 0 && ((uintptr_t)M & 15) == 0)) return pl;
  if (RESID && rows) return pl;
  const int ta = Aout <= 32 ? 32 : 64;
  const long long tn = 8192 / ta;
  MgArgs& a = pl.a;
  a.X = X; a.P = P; a.Bin = Bin; a.Q = Q; a.M = M; a.sa = sa; a.sb = sb; a.Aout = Aout; a.out = out;
  a.B = B;
  a.na = (Aout + ta - 1) / ta;
  a.nt = rows ? (P + tn - 1) / tn : (P * Q + tn - 1) / tn;
  a.nk = (int)((Bin + kMgBK - 1) / kMgBK);
  a.vec = out != nullptr && ((uintptr_t)out & 15) == 0 && (rows ? (Aout & 3) == 0 : true);
  if (!rows && !RESID && !a.vec) return pl;   // the cols stores are 16-byte
  int occ;
  if (rows) occ = mres ? mg_occ<true, true, false>(ta) : mg_occ<true, false, false>(ta);
  else occ = mres ? mg_occ<false, true, RESID>(ta) : mg_occ<false, false, RESID>(ta);
  const long long slots = (long long)mg_sms() * occ;
  const long long per_a = std::max<long long>(1, std::min<long long>(a.nt, slots / a.na));
  pl.grid = a.na * per_a;
  if (pl.grid > 0x7fffffffLL) return pl;
  pl.ok = true;
  pl.rows = rows;
  pl.mres = mres;
  pl.ta = ta;
  return pl;
}

template <bool RESID>
cudaError_t mg_launch(const MgPlan& pl, cudaStream_t s) {
  const unsigned g = (unsigned)pl.grid;
  const bool t32 = pl.ta == 32;
  if (pl.rows) {
    if (pl.mres) t32 ? mg_run<true, true, false, 32>(pl.a, g, s) : mg_run<true, true, false, 64>(pl.a, g, s);
    else t32 ? mg_run<true, false, false, 32>(pl.a, g, s) : mg_run<true, false, false, 64>(pl.a, g, s);
  } else if (pl.mres) {
    t32 ? mg_run<false, true, RESID, 32>(pl.a, g, s) : mg_run<false, true, RESID, 64>(pl.a, g, s);
  } else {
    t32 ? mg_run<false, false, RESID, 32>(pl.a, g, s) : mg_run<false, false, RESID, 64>(pl.a, g, s);
  }
  return cudaGetLastError();
}

}  // namespace

// Number of partial sums launch_mode_resid_gemm writes (0: view not covered).
long long mode_resid_gemm_parts(const float* X, long long P, long long Bin, long long Q, const float* M,
                                long long sa, long long sb, long long Aout, const float* B) {
  MgPlan pl = mg_plan<true>(X, P, Bin, Q, M, sa, sb, Aout, nullptr, B);
  if (pl.ok) return pl.grid;
  if (Q < 64 || P > 65535 || (Aout + 63) / 64 > 65535) return 0;
  return ((Q + 127) / 128) * ((Aout + 63) / 64) * P;
}

cudaError_t launch_mode_resid_gemm(const float* X, long long P, long long Bin, long long Q,
                                   const float* M, long long sa, long long sb, long long Aout,
                                   const float* B, double* part, cudaStream_t s) {
  MgPlan pl = mg_plan<true>(X, P, Bin, Q, M, sa, sb, Aout, nullptr, B);
  if (pl.ok) {
    pl.a.part = part;
    return mg_launch<true>(pl, s);
  }
  if (Q < 64 || P > 65535 || (Aout + 63) / 64 > 65535) return cudaErrorNotSupported;
  const long long gx = (Q + 127) / 128, gy = (Aout + 63) / 64;
  mode_resid_cols<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)P), kGThreads, 0, s>>>(X, Bin, Q, M, sa, sb,
                                                                                   Aout, B, part);
  return cudaGetLastError();
}

bool mode_gemm_gated_ok(const float* X, long long P, long long Bin, long long Q, const float* M, long long sa,
                        long long sb, long long Aout, float* out) {
  return mg_plan<false>(X, P, Bin, Q, M, sa, sb, Aout, out).ok;
}

cudaError_t launch_mode_gemm_gated(const float* X, long long P, long long Bin, long long Q, const float* M,
                                   long long sa, long long sb, long long Aout, float* out, const ModeState* gate,
                                   cudaStream_t s, int every) {
  MgPlan pl = mg_plan<false>(X, P, Bin, Q, M, sa, sb, Aout, out);
  if (!pl.ok) return cudaErrorNotSupported;
  pl.a.gate = gate;
  pl.a.every = every;
  return mg_launch<false>(pl, s);
}

cudaError_t launch_mode_gemm_loss(const float* X, long long P, long long Bin, long long Q, const float* M,
                                  long long sa, long long sb, long long Aout, float* out, const float* tgt,
                                  double* part, long long cap, long long* nparts, cudaStream_t s) {
  MgPlan pl = mg_plan<false>(X, P, Bin, Q, M, sa, sb, Aout, out);
  if (!pl.ok || tgt == nullptr || ((uintptr_t)tgt & 15) != 0 || pl.grid > cap) return cudaErrorNotSupported;
  pl.a.tgt = tgt;
  pl.a.part = part;
  *nparts = pl.grid;
  return mg_launch<false>(pl, s);
}

cudaError_t launch_mode_gemm(const float* X, long long P, long long Bin, long long Q, const float* M,
                             long long sa, long long sb, long long Aout, float* out, cudaStream_t s) {
  if (P < 1 || Bin < 1 || Q < 1 || Aout < 1) return cudaErrorInvalidValue;
  {
    MgPlan pl = mg_plan<false>(X, P, Bin, Q, M, sa, sb, Aout, out);
    if (pl.ok) return mg_launch<false>(pl, s);
  }
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

// ---------------------------------------------------------------------------
// Any-view forms (FP32 and FP64): the fallback where the views above and the
// sweep kernel's PROJECT / GIVEN passes do not apply (long modes in FP64,
// unaligned FP32 views). Plain 32 x 32 shared-memory tiles; the column index
// c = p * Q + q runs over the flattened P x Q positions.
namespace {

template <typename T>
__global__ void __launch_bounds__(256)
    mode_gemm_any(const T* __restrict__ X, long long P, long long Bin, long long Q, const T* __restrict__ M,
                  long long sa, long long sb, long long Aout, T* __restrict__ out) {
  __shared__ T Ms[32][33];   // [k][a]
  __shared__ T Xs[32][33];   // [k][c]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long c = (long long)blockIdx.x * 32 + tx, a0 = (long long)blockIdx.y * 32;
  const bool cok = c < P * Q;
  const long long p = cok ? c / Q : 0, q = cok ? c - p * Q : 0;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (long long k0 = 0; k0 < Bin; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const long long gk = k0 + r, ga = a0 + tx;
      Xs[r][tx] = (cok && gk < Bin) ? X[(p * Bin + gk) * Q + q] : T(0);
      Ms[r][tx] = (ga < Aout && gk < Bin) ? M[ga * sa + gk * sb] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const T x = Xs[k][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma(Ms[k][ty + 8 * i], x, acc[i]);
    }
    __syncthreads();
  }
  if (!cok) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long ga = a0 + ty + 8 * i;
    if (ga < Aout) out[(p * Aout + ga) * Q + q] = acc[i];
  }
}

// part[s][i][r] = sum over columns j of split s of X[p, i, q] V[p, r, q]
// (j = p * Q + q): the factor adjoint X_(n) V_(n)^T in column splits.
template <typename T>
__global__ void __launch_bounds__(256)
    factor_adjoint_any(const T* __restrict__ X, long long P, long long I, long long Q, const T* __restrict__ V,
                       int R, long long jper, T* __restrict__ part) {
  __shared__ T Xs[32][33];   // [j][i]
  __shared__ T Vs[32][33];   // [j][r]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long i0 = (long long)blockIdx.x * 32, r0 = (long long)blockIdx.y * 32;
  const long long J = P * Q;
  const long long jb = (long long)blockIdx.z * jper;
  const long long je = jb + jper < J ? jb + jper : J;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (long long j0 = jb; j0 < je; j0 += 32) {
    const long long j = j0 + tx;
    const bool jok = j < je;
    const long long p = jok ? j / Q : 0, q = jok ? j - p * Q : 0;
    for (int rr = ty; rr < 32; rr += 8) {
      const long long gi = i0 + rr, gr = r0 + rr;
      Xs[tx][rr] = (jok && gi < I) ? X[(p * I + gi) * Q + q] : T(0);
      Vs[tx][rr] = (jok && gr < R) ? V[(p * R + gr) * Q + q] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const T x = Xs[jj][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] = fma(x, Vs[jj][ty + 8 * m], acc[m]);
    }
    __syncthreads();
  }
  const long long gi = i0 + tx;
  if (gi >= I) return;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const long long gr = r0 + ty + 8 * m;
    if (gr < R) part[((long long)blockIdx.z * I + gi) * R + gr] = acc[m];
  }
}

// out[e] = sum_s part[s * n + e], s in order (deterministic).
template <typename T>
__global__ void sum_splits(const T* __restrict__ part, int S, long long n, T* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    T v = part[e];
    for (int s = 1; s < S; ++s) v += part[(long long)s * n + e];
    out[e] = v;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_mode_gemm_any(const T* X, long long P, long long Bin, long long Q, const T* M, long long sa,
                                 long long sb, long long Aout, T* out, cudaStream_t s) {
  if (P < 1 || Bin < 1 || Q < 1 || Aout < 1) return cudaErrorInvalidValue;
  const long long gx = (P * Q + 31) / 32, gy = (Aout + 31) / 32;
  if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorNotSupported;
  mode_gemm_any<T><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(X, P, Bin, Q, M, sa, sb, Aout, out);
  return cudaGetLastError();
}

int factor_adjoint_splits(long long P, long long I, long long Q, int R, int sms) {
  const long long tiles = ((I + 31) / 32) * ((R + 31) / 32);
  long long S = (4LL * sms + tiles - 1) / tiles;
  const long long maxs = (P * Q + 1023) / 1024;   // at least 1024 columns per split
  if (S > maxs) S = maxs;
  if (S > 1024) S = 1024;
  return (int)(S < 1 ? 1 : S);
}

template <typename T>
cudaError_t launch_factor_adjoint_any(const T* X, long long P, long long I, long long Q, const T* V, int R,
                                      int S, T* part, T* Ubar, cudaStream_t s) {
  if (P < 1 || I < 1 || Q < 1 || R < 1 || S < 1) return cudaErrorInvalidValue;
  const long long J = P * Q;
  long long jper = (J + S - 1) / S;
  jper = (jper + 31) / 32 * 32;
  const long long gx = (I + 31) / 32, gy = (R + 31) / 32;
  if (gx > 0x7fffffffLL || gy > 65535 || S > 65535) return cudaErrorNotSupported;
  factor_adjoint_any<T><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)S), 256, 0, s>>>(X, P, I, Q, V, R, jper,
                                                                                    part);
  const long long n = I * R;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  sum_splits<T><<<(unsigned)blocks, 256, 0, s>>>(part, S, n, Ubar);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_adjoint_parts(const T* X, long long P, long long I, long long Q, const T* V, int R,
                                        int S, T* part, cudaStream_t s) {
  if (P < 1 || I < 1 || Q < 1 || R < 1 || S < 1) return cudaErrorInvalidValue;
  const long long J = P * Q;
  long long jper = (J + S - 1) / S;
  jper = (jper + 31) / 32 * 32;
  const long long gx = (I + 31) / 32, gy = (R + 31) / 32;
  if (gx > 0x7fffffffLL || gy > 65535 || S > 65535) return cudaErrorNotSupported;
  factor_adjoint_any<T><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)S), 256, 0, s>>>(X, P, I, Q, V, R, jper,
                                                                                    part);
  return cudaGetLastError();
}

template cudaError_t launch_factor_adjoint_parts<float>(const float*, long long, long long, long long, const float*,
                                                        int, int, float*, cudaStream_t);
template cudaError_t launch_factor_adjoint_parts<double>(const double*, long long, long long, long long,
                                                         const double*, int, int, double*, cudaStream_t);
template cudaError_t launch_mode_gemm_any<float>(const float*, long long, long long, long long, const float*,
                                                 long long, long long, long long, float*, cudaStream_t);
template cudaError_t launch_mode_gemm_any<double>(const double*, long long, long long, long long,
                                                  const double*, long long, long long, long long, double*,
                                                  cudaStream_t);
template cudaError_t launch_factor_adjoint_any<float>(const float*, long long, long long, long long,
                                                      const float*, int, int, float*, float*, cudaStream_t);
template cudaError_t launch_factor_adjoint_any<double>(const double*, long long, long long, long long,
                                                       const double*, int, int, double*, double*,
                                                       cudaStream_t);

}  // namespace tals
