// The fused ALS pass over the mode-n unfolding (CUDA cores, FP32 or FP64).
//
// One CTA walks tiles of kTileCols consecutive unfolding columns j = p*Q + q,
// reading B[p, 0:I, q] in place (never forming a permuted unfolding, Sec. 3
// "row-wise update"). A tile is held as I x (JT + 4); for views with Q = 1,
// whose columns are contiguous rows of the tensor, as JT x (I + 4) (TR). Per tile, with Qb the orthonormal basis of L_k in shared
// memory:
//   step 1  W_t = B_t^T Qb                (kTileCols x RC, K = I)     Alg. 3 R-update
//   step 2  Y  += B_t W_t                 (I x RC, K = kTileCols)     Alg. 3 L-update
// so one read of the tensor gives Y = B B^T Qb (Eq. 2.2). Y stays in registers
// across the CTA's tiles and is written once as a per-CTA partial; the FP64
// reduction over CTAs runs in a second kernel (deterministic order). ||W||^2 is
// accumulated per tile in the compute type and per CTA in FP64, giving
// e_k^2 = ||B||^2 - ||W||^2 for the Eq. 5.01 stop rule. W itself is written in
// the P x R x Q layout, i.e. as the tensor B x_n Qb^T -- the st-HOSVD
// truncation of Alg. 5 without another pass.
//
// Tiles are staged into shared memory with cp.async, two buffers deep, so the
// next tile streams in while the current one is multiplied. The tile is kept
// as Ts[i][c] with 16-byte aligned rows: step 1 reads four columns of a row as
// one vector, step 2 reads four columns of the thread's rows the same way.
//
// Rank is split into chunks of RC columns along gridDim.y: a chunk's W and Y
// columns depend only on the same columns of Qb, so chunks are independent.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace tals {

constexpr int kJT = kTileCols;   // columns per tile
constexpr int kJTP = kJT + 4;    // padded row stride (elements), keeps rows 16-byte aligned

template <typename T>
struct PassArgs {
  const T* X;
  long long P, I, Q, J;
  int R;
  int mode;
  const T* L;
  const T* Win;      // PASS_GIVEN: W read from a tensor in the P x R x Q layout
  T* Ypart;
  double* spart;
  T* Wout;
  uint64_t sketch_state;
  const ModeState* st;
  int w_from_k;
  long long ntiles;
  int nbuf;          // tile buffers (2: cp.async double buffering)
  int vec_ok;        // X is 16-byte aligned and Q keeps rows aligned
  int resid;         // SWEEP: accumulate ||B - Qb W^T||^2 instead of ||W||^2 (one chunk only)
};

template <typename T, int RC, int RPT, int RW, int NT, int JT = kJT>
struct PassShape {
  static constexpr int NRG = RC / RW;              // r-groups of the Y accumulation
  static constexpr int ROWT = NT / NRG;            // row-threads per r-group
  static constexpr int CG = JT / 4;                // step-1 column groups of 4 per warp
  static constexpr int RG = 32 / CG;               // step-1 r-groups per warp
  static constexpr int RL = RC / RG;               // r-columns per lane in step 1
  static constexpr int NW = NT / 32;               // warps (step 1 splits I over them)
  static constexpr int WSP = RC + 4;               // padded row stride of W tiles
  static_assert(RC % RW == 0 && RC % RG == 0 && RW % 4 == 0 && JT % 16 == 0 && JT <= 128,
                "bad chunk");
  static_assert(NT % NRG == 0 && (ROWT % 32) == 0, "r-groups must be warp-uniform");
};

// Rows of slack after the tile buffers: step 2 reads (and discards) rows up to
// rowspan - 1 of the last buffer.
__host__ __device__ inline long long slack_rows(long long I, int rowspan) {
  return rowspan > I ? rowspan - I : 0;
}

// Transposed tile (views with Q = 1, FP32): column c of the tile -- row p = j0 + c
// of the P x I view, contiguous in memory -- is row c of a JT x tr_pitch(I)
// array, copied with 16-byte chunks; step 2's reads past row I - 1 of the last
// column need tr_slack elements after the last buffer.
__host__ __device__ inline long long tr_pitch(long long I) { return I + 4; }
__host__ __device__ inline long long tr_slack(long long I, int rowspan) {
  const long long s = rowspan - tr_pitch(I);
  return s > 0 ? (s + 3) / 4 * 4 : 0;
}

// Step 1 with half-warp row split (FP32, 16-column tiles, rank chunk 32, 256
// threads): a lane holds 4 columns x 8 ranks instead of 4 x 4, so each column
// value it broadcasts feeds four paired FMAs instead of two; the two half-warps
// take alternate rows (alternate groups of four rows for transposed tiles) and
// leave separate partials, doubling the cross-warp reduction buffer.
__host__ __device__ constexpr bool pass_split_rows(bool f32, bool tr, int rc, int nt, int jt) {
  return f32 && rc == 32 && nt == 256 && jt == 16;
}

template <typename T>
__host__ __device__ inline size_t pass_smem_bytes(long long I, int RC, int rowspan, int nbuf,
                                                  int nt = kThreads, int jt = kJT, bool tr = false) {
  const size_t jtp = (size_t)jt + 4;
  size_t ts = tr ? (size_t)nbuf * jt * tr_pitch(I) + (size_t)tr_slack(I, rowspan)
                 : (size_t)nbuf * ((size_t)I * jtp) + (size_t)slack_rows(I, rowspan) * jtp;
  size_t ls = (size_t)I * RC;
  size_t wr = (size_t)(nt / 32) * jt * (RC + 4) *
              (pass_split_rows(sizeof(T) == 4, tr, RC, nt, jt) ? 2 : 1);
  size_t ws = (size_t)jt * (RC + 4);
  return (ts + ls + wr + ws) * sizeof(T) + 32 * sizeof(double);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}
template <int B>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, int src_bytes) {
  if constexpr (B == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Issue the copies of tile t (JT columns) into Tb (I x (JT + 4)). Columns beyond J are zero-filled.
// Column c of the tile is B[p, :, q] with (p, q) stepped from the tile's first
// column: one division per tile, none per element.
template <typename T, int JT = kJT, bool TR = false>
__device__ __forceinline__ void issue_tile(const PassArgs<T>& a, long long t, T* Tb) {
  const long long I = a.I, Q = a.Q;
  const long long j0 = t * JT;
  const int tid = threadIdx.x, nt = blockDim.x;
  if constexpr (TR) {
    // Q = 1: tile column c is the contiguous row j0 + c of the P x I view
    const long long IP = tr_pitch(I);
    if (a.vec_ok) {   // X 16-byte aligned and I % 4 == 0
      constexpr int EPV = 16 / sizeof(T);
      const long long cpr = I / EPV;
      for (long long e = tid; e < JT * cpr; e += nt) {
        const int c = (int)(e / cpr);
        const long long k = e - c * cpr;
        const bool ok = j0 + c < a.J;
        cp_async16(Tb + c * IP + k * EPV, a.X + (ok ? (j0 + c) * I + k * EPV : 0), ok ? 16 : 0);
      }
    } else {
      for (long long e = tid; e < JT * I; e += nt) {
        const int c = (int)(e / I);
        const long long i = e - c * I;
        const bool ok = j0 + c < a.J;
        cp_async_elem<sizeof(T)>(Tb + c * IP + i, a.X + (ok ? (j0 + c) * I + i : 0),
                                 ok ? (int)sizeof(T) : 0);
      }
    }
    return;
  }
  const long long p0 = j0 / Q, q0 = j0 - p0 * Q;
  constexpr int EPV = 16 / sizeof(T);   // elements per 16-byte chunk
  if (a.vec_ok && q0 + JT <= Q && j0 + JT <= a.J) {
    // whole tile inside one p: every row is JT contiguous elements
    const T* base = a.X + p0 * I * Q + q0;
    constexpr int CPR = JT / EPV;      // chunks per row
    for (long long e = tid; e < I * CPR; e += nt) {
      const long long i = e / CPR;
      const int k = (int)(e - i * CPR);
      cp_async16(Tb + i * (JT + 4) + k * EPV, base + i * Q + k * EPV, 16);
    }
  } else if (Q >= JT) {
    // column-fastest element copies; the tile's columns span at most two p
    for (long long e = tid; e < I * JT; e += nt) {
      const long long i = e / JT;
      const int c = (int)(e - i * JT);
      const bool ok = j0 + c < a.J;
      long long q = q0 + c, p = p0;
      if (q >= Q) {
        q -= Q;
        ++p;
      }
      cp_async_elem<sizeof(T)>(Tb + i * (JT + 4) + c, a.X + (ok ? (p * I + i) * Q + q : 0),
                               ok ? (int)sizeof(T) : 0);
    }
  } else {
    // short rows (Q < JT; Q = 1 for the last mode): column by column, consecutive
    // threads read consecutive i (contiguous when Q = 1)
    long long p = p0, q = q0;
    for (int c = 0; c < JT; ++c) {
      const bool ok = j0 + c < a.J;
      const T* col = a.X + (ok ? p * I * Q + q : 0);
      for (long long i = tid; i < I; i += nt)
        cp_async_elem<sizeof(T)>(Tb + i * (JT + 4) + c, col + (ok ? i * Q : 0), ok ? (int)sizeof(T) : 0);
      if (++q == Q) {
        q = 0;
        ++p;
      }
    }
  }
}

// load 4 consecutive T from 16-byte aligned shared memory
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

// One CTA's share of a pass: tiles t_begin, t_begin + t_step, ... of rank chunk
// `rchunk`. Y (this chunk's columns) is written to Yout (I x R, row stride R);
// returns the CTA's FP64 sum (||B||^2, ||W||^2 or ||B - Qb W^T||^2) in thread 0.
template <typename T, int RC, int RPT, int RW, int NT, int JT = kJT, bool TR = false>
__device__ __forceinline__ double pass_cta(const PassArgs<T>& a, long long t_begin, long long t_step,
                                           int rchunk, unsigned char* smem_raw, T* Yout) {
  using S = PassShape<T, RC, RPT, RW, NT, JT>;
  static_assert(!TR || (sizeof(T) == 4 && S::RL % 2 == 0), "transposed tiles: FP32, even RL");
  constexpr int JTP = JT + 4;
  constexpr int WSP = S::WSP;
  const long long I = a.I;
  const long long IP = tr_pitch(I);   // TR: row pitch of the transposed tile
  // elements per tile buffer: [I][JTP], or [JT][IP] for TR
  const size_t TBS = TR ? (size_t)JT * IP : (size_t)I * JTP;
  T* Tbuf = reinterpret_cast<T*>(smem_raw);                                // [nbuf][tile]
  T* Ls = Tbuf + (size_t)a.nbuf * TBS +
          (TR ? (size_t)tr_slack(I, S::ROWT * RPT) : (size_t)slack_rows(I, S::ROWT * RPT) * JTP);  // [I][RC]
  constexpr bool SPLIT = pass_split_rows(sizeof(T) == 4, TR, RC, NT, JT);
  constexpr int NPART = SPLIT ? 2 * S::NW : S::NW;                        // step-1 partial sets
  T* Wred = Ls + (size_t)I * RC;                                           // [NPART][JT][WSP]
  T* Ws = Wred + (size_t)NPART * JT * WSP;                                 // [JT][WSP]
  double* red = reinterpret_cast<double*>(Ws + (size_t)JT * WSP);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = rchunk * RC;
  const bool do_w = a.mode == PASS_SWEEP || a.mode == PASS_PROJECT;
  const bool do_y = a.mode != PASS_PROJECT;
  const bool resid = a.resid && a.mode == PASS_SWEEP;
  const bool cfast = a.Q >= JT;   // W output mapping: q-contiguous or r-contiguous
  bool write_w = a.Wout != nullptr;
  if (write_w && a.st != nullptr)
    write_w = (a.st->k >= a.w_from_k) || (a.st->k + 1 >= a.st->max_sweeps);

  // first tile in flight before anything else
  long long t = t_begin;
  if (t < a.ntiles) issue_tile<T, JT, TR>(a, t, Tbuf);
  cp_async_commit();

  // Qb columns r0 .. r0+RC-1 (zero beyond R) into shared memory.
  if (do_w) {
    for (long long e = tid; e < I * RC; e += NT) {
      const long long i = e / RC;
      const int rl = (int)(e - i * RC);
      const int r = r0 + rl;
      Ls[e] = (r < a.R) ? a.L[i * a.R + r] : T(0);
    }
  }

  T yacc[RPT][RW];
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int v = 0; v < RW; ++v) yacc[k][v] = T(0);
  float2 yacc2[RPT][RW / 2];   // FP32 accumulators of step 2 (paired along r)
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int v = 0; v < RW / 2; ++v) yacc2[k][v] = make_float2(0.f, 0.f);
  double sacc = 0.0;   // this thread's share of the pass's FP64 sum

  const int rgrp = tid / S::ROWT;            // step-2 r-group (warp-uniform)
  const int ti = tid - rgrp * S::ROWT;       // step-2 row-thread index
  // step-1 row slice of this warp (TR: a multiple of 4 rows, for float4 reads along i)
  const long long IW = TR ? ((I + S::NW - 1) / S::NW + 3) / 4 * 4 : (I + S::NW - 1) / S::NW;
  const long long ilo = min(I, warp * IW), ihi = min(I, ilo + IW);
  const int cg = lane % S::CG, rg = lane / S::CG;   // step-1 lane layout: CG col groups x RG r groups

  int buf = 0;
  for (; t < a.ntiles; t += t_step) {
    const long long tn = t + t_step;
    T* Tb = Tbuf + (size_t)buf * TBS;
    cp_async_wait<0>();
    // tile t has landed for every thread, and every thread is done with the
    // previous tile: the other buffer, Wred and Ws are free
    __syncthreads();
    if (a.nbuf > 1) {
      // stream the next tile into the other buffer while this one is used
      if (tn < a.ntiles) issue_tile<T, JT, TR>(a, tn, Tbuf + (size_t)(buf ^ 1) * TBS);
      cp_async_commit();
    }
    const long long j0 = t * JT;
    const int ncol = (int)min((long long)JT, a.J - j0);

    if (a.mode == PASS_INIT && rchunk == 0) {
      if constexpr (sizeof(T) == 4) {
        // ||B||^2 for the stop rule: exact products (x^2 = p + e by FMA) in a
        // Neumaier-compensated FP32 sum, added to the FP64 total per tile
        float hi = 0.f, lo = 0.f;
        for (long long e = tid; e < I * JT; e += NT) {
          const long long i = e / JT;
          const int c = (int)(e - i * JT);
          const float x = (c < ncol) ? Tb[TR ? c * IP + i : i * JTP + c] : 0.f;
          const float pq = x * x, pe = fmaf(x, x, -pq);
          const float tq = hi + pq;
          lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
          hi = tq;
        }
        sacc += (double)hi + (double)lo;
      } else {
        T nacc = T(0);
        for (long long e = tid; e < I * JT; e += NT) {
          const long long i = e / JT;
          const int c = (int)(e - i * JT);
          const T x = Tb[i * JTP + c];
          nacc += (c < ncol) ? x * x : T(0);
        }
        sacc += (double)nacc;
      }
    }

    if (do_w) {
      // ---- step 1: W_t = B_t^T Qb, split over the warps along i ----
      T acc[4][S::RL];
      const T* trow = Tb + cg * 4;
      const T* lrow = Ls + rg * S::RL;
      const int nrow = (int)(ihi - ilo);
      if constexpr (SPLIT) {
        // half-warp h takes rows ilo + h, ilo + h + 2, ... (transposed tiles:
        // groups of four rows); lane (c4, r8) of the half holds four columns x
        // ranks 8 r8 .. 8 r8 + 7
        const int half = lane >> 4, c4 = lane & 3, r8 = (lane >> 2) & 3;
        float2 acc2[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc2[u][v] = make_float2(0.f, 0.f);
        if constexpr (TR) {
          // columns c4 + 4 u, as in the unsplit transposed path
          const int g0 = (int)ilo + 4 * half;
          const float* tc = reinterpret_cast<const float*>(Tb) + (long long)c4 * IP + g0;
          const float* lp = reinterpret_cast<const float*>(Ls) + g0 * RC + r8 * 8;
          const int nh = (nrow / 4 - half + 1) / 2;
#pragma unroll 2
          for (int gg = 0; gg < nh; ++gg) {
            float4 bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              bv[u] = *reinterpret_cast<const float4*>(tc + (long long)u * 4 * IP + 8 * gg);
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
              const float4 qa = *reinterpret_cast<const float4*>(lp + (8 * gg + r4) * RC);
              const float4 qb = *reinterpret_cast<const float4*>(lp + (8 * gg + r4) * RC + 4);
              const float2 l2[4] = {make_float2(qa.x, qa.y), make_float2(qa.z, qa.w),
                                    make_float2(qb.x, qb.y), make_float2(qb.z, qb.w)};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float x = r4 == 0 ? bv[u].x : r4 == 1 ? bv[u].y : r4 == 2 ? bv[u].z : bv[u].w;
                const float2 t2 = make_float2(x, x);
#pragma unroll
                for (int v = 0; v < 4; ++v) acc2[u][v] = __ffma2_rn(t2, l2[v], acc2[u][v]);
              }
            }
          }
        } else {
          const float* tp = reinterpret_cast<const float*>(Tb) + ((int)ilo + half) * JTP + c4 * 4;
          const float* lp = reinterpret_cast<const float*>(Ls) + ((int)ilo + half) * RC + r8 * 8;
          const int nh = (nrow - half + 1) / 2;
#pragma unroll 4
          for (int ii = 0; ii < nh; ++ii) {
            const float4 t4 = *reinterpret_cast<const float4*>(tp + 2 * ii * JTP);
            const float4 qa = *reinterpret_cast<const float4*>(lp + 2 * ii * RC);
            const float4 qb = *reinterpret_cast<const float4*>(lp + 2 * ii * RC + 4);
            const float2 l2[4] = {make_float2(qa.x, qa.y), make_float2(qa.z, qa.w),
                                  make_float2(qb.x, qb.y), make_float2(qb.z, qb.w)};
            const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float2 t2 = make_float2(tv[u], tv[u]);
#pragma unroll
              for (int v = 0; v < 4; ++v) acc2[u][v] = __ffma2_rn(t2, l2[v], acc2[u][v]);
            }
          }
        }
        float* wr = reinterpret_cast<float*>(Wred) + (size_t)(2 * warp + half) * JT * WSP;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float* d = wr + (TR ? c4 + 4 * u : c4 * 4 + u) * WSP + r8 * 8;
          *reinterpret_cast<float4*>(d) = make_float4(acc2[u][0].x, acc2[u][0].y, acc2[u][1].x, acc2[u][1].y);
          *reinterpret_cast<float4*>(d + 4) =
              make_float4(acc2[u][2].x, acc2[u][2].y, acc2[u][3].x, acc2[u][3].y);
        }
      } else if constexpr (TR) {
        // transposed tile: this lane's columns are cg + CG u (u = 0..3), so the
        // four column groups of a warp read different bank groups; rows in
        // fours, one float4 along i per column
        float2 acc2[4][S::RL / 2];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL / 2; ++v) acc2[u][v] = make_float2(0.f, 0.f);
        const float* tc = reinterpret_cast<const float*>(Tb) + (long long)cg * IP + ilo;
        const float* lp = reinterpret_cast<const float*>(lrow) + (int)ilo * RC;
#pragma unroll 2
        for (int ii = 0; ii < nrow; ii += 4) {
          float4 bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) bv[u] = *reinterpret_cast<const float4*>(tc + (long long)u * S::CG * IP + ii);
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            float2 l2[S::RL / 2];
            if constexpr (S::RL % 4 == 0) {
#pragma unroll
              for (int v = 0; v < S::RL; v += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(lp + (ii + r4) * RC + v);
                l2[v / 2] = make_float2(q4.x, q4.y);
                l2[v / 2 + 1] = make_float2(q4.z, q4.w);
              }
            } else {
              l2[0] = *reinterpret_cast<const float2*>(lp + (ii + r4) * RC);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float x = r4 == 0 ? bv[u].x : r4 == 1 ? bv[u].y : r4 == 2 ? bv[u].z : bv[u].w;
              const float2 t2 = make_float2(x, x);
#pragma unroll
              for (int v = 0; v < S::RL / 2; ++v) acc2[u][v] = __ffma2_rn(t2, l2[v], acc2[u][v]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL / 2; ++v) {
            acc[u][2 * v] = acc2[u][v].x;
            acc[u][2 * v + 1] = acc2[u][v].y;
          }
      } else if constexpr (sizeof(T) == 4 && S::RL % 2 == 0) {
        // FP32: paired FMAs (two lanes of r per instruction), same rounding as fmaf
        float2 acc2[4][S::RL / 2];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL / 2; ++v) acc2[u][v] = make_float2(0.f, 0.f);
        const float* tp = reinterpret_cast<const float*>(trow) + (int)ilo * JTP;
        const float* lp = reinterpret_cast<const float*>(lrow) + (int)ilo * RC;
#pragma unroll 4
        for (int ii = 0; ii < nrow; ++ii) {
          const float4 t4 = *reinterpret_cast<const float4*>(tp + ii * JTP);
          float2 l2[S::RL / 2];
          if constexpr (S::RL % 4 == 0) {
#pragma unroll
            for (int v = 0; v < S::RL; v += 4) {
              const float4 q4 = *reinterpret_cast<const float4*>(lp + ii * RC + v);
              l2[v / 2] = make_float2(q4.x, q4.y);
              l2[v / 2 + 1] = make_float2(q4.z, q4.w);
            }
          } else {
            l2[0] = *reinterpret_cast<const float2*>(lp + ii * RC);
          }
          const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 t2 = make_float2(tv[u], tv[u]);
#pragma unroll
            for (int v = 0; v < S::RL / 2; ++v) acc2[u][v] = __ffma2_rn(t2, l2[v], acc2[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL / 2; ++v) {
            acc[u][2 * v] = acc2[u][v].x;
            acc[u][2 * v + 1] = acc2[u][v].y;
          }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL; ++v) acc[u][v] = T(0);
        if (ilo < ihi) {
          T tv[4], lv[S::RL];
          ld4(trow + ilo * JTP, tv);
#pragma unroll
          for (int v = 0; v < S::RL; ++v) lv[v] = lrow[ilo * RC + v];
#pragma unroll 4
          for (long long i = ilo; i < ihi; ++i) {
            // operands of row i+1 are loaded before row i is multiplied
            const long long inx = (i + 1 < ihi) ? i + 1 : i;
            T tn4[4], ln[S::RL];
            ld4(trow + inx * JTP, tn4);
            if constexpr (S::RL % 4 == 0) {
#pragma unroll
              for (int v = 0; v < S::RL; v += 4) {
                T q4[4];
                ld4(lrow + inx * RC + v, q4);
#pragma unroll
                for (int w = 0; w < 4; ++w) ln[v + w] = q4[w];
              }
            } else {
#pragma unroll
              for (int v = 0; v < S::RL; ++v) ln[v] = lrow[inx * RC + v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < S::RL; ++v) acc[u][v] = fma(tv[u], lv[v], acc[u][v]);
#pragma unroll
            for (int u = 0; u < 4; ++u) tv[u] = tn4[u];
#pragma unroll
            for (int v = 0; v < S::RL; ++v) lv[v] = ln[v];
          }
        }
      }
      if constexpr (!SPLIT) {
        T* wr = Wred + (size_t)warp * JT * WSP;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < S::RL; ++v)
            wr[(TR ? cg + S::CG * u : cg * 4 + u) * WSP + rg * S::RL + v] = acc[u][v];
      }
      __syncthreads();
      // final W: consecutive threads -> consecutive q (cfast) or consecutive r
      T wsq = T(0);
      for (int o = tid; o < JT * RC; o += NT) {
        const int c = cfast ? (o % JT) : (o / RC);
        const int rl = cfast ? (o / JT) : (o % RC);
        T w = T(0);
#pragma unroll
        for (int g = 0; g < NPART; ++g) w += Wred[((size_t)g * JT + c) * WSP + rl];
        const int r = r0 + rl;
        const bool valid = (c < ncol) && (r < a.R);
        w = valid ? w : T(0);
        Ws[c * WSP + rl] = w;
        wsq += w * w;
        if (write_w && valid) {
          const long long j = j0 + c, p = j / a.Q, q = j - p * a.Q;
          a.Wout[(p * a.R + r) * a.Q + q] = w;
        }
      }
      if (!resid) sacc += (double)wsq;
      if (resid) {
        // ||B_t - Qb W_t^T||^2 from the tile: no cancellation against ||B||^2
        __syncthreads();
        T racc = T(0);
        for (long long e = tid; e < I * JT; e += NT) {
          const long long i = e / JT;
          const int c = (int)(e - i * JT);
          T dot = T(0);
#pragma unroll
          for (int v = 0; v < RC; v += 4) {
            T l4[4], w4[4];
            ld4(Ls + i * RC + v, l4);
            ld4(Ws + c * WSP + v, w4);
#pragma unroll
            for (int q = 0; q < 4; ++q) dot = fma(l4[q], w4[q], dot);
          }
          const T rsd = Tb[TR ? c * IP + i : i * JTP + c] - dot;
          racc += (c < ncol) ? rsd * rsd : T(0);
        }
        sacc += (double)racc;
      }
    } else if (a.mode == PASS_GIVEN) {
      // W_t read from the given tensor (P x R x Q layout)
      for (int o = tid; o < JT * RC; o += NT) {
        const int c = cfast ? (o % JT) : (o / RC);
        const int rl = cfast ? (o / JT) : (o % RC);
        const int r = r0 + rl;
        T w = T(0);
        if (c < ncol && r < a.R) {
          const long long j = j0 + c, p = j / a.Q, q = j - p * a.Q;
          w = a.Win[(p * a.R + r) * a.Q + q];
        }
        Ws[c * WSP + rl] = w;
      }
    } else {
      // INIT: W_t is the seeded sketch S restricted to the tile's columns
      for (int o = tid; o < JT * RC; o += NT) {
        const int c = o % JT, rl = o / JT;
        const int r = r0 + rl;
        T w = T(0);
        if (c < ncol && r < a.R) w = (T)sketch_entry(a.sketch_state, (uint64_t)(j0 + c), a.R, r);
        Ws[c * WSP + rl] = w;
      }
    }

    if (do_y) {
      __syncthreads();
      // ---- step 2: Y[i, r] += sum_c B_t[i, c] W_t[c, r] ----
      const T* wrow = Ws + rgrp * RW;
      const T* tbase = Tb + (size_t)ti * JTP;
      if constexpr (sizeof(T) == 4) {
        // FP32: paired FMAs along r, same rounding as fmaf
        const float* wp = reinterpret_cast<const float*>(wrow);
        const float* tp = reinterpret_cast<const float*>(tbase);
#pragma unroll
        for (int c4 = 0; c4 < JT; c4 += 4) {
          float tv[RPT][4];
          if constexpr (TR) {
            // transposed tile: consecutive threads read consecutive rows of a column
            const float* tcol = reinterpret_cast<const float*>(Tb) + ti;
#pragma unroll
            for (int k = 0; k < RPT; ++k)
#pragma unroll
              for (int u = 0; u < 4; ++u) tv[k][u] = tcol[(long long)(c4 + u) * IP + k * S::ROWT];
          } else {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
              const float4 x = *reinterpret_cast<const float4*>(tp + k * S::ROWT * JTP + c4);
              tv[k][0] = x.x; tv[k][1] = x.y; tv[k][2] = x.z; tv[k][3] = x.w;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float2 w2[RW / 2];
#pragma unroll
            for (int v = 0; v < RW; v += 4) {
              const float4 q4 = *reinterpret_cast<const float4*>(wp + (c4 + u) * WSP + v);
              w2[v / 2] = make_float2(q4.x, q4.y);
              w2[v / 2 + 1] = make_float2(q4.z, q4.w);
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
              const float2 b2 = make_float2(tv[k][u], tv[k][u]);
#pragma unroll
              for (int v = 0; v < RW / 2; ++v) yacc2[k][v] = __ffma2_rn(b2, w2[v], yacc2[k][v]);
            }
          }
        }
      } else {
#pragma unroll
        for (int c4 = 0; c4 < JT; c4 += 4) {
          T tv[RPT][4];
#pragma unroll
          for (int k = 0; k < RPT; ++k) ld4(tbase + (size_t)k * S::ROWT * JTP + c4, tv[k]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            T wv[RW];
#pragma unroll
            for (int v = 0; v < RW; v += 4) {
              T q4[4];
              ld4(wrow + (c4 + u) * WSP + v, q4);
#pragma unroll
              for (int w = 0; w < 4; ++w) wv[v + w] = q4[w];
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k)
#pragma unroll
              for (int v = 0; v < RW; ++v) yacc[k][v] = fma(tv[k][u], wv[v], yacc[k][v]);
          }
        }
      }
    }
    if (a.nbuf > 1) {
      buf ^= 1;
    } else {
      __syncthreads();   // the single buffer fully consumed before it is refilled
      if (tn < a.ntiles) {
        issue_tile<T, JT, TR>(a, tn, Tbuf);
        cp_async_commit();
      }
    }
  }
  cp_async_wait<0>();

  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
      for (int v = 0; v < RW / 2; ++v) {
        yacc[k][2 * v] = yacc2[k][v].x;
        yacc[k][2 * v + 1] = yacc2[k][v].y;
      }
  }
  if (do_y) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const long long i = ti + (long long)k * S::ROWT;
      if (i < I) {
#pragma unroll
        for (int v = 0; v < RW; ++v) {
          const int r = r0 + rgrp * RW + v;
          if (r < a.R) Yout[i * a.R + r] = yacc[k][v];
        }
      }
    }
  }
  return block_sum(sacc, red);
}

}  // namespace tals
