// Small FP64 linear algebra around the pass (Alg. 3 updates, Remark 2 normal
// equations, the Alg. 4/5 QR step and the Eq. 5.01 stop rule).
//
// Work that is O(I R^2) (Gram matrices, row-wise solves) is spread over many
// CTAs, a few rows each, because FP64 throughput per SM is low on this part;
// only the O(R^3) Cholesky runs in one CTA.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace tals {

// ---------------------------------------------------------------------------
// Reduce per-CTA Y partials to FP64 and form Gram partials of a row block.
// ---------------------------------------------------------------------------
constexpr int kMaxSlices = 16;
constexpr int kReduceThreads = 1024;

template <typename T>
__global__ void reduce_rows_kernel(const T* __restrict__ Ypart, int gx, long long I, int R,
                                   double* __restrict__ Y64, int gram_mode,
                                   const double* __restrict__ L64, double* __restrict__ Gpart,
                                   int rows_per_block, const double* __restrict__ spart, int nsp,
                                   int which, ModeState* st, double* norm_a2, T* YT, int S) {
  if (st != nullptr && st->done) return;
  extern __shared__ double sh[];
  double* Ys = sh;                                   // [rows_per_block][R]
  double* As = sh + (size_t)rows_per_block * R;      // [rows_per_block][R] (L rows for CROSS)
  const long long row0 = (long long)blockIdx.x * rows_per_block;
  const int nrows = (int)min((long long)rows_per_block, I - row0);
  const int nent = nrows * R;
  const size_t stride = (size_t)I * R;
  // The partials are read with many loads in flight: when the block has more
  // threads than entries, each entry's partials are split over S slices
  // (b = sl, sl + S, ...) whose sums are then added in a fixed order.
  double* slice_sum = As + (size_t)rows_per_block * R;   // [S][nent]
  for (int e0 = threadIdx.x; e0 < S * nent; e0 += blockDim.x) {
    const int sl = e0 / nent, e = e0 - sl * nent;
    const long long i = row0 + e / R;
    const int r = e % R;
    const T* src = Ypart + (size_t)i * R + r + (size_t)sl * stride;
    const size_t sstride = (size_t)S * stride;
    const int nb = gx > sl ? (gx - sl + S - 1) / S : 0;
    double s;
    if constexpr (sizeof(T) == 4) {
      // FP32 partials: Neumaier-compensated FP32 sum (the running sum and its
      // exact rounding error), FP64-level accuracy at FP32 arithmetic rates
      float hi = 0.f, lo = 0.f;
      // batches of 8 loads in flight, the last one predicated (adding 0 is exact)
      for (int b = 0; b < nb; b += 8) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = b + u < nb ? src[(size_t)(b + u) * sstride] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float t = hi + x[u];
          lo += fabsf(hi) >= fabsf(x[u]) ? (hi - t) + x[u] : (x[u] - t) + hi;
          hi = t;
        }
      }
      s = (double)hi + (double)lo;
    } else {
      s = 0.0;
      for (int b = 0; b < nb; ++b) s += (double)src[(size_t)b * sstride];
    }
    slice_sum[(size_t)sl * nent + e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nent; e += blockDim.x) {
    const long long i = row0 + e / R;
    const int r = e % R;
    double s = 0.0;
    for (int sl = 0; sl < S; ++sl) s += slice_sum[(size_t)sl * nent + e];
    Ys[e] = s;
    if (Y64 != nullptr) Y64[i * R + r] = s;
    if (YT != nullptr) YT[i * R + r] = (T)s;
    if (gram_mode == 2) As[e] = L64[i * R + r];
  }
  __syncthreads();
  if (gram_mode != 0) {
    const double* A = gram_mode == 1 ? Ys : As;
    double* gp = Gpart + (size_t)blockIdx.x * R * R;
    for (int o = threadIdx.x; o < R * R; o += blockDim.x) {
      const int r = o / R, c = o % R;
      double g = 0.0;
      for (int k = 0; k < nrows; ++k) g = fma(A[k * R + r], Ys[k * R + c], g);
      gp[o] = g;
    }
  }
  if (blockIdx.x == 0 && spart != nullptr) {
    __shared__ double red[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < nsp; k += blockDim.x) v += spart[k];
    // fixed-order tree: per-thread strided sums, then block_sum
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) {
      if (which == 0) {
        st->normM2 = tot;
        if (norm_a2 != nullptr) *norm_a2 = tot;
      } else {
        st->sW = tot;
      }
    }
  }
}

RowPlan row_plan(long long I, int R, int num_sms) {
  RowPlan rp;
  // about one row block per SM, at least one row per block
  long long rpb = (I + num_sms - 1) / num_sms;
  rpb = std::max<long long>(1, std::min<long long>(rpb, 64));
  rp.rows_per_block = (int)rpb;
  rp.blocks = (int)((I + rpb - 1) / rpb);
  return rp;
}

cudaError_t launch_reduce_rows(int dtype, const void* Ypart, int gx, long long I, int R,
                               double* Y64, int gram_mode, const double* L64, double* Gpart,
                               const RowPlan& rp, const double* spart, int nsp, int which,
                               ModeState* st, double* norm_a2, cudaStream_t s, void* YT) {
  const int nent = rp.rows_per_block * R;
  int S = std::max(1, std::min(kMaxSlices, kReduceThreads / std::max(1, nent)));
  while (S > 1 && ((size_t)2 + S) * nent * sizeof(double) > 200 * 1024) --S;
  const size_t sm = ((size_t)2 + S) * nent * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(dtype == 1 ? (const void*)reduce_rows_kernel<float>
                                                    : (const void*)reduce_rows_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (dtype == 1)
    reduce_rows_kernel<float><<<rp.blocks, kReduceThreads, sm, s>>>((const float*)Ypart, gx, I, R, Y64,
                                                         gram_mode, L64, Gpart,
                                                         rp.rows_per_block, spart, nsp, which,
                                                         st, norm_a2, (float*)YT, S);
  else
    reduce_rows_kernel<double><<<rp.blocks, kReduceThreads, sm, s>>>((const double*)Ypart, gx, I, R, Y64,
                                                          gram_mode, L64, Gpart,
                                                          rp.rows_per_block, spart, nsp, which,
                                                          st, norm_a2, (double*)YT, S);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-CTA kernel: Gram sum, Eq. 5.01 stop rule, Cholesky.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;
constexpr int kMaxR = 64;                                              // rank limit of the solves

__global__ void __launch_bounds__(kSmallThreads) small_kernel(const double* __restrict__ Gpart,
                                                              int nb, int R, int op,
                                                              double* __restrict__ F,
                                                              ModeState* st,
                                                              const double* norm_a2,
                                                              cudaGraphConditionalHandle cond,
                                                              int has_cond,
                                                              const double* __restrict__ GL,
                                                              int f32) {
  const int tid = threadIdx.x;
  // R <= 32, FP32 factor: warp 0 factors in registers (row `lane` of the
  // symmetrised Gram per lane, identity beyond R). Its row is loaded here, in
  // the same round trip as the done flag.
  const bool reg32 = f32 && R <= 32 && nb == 1;
  float srow[32];
  if (reg32 && tid < 32) {
    const float* G32 = reinterpret_cast<const float*>(Gpart + R * R);   // FP32 copy (gram_sum)
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const bool in = tid < R && j < R;
      const float a = in ? G32[tid * R + j] : 0.f, b = in ? G32[j * R + tid] : 0.f;
      srow[j] = in ? 0.5f * (a + b) : (tid == j ? 1.f : 0.f);
    }
  }
  if (st->done) {
    if (has_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  __shared__ int fail;

  if (op == 1 || op == 2) {
    // Eq. 5.01 on e_k^2 = ||B_(n)||^2 - ||W||^2 (W = B^T Q_k is the LS optimum for Q_k),
    // plus tr((Q'^T Q' - I) X), the first-order term of the projector onto the
    // rounded basis Q' actually used, X = Q^T B B^T Q' (the cross Gram below)
    __shared__ int stop, phase_end;
    __shared__ double red[32];
    if (tid == 0) phase_end = 0;
    // a split sweep took its test on W alone (split_test_kernel) before Y existed;
    // here only the prediction for the next sweep and the L-update's factor remain
    const bool pre = op == 1 && st->split;
    double c = 0.0;
    if (GL != nullptr && !pre) {
      // a thread's first four entries: their loads issued together, then summed in
      // the order of the plain loop
      double g[4], x[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int o = tid + m * kSmallThreads;
        g[m] = o < R * R ? GL[o] : 0.0;
        x[m] = o < R * R ? Gpart[o] : 0.0;
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int o = tid + m * kSmallThreads;
        if (o < R * R) c += (g[m] - (o / R == o % R ? 1.0 : 0.0)) * x[m];
      }
      for (int o = tid + 4 * kSmallThreads; o < R * R; o += kSmallThreads) {
        const int r = o / R, q = o % R;
        c += (GL[o] - (r == q ? 1.0 : 0.0)) * Gpart[o];
      }
    }
    const double corr = block_sum(c, red);
    if (tid == 0 && pre) {
      stop = st->done;
      if (!stop) als_predict_split(st, sqrt(*norm_a2));
    } else if (tid == 0) {
      const bool rs = st->resid && op == 1;
      st->corr = rs ? 0.0 : corr;
      const double e2 = rs ? st->sW : st->normM2 - st->sW + corr;
      const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
      const int k = st->k;
      const double norm_a = sqrt(*norm_a2);
      int s = 0;
      if (op == 2) {
        // mixed-precision bulk phase: e from ||B||^2 - ||W||^2 is below BF16
        // resolution, so leave the phase once ||W||^2 = tr(Q^T B B^T Q) stops moving
        // at BF16 resolution (2^-9 relative), or after bulk_max sweeps; the stop
        // rule itself is only taken on the FP32 sweeps that follow
        const bool flat = st->bulk >= 1 && fabs(st->sW - st->sw_prev) <= 0.001953125 * st->sW;
        st->sw_prev = st->sW;
        if (flat || st->bulk + 1 >= st->bulk_max) {
          st->bulk_mode = 0;
          st->kf = 0;
          phase_end = 1;
        }
        st->bulk += 1;
      } else {
        s = als_stop_step(st, e, norm_a);
        if (!s) als_predict_split(st, norm_a);
      }
      if (op == 2) {
        if (k + 1 >= st->max_sweeps) s = 1;
        st->e_prev = e;
        st->e_cur = e;
        st->k = k + 1;
        if (s) st->done = 1;
      }
      stop = s;
    }
    __syncthreads();
    if (stop) {
      if (has_cond && tid == 0) cudaGraphSetConditional(cond, 0u);
      return;
    }
    // the bulk loop ends after this sweep; its L-update still runs below
    if (phase_end && has_cond && tid == 0) cudaGraphSetConditional(cond, 0u);
  }

  // Right-looking Cholesky in LDL^T form on the symmetrised Gram S (lower
  // triangle in shared memory). FP64 on this part is slow per instruction
  // (~64-cycle latency; a warp instruction holds an SMSP's FP64 pipe ~76
  // cycles whatever its active lanes), so the serial chain per step is kept
  // short: warp 0 finishes column k+1 (one FMA per lane), takes the pivot's
  // reciprocal (FP32 seed, one third-order FP64 correction) and forms
  // L_j = S[j][k+1] / d_{k+1}, while warps 1.. update the rest of the trailing
  // block, densely enumerated -- one barrier per step. Square roots come at
  // the end, in parallel: C[i][k] = S_k[i][k] / sqrt(d_k).
  __shared__ double S[kMaxR * kMaxR];
  __shared__ double Lc[2][kMaxR];
  __shared__ double rs[kMaxR];
  __shared__ long long tiny_bits;
  // (i', j') of dense index a = i'(i'+1)/2 + j' over a lower triangle, packed
  // 16:16; the trailing block of every step enumerates a prefix of it
  __shared__ int tri[(kMaxR - 1) * kMaxR / 2];
  for (int a = tid; a < (R - 1) * R / 2; a += kSmallThreads) {
    int ip = (int)((sqrtf(8.f * (float)a + 1.f) - 1.f) * 0.5f);
    while (ip * (ip + 1) / 2 > a) --ip;
    while ((ip + 1) * (ip + 2) / 2 <= a) ++ip;
    tri[a] = (ip << 16) | (a - ip * (ip + 1) / 2);
  }
  if (reg32) {
    // LDL^T in FP32 registers, one warp, no block barriers: at step k lane i
    // holds row i of S_k; the pivot d_k comes from lane k and every S_k[j][k]
    // from lane j by shuffle. The full symmetric matrix is carried (each lane
    // updates its whole row), so no transposes are needed.
    __shared__ int bad_r;
    if (tid < 32) {
      const int lane = tid;
      float dl = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) dl = j == lane ? srow[j] : dl;
      float dmax = lane < R ? dl : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      const int tiny = __float_as_int(64.f * 1.1920929e-7f * dmax);
      int bad = 0;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float d = __shfl_sync(0xffffffffu, srow[k], k);
        const int b = __float_as_int(d);
        bad |= (k < R) && !(b > tiny && ((b >> 23) & 0xff) != 0xff);
        const float l = srow[k] * __frcp_rn(d);
#pragma unroll
        for (int j = k + 1; j < 32; ++j) srow[j] = fmaf(-l, __shfl_sync(0xffffffffu, srow[k], j), srow[j]);
      }
      if (!bad) {
        // C = L D^{1/2}: C[i][j] = S_j[i][j] / sqrt(d_j), staged in FP32
        float* C32 = reinterpret_cast<float*>(S);
#pragma unroll
        for (int j = 0; j < 32; ++j) dl = j == lane ? srow[j] : dl;
        const float rsl = rsqrtf(dl);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float rsj = __shfl_sync(0xffffffffu, rsl, j);
          const float c = j < lane ? srow[j] * rsj : (j == lane ? dl * rsl : 0.f);
          if (lane < R && j < R) C32[lane * R + j] = c;
        }
      }
      if (lane == 0) bad_r = bad;
    }
    __syncthreads();
    if (!bad_r) {
      // the FP64 factor block, spread over all warps (each FP64 warp instruction
      // holds an SMSP's FP64 pipe ~76 cycles: one warp alone would take ~4x longer)
      const float* C32 = reinterpret_cast<const float*>(S);
      __shared__ double dinv_r[32];
      if (tid < R) dinv_r[tid] = 1.0 / (double)C32[tid * R + tid];
      __syncthreads();
      for (int o = tid; o < R * R; o += kSmallThreads) {
        const int r = o / R, c = o % R;
        const double cv = (double)C32[o];
        F[o] = cv;
        F[R * R + o] = cv * dinv_r[r];
        F[2 * R * R + o] = cv * dinv_r[c];
      }
      if (tid < R) F[3 * R * R + tid] = dinv_r[tid];
      return;
    }
    // a pivot failed in FP32: the FP64 factorization below
  } else if (f32) {
    // The same LDL^T in FP32 (4-cycle latency instead of 64), for factors that
    // only have to be invertible and well scaled -- chol(X) of the L-update on
    // FP32 data: the row solves apply it exactly in FP64, so Y X^-1 keeps the
    // span of Y, and the basis rotates by O(eps32 cond(X)) at most. A pivot
    // that fails in FP32 falls back to the FP64 factorization below.
    float* S32 = reinterpret_cast<float*>(S);   // the FP64 array's storage
    __shared__ float Lc32[2][kMaxR];
    __shared__ float rs32[kMaxR];
    __shared__ int tiny32, fail32;
    for (int o = tid; o < R * R; o += kSmallThreads) {
      const int r = o / R, c = o % R;
      if (c <= r) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nb; ++q) {
          a += Gpart[(size_t)q * R * R + r * R + c];
          b += Gpart[(size_t)q * R * R + c * R + r];
        }
        S32[r * R + c] = (float)(0.5 * (a + b));
      }
    }
    if (tid == 0) fail32 = 0;
    __syncthreads();
    if (tid < 32) {
      float dmax = 0.f;
      for (int r = tid; r < R; r += 32) dmax = fmaxf(dmax, S32[r * R + r]);
      for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      if (tid == 0) tiny32 = __float_as_int(64.f * 1.1920929e-7f * dmax);
    }
    __syncthreads();
    const int lane32 = tid & 31, warp32 = tid >> 5;
    auto ok32 = [&](float d) {
      const int b = __float_as_int(d);
      return b > tiny32 && ((b >> 23) & 0xff) != 0xff;
    };
    if (warp32 == 0) {
      const float d = S32[0];
      if (lane32 == 0 && !ok32(d)) fail32 = 1;
      const float dinv = __frcp_rn(d);
      for (int j = 1 + lane32; j < R; j += 32) Lc32[0][j] = S32[j * R] * dinv;
    }
    __syncthreads();
    for (int k = 0; k + 1 < R; ++k) {
      const int cb = k & 1, c1 = k + 1;
      if (warp32 == 0) {
        const float lk = Lc32[cb][c1];
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = c1 + lane32 + 32 * h;
          v[h] = i < R ? fmaf(-S32[i * R + k], lk, S32[i * R + c1]) : 0.f;
        }
        const float d = __shfl_sync(0xffffffffu, v[0], 0);
        if (lane32 == 0 && !ok32(d)) fail32 = 1;
        const float dinv = __frcp_rn(d);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = c1 + lane32 + 32 * h;
          if (i < R) {
            S32[i * R + c1] = v[h];
            if (i > c1) Lc32[cb ^ 1][i] = v[h] * dinv;
          }
        }
      } else {
        const int m = R - 2 - k;
        const int na = m * (m + 1) / 2;
        for (int a = tid - 32; a < na; a += kSmallThreads - 32) {
          const int ij = tri[a];
          const int i = k + 2 + (ij >> 16), j = k + 2 + (ij & 0xffff);
          S32[i * R + j] = fmaf(-S32[i * R + k], Lc32[cb][j], S32[i * R + j]);
        }
      }
      __syncthreads();
    }
    if (!fail32) {
      __shared__ double dinv32[kMaxR];
      for (int r = tid; r < R; r += kSmallThreads) {
        rs32[r] = rsqrtf(S32[r * R + r]);
        dinv32[r] = 1.0 / (double)(S32[r * R + r] * rs32[r]);
      }
      __syncthreads();
      for (int o = tid; o < R * R; o += kSmallThreads) {
        const int r = o / R, c = o % R;
        const double cv = c <= r ? (double)(S32[o] * rs32[c]) : 0.0;
        F[o] = cv;
        F[R * R + o] = cv * dinv32[r];
        F[2 * R * R + o] = cv * dinv32[c];
      }
      for (int r = tid; r < R; r += kSmallThreads) F[3 * R * R + r] = dinv32[r];
      return;
    }
    __syncthreads();   // every thread is past its last read of S32 before the FP64 reload
  }
  if (nb == 1) {
    // the summed Gram: four entries' loads in flight per thread and round
    for (int m0 = 0; m0 < R * R; m0 += 4 * kSmallThreads) {
      double a[4], b[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int o = m0 + tid + m * kSmallThreads;
        const int r = o / R, c = o % R;
        const bool in = o < R * R && c <= r;
        a[m] = in ? Gpart[r * R + c] : 0.0;
        b[m] = in ? Gpart[c * R + r] : 0.0;
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int o = m0 + tid + m * kSmallThreads;
        const int r = o / R, c = o % R;
        // symmetrise (the cross Gram Q^T B B^T Q is symmetric in exact arithmetic)
        if (o < R * R && c <= r) S[r * R + c] = 0.5 * (a[m] + b[m]);
      }
    }
  } else {
    for (int o = tid; o < R * R; o += kSmallThreads) {
      const int r = o / R, c = o % R;
      if (c <= r) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nb; ++q) {
          a += Gpart[(size_t)q * R * R + r * R + c];
          b += Gpart[(size_t)q * R * R + c * R + r];
        }
        S[r * R + c] = 0.5 * (a + b);
      }
    }
  }
  if (tid == 0) fail = 0;
  // largest diagonal entry, from the high words of the (positive) doubles
  if (tid < 32) {
    int hmax = 0;
    for (int r = tid; r < R; r += 32) hmax = max(hmax, __double2hiint(Gpart[r * R + r]));
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    if (tid == 0)
      tiny_bits = __double_as_longlong(64.0 * 2.220446049250313e-16 * __hiloint2double(hmax, 0));
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  // column 0: pivot and L_j = S[j][0] / d_0 (warp 0)
  if (warp == 0) {
    double d = S[0];
    if (lane == 0 && !pivot_ok(d, tiny_bits)) {
      d = 1.0;
      S[0] = 1.0;
      fail = 1;
    }
    const double dinv = __shfl_sync(0xffffffffu, lane == 0 ? fast_rcp64(d) : 0.0, 0);
    for (int j = 1 + lane; j < R; j += 32) Lc[0][j] = S[j * R] * dinv;
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; ++k) {
    const int cb = k & 1;
    const int c1 = k + 1;   // the column finished this step
    if (warp == 0) {
      // column k+1: S[i][k+1] -= S[i][k] L_{k+1}, i >= k+1
      const double lk = Lc[cb][c1];
      // the second row of each lane only exists for R > 32 (a uniform branch:
      // a predicated-off FP64 instruction would still hold the pipe)
      double v[2];
      v[0] = c1 + lane < R ? fma(-S[(c1 + lane) * R + k], lk, S[(c1 + lane) * R + c1]) : 0.0;
      v[1] = 0.0;
      if (R > 32) {
        const int i = c1 + lane + 32;
        v[1] = i < R ? fma(-S[i * R + k], lk, S[i * R + c1]) : 0.0;
      }
      // every lane takes the pivot's reciprocal (one warp instruction either
      // way; no divergent branch and no shuffle after it)
      double d = __shfl_sync(0xffffffffu, v[0], 0);
      if (!pivot_ok(d, tiny_bits)) {
        d = 1.0;
        if (lane == 0) {
          v[0] = 1.0;
          fail = 1;
        }
      }
      const double dinv = fast_rcp64_newton(d);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && R <= 32) break;
        const int i = c1 + lane + 32 * h;
        if (i < R) {
          S[i * R + c1] = v[h];
          if (i > c1) Lc[cb ^ 1][i] = v[h] * dinv;
        }
      }
    } else if (warp != 4) {
      // the rest of the trailing block: i >= j >= k+2, on the warps that do not
      // share warp 0's SMSP (warp w runs on SMSP w % 4): its FP64 pipe stays free
      // for the serial chain
      const int m = R - 2 - k;
      const int na = m * (m + 1) / 2;
      const int tt = tid < 128 ? tid - 32 : tid - 64;   // 0 .. 191
      for (int a = tt; a < na; a += kSmallThreads - 64) {
        const int ij = tri[a];
        const int i = k + 2 + (ij >> 16), j = k + 2 + (ij & 0xffff);
        S[i * R + j] = fma(-S[i * R + k], Lc[cb][j], S[i * R + j]);
      }
    }
    __syncthreads();
  }
  __shared__ double dinv64[kMaxR];
  for (int r = tid; r < R; r += kSmallThreads) {
    rs[r] = rsqrt(S[r * R + r]);
    dinv64[r] = 1.0 / (S[r * R + r] * rs[r]);
  }
  __syncthreads();
  for (int o = tid; o < R * R; o += kSmallThreads) {
    const int r = o / R, c = o % R;
    const double cv = c <= r ? S[o] * rs[c] : 0.0;   // C[r][c]; sqrt(d_c) on the diagonal
    F[o] = cv;
    F[R * R + o] = cv * dinv64[r];       // forward-solve copy, rows scaled by 1 / C[r][r]
    F[2 * R * R + o] = cv * dinv64[c];   // backward-solve copy, columns scaled by 1 / C[c][c]
  }
  for (int r = tid; r < R; r += kSmallThreads) F[3 * R * R + r] = dinv64[r];
  if (tid == 0 && fail) {
    st->status = 4;   // TALS_ESINGULAR: Gram not numerically SPD (Remark 3)
    st->fail_stage = op == 1 ? 1 : 2;
    st->done = 1;
    if (has_cond) cudaGraphSetConditional(cond, 0u);
  }
}

cudaError_t launch_small(const double* Gpart, int nb, int R, int op, double* F, ModeState* st,
                         const double* norm_a2, unsigned long long cond, int has_cond,
                         cudaStream_t s, const double* GL, int f32) {
  if (R > kMaxR) return cudaErrorInvalidValue;
  small_kernel<<<1, kSmallThreads, 0, s>>>(Gpart, nb, R, op, F, st, norm_a2,
                                            (cudaGraphConditionalHandle)cond, has_cond, GL, f32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row-wise triangular solves: one warp per row, lane j owns columns j and j+32
// (R <= 64). The factor's rows (forward) and columns (backward) are scaled by
// the pivot reciprocals once per block; each solved entry is broadcast with a
// shuffle and every lane updates its own scaled running value, so the
// dependent chain per row is R steps of one shuffle and one FMA. WIDE (R > 32)
// adds the second column per lane; below that it is not issued at all (a
// predicated-off FP64 instruction still holds the FP64 pipe).
// ---------------------------------------------------------------------------
template <typename T, bool WIDE>
__global__ void row_solve_kernel(const double* __restrict__ In, long long I, int R,
                                 const double* __restrict__ F, int op, double* __restrict__ Out,
                                 T* __restrict__ OutT, double* __restrict__ Gpart,
                                 int rows_per_block, const ModeState* st, int gram_rounded) {
  const int done = st != nullptr ? st->done : 0;   // read in the same round trip as the factor
  extern __shared__ double sh[];
  double* Ff = sh;                                   // [R][R] F[j][c] / F[j][j]  (forward)
  double* Fb = Ff + (size_t)R * R;                   // [R][R] F[c][j] / F[j][j]  (backward)
  double* dinv = Fb + (size_t)R * R;                 // [R]
  double* Os = dinv + R;                             // [rows_per_block][R]
  // the factor block [C | Ff | Fb | dinv] written by the small kernel: Ff, Fb
  // and dinv are contiguous, staged as one array by asynchronous 8-byte copies,
  // all in flight at once (one round trip to L2 instead of one per batch of loads)
  {
    const double* src = F + (size_t)R * R;
    const int n = 2 * R * R + R;
    for (int o = threadIdx.x; o < n; o += blockDim.x)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(sh + o)), "l"(src + o));
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
  }
  __syncthreads();
  if (done) return;
  const long long row0 = (long long)blockIdx.x * rows_per_block;
  const int nrows = (int)min((long long)rows_per_block, I - row0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int j0 = lane, j1 = lane + 32;
  for (int lr = warp; lr < nrows; lr += nwarp) {
    const long long i = row0 + lr;
    // Lane j keeps e_j = (b_j - sum_{c<j, solved} F[j][c] x_c) / F[j][j], updated
    // as each x_c is broadcast; e_r is final when step r begins, so x_r = e_r and
    // each step's serial chain is one shuffle and one FMA.
    double e0 = j0 < R ? In[i * R + j0] * dinv[j0] : 0.0;
    double e1 = (WIDE && j1 < R) ? In[i * R + j1] * dinv[j1] : 0.0;
    double x0 = 0.0, x1 = 0.0;   // solved entries owned by this lane
    // forward: F x^T = b^T
    for (int r = 0; r < R; ++r) {
      const int owner = r & 31;
      const double v = __shfl_sync(0xffffffffu, (!WIDE || r < 32) ? e0 : e1, owner);
      if (lane == owner) {
        if (!WIDE || r < 32) x0 = v; else x1 = v;
      }
      if (j0 > r && j0 < R) e0 = fma(-Ff[j0 * R + r], v, e0);
      if constexpr (WIDE)
        if (j1 > r && j1 < R) e1 = fma(-Ff[j1 * R + r], v, e1);
    }
    if (op == 1) {
      // backward: F^T z^T = x^T, z_r = (x_r - sum_{c>r} F[c][r] z_c) / F[r][r]
      e0 = j0 < R ? x0 * dinv[j0] : 0.0;
      e1 = (WIDE && j1 < R) ? x1 * dinv[j1] : 0.0;
      for (int r = R - 1; r >= 0; --r) {
        const int owner = r & 31;
        const double v = __shfl_sync(0xffffffffu, (!WIDE || r < 32) ? e0 : e1, owner);
        if (lane == owner) {
          if (!WIDE || r < 32) x0 = v; else x1 = v;
        }
        if (j0 < r) e0 = fma(-Fb[r * R + j0], v, e0);
        if constexpr (WIDE)
          if (j1 < r && j1 < R) e1 = fma(-Fb[r * R + j1], v, e1);
      }
    }
    double* xs = Os + (size_t)lr * R;
    if (j0 < R) {
      Out[i * R + j0] = x0;
      double g = x0;
      if (OutT != nullptr) {
        const T q = (T)x0;
        OutT[i * R + j0] = q;
        if (gram_rounded) g = (double)q;   // the Gram below is of the stored basis
      }
      xs[j0] = g;
    }
    if (WIDE && j1 < R) {
      Out[i * R + j1] = x1;
      double g = x1;
      if (OutT != nullptr) {
        const T q = (T)x1;
        OutT[i * R + j1] = q;
        if (gram_rounded) g = (double)q;
      }
      xs[j1] = g;
    }
  }
  if (Gpart != nullptr) {
    __syncthreads();
    double* gp = Gpart + (size_t)blockIdx.x * R * R;
    for (int o = threadIdx.x; o < R * R; o += blockDim.x) {
      const int r = o / R, c = o % R;
      double g0 = 0.0, g1 = 0.0;
      int k = 0;
      for (; k + 1 < nrows; k += 2) {
        g0 = fma(Os[k * R + r], Os[k * R + c], g0);
        g1 = fma(Os[(k + 1) * R + r], Os[(k + 1) * R + c], g1);
      }
      if (k < nrows) g0 = fma(Os[k * R + r], Os[k * R + c], g0);
      gp[o] = g0 + g1;
    }
  }
}

cudaError_t launch_row_solve(int dtype, const double* In, long long I, int R, const double* F,
                             int op, double* Out, void* OutT, double* Gpart, const RowPlan& rp,
                             const ModeState* st, cudaStream_t s, int gram_rounded) {
  if (R > 64) return cudaErrorInvalidValue;
  const size_t sm = ((size_t)2 * R * R + R + (size_t)rp.rows_per_block * R) * sizeof(double);
  const int threads = 32 * std::max(1, std::min(8, rp.rows_per_block));
  auto go = [&](auto kern, auto* outT) {
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    kern<<<rp.blocks, threads, sm, s>>>(In, I, R, F, op, Out, outT, Gpart, rp.rows_per_block, st,
                                        gram_rounded);
    return cudaGetLastError();
  };
  if (dtype == 1)
    return R > 32 ? go(row_solve_kernel<float, true>, (float*)OutT)
                  : go(row_solve_kernel<float, false>, (float*)OutT);
  return R > 32 ? go(row_solve_kernel<double, true>, (double*)OutT)
                : go(row_solve_kernel<double, false>, (double*)OutT);
}

// ---------------------------------------------------------------------------
// Deterministic multi-CTA sum of Gram partials: Gfin[o] = sum_b Gpart[b][o].
// ---------------------------------------------------------------------------
constexpr int kGramSumThreads = 1024;   // 32 groups x 32 entries per block

__global__ void gram_sum_kernel(const double* __restrict__ Gpart, int nb, int RR,
                                double* __restrict__ Gfin, const ModeState* st, int write32) {
  if (st != nullptr && st->done) return;
  __shared__ double part[32][33];
  __shared__ double red[4][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (o < RR) {
    int b = grp;
    // four loads in flight, then their sum in order
    for (; b + 96 < nb; b += 128) {
      const double v0 = Gpart[(size_t)b * RR + o], v1 = Gpart[(size_t)(b + 32) * RR + o],
                   v2 = Gpart[(size_t)(b + 64) * RR + o], v3 = Gpart[(size_t)(b + 96) * RR + o];
      s += v0;
      s += v1;
      s += v2;
      s += v3;
    }
    for (; b < nb; b += 32) s += Gpart[(size_t)b * RR + o];
  }
  part[grp][lane] = s;
  __syncthreads();
  // fixed-order tree over the 32 groups: four sums of eight, then their sum
  if (grp < 4) {
    double t = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) t += part[grp * 8 + g][lane];
    red[grp][lane] = t;
  }
  __syncthreads();
  if (grp == 0 && o < RR) {
    const double t = (red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane]);
    Gfin[o] = t;
    if (write32) reinterpret_cast<float*>(Gfin + RR)[o] = (float)t;   // FP32 copy after the matrix
  }
}

cudaError_t launch_gram_sum(const double* Gpart, int nb, int R, double* Gfin,
                            const ModeState* st, cudaStream_t s, int write32) {
  const int RR = R * R;
  gram_sum_kernel<<<(RR + 31) / 32, kGramSumThreads, 0, s>>>(Gpart, nb, RR, Gfin, st, write32);
  return cudaGetLastError();
}

__global__ void state_init_kernel(ModeState* st, double eta, int max_sweeps, int resid,
                                  int bulk_max, int tc, int split_ok, int prod) {
  ModeState z = {};
  z.tc_resid = tc;
  z.split_ok = split_ok;
  z.prod = prod;
  z.d_cur = -1.0;
  z.d_prev = -1.0;
  z.eta = eta;
  z.max_sweeps = max_sweeps;
  z.resid = resid;
  z.bulk_mode = bulk_max > 0 ? 1 : 0;
  z.bulk_max = bulk_max;
  *st = z;
}

cudaError_t launch_state_init(ModeState* st, double eta, int max_sweeps, int resid, cudaStream_t s,
                              int bulk_max, int tc, int split_ok, int prod) {
  state_init_kernel<<<1, 1, 0, s>>>(st, eta, max_sweeps, resid, bulk_max, tc, split_ok, prod);
  return cudaGetLastError();
}

}  // namespace tals

namespace tals {

template <typename T>
__global__ void transpose_kernel(const T* __restrict__ In, long long rows, long long cols,
                                 T* __restrict__ Out) {
  __shared__ T tile[32][33];
  const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = In[r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) Out[c * rows + r] = tile[threadIdx.x][k];
  }
}

// Device-to-device copy by the SMs: leaves the decomposition's graph no
// copy-engine work before its final small downloads, so that no step in the
// middle of it can wait behind a host upload queued on a copy engine by
// another stream.
__global__ void copy_words_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                  size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

cudaError_t launch_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if ((((uintptr_t)dst | (uintptr_t)src | bytes) & 3) != 0) return cudaErrorInvalidValue;
  const size_t n = bytes / 4;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
  copy_words_kernel<<<blocks, 256, 0, s>>>((const uint32_t*)src, (uint32_t*)dst, n);
  return cudaGetLastError();
}

cudaError_t launch_transpose(int dtype, const void* In, long long rows, long long cols, void* Out,
                             cudaStream_t s) {
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
  if (dtype == 1)
    transpose_kernel<float><<<grid, block, 0, s>>>((const float*)In, rows, cols, (float*)Out);
  else
    transpose_kernel<double><<<grid, block, 0, s>>>((const double*)In, rows, cols, (double*)Out);
  return cudaGetLastError();
}

}  // namespace tals

namespace tals {

// ---------------------------------------------------------------------------
// Exact e_k^2 = ||B_(n) - Q W^T||^2 of a sweep from the tensor, the sweep's W
// (P x R x Q layout) and the FP32 basis Q it used: for modes whose rank is split
// across CTAs, so the pass cannot form the residual itself and ||B||^2 - ||W||^2
// would cancel. Generic views: columns in tiles of 32, W tile in shared memory,
// 8 row groups; exact squares in compensated FP32 per thread, FP64 per block.
// ---------------------------------------------------------------------------
__global__ void mode_residual_kernel(const float* __restrict__ X, long long P, long long I,
                                     long long Q, int R, const float* __restrict__ W,
                                     const float* __restrict__ L, double* __restrict__ part,
                                     const ModeState* st) {
  extern __shared__ float Wt[];   // [32][R + 1]
  __shared__ double red[32];
  const long long J = P * Q;
  const int tid = threadIdx.x, c = tid & 31, rg = tid >> 5, nrg = blockDim.x >> 5;
  float hi = 0.f, lo = 0.f;
  for (long long t = blockIdx.x; t * 32 < J; t += gridDim.x) {
    const long long j0 = t * 32;
    __syncthreads();
    for (int e = tid; e < 32 * R; e += blockDim.x) {
      const int cc = e & 31, r = e >> 5;
      const long long j = j0 + cc;
      float w = 0.f;
      if (j < J) {
        const long long p = j / Q, q = j - p * Q;
        w = W[(p * R + r) * Q + q];
      }
      Wt[cc * (R + 1) + r] = w;
    }
    __syncthreads();
    const long long j = j0 + c;
    if (j < J) {
      const long long p = j / Q, q = j - p * Q;
      const float* xcol = X + p * I * Q + q;
      const float* wc = Wt + c * (R + 1);
      for (long long i = rg; i < I; i += nrg) {
        float y = xcol[i * Q];
        const float* lrow = L + i * R;
        for (int r = 0; r < R; ++r) y = fmaf(-lrow[r], wc[r], y);
        const float pq = y * y, pe = fmaf(y, y, -pq);
        const float tq = hi + pq;
        lo += (hi >= pq ? (hi - tq) + pq : (pq - tq) + hi) + pe;
        hi = tq;
      }
    }
  }
  const double tot = block_sum((double)hi + (double)lo, red);
  if (tid == 0) part[blockIdx.x] = tot;
}

// Sum of the n residual partials into the mode state: per sweep into sW (the
// TEST kernel's e^2 for modes that measure the residual), unless the mode is done.
__global__ void mode_residual_finish(const double* __restrict__ part, long long n, ModeState* st) {
  if (st->done) return;
  __shared__ double red[32];
  double v = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  const double tot = block_sum(v, red);
  if (threadIdx.x == 0) st->sW = tot;
}

// st->sw_tc = sum of n partials (unless the mode is done): ||W||^2 of the W the
// split-precision W pass stored.
__global__ void state_sum_kernel(const double* __restrict__ part, int n, ModeState* st) {
  if (st->done) return;
  __shared__ double red[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  const double tot = block_sum(v, red);
  if (threadIdx.x == 0) st->sw_tc = tot;
}

cudaError_t launch_state_sum(const double* part, int n, ModeState* st, cudaStream_t s) {
  state_sum_kernel<<<1, 256, 0, s>>>(part, n, st);
  return cudaGetLastError();
}

cudaError_t launch_mode_residual(const float* X, const ModeView& v, int R, const float* W,
                                 const float* L, double* part, long long cap, ModeState* st,
                                 cudaStream_t s) {
  // the tiled GEMM form where the view has long rows (Q >= 64)
  const long long ng = mode_resid_gemm_parts(W, v.P, R, v.Q, L, R, 1, v.I, X);
  if (ng > 0 && ng <= cap) {
    cudaError_t e = launch_mode_resid_gemm(W, v.P, R, v.Q, L, R, 1, v.I, X, part, s);
    if (e != cudaSuccess) return e;
    mode_residual_finish<<<1, 256, 0, s>>>(part, ng, st);
    return cudaGetLastError();
  }
  const long long tiles = (v.J() + 31) / 32;
  const int grid = (int)std::max<long long>(1, std::min<long long>(std::min<long long>(cap, 1024), tiles));
  const size_t sm = (size_t)32 * (R + 1) * sizeof(float);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(mode_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  mode_residual_kernel<<<grid, 256, sm, s>>>(X, v.P, v.I, v.Q, R, W, L, part, st);
  mode_residual_finish<<<1, 256, 0, s>>>(part, grid, st);
  return cudaGetLastError();
}

}  // namespace tals
