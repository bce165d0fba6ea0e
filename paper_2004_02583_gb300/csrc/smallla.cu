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
template <typename T>
__global__ void reduce_rows_kernel(const T* __restrict__ Ypart, int gx, long long I, int R,
                                   double* __restrict__ Y64, int gram_mode,
                                   const double* __restrict__ L64, double* __restrict__ Gpart,
                                   int rows_per_block, const double* __restrict__ spart, int nsp,
                                   int which, ModeState* st, double* norm_a2, T* YT) {
  if (st != nullptr && st->done) return;
  extern __shared__ double sh[];
  double* Ys = sh;                                   // [rows_per_block][R]
  double* As = sh + (size_t)rows_per_block * R;      // [rows_per_block][R] (L rows for CROSS)
  const long long row0 = (long long)blockIdx.x * rows_per_block;
  const int nrows = (int)min((long long)rows_per_block, I - row0);
  const int nent = nrows * R;
  for (int e = threadIdx.x; e < nent; e += blockDim.x) {
    const long long i = row0 + e / R;
    const int r = e % R;
    double s = 0.0;
    for (int b = 0; b < gx; ++b) s += (double)Ypart[((size_t)b * I + i) * R + r];
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
  const size_t sm = (size_t)2 * rp.rows_per_block * R * sizeof(double);
  if (dtype == 1)
    reduce_rows_kernel<float><<<rp.blocks, 256, sm, s>>>((const float*)Ypart, gx, I, R, Y64,
                                                         gram_mode, L64, Gpart,
                                                         rp.rows_per_block, spart, nsp, which,
                                                         st, norm_a2, (float*)YT);
  else
    reduce_rows_kernel<double><<<rp.blocks, 256, sm, s>>>((const double*)Ypart, gx, I, R, Y64,
                                                          gram_mode, L64, Gpart,
                                                          rp.rows_per_block, spart, nsp, which,
                                                          st, norm_a2, (double*)YT);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-CTA kernel: Gram sum, Eq. 5.01 stop rule, Cholesky.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;

__global__ void __launch_bounds__(kSmallThreads) small_kernel(const double* __restrict__ Gpart,
                                                              int nb, int R, int op,
                                                              double* __restrict__ F,
                                                              ModeState* st,
                                                              const double* norm_a2,
                                                              cudaGraphConditionalHandle cond,
                                                              int has_cond,
                                                              const double* __restrict__ GL) {
  if (st->done) {
    if (has_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  extern __shared__ double G[];   // [R][R]
  __shared__ int fail;
  const int tid = threadIdx.x;

  if (op == 1 || op == 2) {
    // Eq. 5.01 on e_k^2 = ||B_(n)||^2 - ||W||^2 (W = B^T Q_k is the LS optimum for Q_k),
    // plus tr((Q'^T Q' - I) X), the first-order term of the projector onto the
    // rounded basis Q' actually used, X = Q^T B B^T Q' (the cross Gram below)
    __shared__ int stop;
    __shared__ double red[32];
    double c = 0.0;
    if (GL != nullptr)
      for (int o = tid; o < R * R; o += kSmallThreads) {
        const int r = o / R, q = o % R;
        c += (GL[o] - (r == q ? 1.0 : 0.0)) * Gpart[o];
      }
    const double corr = block_sum(c, red);
    if (tid == 0) {
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
        }
        st->bulk += 1;
      } else {
        if (st->kf >= 1 && fabs(st->e_prev - e) <= st->eta * norm_a) {
          s = 1;
          st->converged = 1;
        }
        st->kf += 1;
      }
      if (k + 1 >= st->max_sweeps) s = 1;
      st->e_prev = e;
      st->e_cur = e;
      st->k = k + 1;
      if (s) st->done = 1;
      stop = s;
    }
    __syncthreads();
    if (stop) {
      if (has_cond && tid == 0) cudaGraphSetConditional(cond, 0u);
      return;
    }
  }

  for (int o = tid; o < R * R; o += kSmallThreads) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += Gpart[(size_t)b * R * R + o];   // nb = 1 after gram_sum
    G[o] = s;
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  // symmetrise (the cross Gram Q^T B B^T Q is symmetric in exact arithmetic)
  for (int o = tid; o < R * R; o += kSmallThreads) {
    const int r = o / R, c = o % R;
    if (r > c) {
      const double v = 0.5 * (G[r * R + c] + G[c * R + r]);
      G[r * R + c] = v;
      G[c * R + r] = v;
    }
  }
  __syncthreads();
  double maxd = 0.0;
  for (int r = 0; r < R; ++r) maxd = fmax(maxd, G[r * R + r]);
  const double tiny = 64.0 * 2.220446049250313e-16 * maxd;
  // right-looking Cholesky, lower factor in place
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {
      const double d = G[k * R + k];
      if (!(d > tiny)) {
        fail = 1;
        G[k * R + k] = 1.0;
      } else {
        G[k * R + k] = sqrt(d);
      }
    }
    __syncthreads();
    const double rk = 1.0 / G[k * R + k];
    for (int i = k + 1 + tid; i < R; i += kSmallThreads) G[i * R + k] *= rk;
    __syncthreads();
    const int m = R - k - 1;
    for (int o = tid; o < m * m; o += kSmallThreads) {
      const int i = k + 1 + o / m, j = k + 1 + o % m;
      if (j <= i) G[i * R + j] -= G[i * R + k] * G[j * R + k];
    }
    __syncthreads();
  }
  for (int o = tid; o < R * R; o += kSmallThreads) {
    const int r = o / R, c = o % R;
    F[o] = (c <= r) ? G[o] : 0.0;
  }
  if (tid == 0 && fail) {
    st->status = 4;   // TALS_ESINGULAR: Gram not numerically SPD (Remark 3)
    st->fail_stage = op == 1 ? 1 : 2;
    st->done = 1;
    if (has_cond) cudaGraphSetConditional(cond, 0u);
  }
}

cudaError_t launch_small(const double* Gpart, int nb, int R, int op, double* F, ModeState* st,
                         const double* norm_a2, unsigned long long cond, int has_cond,
                         cudaStream_t s, const double* GL) {
  const size_t sm = (size_t)R * R * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
  }
  small_kernel<<<1, kSmallThreads, sm, s>>>(Gpart, nb, R, op, F, st, norm_a2,
                                            (cudaGraphConditionalHandle)cond, has_cond, GL);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row-wise triangular solves: one warp per row, lane j owns columns j and j+32
// (R <= 64). Each solved entry is broadcast with a shuffle and every lane
// updates its own running sums, so the dependent chain per row is R short steps
// (no per-thread R^2 chain). Pivot reciprocals are taken once per block.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void row_solve_kernel(const double* __restrict__ In, long long I, int R,
                                 const double* __restrict__ F, int op, double* __restrict__ Out,
                                 T* __restrict__ OutT, double* __restrict__ Gpart,
                                 int rows_per_block, const ModeState* st, int gram_rounded) {
  if (st != nullptr && st->done) return;
  extern __shared__ double sh[];
  double* Fs = sh;                                   // [R][R]
  double* dinv = sh + (size_t)R * R;                 // [R]
  double* Os = dinv + R;                             // [rows_per_block][R]
  for (int o = threadIdx.x; o < R * R; o += blockDim.x) Fs[o] = F[o];
  for (int r = threadIdx.x; r < R; r += blockDim.x) dinv[r] = 1.0 / F[r * R + r];
  __syncthreads();
  const long long row0 = (long long)blockIdx.x * rows_per_block;
  const int nrows = (int)min((long long)rows_per_block, I - row0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int j0 = lane, j1 = lane + 32;
  for (int lr = warp; lr < nrows; lr += nwarp) {
    const long long i = row0 + lr;
    double b0 = j0 < R ? In[i * R + j0] : 0.0, b1 = j1 < R ? In[i * R + j1] : 0.0;
    double a0 = 0.0, a1 = 0.0;   // running sums of the solve
    double x0 = 0.0, x1 = 0.0;   // solved entries owned by this lane
    // forward: F x^T = b^T, x_r = (b_r - sum_{c<r} F[r][c] x_c) / F[r][r]
    for (int r = 0; r < R; ++r) {
      const int owner = r & 31;
      double v = 0.0;
      if (lane == owner) v = ((r < 32 ? b0 : b1) - (r < 32 ? a0 : a1)) * dinv[r];
      v = __shfl_sync(0xffffffffu, v, owner);
      if (lane == owner) {
        if (r < 32) x0 = v; else x1 = v;
      }
      if (j0 > r && j0 < R) a0 = fma(Fs[j0 * R + r], v, a0);
      if (j1 > r && j1 < R) a1 = fma(Fs[j1 * R + r], v, a1);
    }
    if (op == 1) {
      // backward: F^T z^T = x^T, z_r = (x_r - sum_{c>r} F[c][r] z_c) / F[r][r]
      b0 = x0;
      b1 = x1;
      a0 = 0.0;
      a1 = 0.0;
      for (int r = R - 1; r >= 0; --r) {
        const int owner = r & 31;
        double v = 0.0;
        if (lane == owner) v = ((r < 32 ? b0 : b1) - (r < 32 ? a0 : a1)) * dinv[r];
        v = __shfl_sync(0xffffffffu, v, owner);
        if (lane == owner) {
          if (r < 32) x0 = v; else x1 = v;
        }
        if (j0 < r) a0 = fma(Fs[r * R + j0], v, a0);
        if (j1 < r && j1 < R) a1 = fma(Fs[r * R + j1], v, a1);
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
    if (j1 < R) {
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
  const size_t sm = ((size_t)R * R + R + (size_t)rp.rows_per_block * R) * sizeof(double);
  const int threads = 32 * std::max(1, std::min(8, rp.rows_per_block));
  if (dtype == 1) {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(row_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    row_solve_kernel<float><<<rp.blocks, threads, sm, s>>>(In, I, R, F, op, Out, (float*)OutT,
                                                           Gpart, rp.rows_per_block, st,
                                                           gram_rounded);
  } else {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(row_solve_kernel<double>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    row_solve_kernel<double><<<rp.blocks, threads, sm, s>>>(In, I, R, F, op, Out, (double*)OutT,
                                                            Gpart, rp.rows_per_block, st,
                                                            gram_rounded);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic multi-CTA sum of Gram partials: Gfin[o] = sum_b Gpart[b][o].
// ---------------------------------------------------------------------------
__global__ void gram_sum_kernel(const double* __restrict__ Gpart, int nb, int RR,
                                double* __restrict__ Gfin, const ModeState* st) {
  if (st != nullptr && st->done) return;
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;   // 8 groups x 32 entries
  const int o = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (o < RR)
    for (int b = grp; b < nb; b += 8) s += Gpart[(size_t)b * RR + o];
  part[grp][lane] = s;
  __syncthreads();
  if (grp == 0 && o < RR) {
    double t = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) t += part[g][lane];
    Gfin[o] = t;
  }
}

cudaError_t launch_gram_sum(const double* Gpart, int nb, int R, double* Gfin,
                            const ModeState* st, cudaStream_t s) {
  const int RR = R * R;
  gram_sum_kernel<<<(RR + 31) / 32, 256, 0, s>>>(Gpart, nb, RR, Gfin, st);
  return cudaGetLastError();
}

__global__ void state_init_kernel(ModeState* st, double eta, int max_sweeps, int resid,
                                  int bulk_max) {
  ModeState z = {};
  z.eta = eta;
  z.max_sweeps = max_sweeps;
  z.resid = resid;
  z.bulk_mode = bulk_max > 0 ? 1 : 0;
  z.bulk_max = bulk_max;
  *st = z;
}

cudaError_t launch_state_init(ModeState* st, double eta, int max_sweeps, int resid, cudaStream_t s,
                              int bulk_max) {
  state_init_kernel<<<1, 1, 0, s>>>(st, eta, max_sweeps, resid, bulk_max);
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
