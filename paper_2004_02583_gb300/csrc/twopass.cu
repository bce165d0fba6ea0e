// Two-pass ALS sweep (Alg. 3) for mode views whose size I_n is above what the
// fused pass can hold: the fused pass keeps an I_n x (columns per tile) slab of
// B_(n) in shared memory, which caps I_n near 1920 (FP32) and 852 (FP64). The
// long modes of the paper's synthetic workloads (the third mode K = 100 I of the
// CP model, Sec. 6.1.1; I_1 up to 5000 in the Tucker model, Sec. 6.1.2) go through
// two reads of the tensor per sweep instead, each a tiled product that streams
// B once:
//   W = B_(n)^T Q_k, written as the tensor B x_n Q_k^T (P x R x Q layout) -- the
//       R-update of Alg. 3 for the orthonormal Q_k -- by the mode-product GEMM;
//   Y = B_(n) W, by the split-K row-tile kernel of adjoint.cu where the view has
//       16-column rows (else the any-view factor adjoint), column splits of at most
//       2048 columns added in FP64 in order;
//   ||W||^2 from W, or (FP32 tensors up to a quarter of the input) the explicit
//   residual ||B - Q_k W^T||^2 as e_k^2.
// The initial guess of Sec. 4 is Y_0 = B_(n) S with S written out in the same
// P x R x Q layout and the same counter-based entries as the fused pass draws.
// Everything after the products (the reduction, the FP64 Grams, CholeskyQR, the
// Eq. 5.01 test) is the fused path's own chain.
#include <algorithm>

#include "internal.h"

namespace tals {

namespace {

constexpr int kSqThreads = 256;

// ||x||^2 partials in FP64 over a fixed grid of kSumsqParts blocks.
template <typename T>
__global__ void __launch_bounds__(kSqThreads) sumsq_part_kernel(const T* __restrict__ x, size_t n,
                                                                double* __restrict__ part) {
  __shared__ double red[kSqThreads];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * kSqThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kSqThreads) {
    const double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kSqThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kSqThreads) sum_parts_kernel(const double* __restrict__ part, int nb,
                                                               double* __restrict__ out) {
  __shared__ double red[kSqThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += kSqThreads) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kSqThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// S[p, r, q] = entry (j = p Q + q, r) of the Sec. 4 sketch.
template <typename T>
__global__ void __launch_bounds__(256) sketch_prq_kernel(T* __restrict__ S, long long P, long long Q, int R,
                                                         uint64_t state) {
  const long long tot = P * R * Q;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long q = e % Q;
    const long long pr = e / Q;
    const int r = (int)(pr % R);
    const long long p = pr / R;
    S[e] = (T)sketch_entry(state, (uint64_t)(p * Q + q), R, r);
  }
}

// out[e] = sum over s of part[s * n + e], in FP64, in order.
template <typename T>
__global__ void __launch_bounds__(256) sum_parts_f64_kernel(const T* __restrict__ part, int S, long long n,
                                                            T* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += (double)part[(long long)s * n + e];
    out[e] = (T)v;
  }
}

unsigned elem_grid(long long n, int sms) {
  const long long want = (n + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(want, (long long)std::max(sms, 1) * 16));
}

}  // namespace

cudaError_t launch_sumsq_parts(int dtype, const void* x, size_t n, double* part, cudaStream_t s) {
  if (dtype == TALS_F32)
    sumsq_part_kernel<float><<<kSumsqParts, kSqThreads, 0, s>>>((const float*)x, n, part);
  else
    sumsq_part_kernel<double><<<kSumsqParts, kSqThreads, 0, s>>>((const double*)x, n, part);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(int dtype, const void* x, size_t n, double* part, double* out, cudaStream_t s) {
  cudaError_t e = launch_sumsq_parts(dtype, x, n, part, s);
  if (e != cudaSuccess) return e;
  sum_parts_kernel<<<1, kSqThreads, 0, s>>>(part, kSumsqParts, out);
  return cudaGetLastError();
}

cudaError_t launch_sketch_prq(int dtype, void* S, const ModeView& v, int R, uint64_t state, int sms,
                              cudaStream_t s) {
  const unsigned g = elem_grid(v.P * R * v.Q, sms);
  if (dtype == TALS_F32)
    sketch_prq_kernel<float><<<g, 256, 0, s>>>((float*)S, v.P, v.Q, R, state);
  else
    sketch_prq_kernel<double><<<g, 256, 0, s>>>((double*)S, v.P, v.Q, R, state);
  return cudaGetLastError();
}

cudaError_t launch_mode_project_any(int dtype, const void* X, const ModeView& v, const void* U, int R, void* out,
                                    cudaStream_t s) {
  // out[p, a, q] = sum_i U[i, a] X[p, i, q]: M = U^T, element (a, i) at U[i * R + a]
  if (dtype == TALS_F32) {
    cudaError_t e = launch_mode_gemm((const float*)X, v.P, v.I, v.Q, (const float*)U, 1, R, R, (float*)out, s);
    if (e != cudaErrorNotSupported) return e;
    return launch_mode_gemm_any((const float*)X, v.P, v.I, v.Q, (const float*)U, 1, R, R, (float*)out, s);
  }
  return launch_mode_gemm_any((const double*)X, v.P, v.I, v.Q, (const double*)U, 1, R, R, (double*)out, s);
}

int twopass_splits(const ModeView& v, int R, int sms) {
  const long long by_len = (v.J() + 2047) / 2048;   // at most 2048 columns per FP32 sum
  long long S = std::max<long long>(factor_adjoint_splits(v.P, v.I, v.Q, R, sms), by_len);
  return (int)std::min<long long>(S, 4096);
}

cudaError_t launch_mode_adjoint_any(int dtype, const void* X, const ModeView& v, const void* W, int R, int S,
                                    void* part, void* Y, cudaStream_t s) {
  cudaError_t e;
  const long long n = v.I * R;
  const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096));
  if (dtype == TALS_F32) {
    // the split-K register-tiled kernel where the view allows it (rows of 16
    // columns: Q % 16 == 0, R <= 64, aligned), else the any-view tiles
    if (adjoint_rows_ok(v, R, X, W))
      e = launch_adjoint_rows((const float*)X, v, (const float*)W, R, S, (float*)part, nullptr, nullptr, s);
    else
      e = launch_factor_adjoint_parts((const float*)X, v.P, v.I, v.Q, (const float*)W, R, S, (float*)part, s);
    if (e != cudaSuccess) return e;
    sum_parts_f64_kernel<float><<<g, 256, 0, s>>>((const float*)part, S, n, (float*)Y);
  } else {
    e = launch_factor_adjoint_parts((const double*)X, v.P, v.I, v.Q, (const double*)W, R, S, (double*)part, s);
    if (e != cudaSuccess) return e;
    sum_parts_f64_kernel<double><<<g, 256, 0, s>>>((const double*)part, S, n, (double*)Y);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host side: the mode's init and sweep in the two-pass form. Y goes to Ypart as
// one partial (gx = 1), the factor adjoint's column-split partials right after it.
// ---------------------------------------------------------------------------
#define TALS_CK(x) \
  if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x);

tals_status twopass_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const size_t ir = (size_t)j.v.I * R;
  cudaError_t e;
  TALS_CK(launch_sketch_prq(c->dtype, j.Wt, j.v, R, sketch_state(c->opts.seed, j.n), c->sms, s));
  TALS_CK(launch_mode_adjoint_any(c->dtype, j.X, j.v, j.Wt, R, j.splits, (char*)c->Ypart + ir * c->esz, c->Ypart,
                                  s));
  TALS_CK(launch_sumsq_parts(c->dtype, j.X, (size_t)(j.v.P * j.v.I * j.v.Q), c->spart, s));
  return mode_init_tail(c, j, set_norm_a, 1, c->spart, kSumsqParts);
}

tals_status twopass_sweep_launch(tals_ctx* c, const ModeJob& j) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const size_t ir = (size_t)j.v.I * R;
  cudaError_t e;
  // R-update: W = B_(n)^T Q_k as B x_n Q_k^T, then ||W||^2 and Y = B_(n) W
  TALS_CK(launch_mode_project_any(c->dtype, j.X, j.v, c->Lt, R, j.Wt, s));
  TALS_CK(launch_sumsq_parts(c->dtype, j.Wt, (size_t)(j.v.P * j.v.Q) * R, c->spart, s));
  TALS_CK(launch_mode_adjoint_any(c->dtype, j.X, j.v, j.Wt, R, j.splits, (char*)c->Ypart + ir * c->esz, c->Ypart,
                                  s));
  return mode_sweep_tail(c, j, 1, kSumsqParts, 1);
}

// out = X x_n U^T by the fused pass in projection mode where it applies, else by
// the tiled mode product; *nsp partial sums of ||out||^2 are left in c->spart.
tals_status project_mode(tals_ctx* c, const void* X, const ModeView& v, int R, const void* U, void* out, int* nsp) {
  const PassConfig pc = pass_config(c->dtype, v, R, c->sms);
  cudaError_t e;
  if (pc.ok && (size_t)pc.grid_x * pc.grid_y <= c->spart_n) {
    TALS_CK(launch_pass(c->dtype, pc, PASS_PROJECT, X, v, R, U, nullptr, c->spart, out, 0, nullptr, 0, c->stream));
    *nsp = pc.grid_x * pc.grid_y;
    return TALS_OK;
  }
  if (c->spart_n < (size_t)kSumsqParts) return fail(TALS_ENOTSUP, "projection: workspace too small");
  TALS_CK(launch_mode_project_any(c->dtype, X, v, U, R, out, c->stream));
  TALS_CK(launch_sumsq_parts(c->dtype, out, (size_t)(v.P * v.Q) * R, c->spart, c->stream));
  *nsp = kSumsqParts;
  return TALS_OK;
}

#undef TALS_CK

}  // namespace tals
