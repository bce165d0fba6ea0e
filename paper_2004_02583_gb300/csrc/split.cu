// The split sweep: a sweep whose stop test (Eq. 5.01) is likely to fire forms W
// alone first and Y only if the loop goes on.
//
// The fused pass forms W = B_(n)^T Q_k and Y = B_(n) W from one read of B; on the
// sweep where the test stops the mode only W (the st-HOSVD truncation, Alg. 5)
// and ||W||^2 (for e_k) are used. A sweep the TEST kernel predicts to be the last
// (als_predict_split) therefore runs: the fused pass exits at once; the
// register-tiled mode product writes W = B x_n Q_k^T; wstats_kernel forms, per
// CTA, ||W||^2 (compensated FP32, FP64 across threads) and w^T (Q'^T Q' - I) w
// summed over W's columns -- tr((Q'^T Q' - I) W^T W), the rounded-basis term of
// e_k, W^T W being the cross Gram X of the fused path for Q = Q'; split_test_kernel
// adds the partials in a fixed order and takes the same Eq. 5.01 step; the
// factor-adjoint pass forms Y = B_(n) W only if the mode is not done. Every kernel
// reads the mode state and exits at once when the sweep is not split (or is done),
// so one captured sweep serves both forms.
#include <algorithm>

#include "internal.h"

namespace tals {

namespace {

constexpr int kWsThreads = 256;

// Neumaier-compensated FP32 sum of exact squares (x^2 = p + e by FMA).
__device__ __forceinline__ void add_sq(float x, float& s, float& c) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  const float t = s + p;
  c += (fabsf(s) >= fabsf(p)) ? (s - t) + p : (p - t) + s;
  c += e;
  s = t;
}

// Per CTA: part[2 b] = sum of ||w||^2 and part[2 b + 1] = sum of w^T D w over the
// CTA's columns j = p Q + q of W (P x R x Q), D = GL - I (the stored basis' Gram
// minus the identity; RP = R rounded up to 16, zeros beyond R). One thread per
// column: the column in registers for the inner products with D's rows (read as
// float4 broadcasts) and in the thread's own shared-memory slot for the outer sum.
template <int RP>
__global__ void __launch_bounds__(kWsThreads) wstats_kernel(const float* __restrict__ W, long long P, int R,
                                                            long long Q, const double* __restrict__ GL,
                                                            const ModeState* __restrict__ st,
                                                            double* __restrict__ part) {
  if (!st->split || st->done) return;
  extern __shared__ __align__(16) float ws_dyn[];
  float* D = ws_dyn;                   // [RP][RP]
  float* Vs = ws_dyn + RP * RP;        // each thread's column, [a][thread]
  __shared__ double red[2][kWsThreads / 32];
  for (int e = threadIdx.x; e < RP * RP; e += kWsThreads) {
    const int a = e / RP, b = e % RP;
    D[e] = (a < R && b < R) ? (float)(GL[a * R + b] - (a == b ? 1.0 : 0.0)) : 0.f;
  }
  __syncthreads();
  float s = 0.f, c = 0.f, qsum = 0.f;
  const long long J = P * Q;
  for (long long j = (long long)blockIdx.x * kWsThreads + threadIdx.x; j < J;
       j += (long long)gridDim.x * kWsThreads) {
    const long long p = j / Q, q = j - p * Q;
    const float* w = W + p * R * Q + q;
    float v[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      v[r] = r < R ? w[(long long)r * Q] : 0.f;
      Vs[r * kWsThreads + threadIdx.x] = v[r];
    }
#pragma unroll
    for (int r = 0; r < RP; ++r) add_sq(v[r], s, c);
    float qa = 0.f;
#pragma unroll 1
    for (int a = 0; a < R; ++a) {
      float t = 0.f;
#pragma unroll
      for (int b = 0; b < RP; b += 4) {
        const float4 d = *reinterpret_cast<const float4*>(&D[a * RP + b]);
        t = fmaf(d.x, v[b], t);
        t = fmaf(d.y, v[b + 1], t);
        t = fmaf(d.z, v[b + 2], t);
        t = fmaf(d.w, v[b + 3], t);
      }
      qa = fmaf(Vs[a * kWsThreads + threadIdx.x], t, qa);
    }
    qsum += qa;
  }
  double ws = (double)s + (double)c, wq = (double)qsum;
  for (int o = 16; o > 0; o >>= 1) {
    ws += __shfl_down_sync(0xffffffffu, ws, o);
    wq += __shfl_down_sync(0xffffffffu, wq, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = ws;
    red[1][warp] = wq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int k = 0; k < kWsThreads / 32; ++k) {
      x += red[0][k];
      y += red[1][k];
    }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

// The split sweep's Eq. 5.01 step: e_k^2 = ||B||^2 - ||W||^2 + tr((Q'^T Q' - I) W^T W).
__global__ void __launch_bounds__(256) split_test_kernel(const double* __restrict__ part, int nb, ModeState* st,
                                                         const double* __restrict__ norm_a2,
                                                         unsigned long long cond, int has_cond) {
  if (!st->split || st->done) return;
  __shared__ double r0[256], r1[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r0[threadIdx.x] += r0[threadIdx.x + w];
      r1[threadIdx.x] += r1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->nsplit += 1;
    st->sW = r0[0];
    st->corr = r1[0];
    const double e2 = st->normM2 - r0[0] + r1[0];
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    if (als_stop_step(st, e, sqrt(*norm_a2)) && has_cond)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

template <int RP>
cudaError_t run_wstats(const float* W, const ModeView& v, int R, const double* GL, const ModeState* st,
                       double* part, int nb, cudaStream_t s) {
  constexpr int smem = (RP * RP + RP * kWsThreads) * (int)sizeof(float);
  // the attribute belongs to the current device: set on every call
  cudaError_t e = cudaFuncSetAttribute(wstats_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  wstats_kernel<RP><<<nb, kWsThreads, smem, s>>>(W, v.P, R, v.Q, GL, st, part);
  return cudaGetLastError();
}

}  // namespace

int split_stat_blocks(const ModeView& v, int sms) {
  const long long want = (v.J() + kWsThreads - 1) / kWsThreads;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * 2));
}

cudaError_t launch_split_stats(const float* W, const ModeView& v, int R, const double* GL, const ModeState* st,
                               double* part, int nb, cudaStream_t s) {
  if (R < 1 || R > 64) return cudaErrorInvalidValue;
  if (R <= 16) return run_wstats<16>(W, v, R, GL, st, part, nb, s);
  if (R <= 32) return run_wstats<32>(W, v, R, GL, st, part, nb, s);
  if (R <= 48) return run_wstats<48>(W, v, R, GL, st, part, nb, s);
  return run_wstats<64>(W, v, R, GL, st, part, nb, s);
}

cudaError_t launch_split_test(const double* part, int nb, ModeState* st, const double* norm_a2,
                              unsigned long long cond, int has_cond, cudaStream_t s) {
  split_test_kernel<<<1, 256, 0, s>>>(part, nb, st, norm_a2, cond, has_cond);
  return cudaGetLastError();
}

}  // namespace tals
