// Shared device-side definitions of the tals library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tals {

constexpr int kThreads = 256;       // threads per CTA of the pass and row kernels
constexpr int kTileCols = 16;       // unfolding columns per tile of the pass kernel

// Per-mode ALS state, resident in device memory. Written only by the single-CTA
// small kernels, read by every kernel of the sweep to skip work once the stop
// rule has fired.
struct ModeState {
  double normM2;      // ||B_(n)||^2, from the initial pass
  double normA;       // ||A||_F of the original input (reading of Eq. 5.01's norm)
  double eta;         // stop tolerance (negative: never stop early)
  double e_prev;      // e_{k-1}
  double e_cur;       // e_k
  double sW;          // ||W||^2 = ||Q_k^T B_(n)||^2 of the last sweep
  int k;              // completed R-updates
  int max_sweeps;
  int done;           // stop rule fired or sweep budget exhausted
  int converged;      // stop rule fired
  int status;         // 0 ok, else a tals_status code
  int fail_stage;     // where a factorisation failed (diagnostics)
  int bulk;           // sweeps run on the bulk (BF16) path
  int resid;          // sW holds ||B - Q W^T||^2 (the error itself) instead of ||W||^2
  double corr;        // tr((Q'^T Q' - I) X): first-order term for the rounded basis Q'
  int bulk_mode;      // 1 while the mixed-precision bulk (BF16) sweeps run
  int kf;             // sweeps of the current (final-precision) phase
  int bulk_max;       // at most this many bulk sweeps
  int tc_resid;       // products on the tensor cores: e_k from the explicit residual, and
                      // sw_tc holds ||W||^2 of the stored W
  double sw_prev;     // ||W||^2 of the previous bulk sweep
  double sw_tc;       // tensor-core modes: ||W||^2 of the W last written
  int split_ok;       // the mode may run a sweep split (W alone, the test, then Y if needed)
  int split;          // this sweep runs split (set for the next sweep by the TEST kernel)
  double d_cur;       // |e_{k-1} - e_k| of the last test (negative: no comparison yet)
  double d_prev;      // the one before
  int nsplit;         // sweeps that ran split
  int prod;           // FP32 sweeps as two products (mode product W, split-K Y)
};

// The Eq. 5.01 step of an FP32-phase sweep, given e_k (thread 0 of a single-CTA
// kernel): the test on |e_{k-1} - e_k| from the second sweep of the phase on, the
// sweep budget, and the state's counters. Returns 1 when the mode is done.
__device__ inline int als_stop_step(ModeState* st, double e, double norm_a) {
  int s = 0;
  st->d_cur = -1.0;
  if (st->kf >= 1) {
    const double d = fabs(st->e_prev - e);
    st->d_cur = d;
    if (d <= st->eta * norm_a) {
      s = 1;
      st->converged = 1;
    }
  }
  st->kf += 1;
  if (st->k + 1 >= st->max_sweeps) s = 1;
  st->e_prev = e;
  st->e_cur = e;
  st->k += 1;
  if (s) st->done = 1;
  return s;
}

// Whether the next sweep runs split (thread 0, after a test that did not stop):
// the mixed path's second FP32 sweep (the first one the test can stop), a sweep
// whose predicted change rho |e_{k-1} - e_k| (rho = the last two changes' ratio)
// is within the tolerance, or the budget's last sweep.
__device__ inline void als_predict_split(ModeState* st, double norm_a) {
  int nxt = 0;
  if (st->split_ok) {
    if (st->bulk > 0 && st->kf == 1) nxt = 1;
    if (st->d_cur >= 0.0 && st->d_prev > 0.0 && st->d_cur * st->d_cur <= st->eta * norm_a * st->d_prev) nxt = 1;
    if (st->k + 1 >= st->max_sweeps) nxt = 1;
  }
  st->d_prev = st->d_cur;
  st->split = nxt;
}

// splitmix64 output number c of the stream seeded with `state`:
// mix(state + (c + 1) * 0x9E3779B97F4A7C15) (Steele, Lea, Flood 2014; Vigna).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t state, uint64_t c) {
  uint64_t z = state + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry (j, r) of the initial sketch S: top 24 bits of output j*R + r, scaled
// to [0, 1) (exactly representable in FP32 and FP64).
__device__ __forceinline__ float sketch_entry(uint64_t state, uint64_t j, int R, int r) {
  uint64_t z = splitmix64_at(state, j * (uint64_t)R + (uint64_t)r);
  return (float)(uint32_t)(z >> 40) * (1.0f / 16777216.0f);
}

// d > tiny for a pivot, on the bit patterns (both non-negative; NaN fails):
// integer compares keep FP64 instructions off the serial chain.
__device__ __forceinline__ bool pivot_ok(double d, long long tiny_bits) {
  const long long b = __double_as_longlong(d);
  return b > tiny_bits && ((b >> 52) & 0x7ff) != 0x7ff;
}

// 1/d for a positive normal double: FP32 reciprocal of the leading bits, then
// x = x0 (1 + e + e^2) with e = 1 - d x0 (Newton's method continued to third
// order), ~2^-66 relative before the last rounding. Three dependent FP64
// operations instead of a full double division.
__device__ __forceinline__ double fast_rcp64(double d) {
  const int hi = __double2hiint(d);
  const int ex = ((hi >> 20) & 0x7ff) - 1023;
  if (ex < -120 || ex > 120) return 1.0 / d;   // callers pass d > 0
  const unsigned lo = (unsigned)__double2loint(d);
  const float f = __int_as_float(((ex + 127) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29));
  const float rf = __frcp_rn(f);
  const int rb = __float_as_int(rf);
  const int rex = ((rb >> 23) & 0xff) - 127;
  const double x0 = __hiloint2double(((rex + 1023) << 20) | ((rb & 0x7fffff) >> 3), (rb & 7) << 29);
  const double e = fma(-d, x0, 1.0);
  const double e2 = fma(e, e, e);
  return fma(x0, e2, x0);
}

// As fast_rcp64 with one Newton step instead of the third-order one: relative
// error below 2^-46 from the 24-bit seed, one dependent FP64 instruction less.
__device__ __forceinline__ double fast_rcp64_newton(double d) {
  const int hi = __double2hiint(d);
  const int ex = ((hi >> 20) & 0x7ff) - 1023;
  if (ex < -120 || ex > 120) return 1.0 / d;   // callers pass d > 0
  const unsigned lo = (unsigned)__double2loint(d);
  const float f = __int_as_float(((ex + 127) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29));
  const float rf = __frcp_rn(f);
  const int rb = __float_as_int(rf);
  const int rex = ((rb >> 23) & 0xff) - 127;
  const double x0 = __hiloint2double(((rex + 1023) << 20) | ((rb & 0x7fffff) >> 3), (rb & 7) << 29);
  return fma(x0, fma(-d, x0, 1.0), x0);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red /* >= 32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

}  // namespace tals
