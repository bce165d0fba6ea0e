// Batched st-HOSVD-ALS (Alg. 5) over thousands of small third-order FP32
// tensors of uneven sizes and ranks, in one persistent launch.
//
// Each CTA takes whole tensors from an atomic work queue and runs the complete
// decomposition of a tensor by itself: per mode the Sec. 4 initial guess, the
// ALS sweeps (Alg. 3, one read of the tensor per sweep through the same fused
// pass as the single-tensor path, at CTA scope), the Eq. 5.01 stop rule, the
// factor QR and the truncation written straight from the last sweep's W. The
// small linear algebra (Grams, Cholesky, row solves) runs in FP64 in shared
// memory. No CTA ever waits on another: the only inter-CTA interaction is the
// atomicAdd on the queue head. The launch (queue reset + kernel) is captured in
// a CUDA graph and replayed; an autotuner times the candidate tile shapes and
// CTA counts on first use and keeps the fastest for that batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "pass_impl.cuh"

namespace tals {

constexpr int kBatchMaxI = 128;
constexpr int kBatchMaxR = 16;

struct BatchStat {
  double e[3];
  double norm_a2;
  double corr[3];
  int sweeps[3];
  int converged[3];
  int order[3];
  int status;
};

struct BatchArgs {
  int count;
  const float* const* A;
  const long long* dims;   // [3 count]
  const int* ranks;        // [3 count]
  float* const* G;
  float* const* U;         // [3 count]
  float* scratch;          // per CTA: 2 x scratch_elems floats
  long long scratch_elems;
  BatchStat* stats;
  int* queue;
  double eta;
  int max_sweeps;
  uint64_t seed;
};

namespace {

// ---- CTA-scope FP64 helpers (blockDim.x == kThreads) ----
// FP64 on this part has ~64-cycle latency and a warp FP64 instruction holds an
// SMSP's FP64 pipe ~76 cycles: the helpers keep several independent chains per
// thread, skip the mirrored half of symmetric products and take no division
// inside a dependent chain.

// out = A^T B (R x R). sym: A == B, only s <= r computed and mirrored.
__device__ void cta_gram(const double* A, const double* B, int I, int R, double* out, bool sym) {
  const int n = sym ? R * (R + 1) / 2 : R * R;
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    int r, c;
    if (sym) {
      r = (int)((sqrtf(8.f * (float)o + 1.f) - 1.f) * 0.5f);
      while (r * (r + 1) / 2 > o) --r;
      while ((r + 1) * (r + 2) / 2 <= o) ++r;
      c = o - r * (r + 1) / 2;
    } else {
      r = o / R;
      c = o % R;
    }
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
    int i = 0;
    for (; i + 4 <= I; i += 4) {
      g0 = fma(A[i * R + r], B[i * R + c], g0);
      g1 = fma(A[(i + 1) * R + r], B[(i + 1) * R + c], g1);
      g2 = fma(A[(i + 2) * R + r], B[(i + 2) * R + c], g2);
      g3 = fma(A[(i + 3) * R + r], B[(i + 3) * R + c], g3);
    }
    for (; i < I; ++i) g0 = fma(A[i * R + r], B[i * R + c], g0);
    const double g = (g0 + g1) + (g2 + g3);
    out[r * R + c] = g;
    if (sym) out[c * R + r] = g;
  }
  __syncthreads();
}

// Lower Cholesky factor of the (symmetrised) R x R matrix G in place (R <= 16);
// returns 1 on failure. Right-looking LDL^T: warp 0 finishes column k+1 and
// takes its pivot reciprocal, the other warps update the rest of the trailing
// block; square roots at the end. `w` holds 2 R doubles of scratch.
__device__ int cta_chol(double* G, int R, int* flag, double* w) {
  double* Lc = w;          // [2][kBatchMaxR]
  __shared__ double rs[kBatchMaxR];
  __shared__ long long tiny_bits;
  __shared__ int tri[(kBatchMaxR - 1) * kBatchMaxR / 2];   // packed (i', j') of a dense index
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int a = tid; a < (R - 1) * R / 2; a += blockDim.x) {
    int ip = (int)((sqrtf(8.f * (float)a + 1.f) - 1.f) * 0.5f);
    while (ip * (ip + 1) / 2 > a) --ip;
    while ((ip + 1) * (ip + 2) / 2 <= a) ++ip;
    tri[a] = (ip << 16) | (a - ip * (ip + 1) / 2);
  }
  for (int o = tid; o < R * R; o += blockDim.x) {
    const int r = o / R, c = o % R;
    if (r > c) G[r * R + c] = 0.5 * (G[r * R + c] + G[c * R + r]);
  }
  if (tid == 0) *flag = 0;
  if (tid < 32) {
    const int hmax = __reduce_max_sync(0xffffffffu, lane < R ? max(0, __double2hiint(G[lane * R + lane])) : 0);
    if (lane == 0)
      tiny_bits = __double_as_longlong(64.0 * 2.220446049250313e-16 * __hiloint2double(hmax, 0));
  }
  __syncthreads();
  if (warp == 0) {
    double d = G[0];
    if (lane == 0 && !pivot_ok(d, tiny_bits)) {
      d = 1.0;
      G[0] = 1.0;
      *flag = 1;
    }
    const double dinv = __shfl_sync(0xffffffffu, lane == 0 ? fast_rcp64(d) : 0.0, 0);
    if (lane >= 1 && lane < R) Lc[lane] = G[lane * R] * dinv;
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; ++k) {
    const int cb = (k & 1) * kBatchMaxR, c1 = k + 1;
    if (warp == 0) {
      const int i = c1 + lane;
      double v = i < R ? fma(-G[i * R + k], Lc[cb + c1], G[i * R + c1]) : 0.0;
      double d = __shfl_sync(0xffffffffu, v, 0);
      if (!pivot_ok(d, tiny_bits)) {
        d = 1.0;
        if (lane == 0) {
          v = 1.0;
          *flag = 1;
        }
      }
      const double dinv = fast_rcp64(d);
      if (i < R) {
        G[i * R + c1] = v;
        if (i > c1) Lc[(kBatchMaxR - cb) + i] = v * dinv;
      }
    } else if (warp != 4) {
      // warps sharing warp 0's SMSP stay off the FP64 pipe the serial chain uses
      const int m = R - 2 - k, na = m * (m + 1) / 2;
      const int tt = tid < 128 ? tid - 32 : tid - 64;
      for (int a = tt; a < na; a += blockDim.x - 64) {
        const int ij = tri[a];
        const int i = k + 2 + (ij >> 16), j = k + 2 + (ij & 0xffff);
        G[i * R + j] = fma(-G[i * R + k], Lc[cb + j], G[i * R + j]);
      }
    }
    __syncthreads();
  }
  for (int r = tid; r < R; r += blockDim.x) rs[r] = rsqrt(G[r * R + r]);
  __syncthreads();
  for (int o = tid; o < R * R; o += blockDim.x) {
    const int r = o / R, c = o % R;
    G[o] = c <= r ? G[o] * rs[c] : 0.0;
  }
  __syncthreads();
  const int f = *flag;
  __syncthreads();
  return f;
}

// Row solves with the lower factor F: op 0: Out = In F^-T, op 1: Out = In (F F^T)^-1.
// One thread per row, right-looking so each step's chain is one FMA; the factor
// is scaled by its pivot reciprocals first (no division in the chains); the
// row lives in registers (loops unrolled to the rank limit). `w` holds
// 2 R^2 + R doubles of scratch.
__device__ void cta_rowsolve(const double* In, const double* F, int op, double* Out, int I, int R,
                             double* w) {
  double* Ff = w;                          // F[r][c] / F[r][r]
  double* Fb = w + kBatchMaxR * kBatchMaxR;  // F[c][r] / F[r][r], stored at [c][r]
  double* dinv = Fb + kBatchMaxR * kBatchMaxR;
  for (int r = threadIdx.x; r < R; r += blockDim.x) dinv[r] = 1.0 / F[r * R + r];
  __syncthreads();
  for (int o = threadIdx.x; o < R * R; o += blockDim.x) {
    const int r = o / R, c = o % R;
    Ff[r * kBatchMaxR + c] = F[o] * dinv[r];
    Fb[r * kBatchMaxR + c] = F[o] * dinv[c];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    double s[kBatchMaxR];
#pragma unroll
    for (int r = 0; r < kBatchMaxR; ++r) s[r] = r < R ? In[i * R + r] * dinv[r] : 0.0;
    // forward: F x^T = b^T
#pragma unroll
    for (int c = 0; c < kBatchMaxR; ++c) {
      if (c < R) {
        const double xc = s[c];
#pragma unroll
        for (int r = c + 1; r < kBatchMaxR; ++r)
          if (r < R) s[r] = fma(-Ff[r * kBatchMaxR + c], xc, s[r]);
      }
    }
    if (op == 1) {
      // backward: F^T z^T = x^T
#pragma unroll
      for (int r = 0; r < kBatchMaxR; ++r) s[r] = r < R ? s[r] * dinv[r] : 0.0;
#pragma unroll
      for (int c = kBatchMaxR - 1; c >= 0; --c) {
        if (c < R) {
          const double zc = s[c];
#pragma unroll
          for (int r = 0; r < c; ++r) s[r] = fma(-Fb[c * kBatchMaxR + r], zc, s[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kBatchMaxR; ++r)
      if (r < R) Out[i * R + r] = s[r];
  }
  __syncthreads();
}

struct LaSmem {
  double* Y;    // [I][R]
  double* L;    // [I][R]
  double* Z;    // [I][R]
  double* X;    // [R][R]
  double* GL;   // [R][R]
  float* Yf;    // [I][R]
  float* Lt;    // [I][R]
  double* work; // [2 R^2 + R] for the solves and the Cholesky
  int* flag;
};

// Bytes of the small algebra's scratch (aliasing the pass buffers) and of the
// buffers that live across passes.
__host__ __device__ constexpr size_t la_scratch_bytes() {
  return ((2 * (size_t)kBatchMaxI * kBatchMaxR + 4 * kBatchMaxR * kBatchMaxR + kBatchMaxR) * sizeof(double) + 16 +
          15) / 16 * 16;
}
__host__ __device__ constexpr size_t la_live_bytes() {
  return (size_t)kBatchMaxI * kBatchMaxR * (sizeof(double) + 2 * sizeof(float));
}

// Q = orthonormal basis of In by CholeskyQR (one round): L = In F^-T; the
// FP32 copy Lt and the Gram of its stored values GL. Returns failure.
__device__ int cta_cholqr(const double* In, LaSmem& m, int I, int R, double* Out) {
  cta_gram(In, In, I, R, m.X, true);
  if (cta_chol(m.X, R, m.flag, m.work)) return 1;
  cta_rowsolve(In, m.X, 0, Out, I, R, m.work);
  return 0;
}

template <int RC, int RPT, int RW, int JT>
__device__ void run_tensor(const BatchArgs& b, int t, unsigned char* smem, size_t pass_bytes) {
  const long long* dd = b.dims + 3 * (size_t)t;
  const int* rr = b.ranks + 3 * (size_t)t;
  long long d[3] = {dd[0], dd[1], dd[2]};
  int R[3] = {rr[0], rr[1], rr[2]};
  int order[3] = {0, 1, 2};
  // ascending rank, ties by mode index (Prop. 1)
  for (int a = 0; a < 3; ++a)
    for (int c = a + 1; c < 3; ++c)
      if (R[order[c]] < R[order[a]] || (R[order[c]] == R[order[a]] && order[c] < order[a])) {
        const int x = order[a];
        order[a] = order[c];
        order[c] = x;
      }
  // The pass's buffers and the FP64 scratch of the small algebra (Y, Z, X, GL,
  // work) are never live together: both start at offset 0. L, Lt and Yf cross
  // the passes and sit above the larger of the two.
  LaSmem m;
  const int IR = kBatchMaxI * kBatchMaxR;
  m.Y = reinterpret_cast<double*>(smem);
  m.Z = m.Y + IR;
  m.X = m.Z + IR;
  m.GL = m.X + kBatchMaxR * kBatchMaxR;
  m.work = m.GL + kBatchMaxR * kBatchMaxR;
  m.flag = reinterpret_cast<int*>(m.work + 2 * kBatchMaxR * kBatchMaxR + kBatchMaxR);
  unsigned char* live = smem + (pass_bytes > la_scratch_bytes() ? pass_bytes : la_scratch_bytes());
  m.L = reinterpret_cast<double*>(live);
  m.Yf = reinterpret_cast<float*>(m.L + IR);
  m.Lt = m.Yf + IR;
  __shared__ double s_norm;
  __shared__ int s_stop;

  float* scr = b.scratch + (size_t)blockIdx.x * 2 * b.scratch_elems;
  const float* cur = b.A[t];
  BatchStat stat;
  memset(&stat, 0, sizeof(stat));
  double norm_a = 0.0;
  for (int idx = 0; idx < 3; ++idx) {
    const int n = order[idx];
    stat.order[idx] = n;
    ModeView v = {1, d[n], 1};
    for (int q = 0; q < n; ++q) v.P *= d[q];
    for (int q = n + 1; q < 3; ++q) v.Q *= d[q];
    const int Rn = R[n];
    const int I = (int)v.I;
    float* dest = idx == 2 ? b.G[t] : scr + (size_t)idx * b.scratch_elems;
    PassArgs<float> a{};
    a.X = cur;
    a.P = v.P;
    a.I = v.I;
    a.Q = v.Q;
    a.J = v.J();
    a.R = Rn;
    a.ntiles = (a.J + JT - 1) / JT;
    a.nbuf = 2;
    a.vec_ok = (((uintptr_t)cur % 16) == 0) && ((v.Q * 4) % 16 == 0);
    a.st = nullptr;
    a.resid = 1;   // small tensors: e_k from the explicit residual
    // ---- Sec. 4: Y0 = B_(n) S, ||B_(n)||^2; L0 = Q of QR(Y0) by CholeskyQR2 ----
    a.mode = PASS_INIT;
    a.sketch_state = b.seed ^ ((uint64_t)n << 56);
    double nrm = pass_cta<float, RC, RPT, RW, kThreads, JT>(a, 0, 1, 0, smem, m.Yf);
    __syncthreads();   // the scratch below overlays the pass's tiles
    if (threadIdx.x == 0) s_norm = nrm;
    __syncthreads();
    const double normM2 = s_norm;
    if (idx == 0) norm_a = sqrt(normM2);
    for (int e = threadIdx.x; e < I * Rn; e += blockDim.x) m.Y[e] = (double)m.Yf[e];
    __syncthreads();
    int fail = cta_cholqr(m.Y, m, I, Rn, m.Z);
    if (!fail) fail = cta_cholqr(m.Z, m, I, Rn, m.L);
    int k = 0, converged = 0;
    double e_prev = 0.0, e_cur = 0.0;
    while (!fail) {
      for (int e = threadIdx.x; e < I * Rn; e += blockDim.x) m.Lt[e] = (float)m.L[e];
      __syncthreads();
      // ---- one read of B: W = B^T Q, Y = B W and ||B - Q W^T||^2; W written
      // when it may be the final one ----
      a.mode = PASS_SWEEP;
      a.L = m.Lt;
      a.Wout = (k >= 1 || k + 1 >= b.max_sweeps) ? dest : nullptr;
      const double rs = pass_cta<float, RC, RPT, RW, kThreads, JT>(a, 0, 1, 0, smem, m.Yf);
      __syncthreads();   // the scratch below overlays the pass's tiles
      for (int e = threadIdx.x; e < I * Rn; e += blockDim.x) m.Y[e] = (double)m.Yf[e];
      // e_k and the Eq. 5.01 stop rule
      if (threadIdx.x == 0) {
        const double e = sqrt(rs > 0.0 ? rs : 0.0);
        int stop = 0;
        if (k >= 1 && fabs(e_prev - e) <= b.eta * norm_a) {
          stop = 1;
          converged = 1;
        }
        if (k + 1 >= b.max_sweeps) stop = 1;
        s_stop = stop;
        s_norm = e;
      }
      __syncthreads();
      e_cur = s_norm;
      e_prev = e_cur;
      ++k;
      if (s_stop) break;
      // ---- L_{k+1} = Y X^-1 with X = Q^T Y, then its Q factor ----
      cta_gram(m.L, m.Y, I, Rn, m.X, false);
      if (cta_chol(m.X, Rn, m.flag, m.work)) {
        fail = 1;
        break;
      }
      cta_rowsolve(m.Y, m.X, 1, m.Z, I, Rn, m.work);
      fail = cta_cholqr(m.Z, m, I, Rn, m.L);
    }
    if (threadIdx.x == 0) converged = s_stop ? converged : 0;
    stat.e[n] = e_cur;
    stat.sweeps[n] = k;
    stat.converged[n] = converged;
    if (fail) stat.status = 4;   // TALS_ESINGULAR
    // factor U^(n) = the stored basis of the last sweep
    float* U = b.U[3 * (size_t)t + n];
    for (int e = threadIdx.x; e < I * Rn; e += blockDim.x) U[e] = m.Lt[e];
    __syncthreads();
    if (fail) break;
    cur = dest;
    d[n] = Rn;
  }
  if (threadIdx.x == 0) {
    stat.norm_a2 = norm_a * norm_a;
    b.stats[t] = stat;
  }
  __syncthreads();
}

template <int RC, int RPT, int RW, int JT>
__global__ void __launch_bounds__(kThreads, 2) batched_kernel(BatchArgs b, size_t pass_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_t;
  while (true) {
    if (threadIdx.x == 0) s_t = atomicAdd(b.queue, 1);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= b.count) return;
    run_tensor<RC, RPT, RW, JT>(b, t, smem_raw, pass_bytes);
  }
}

struct Variant {
  int rc, rpt, rw, jt;
  void* fn;
};

template <int RC, int RPT, int RW, int JT>
Variant make_variant() {
  return Variant{RC, RPT, RW, JT, reinterpret_cast<void*>(&batched_kernel<RC, RPT, RW, JT>)};
}

std::vector<Variant> variants() {
  // tile shapes the autotuner chooses between (all cover I <= 128, R <= 16);
  // 32-column tiles halve the per-tile latency a CTA pays on a small tensor
  return {make_variant<16, 2, 4, 16>(), make_variant<16, 1, 8, 16>(), make_variant<16, 2, 8, 16>(),
          make_variant<16, 2, 4, 32>(), make_variant<16, 2, 8, 32>()};
}

size_t pass_region(const Variant& v) {
  const int rowt = kThreads / (v.rc / v.rw);
  size_t b = pass_smem_bytes<float>(kBatchMaxI, v.rc, rowt * v.rpt, 2, kThreads, v.jt);
  // slack rows are sized for the smallest I the shape serves
  b += (size_t)slack_rows(16, rowt * v.rpt) * (v.jt + 4) * sizeof(float);
  return (b + 15) / 16 * 16;
}

// Dynamic shared memory of a variant: max(pass buffers, small-algebra scratch) + live buffers.
size_t batch_smem(size_t pass_bytes) {
  return std::max(pass_bytes, la_scratch_bytes()) + la_live_bytes();
}

struct Plan {
  int variant = -1;
  int ctas_per_sm = 1;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
};

struct BatchCache {
  std::mutex mu;
  std::map<std::vector<long long>, Plan> plans;
  // device buffers reused across calls
  void* dev = nullptr;
  size_t dev_bytes = 0;
  float* scratch = nullptr;
  size_t scratch_bytes = 0;
  BatchStat* hstats = nullptr;
  size_t hstats_n = 0;
};

BatchCache& cache() {
  static BatchCache c;
  return c;
}

}  // namespace

}  // namespace tals

using namespace tals;

extern "C" tals_status tals_batched_st_hosvd(int count, void* const* A_ptrs, const int64_t* dims,
                                             const int* ranks, const tals_opts* opts,
                                             void* const* G_ptrs, void* const* U_ptrs,
                                             tals_stats* stats, void* stream) {
  if (count < 0 || (count > 0 && (!A_ptrs || !dims || !ranks || !G_ptrs || !U_ptrs)))
    return fail(TALS_EINVAL, "bad batched arguments");
  if (count == 0) return TALS_OK;
  tals_opts o;
  if (opts) o = *opts; else tals_default_opts(&o);
  if (o.max_sweeps < 1) return fail(TALS_EINVAL, "max_sweeps must be >= 1");
  if (o.precision != TALS_PREC_NATIVE) return fail(TALS_ENOTSUP, "batched runs in FP32 only");
  long long scratch_elems = 1;
  for (int t = 0; t < count; ++t) {
    const int64_t* d = dims + 3 * (size_t)t;
    const int* r = ranks + 3 * (size_t)t;
    for (int n = 0; n < 3; ++n) {
      if (d[n] < 1 || d[n] > kBatchMaxI || r[n] < 1 || r[n] > d[n] || r[n] > kBatchMaxR)
        return fail(TALS_EINVAL, "tensor %d mode %d: need 1 <= R <= I <= %d and R <= %d", t, n,
                    kBatchMaxI, kBatchMaxR);
      if ((long long)r[n] > (long long)r[(n + 1) % 3] * r[(n + 2) % 3])
        return fail(TALS_EINVAL, "tensor %d: rank %d exceeds the product of the others", t, n);
    }
    // intermediates after the first and second truncation, any order
    long long mx = 0;
    for (int n = 0; n < 3; ++n) {
      long long j = 1;
      for (int m = 0; m < 3; ++m) j *= (m == n) ? r[n] : d[m];
      mx = std::max(mx, j);
    }
    scratch_elems = std::max(scratch_elems, mx);
  }
  cudaStream_t s = (cudaStream_t)stream;
  BatchCache& bc = cache();
  std::lock_guard<std::mutex> lock(bc.mu);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int max_ctas = sms * 2;
  cudaError_t e;
  // device copies of the descriptors: [A ptrs][G ptrs][U ptrs][dims][ranks][stats][queue]
  const size_t off_A = 0, off_G = off_A + count * sizeof(void*), off_U = off_G + count * sizeof(void*),
               off_d = off_U + 3 * (size_t)count * sizeof(void*),
               off_r = off_d + 3 * (size_t)count * sizeof(long long),
               off_s = ((off_r + 3 * (size_t)count * sizeof(int) + 15) / 16) * 16,
               off_q = off_s + (size_t)count * sizeof(BatchStat), total = off_q + 16;
  if (bc.dev_bytes < total) {
    if (bc.dev) cudaFree(bc.dev);
    if ((e = cudaMalloc(&bc.dev, total)) != cudaSuccess) return cuda_fail(e, "batched descriptors");
    bc.dev_bytes = total;
    for (auto& kv : bc.plans)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    bc.plans.clear();
  }
  const size_t sbytes = (size_t)max_ctas * 2 * scratch_elems * sizeof(float);
  if (bc.scratch_bytes < sbytes) {
    if (bc.scratch) cudaFree(bc.scratch);
    if ((e = cudaMalloc((void**)&bc.scratch, sbytes)) != cudaSuccess)
      return cuda_fail(e, "batched scratch");
    bc.scratch_bytes = sbytes;
    for (auto& kv : bc.plans)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    bc.plans.clear();
  }
  if (bc.hstats_n < (size_t)count) {
    if (bc.hstats) cudaFreeHost(bc.hstats);
    if ((e = cudaMallocHost((void**)&bc.hstats, count * sizeof(BatchStat))) != cudaSuccess)
      return cuda_fail(e, "batched stats");
    bc.hstats_n = count;
  }
  unsigned char* dv = (unsigned char*)bc.dev;
  std::vector<long long> d64(3 * (size_t)count);
  for (size_t i = 0; i < d64.size(); ++i) d64[i] = dims[i];
  e = cudaMemcpyAsync(dv + off_A, A_ptrs, count * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dv + off_G, G_ptrs, count * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dv + off_U, U_ptrs, 3 * (size_t)count * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dv + off_d, d64.data(), d64.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dv + off_r, ranks, 3 * (size_t)count * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "batched descriptor upload");

  BatchArgs a;
  a.count = count;
  a.A = (const float* const*)(dv + off_A);
  a.G = (float* const*)(dv + off_G);
  a.U = (float* const*)(dv + off_U);
  a.dims = (const long long*)(dv + off_d);
  a.ranks = (const int*)(dv + off_r);
  a.stats = (BatchStat*)(dv + off_s);
  a.queue = (int*)(dv + off_q);
  a.scratch = bc.scratch;
  a.scratch_elems = scratch_elems;
  a.eta = o.eta;
  a.max_sweeps = o.max_sweeps;
  a.seed = o.seed;

  const std::vector<Variant> vs = variants();
  auto launch = [&](int vi, int per_sm, cudaStream_t st) -> cudaError_t {
    const Variant& v = vs[vi];
    const size_t pr = pass_region(v);
    const size_t smem = batch_smem(pr);
    cudaError_t err = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, kThreads, smem);
    if (err != cudaSuccess) return err;
    const int grid = std::min(count, sms * std::max(1, std::min(occ, per_sm)));
    err = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
    if (err != cudaSuccess) return err;
    BatchArgs aa = a;
    size_t prb = pr;
    void* args[] = {&aa, &prb};
    return cudaLaunchKernel(v.fn, dim3(grid), dim3(kThreads), args, smem, st);
  };

  // autotune key: batch size and the histogram of (max I, max R)
  std::vector<long long> key = {count, scratch_elems};
  for (int t = 0; t < count; t += std::max(1, count / 64)) {
    key.push_back(dims[3 * t] * 10007 + dims[3 * t + 1] * 101 + dims[3 * t + 2]);
    key.push_back(ranks[3 * t] * 289 + ranks[3 * t + 1] * 17 + ranks[3 * t + 2]);
  }
  Plan& plan = bc.plans[key];
  if (plan.variant < 0) {
    // time every (tile shape, CTAs per SM) once and keep the fastest
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int vi = 0; vi < (int)vs.size(); ++vi)
      for (int per_sm = 1; per_sm <= 2; ++per_sm) {
        cudaEventRecord(e0, s);
        e = launch(vi, per_sm, s);
        cudaEventRecord(e1, s);
        if (e != cudaSuccess) continue;
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          plan.variant = vi;
          plan.ctas_per_sm = per_sm;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (plan.variant < 0) return cuda_fail(cudaGetLastError(), "batched kernel launch");
    // capture queue reset + kernel into a graph
    cudaStream_t cs;
    cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t le = launch(plan.variant, plan.ctas_per_sm, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      if (le != cudaSuccess) e = le;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&plan.exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "batched graph");
  }
  e = cudaGraphLaunch(plan.exec, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bc.hstats, dv + off_s, count * sizeof(BatchStat), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "batched run");
  int worst = 0;
  for (int t = 0; t < count; ++t) {
    const BatchStat& b = bc.hstats[t];
    if (b.status && !worst) worst = b.status;
    if (stats) {
      tals_stats& st = stats[t];
      std::memset(&st, 0, sizeof(st));
      double e2 = 0.0;
      for (int n = 0; n < 3; ++n) {
        st.err_per_mode[n] = b.e[n];
        st.sweeps[n] = b.sweeps[n];
        st.converged[n] = b.converged[n];
        st.order[n] = b.order[n];
        e2 += b.e[n] * b.e[n];
      }
      st.norm_a = std::sqrt(b.norm_a2);
      st.rel_err = b.norm_a2 > 0 ? std::sqrt(e2 / b.norm_a2) : 0.0;
      st.status = b.status;
    }
  }
  if (worst)
    return fail((tals_status)worst, "a tensor of the batch had a Gram matrix that is not positive "
                                    "definite (truncation above the numerical rank, Remark 3)");
  return TALS_OK;
}
