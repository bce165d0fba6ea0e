// Y = B_(n) W for a mode view whose columns j = p Q + q come in runs of 16 along
// q (Q % 16 == 0): the L-update product of Alg. 3 (Y = A R_k) as a register-tiled
// GEMM with the long contraction (the J unfolding columns) split across CTAs.
//
// C (I x R) = A (I x J) . Wm (R x J)^T with A[i][j] = X[p, i, q] and Wm[r][j] =
// W[p, r, q] (W in the P x R x Q layout of the R-update's output). CTA (bx, s)
// computes rows bx*256 .. +255 of C over columns [s*kper, (s+1)*kper) and writes
// them as partial s: part[s][i][r] -- the per-CTA Y partials the fused pass
// writes, summed in FP64 by the same reduction. The CTAs of row tile 0 also sum
// ||W||^2 over their columns (exact squares, compensated), one FP64 partial per
// split; a CTA exits at once when the gate's mode is done. Tiles of 16 columns
// move through a three-stage cp.async ring: the A tile row-major (each row's 16
// columns contiguous, row stride 20 floats: 5 chunks of 16 bytes, so a warp's
// 16-byte row reads are conflict-free), the Wm tile column-major (16 rows of RP
// ranks, copied element-wise). A thread holds 8 rows x 8 ranks (rows lane + 32 m,
// ranks 8 w .. 8 w + 7 of warp w) as rank pairs, updated by paired FP32 FMAs
// (__ffma2_rn, each pair rounded like two fmaf): per 4 columns, 8 row reads and 8
// broadcast rank reads of 16 bytes feed 128 paired FMAs.
#include <algorithm>

#include "internal.h"

namespace tals {

namespace {

constexpr int kAdjTI = 256;      // rows per CTA
constexpr int kAdjKC = 16;       // columns per tile
constexpr int kAdjLD = kAdjKC + 4;
constexpr int kAdjStages = 3;

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint32_t sptr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void add_sq_c(float x, float& s, float& c) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  const float t = s + p;
  c += (fabsf(s) >= fabsf(p)) ? (s - t) + p : (p - t) + s;
  c += e;
  s = t;
}

__device__ __forceinline__ float comp(const float4& v, int u) {
  return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w;
}

// RP ranks (32 or 64): RP / 8 warps; three (RP = 32) or two CTAs per SM.
template <int RP>
__global__ void __launch_bounds__(RP * 4, RP == 32 ? 3 : 2) adjoint_rows_kernel(const float* __restrict__ X, long long I,
                                                              long long Q, const float* __restrict__ W,
                                                              int R, long long J, long long kper,
                                                              float* __restrict__ part, double* __restrict__ wsq,
                                                              const ModeState* __restrict__ gate) {
  if (gate != nullptr && gate->done) return;   // uniform, before any barrier
  constexpr int NT = RP * 4;
  extern __shared__ __align__(16) float adj_sm[];
  float* As = adj_sm;                                      // [stages][TI][LD]
  float* Bs = adj_sm + kAdjStages * kAdjTI * kAdjLD;       // [stages][KC][RP]
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long i0 = (long long)blockIdx.x * kAdjTI;
  const long long kb = (long long)blockIdx.y * kper;
  const long long ke = kb + kper < J ? kb + kper : J;
  const int nch = (int)((ke - kb + kAdjKC - 1) / kAdjKC);
  const bool wsum = blockIdx.x == 0 && wsq != nullptr;

  // one tile: A rows i0 .. i0 + 255 and the RP rows of Wm, columns j0 .. j0 + 15
  auto load = [&](int c, int st) {
    const long long j0 = kb + (long long)c * kAdjKC;
    const long long p = j0 / Q, q = j0 - p * Q;   // a tile stays within one p (Q % 16 == 0)
    const bool jin = j0 < ke;
    float* as = As + st * kAdjTI * kAdjLD;
    float* bs = Bs + st * kAdjKC * RP;
    const float* xa = X + (p * I + i0) * Q + q;
#pragma unroll
    for (int t = 0; t < kAdjTI * 4 / NT; ++t) {
      const int e = tid + t * NT;
      const int r = e >> 2, c4 = e & 3;
      const bool ok = jin && i0 + r < I;
      cp16(sptr(as + r * kAdjLD + c4 * 4), ok ? xa + (long long)r * Q + c4 * 4 : X, ok ? 16u : 0u);
    }
    // Wm column-major: consecutive threads, consecutive ranks of one column
    const float* wa = W + p * R * Q + q;
#pragma unroll
    for (int t = 0; t < kAdjKC * RP / NT; ++t) {
      const int e = tid + t * NT;
      const int r = e % RP, k = e / RP;
      const bool ok = jin && r < R;
      cp4(sptr(bs + k * RP + r), ok ? wa + (long long)r * Q + k : W, ok ? 4u : 0u);
    }
  };

  float2 acc[8][4];
#pragma unroll
  for (int m = 0; m < 8; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n) acc[m][n] = make_float2(0.f, 0.f);
  float ws = 0.f, wc = 0.f;

#pragma unroll
  for (int st = 0; st < kAdjStages - 1; ++st) {
    if (st < nch) load(st, st);
    cp_commit();
  }
  for (int c = 0; c < nch; ++c) {
    cp_wait<kAdjStages - 2>();
    __syncthreads();
    // refill the stage consumed two tiles ago (its readers passed the barrier above)
    if (c + kAdjStages - 1 < nch) load(c + kAdjStages - 1, (c + kAdjStages - 1) % kAdjStages);
    cp_commit();
    const int st = c % kAdjStages;
    const float* as = As + st * kAdjTI * kAdjLD;
    const float* bs = Bs + st * kAdjKC * RP;
    if (wsum) {
      // the warp's 8 ranks x 16 columns: 4 values per lane
#pragma unroll
      for (int u = 0; u < 4; ++u) add_sq_c(bs[((lane >> 3) + 4 * u) * RP + warp * 8 + (lane & 7)], ws, wc);
    }
#pragma unroll
    for (int kk = 0; kk < kAdjKC; kk += 4) {
      float4 a[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) a[m] = *reinterpret_cast<const float4*>(as + (lane + 32 * m) * kAdjLD + kk);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 b0 = *reinterpret_cast<const float4*>(bs + (kk + u) * RP + warp * 8);
        const float4 b1 = *reinterpret_cast<const float4*>(bs + (kk + u) * RP + warp * 8 + 4);
        const float2 bp[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float av = comp(a[m], u);
          const float2 a2 = make_float2(av, av);
#pragma unroll
          for (int n = 0; n < 4; ++n) acc[m][n] = __ffma2_rn(a2, bp[n], acc[m][n]);
        }
      }
    }
  }
  cp_wait<0>();
  // partial s: rows lane + 32 m, ranks 8 warp .. 8 warp + 7
  float* out = part + (size_t)blockIdx.y * (size_t)I * R;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const long long i = i0 + lane + 32 * m;
    if (i >= I) continue;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int r = warp * 8 + 2 * n;
      if (r < R) out[i * R + r] = acc[m][n].x;
      if (r + 1 < R) out[i * R + r + 1] = acc[m][n].y;
    }
  }
  if (wsum) {
    double t = (double)ws + (double)wc;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      wsq[blockIdx.y] = t;
    }
  }
}

template <int RP>
size_t adjoint_smem() {
  return (size_t)kAdjStages * ((size_t)kAdjTI * kAdjLD + (size_t)kAdjKC * RP) * sizeof(float);
}

}  // namespace

bool adjoint_rows_ok(const ModeView& v, int R, const void* X, const void* W) {
  return R >= 1 && R <= 64 && v.Q % 16 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)W & 15) == 0;
}

int adjoint_rows_splits(const ModeView& v, int R, int sms) {
  // about three CTAs per SM, each at least 32 tiles of columns
  const long long tiles_i = (v.I + kAdjTI - 1) / kAdjTI;
  long long S = std::max<long long>(1, (3LL * sms + tiles_i - 1) / tiles_i);
  const long long maxs = std::max<long long>(1, v.J() / (32 * kAdjKC));
  S = std::min(S, maxs);
  return (int)std::min<long long>(S, 65535);
}

cudaError_t launch_adjoint_rows(const float* X, const ModeView& v, const float* W, int R, int S, float* part,
                                double* wsq, const ModeState* gate, cudaStream_t s) {
  if (!adjoint_rows_ok(v, R, X, W) || S < 1) return cudaErrorInvalidValue;
  const long long J = v.J();
  long long kper = (J + S - 1) / S;
  kper = (kper + kAdjKC - 1) / kAdjKC * kAdjKC;
  const dim3 grid((unsigned)((v.I + kAdjTI - 1) / kAdjTI), (unsigned)S);
  if (R <= 32) {
    // the attribute belongs to the current device: set on every call
    const size_t sm = adjoint_smem<32>();
    cudaError_t e = cudaFuncSetAttribute(adjoint_rows_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    adjoint_rows_kernel<32><<<grid, 128, sm, s>>>(X, v.I, v.Q, W, R, J, kper, part, wsq, gate);
  } else {
    const size_t sm = adjoint_smem<64>();
    cudaError_t e = cudaFuncSetAttribute(adjoint_rows_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    adjoint_rows_kernel<64><<<grid, 256, sm, s>>>(X, v.I, v.Q, W, R, J, kper, part, wsq, gate);
  }
  return cudaGetLastError();
}

}  // namespace tals
