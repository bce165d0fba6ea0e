// Fused ALS sweep pass on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory.
//
// Same computation as the CUDA-core pass (Alg. 3 R-update and L-update fused
// as in Eq. 2.2): per tile of 128 unfolding columns,
//   GEMM1  W_t (128 x R) = B_t^T (128 x I) . Q (I x R)      -> TMEM, fp32
//   GEMM2  Y   (I x R)  += B_t  (I x 128) . W_t (128 x R)   -> TMEM, fp32
// B_t is a BF16 copy of the tensor, staged by TMA with 128-byte swizzle in
// 128 x 128 chunks (two 64-column boxes). One staged chunk is read by GEMM1 as
// an MN-major A operand (m = column, k = row i) and by GEMM2 as a K-major A
// operand (m = row i, k = column): for 16-bit types the 128B-swizzled layout
// with 128-byte rows is a canonical layout for both majors. W_t goes TMEM ->
// registers -> BF16 -> shared memory (K-major, 128B swizzle) between the two
// GEMMs; Y stays in TMEM across all the CTA's tiles and is written once as a
// per-CTA FP32 partial, reduced in FP64 by the same kernel as the CUDA-core path.
//
// One thread issues every TMA load and every MMA; completion is tracked with
// mbarriers (tcgen05.commit for the MMAs). Every wait is bounded: on timeout
// the CTA records an error code, stops issuing work, waits (again bounded) for
// what it already issued and frees its tensor memory before it returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace tals {

constexpr int kTcCols = 128;     // unfolding columns per tile (GEMM1 M, GEMM2 K)
constexpr int kTcRows = 128;     // rows i per staged chunk (GEMM1 K block, GEMM2 M)
constexpr int kTcThreads = 128;  // one warpgroup: thread 0 issues, all four warps drain TMEM
constexpr int kChunkBytes = kTcCols * kTcRows * 2;   // 32 KiB
constexpr int kHalfBytes = kChunkBytes / 2;           // one 64-column box
constexpr unsigned kWaitLimit = 1u << 26;

struct TcArgs {
  int I, R, RP;                // R padded to RP (multiple of 16)
  long long P, Q, J, ntiles;
  const float* L;              // basis I x R (FP32)
  float* Ypart;                // [gridDim.x][I][R]
  double* spart;               // [gridDim.x]
  int* err;                    // error flag (timeout)
};

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, LBO, SBO (bytes), SM100
// version bit, 128-byte swizzle.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, majors, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(map), "r"(mbar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 32 columns of fp32 from tensor memory.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Byte offset of element (row, col) in a K-major 128B-swizzled operand block
// whose rows are 128 bytes (64 bf16 of K) and whose 8-row groups are 1024 B apart.
__device__ __forceinline__ uint32_t sw128_off(int row, int kcol) {
  return (uint32_t)(row * 128 + ((((kcol * 2) >> 4) ^ (row & 7)) << 4) + ((kcol * 2) & 15));
}

}  // namespace

template <int RP>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_pass_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up: [4 chunks][Q operand][W operand][barriers]
  unsigned char* base = smem_raw;
  const uint32_t b0 = su32(base);
  const uint32_t pad = (1024u - (b0 & 1023u)) & 1023u;
  base += pad;
  const int nchunk = a.I / kTcRows;
  unsigned char* chunks = base;                                    // nchunk x 32 KiB
  unsigned char* qop = chunks + (size_t)nchunk * kChunkBytes;     // (I/64) x RP x 128 B
  unsigned char* wop = qop + (size_t)(a.I / 64) * RP * 128;        // 2 x RP x 128 B
  uint64_t* bars = reinterpret_cast<uint64_t*>(wop + 2 * RP * 128);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 4);
  __shared__ double red[32];
  __shared__ int s_fail;
  __shared__ uint32_t s_pend_bar, s_pend_par;   // barrier phase outstanding after a timeout

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_tma = su32(&bars[0]), bar_g1 = su32(&bars[1]), bar_g2 = su32(&bars[2]);
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_g1, 1);
    mbar_init(bar_g2, 1);
    s_fail = 0;
    s_pend_bar = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tensor memory: W (RP columns) + Y (nchunk x RP columns), power of two >= 32
  const uint32_t need = (uint32_t)(RP + nchunk * RP);
  uint32_t ncols = 32;
  while (ncols < need) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // Q operand (B of GEMM1: n = r, k = i), K-major, 128B swizzle, bf16
  for (int e = tid; e < a.I * RP; e += kTcThreads) {
    const int i = e / RP, r = e % RP;
    const float v = r < a.R ? a.L[(size_t)i * a.R + r] : 0.f;
    const int katom = i >> 6;
    __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(qop + (size_t)katom * RP * 128 +
                                                          sw128_off(r, i & 63));
    *dst = __float2bfloat16_rn(v);
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;
  const uint32_t t_w = tmem;                 // W: columns [0, RP)
  const uint32_t t_y = tmem + RP;            // Y chunk c: columns [RP + c*RP, ...)
  constexpr uint32_t kIdesc = idesc_bf16(128, RP, 0, 0);
  constexpr uint32_t kIdescMN = idesc_bf16(128, RP, 1, 0);
  double wsq = 0.0;
  uint32_t ph_tma = 0, ph_g1 = 0, ph_g2 = 0;
  int first = 1;

  for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const long long j0 = t * kTcCols;
    const long long p = j0 / a.Q, q0 = j0 - p * a.Q;
    // ---- TMA: the tile's nchunk chunks, two 64-column boxes each ----
    if (tid == 0 && !s_fail) {
      mbar_expect_tx(bar_tma, (uint32_t)(nchunk * kChunkBytes));
      for (int c = 0; c < nchunk; ++c)
        for (int h = 0; h < 2; ++h)
          tma_load_3d(su32(chunks + (size_t)c * kChunkBytes + h * kHalfBytes), &tmap, bar_tma,
                      (int)(q0 + h * 64), c * kTcRows, (int)p);
    }
    if (!mbar_wait(bar_tma, ph_tma) && tid == 0) {
      s_fail = 1;
      s_pend_bar = bar_tma;
      s_pend_par = ph_tma;
    }
    ph_tma ^= 1;
    // ---- GEMM1: W = B_t^T Q (M = 128 columns, K = I) ----
    if (tid == 0 && !s_fail) {
      fence_after();
      for (int c = 0; c < nchunk; ++c)
        for (int ks = 0; ks < kTcRows / 16; ++ks) {
          const uint32_t a_addr = su32(chunks + (size_t)c * kChunkBytes) + ks * 16 * 128;
          const uint64_t ad = desc_sw128(a_addr, kHalfBytes, 1024);   // MN-major: LBO = next 64 columns
          const int k = c * kTcRows + ks * 16;                          // global i
          const uint32_t b_addr = su32(qop) + (uint32_t)((k >> 6) * RP * 128 + ((k & 63) >> 4) * 32);
          const uint64_t bd = desc_sw128(b_addr, 16, 1024);
          mma_bf16(t_w, ad, bd, kIdescMN, (c | ks) ? 1u : 0u);
        }
      mma_commit(bar_g1);
    }
    __syncthreads();
    if (!mbar_wait(bar_g1, ph_g1) && tid == 0) {
      s_fail = 1;
      s_pend_bar = bar_g1;
      s_pend_par = ph_g1;
    }
    ph_g1 ^= 1;
    fence_after();
    // ---- W: TMEM -> registers -> bf16 K-major operand (n = r, k = column) ----
    {
      const int col = warp * 32 + lane;   // this thread's tile column (TMEM lane)
      const bool valid = j0 + col < a.J;
#pragma unroll
      for (int rb = 0; rb < RP; rb += 32) {
        float v[32];
        tmem_ld32(t_w + ((uint32_t)(warp * 32) << 16) + rb, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int r = rb + k;
          if (r >= RP) break;
          const float w = (valid && r < a.R) ? v[k] : 0.f;
          wsq += (double)w * w;
          __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(
              wop + (size_t)(col >> 6) * RP * 128 + sw128_off(r, col & 63));
          *dst = __float2bfloat16_rn(w);
        }
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    // ---- GEMM2: Y += B_t W (M = 128 rows per chunk, K = 128 columns) ----
    if (tid == 0 && !s_fail) {
      fence_after();
      for (int c = 0; c < nchunk; ++c)
        for (int ks = 0; ks < kTcCols / 16; ++ks) {
          const uint32_t a_addr = su32(chunks + (size_t)c * kChunkBytes) + (ks >> 2) * kHalfBytes +
                                  (ks & 3) * 32;
          const uint64_t ad = desc_sw128(a_addr, 16, 1024);
          const uint32_t b_addr = su32(wop) + (ks >> 2) * RP * 128 + (ks & 3) * 32;
          const uint64_t bd = desc_sw128(b_addr, 16, 1024);
          mma_bf16(t_y + c * RP, ad, bd, kIdesc, (first && ks == 0) ? 0u : 1u);
        }
      mma_commit(bar_g2);
    }
    __syncthreads();
    if (!mbar_wait(bar_g2, ph_g2) && tid == 0) {
      s_fail = 1;
      s_pend_bar = bar_g2;
      s_pend_par = ph_g2;
    }
    ph_g2 ^= 1;
    fence_after();
    first = 0;
    __syncthreads();
    if (s_fail) break;
  }

  // ---- Y partial: TMEM -> FP32 Ypart[bx][i][r] ----
  if (!s_fail && !first) {
    float* yp = a.Ypart + (size_t)blockIdx.x * a.I * a.R;
    for (int c = 0; c < nchunk; ++c) {
      const int i = c * kTcRows + warp * 32 + lane;
#pragma unroll
      for (int rb = 0; rb < RP; rb += 32) {
        float v[32];
        tmem_ld32(t_y + c * RP + ((uint32_t)(warp * 32) << 16) + rb, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int r = rb + k;
          if (r < a.R) yp[(size_t)i * a.R + r] = v[k];
        }
      }
    }
  } else if (first) {
    // no tile: the partial is zero
    float* yp = a.Ypart + (size_t)blockIdx.x * a.I * a.R;
    for (int e = tid; e < a.I * a.R; e += kTcThreads) yp[e] = 0.f;
  }
  const double tot = block_sum(wsq, red);
  if (tid == 0) {
    a.spart[blockIdx.x] = tot;
    if (s_fail) {
      atomicExch(a.err, 5);   // TALS_ETIMEOUT
      // let the copy or MMA group that timed out finish (bounded) before the
      // shared and tensor memory it targets is released
      if (s_pend_bar) mbar_wait(s_pend_bar, s_pend_par);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

bool tc_supported(const ModeView& v, int R) {
  return v.I % kTcRows == 0 && v.I <= 512 && v.Q % kTcCols == 0 && R >= 1 && R <= 64;
}

size_t tc_smem_bytes(long long I, int RP) {
  return 1024 + (size_t)(I / kTcRows) * kChunkBytes + (size_t)(I / 64) * RP * 128 +
         2 * (size_t)RP * 128 + 64;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

// Tensor map of a BF16 tensor viewed as (Q, I, P), boxes of 64 x 128 x 1, 128B swizzle.
bool tc_make_map(const void* Xb, const ModeView& v, CUtensorMap* map) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if ((uintptr_t)Xb % 16 != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)v.Q, (cuuint64_t)v.I, (cuuint64_t)v.P};
  cuuint64_t strides[2] = {(cuuint64_t)v.Q * 2, (cuuint64_t)v.I * v.Q * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)kTcRows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(Xb), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_tc_pass(const void* Xb, const ModeView& v, int R, const float* L, float* Ypart,
                           double* spart, int* err, int grid, cudaStream_t s) {
  if (!tc_supported(v, R)) return cudaErrorInvalidValue;
  CUtensorMap map;
  if (!tc_make_map(Xb, v, &map)) return cudaErrorInvalidValue;
  const int RP = ((R + 15) / 16) * 16;
  TcArgs a;
  a.I = (int)v.I;
  a.R = R;
  a.RP = RP;
  a.P = v.P;
  a.Q = v.Q;
  a.J = v.J();
  a.ntiles = (v.J() + kTcCols - 1) / kTcCols;
  a.L = L;
  a.Ypart = Ypart;
  a.spart = spart;
  a.err = err;
  const size_t smem = tc_smem_bytes(v.I, RP);
  void* fn = nullptr;
  switch (RP) {
    case 16: fn = (void*)&tc_pass_kernel<16>; break;
    case 32: fn = (void*)&tc_pass_kernel<32>; break;
    case 48: fn = (void*)&tc_pass_kernel<48>; break;
    case 64: fn = (void*)&tc_pass_kernel<64>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  grid = (int)std::min<long long>(grid, a.ntiles);
  void* args[] = {&map, &a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), args, smem, s);
}

// FP32 -> BF16 copy (round to nearest even), vectorised by 4.
__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, size_t n) {
  const size_t i4 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t i = i4; i < n; i += stride) {
    if (i + 3 < n) {
      const float4 v = *reinterpret_cast<const float4*>(x + i);
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
      *reinterpret_cast<__nv_bfloat162*>(y + i) = lo;
      *reinterpret_cast<__nv_bfloat162*>(y + i + 2) = hi;
    } else {
      for (size_t k = i; k < n; ++k) y[k] = __float2bfloat16_rn(x[k]);
    }
  }
}

cudaError_t launch_to_bf16(const float* x, void* y, size_t n, int sms, cudaStream_t s) {
  const int threads = 256;
  const long long blocks = std::min<long long>((long long)sms * 8, (long long)((n / 4 + threads - 1) / threads) + 1);
  to_bf16_kernel<<<(unsigned)blocks, threads, 0, s>>>(x, (__nv_bfloat16*)y, n);
  return cudaGetLastError();
}

}  // namespace tals
