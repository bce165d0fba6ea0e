// Fused ALS sweep pass on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory.
//
// Same computation as the CUDA-core pass (Alg. 3 R-update and L-update fused
// as in Eq. 2.2): per tile of 64 unfolding columns,
//   GEMM1  W_t (64 x R) = B_t^T (64 x I) . Q (I x R)      -> TMEM, fp32 (M = 64)
//   GEMM2  Y   (I x R) += B_t  (I x 64) . W_t (64 x R)    -> TMEM, fp32 (M = 128)
// B_t is a BF16 copy of the tensor, staged by TMA with 128-byte swizzle in
// 64-column x 128-row chunks (one box, 16 KiB). The staged chunk is read by
// GEMM1 as an MN-major A operand (m = column, k = row i) and by GEMM2 as a
// K-major A operand (m = row i, k = column): for 16-bit types the 128B-swizzled
// layout with 128-byte rows is a canonical layout for both majors. A tile stays
// in shared memory from its load until GEMM2 has used it, so the tensor crosses
// HBM -> SM exactly once per sweep. W_t goes TMEM -> registers -> BF16 ->
// shared memory (K-major, 128B swizzle) between the two GEMMs; Y stays in TMEM
// across all the CTA's tiles and is written once as a per-CTA FP32 partial,
// reduced in FP64 by the same kernel as the CUDA-core path.
//
// Warp-specialised: one producer warp issues the TMA loads, two MMA warps issue
// the two GEMMs, four warps run the epilogue; completion is tracked with
// mbarriers (tcgen05.commit for the MMAs). Every wait is bounded: on timeout
// the CTA records an error code, stops issuing work, waits (again bounded) for
// the copies and MMAs it already issued and frees its tensor memory before it
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tcgen05.cuh"

namespace tals {

constexpr int kTcCols = 64;      // unfolding columns per tile (GEMM1 M, GEMM2 K)
constexpr int kTcRows = 128;     // rows i per staged chunk (GEMM1 K block, GEMM2 M)
constexpr int kChunkBytes = kTcCols * kTcRows * 2;   // 16 KiB, one TMA box

struct TcArgs {
  int I, R, RP;                // R padded to RP (multiple of 16)
  long long P, Q, J, ntiles;
  const float* L;              // basis I x R (FP32)
  float* Ypart;                // [gridDim.x][I][R]
  double* spart;               // [gridDim.x]
  int* err;                    // error flag (timeout)
  int init;                    // Sec. 4 init: W_t is the seeded sketch S_t, no GEMM1
  uint64_t sketch;             // sketch state (seed and mode)
};

using namespace tc;

namespace {

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return idesc(kFmtBF16, M, N, a_mn, b_mn);
}

}  // namespace

// Warp roles (224 threads):
//   warps 0-3  epilogue: W_t (TMEM) -> bf16 operand and ||W||^2; final Y
//   warp 4     producer: TMA of tile t's chunks into the chunk ring
//   warp 5     GEMM1 issuer (W_t into TMEM W buffer t % 2)
//   warp 6     GEMM2 issuer (Y += B_t W_t); it releases the tile's ring slots
// A ring slot is held from its load until GEMM2 has used it; the producer runs
// ahead by whatever the ring holds beyond the tile waiting for GEMM2.
// An M = 64 accumulator puts row m in TMEM lane (m / 16) * 32 + m % 16, so
// lanes 0-15 of each epilogue warp hold W_t's rows.
constexpr int kTcThreads = 224;
constexpr int kMaxSlots = 16;

template <int RP>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_pass_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap ymap,
                   TcArgs a, int ns, int y_tma) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw;
  base += (1024u - (su32(base) & 1023u)) & 1023u;
  const int nchunk = a.I / kTcRows;
  unsigned char* ring = base;                                           // ns x 16 KiB
  unsigned char* qop = ring + (size_t)ns * kChunkBytes;                 // (I/64) x RP x 128 B
  unsigned char* wop = qop + (size_t)(a.I / 64) * RP * 128;             // 2 x RP x 128 B
  uint64_t* bars = reinterpret_cast<uint64_t*>(wop + 2 * RP * 128);
  uint64_t* full = bars;                     // [kMaxSlots] chunk landed
  uint64_t* empty = bars + kMaxSlots;        // [kMaxSlots] GEMM2 done with the chunk
  uint64_t* wfull = bars + 2 * kMaxSlots;    // [2] GEMM1 done -> W in TMEM buffer
  uint64_t* wfree = wfull + 2;               // [2] epilogue read the TMEM W buffer
  uint64_t* opfull = wfree + 2;              // [2] bf16 W operand written
  uint64_t* opfree = opfull + 2;             // [2] GEMM2 done reading the operand
  uint64_t* ydone = opfree + 2;              // [1] all GEMM2 MMAs done
  uint64_t* g1done = ydone + 1;              // [1] all GEMM1 MMAs done
  uint64_t* ystaged = g1done + 1;            // [1] final Y staged in shared memory
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(ystaged + 1);
  __shared__ double red[32];
  __shared__ int s_fail;
  volatile int* vfail = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nt = a.ntiles > blockIdx.x ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (tid == 0) {
    for (int k = 0; k < kMaxSlots; ++k) {
      mbar_init(su32(&full[k]), 1);
      mbar_init(su32(&empty[k]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&wfull[b]), 1);
      mbar_init(su32(&wfree[b]), 128);
      mbar_init(su32(&opfull[b]), 128);
      mbar_init(su32(&opfree[b]), 1);
    }
    mbar_init(su32(ydone), 1);
    mbar_init(su32(g1done), 1);
    mbar_init(su32(ystaged), 128);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t need = (uint32_t)(2 * RP + nchunk * RP);
  uint32_t ncols = 32;
  while (ncols < need) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;
  const uint32_t t_w0 = tmem, t_y = tmem + 2 * RP;   // W buffers at 0 and RP; Y chunks after
  double wsq = 0.0;

  if (warp != 4) {
    // The basis as GEMM1's B operand (K-major, 128B swizzle): every warp but the
    // producer, which starts streaming at once. One unit = 8 consecutive rows i
    // of one column r -> one 16-byte store; lanes take consecutive r, so each of
    // the 8 loads of a unit is coalesced across the warp.
    const int ft = tid < 128 ? tid : tid - 32;   // 0..191
    constexpr int kFill = kTcThreads - 32;
    constexpr int kUn = 4;
    const int nunits = a.init ? 0 : (a.I / 8) * RP;   // no basis operand in the init pass
    for (int u0 = ft; u0 < nunits; u0 += kFill * kUn) {
      float x[kUn][8];
#pragma unroll
      for (int w = 0; w < kUn; ++w) {
        const int u = u0 + w * kFill;
        const int r = u % RP, i0 = (u / RP) * 8;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          x[w][k] = (u < nunits && r < a.R) ? __ldg(a.L + (size_t)(i0 + k) * a.R + r) : 0.f;
      }
#pragma unroll
      for (int w = 0; w < kUn; ++w) {
        const int u = u0 + w * kFill;
        if (u >= nunits) break;
        const int r = u % RP, i0 = (u / RP) * 8;
        uint4 pk;
        pk.x = pack_bf16(x[w][0], x[w][1]);
        pk.y = pack_bf16(x[w][2], x[w][3]);
        pk.z = pack_bf16(x[w][4], x[w][5]);
        pk.w = pack_bf16(x[w][6], x[w][7]);
        *reinterpret_cast<uint4*>(qop + (size_t)(i0 >> 6) * RP * 128 + r * 128 +
                                  ((((i0 & 63) >> 3) ^ (r & 7)) << 4)) = pk;
      }
    }
    fence_async_smem();
    asm volatile("bar.sync 1, %0;" ::"r"(kFill) : "memory");
  }

  if (warp == 4) {
    // ---------------- producer (whole warp waits, lane 0 issues) ----------------
    int slot = 0;
    uint32_t ph = 0;
    long long fills = 0;
    bool ok = true;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      const long long j0 = (blockIdx.x + lt * gridDim.x) * kTcCols;
      const long long p = j0 / a.Q, q0 = j0 - p * a.Q;
      for (int c = 0; c < nchunk && ok; ++c) {
        ok = mbar_wait_b(su32(&empty[slot]), ph ^ 1u, vfail);
        if (!ok) break;
        if (lane == 0) {
          mbar_expect_tx(su32(&full[slot]), (uint32_t)kChunkBytes);
          tma_load_3d(su32(ring + (size_t)slot * kChunkBytes), &tmap, su32(&full[slot]), (int)q0,
                      c * kTcRows, (int)p);
        }
        __syncwarp();
        ++fills;
        if (++slot == ns) {
          slot = 0;
          ph ^= 1u;
        }
      }
    }
    // every copy issued must have landed before the shared memory is released
    if (lane == 0) {
      for (int sl = 0; sl < ns && sl < fills; ++sl) {
        const long long nfill = fills / ns + (sl < fills % ns ? 1 : 0);
        const uint32_t par = (uint32_t)((nfill - 1) & 1);
        const long long t0 = clock64();
        while (!mbar_try(su32(&full[sl]), par) && clock64() - t0 < (1ll << 30)) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 5) {
    // ---------------- GEMM1 issuer: W_t = B_t^T Q (M = 64 columns) ----------------
    constexpr uint32_t kIdesc1 = idesc_bf16(64, RP, 1, 0);
    int slot = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (long long lt = 0; lt < nt && ok && !a.init; ++lt) {
      const int wb = (int)(lt & 1);
      const uint32_t use = (uint32_t)(lt >> 1);
      if (lt >= 2) ok = mbar_wait_b(su32(&wfree[wb]), (use - 1) & 1u, vfail);
      fence_after();
      for (int c = 0; c < nchunk && ok; ++c) {
        ok = mbar_wait_b(su32(&full[slot]), ph, vfail);
        if (!ok) break;
        fence_after();
        if (lane == 0) {
          const uint32_t abase = su32(ring + (size_t)slot * kChunkBytes);
#pragma unroll
          for (int ks = 0; ks < kTcRows / 16; ++ks) {
            const uint64_t ad = desc_sw128(abase + ks * 16 * 128, kChunkBytes, 1024);
            const int k = c * kTcRows + ks * 16;
            const uint64_t bd = desc_sw128(
                su32(qop) + (uint32_t)((k >> 6) * RP * 128 + ((k & 63) >> 4) * 32), 16, 1024);
            mma_bf16(t_w0 + wb * RP, ad, bd, kIdesc1, (c | ks) ? 1u : 0u);
          }
        }
        __syncwarp();
        if (++slot == ns) {
          slot = 0;
          ph ^= 1u;
        }
      }
      if (ok && lane == 0) mma_commit(su32(&wfull[wb]));
      __syncwarp();
    }
    if (lane == 0) mma_commit(su32(g1done));
    __syncwarp();
  } else if (warp == 6) {
    // ---------------- GEMM2 issuer: Y += B_t W_t (M = 128 rows) ----------------
    constexpr uint32_t kIdesc2 = idesc_bf16(128, RP, 0, 0);
    int slot = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      const int wb = (int)(lt & 1);
      const uint32_t use = (uint32_t)(lt >> 1);
      ok = mbar_wait_b(su32(&opfull[wb]), use & 1u, vfail);
      fence_after();
      const uint32_t bbase = su32(wop + (size_t)wb * RP * 128);
      for (int c = 0; c < nchunk && ok; ++c) {
        // already complete (GEMM1 waited on it; the slot is not refilled before
        // this warp releases it): makes the TMA data visible to this thread too
        ok = mbar_wait_b(su32(&full[slot]), ph, vfail);
        if (!ok) break;
        fence_after();
        if (lane == 0) {
          const uint32_t abase = su32(ring + (size_t)slot * kChunkBytes);
#pragma unroll
          for (int ks = 0; ks < kTcCols / 16; ++ks) {
            const uint64_t ad = desc_sw128(abase + ks * 32, 16, 1024);
            const uint64_t bd = desc_sw128(bbase + ks * 32, 16, 1024);
            mma_bf16(t_y + c * RP, ad, bd, kIdesc2, (lt == 0 && ks == 0) ? 0u : 1u);
          }
          mma_commit(su32(&empty[slot]));
        }
        __syncwarp();
        if (++slot == ns) {
          slot = 0;
          ph ^= 1u;
        }
      }
      if (ok && lane == 0) mma_commit(su32(&opfree[wb]));
      __syncwarp();
    }
    if (lane == 0) mma_commit(su32(ydone));
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 0-3 ----------------
    const bool wrow = lane < 16;               // this lane holds a row of W_t
    const int m = warp * 16 + (lane & 15);     // tile column of that row
    bool ok = true;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      const int wb = (int)(lt & 1);
      const uint32_t use = (uint32_t)(lt >> 1);
      if (a.init) {
        // Sec. 4: W_t = S restricted to the tile's columns, drawn from the
        // counter-based generator (entry (j, r) from output j R + r)
        if (lt >= 2) ok = mbar_wait_b(su32(&opfree[wb]), (use - 1) & 1u, vfail);
        if (!ok) break;
        {
          // lanes l and l + 16 share row m of W_t, half of its ranks each: the
          // generator is integer-heavy, and every tile of the pass waits for it
          const long long j = (blockIdx.x + lt * gridDim.x) * kTcCols + m;
          unsigned char* wrowp = wop + (size_t)wb * RP * 128 + (m & 7) * 2;
          const int c8 = m >> 3;
          const int rbeg = (lane >> 4) * (RP / 2);
#pragma unroll 4
          for (int rr = 0; rr < RP / 2; ++rr) {
            const int r = rbeg + rr;
            const float w = r < a.R ? sketch_entry(a.sketch, (uint64_t)j, a.R, r) : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(wrowp + r * 128 + ((c8 ^ (r & 7)) << 4)) =
                __float2bfloat16_rn(w);
          }
        }
        fence_async_smem();
        mbar_arrive(su32(&opfull[wb]));
        continue;
      }
      ok = mbar_wait_b(su32(&wfull[wb]), use & 1u, vfail);
      if (!ok) break;
      fence_after();
      float v[RP];
#pragma unroll
      for (int rb = 0; rb < RP; rb += 32) {
        float t32[32];
        tmem_ld32(t_w0 + wb * RP + ((uint32_t)(warp * 32) << 16) + rb, t32);
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (rb + k < RP) v[rb + k] = t32[k];
      }
      fence_before();
      mbar_arrive(su32(&wfree[wb]));
      if (lt >= 2) ok = mbar_wait_b(su32(&opfree[wb]), (use - 1) & 1u, vfail);
      if (!ok) break;
      if (wrow) {
        unsigned char* wrowp = wop + (size_t)wb * RP * 128 + (m & 7) * 2;
        const int c8 = m >> 3;
        float tsq = 0.f;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const float w = r < a.R ? v[r] : 0.f;
          tsq = fmaf(w, w, tsq);
          *reinterpret_cast<__nv_bfloat16*>(wrowp + r * 128 + ((c8 ^ (r & 7)) << 4)) =
              __float2bfloat16_rn(w);
        }
        wsq += (double)tsq;
      }
      fence_async_smem();
      mbar_arrive(su32(&opfull[wb]));
    }
    // final Y: wait for every GEMM2, then TMEM -> FP32 partials
    float* yp = a.Ypart + (size_t)blockIdx.x * a.I * a.R;
    if (ok && mbar_wait_b(su32(ydone), 0u, vfail)) {
      fence_after();
      if (y_tma) {
        // Stage 128 x 32 boxes with 128B swizzle in the (now idle) ring and
        // operand memory, then one thread stores them with TMA; the swizzle
        // spreads each warp's 16-byte writes over all banks.
        const int nxb = (a.R + 31) / 32;
        const int row = warp * 32 + lane;
        for (int c = 0; c < nchunk; ++c) {
#pragma unroll
          for (int rb = 0; rb < RP; rb += 32) {
            if (rb / 32 >= nxb) break;
            float t32[32];
            tmem_ld32(t_y + c * RP + ((uint32_t)(warp * 32) << 16) + rb, t32);
            unsigned char* box = base + (size_t)(c * nxb + rb / 32) * 16384 + row * 128;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<float4*>(box + ((j ^ (row & 7)) << 4)) =
                  make_float4(t32[4 * j], t32[4 * j + 1], t32[4 * j + 2], t32[4 * j + 3]);
          }
        }
        fence_async_smem();
        mbar_arrive(su32(ystaged));
        if (tid == 0 && mbar_wait_b(su32(ystaged), 0u, vfail)) {
          for (int c = 0; c < nchunk; ++c)
            for (int xb = 0; xb < nxb; ++xb)
              tma_store_2d(&ymap, su32(base + (size_t)(c * nxb + xb) * 16384), xb * 32,
                           (int)(blockIdx.x * a.I + c * kTcRows));
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
      } else {
        for (int c = 0; c < nchunk; ++c) {
          const int i = c * kTcRows + warp * 32 + lane;
#pragma unroll
          for (int rb = 0; rb < RP; rb += 32) {
            float t32[32];
            tmem_ld32(t_y + c * RP + ((uint32_t)(warp * 32) << 16) + rb, t32);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int r = rb + k;
              if (r < a.R) yp[(size_t)i * a.R + r] = t32[k];
            }
          }
        }
      }
    }
  }
  const double tot = block_sum(wsq, red);
  if (tid == 0) {
    a.spart[blockIdx.x] = tot;
    if (*vfail) atomicExch(a.err, 5);   // TALS_ETIMEOUT
  }
  // nothing may still write the shared or tensor memory released below: after a
  // failure, wait (bounded) for both MMA groups issued so far
  if (*vfail && (tid == 160 || tid == 192)) {
    const uint32_t b = tid == 160 ? su32(g1done) : su32(ydone);
    const long long t0 = clock64();
    while (!mbar_try(b, 0u) && clock64() - t0 < (1ll << 30)) {
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

int tc_slots(long long I, int RP);

bool tc_supported(const ModeView& v, int R) {
  return v.I % kTcRows == 0 && v.I <= 512 && v.Q % kTcCols == 0 && R >= 1 && R <= 64 &&
         tc_slots(v.I, ((R + 15) / 16) * 16) >= v.I / kTcRows;
}

size_t tc_smem_bytes(long long I, int RP, int ns) {
  return 1024 + (size_t)ns * kChunkBytes + (size_t)(I / 64) * RP * 128 + 2 * (size_t)RP * 128 +
         (2 * kMaxSlots + 11) * 8 + 16;
}

// Ring slots that fit next to the operands (at least one tile's worth is needed).
int tc_slots(long long I, int RP) {
  const size_t fixed = 1024 + (size_t)(I / 64) * RP * 128 + 2 * (size_t)RP * 128 + 512;
  const size_t cap = 227 * 1024 - 2048;   // dynamic smem budget (static smem: red + flag)
  if (fixed >= cap) return 0;
  return (int)std::min<size_t>(kMaxSlots, (cap - fixed) / kChunkBytes);
}

EncodeTiledFn tma_encode_fn() {
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

// Tensor map of a BF16 tensor viewed as (Q, I, P), boxes of 64 x 128 x 1, 128B swizzle.
bool tc_make_map(const void* Xb, const ModeView& v, CUtensorMap* map) {
  EncodeTiledFn fn = tma_encode_fn();
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

// Tensor map of the per-CTA FP32 partials Ypart viewed as (R, rows), boxes of
// 32 x 128 with 128B swizzle (the staging layout of the final Y store).
bool tc_make_ymap(float* Ypart, int R, long long rows, CUtensorMap* map) {
  EncodeTiledFn fn = tma_encode_fn();
  if (!fn) return false;
  if ((uintptr_t)Ypart % 16 != 0 || R % 4 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)R * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)kTcRows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Ypart, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_tc_pass(const void* Xb, const ModeView& v, int R, const float* L, float* Ypart,
                           double* spart, int* err, int grid, cudaStream_t s, int init,
                           uint64_t sketch) {
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
  a.init = init;
  a.sketch = sketch;
  const int ns = tc_slots(v.I, RP);
  if (ns < v.I / kTcRows) return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes(v.I, RP, ns);
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
  // final Y through TMA when the rows are 16-byte multiples and the staged
  // boxes fit in the ring and basis-operand memory
  CUtensorMap ymap;
  std::memset(&ymap, 0, sizeof(ymap));
  const size_t nbox = (size_t)(v.I / kTcRows) * ((R + 31) / 32);
  const size_t region = (size_t)ns * kChunkBytes + (size_t)(v.I / 64) * RP * 128;
  int y_tma = (nbox * 16384 <= region && tc_make_ymap(Ypart, R, (long long)grid * v.I, &ymap)) ? 1 : 0;
  int ns_ = ns;
  void* args[] = {&map, &ymap, &a, (void*)&ns_, (void*)&y_tma};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), args, smem, s);
}

// FP32 -> BF16 copy (round to nearest even), vectorised by 4.
// FP32 -> BF16 copy (round to nearest even), vectorised by 4. With sq != null
// each block also writes the FP64 sum of squares of the FP32 elements it read
// (||B||^2 for the stop rule, from the original data): exact products
// (x^2 = p + e via FMA) in a Neumaier-compensated FP32 sum per thread, then a
// fixed-order FP64 block sum.
__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, size_t n,
                               double* __restrict__ sq) {
  __shared__ double red[32];
  const size_t i4 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x * 4;
  float hi = 0.f, lo = 0.f;
  auto acc = [&](float v) {
    const float p = v * v, pe = fmaf(v, v, -p);
    const float t = hi + p;
    lo += (hi >= p ? (hi - t) + p : (p - t) + hi) + pe;
    hi = t;
  };
  for (size_t i = i4; i < n; i += stride) {
    if (i + 3 < n) {
      const float4 v = *reinterpret_cast<const float4*>(x + i);
      __nv_bfloat162 l2 = __floats2bfloat162_rn(v.x, v.y), h2 = __floats2bfloat162_rn(v.z, v.w);
      *reinterpret_cast<__nv_bfloat162*>(y + i) = l2;
      *reinterpret_cast<__nv_bfloat162*>(y + i + 2) = h2;
      if (sq) {
        acc(v.x);
        acc(v.y);
        acc(v.z);
        acc(v.w);
      }
    } else {
      for (size_t k = i; k < n; ++k) {
        y[k] = __float2bfloat16_rn(x[k]);
        if (sq) acc(x[k]);
      }
    }
  }
  if (sq) {
    const double t = block_sum((double)hi + (double)lo, red);
    if (threadIdx.x == 0) sq[blockIdx.x] = t;
  }
}

// Failure path of the bounded waits, exercised on purpose: one thread waits on
// an initialised mbarrier that nothing arrives at (phase 0 never completes),
// gives up after `limit` cycles through the same helper as the pass, records
// TALS_ETIMEOUT and the kernel returns normally.
__global__ void wait_timeout_probe(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    mbar_init(su32(&bar), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* vf = &s_fail;
    if (!mbar_wait_limit(su32(&bar), 0u, vf, limit)) atomicExch(err, 5);   // TALS_ETIMEOUT
  }
}

cudaError_t launch_wait_timeout_probe(int* err, long long limit_cycles, cudaStream_t s) {
  wait_timeout_probe<<<1, 32, 0, s>>>(err, limit_cycles);
  return cudaGetLastError();
}

int to_bf16_blocks(size_t n, int sms) {
  const int threads = 256;
  return (int)std::min<long long>((long long)sms * 8, (long long)((n / 4 + threads - 1) / threads) + 1);
}

cudaError_t launch_to_bf16(const float* x, void* y, size_t n, int sms, cudaStream_t s, double* sq) {
  to_bf16_kernel<<<(unsigned)to_bf16_blocks(n, sms), 256, 0, s>>>(x, (__nv_bfloat16*)y, n, sq);
  return cudaGetLastError();
}

}  // namespace tals
