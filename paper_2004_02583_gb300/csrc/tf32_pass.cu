// Split-precision (3xTF32) ALS sweep on the 5th-generation tensor cores.
//
// The FP32 products of Alg. 3 -- the R-update W = B_(n)^T Q and the L-update
// Y = B_(n) W, which together form B B^T Q of Eq. 2.2 -- run on tcgen05
// (kind::tf32) at FP32-level accuracy: every operand x is split as x = hi + lo
// with hi = tf32(x) and lo = tf32(x - hi) (round to nearest), and a product a b
// is formed as a_hi b_hi + a_hi b_lo + a_lo b_hi (the omitted a_lo b_lo term is
// below 2^-22 |a b|), accumulated in FP32 in tensor memory.
//
// Two passes per sweep, each streaming the tensor once through TMA:
//   pass 1 (W pass)  W = B_(n)^T Q. Tiles of 128 unfolding columns (MMA M = 128),
//                    K = I in stages of 32 rows; the split basis [Q_hi | Q_lo]
//                    (N = 2 RP) streams beside each stage. The tensor cores
//                    round each FP32 result toward zero (measured: a relative
//                    bias of about 3e-8 per accumulating MMA, -4e-6 on ||W||^2
//                    over K = 512, with sweep-to-sweep noise large enough to
//                    move the Eq. 5.01 stop rule), so every K-step's products
//                    land in a fresh tensor-memory buffer, the two correction
//                    terms in columns of their own, and the epilogue sums them
//                    in registers with rounding to nearest. W is written
//                    in the P x R x Q layout, i.e. as the tensor B x_n Q^T
//                    (Alg. 5's truncation), with ||W||^2.
//   pass 2 (Y pass)  Y = B_(n) W. Blocks of 32 columns (MMA K), rows in stages of
//                    128 (MMA M); Y stays in tensor memory for every row of the
//                    mode and is written once as a per-CTA FP32 partial. In init
//                    mode the W block is the Sec. 4 sketch S and the pass also
//                    sums ||B||^2.
// The split of each staged tile into hi and lo planes runs on four warps of
// CUDA cores between the TMA landing and the MMAs. The single-read fused form
// of the BF16 pass does not fit here: a resident FP32 tile at I = 512 beside
// the split basis exceeds the shared memory of an SM.
//
// Views: the mode's unfolding columns j = p Q + q with Q a multiple of 32, so a
// 32-column box never crosses p; the tensor is read in place through a 3-D map
// (Q, I, P). Both MMA operands are K-major (kind::tf32 takes no MN-major
// operand here): pass 1's split step also transposes each landed stage. Warp
// roles: warps 0-3 read tensor memory (W tiles, final Y), warps 4-7 split the
// staged tiles, warp 8 issues TMA, warp 9 issues the MMAs; in pass 2 warps 10-11
// prepare the W blocks. Every wait is clock-bounded: on timeout the CTA records
// TALS_ETIMEOUT, stops issuing, waits (bounded) for its copies and MMAs and
// frees its tensor memory.
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tcgen05.cuh"

namespace tals {

using namespace tc;

namespace {

constexpr int kT32Threads = 320;    // pass 1
constexpr int kT32Threads2 = 384;   // pass 2: two more warps prepare the W blocks
constexpr int kMaxStages = 8;
constexpr int kKC = 32;                      // pass 1: rows per stage (4 MMA K-steps of 8)
constexpr int kBox1 = 32 * kKC * 4;          // pass 1: one 32-column box, 4 KiB
constexpr int kStage1 = 4 * kBox1;           // pass 1: 128 columns x 32 rows, 16 KiB
constexpr int kRows2 = 128;                  // pass 2: rows per stage (MMA M)
constexpr int kStage2 = 32 * kRows2 * 4;     // pass 2: 32 columns x 128 rows, 16 KiB
constexpr int kSmemCap = 227 * 1024;
constexpr int kMaxDB = 4;                    // pass 1: K-step product buffers in tensor memory

struct T32Args {
  int I, R, RP;
  long long P, Q, J;
  int nkc;              // pass 1: stages per tile, ceil(I / 32)
  int nch;              // pass 2: 128-row chunks, ceil(I / 128) (one per CTA row of the grid)
  long long ntiles;     // pass 1: 128-column tiles; pass 2: 32-column blocks
  const float* QS;      // pass 1: split basis, nkc x [2 RP rows][32] (128B-swizzled)
  const float* L;       // pass 2: the FP32 basis Q (I x R), for the residual
  float* W;             // pass 1: W (P x R x Q)
  float* Ypart;         // pass 2: [gridDim.y][I][R]
  double* spart;        // pass 1: [gridDim.x] ||W||^2; pass 2: [gridDim.y][gridDim.x] the
                        // residual ||B - Q W^T||^2 (init: ||B||^2)
  int* err;
  int init;             // pass 2: W block = sketch S (Sec. 4)
  uint64_t sketch;
  const ModeState* st;  // skip the pass once the mode's stop rule has fired (may be null)
  int flush;            // K-steps (of 8) accumulated in tensor memory before the registers take them
};

// Optional cycle trace of the passes' roles (builds with -DT32_TRACE only): per
// kernel, warp and wait site, the clock cycles spent, summed over CTAs.
#ifdef T32_TRACE
__device__ unsigned long long g_t32_trace[2][12][12];
#define T32_TRACE_DECL long long trc[12] = {}; const long long trc0 = clock64();
#define TWAIT(site, call)                                   \
  ([&]() {                                                  \
    const long long _t0 = clock64();                        \
    const bool _r = (call);                                 \
    trc[site] += clock64() - _t0;                           \
    return _r;                                              \
  }())
#define T32_TRACE_FLUSH(kern)                                                        \
  trc[11] = clock64() - trc0;                                                        \
  if ((threadIdx.x & 31) == 0)                                                       \
    for (int _k = 0; _k < 12; ++_k)                                                  \
      atomicAdd(&g_t32_trace[kern][threadIdx.x >> 5][_k], (unsigned long long)trc[_k]);
#else
#define T32_TRACE_DECL
#define TWAIT(site, call) (call)
#define T32_TRACE_FLUSH(kern)
#endif

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return p + ((1024u - (su32(p) & 1023u)) & 1023u);
}

// Exact square x^2 = p + e (FMA) into a Neumaier-compensated FP32 sum.
__device__ __forceinline__ void acc_sq(float x, float& hi, float& lo) {
  const float p = x * x, pe = fmaf(x, x, -p);
  const float t = hi + p;
  lo += (hi >= p ? (hi - t) + p : (p - t) + hi) + pe;
  hi = t;
}

__device__ __forceinline__ float4 split4(float4& x) {
  float4 l;
  float h;
  h = to_tf32(x.x); l.x = to_tf32(x.x - h); x.x = h;
  h = to_tf32(x.y); l.y = to_tf32(x.y - h); x.y = h;
  h = to_tf32(x.z); l.z = to_tf32(x.z - h); x.z = h;
  h = to_tf32(x.w); l.w = to_tf32(x.w - h); x.w = h;
  return l;
}

// Split `nf` floats of a staged tile (layout-agnostic: the lo plane has the hi
// plane's layout) by the 128 split threads (t = 0..127): hi in place, lo beside.
// With norm, the squares of the original values go into (sh, sl).
template <int NF>
__device__ __forceinline__ void split_tile(float* hi, float* lo, int t, bool norm, float& sh,
                                           float& sl) {
  static_assert(NF % (128 * 4 * 8) == 0, "tile size");
#pragma unroll 1
  for (int e0 = t * 4; e0 < NF; e0 += 128 * 4 * 8) {
    float4 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = *reinterpret_cast<const float4*>(hi + e0 + u * 512);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (norm) {
        acc_sq(x[u].x, sh, sl);
        acc_sq(x[u].y, sh, sl);
        acc_sq(x[u].z, sh, sl);
        acc_sq(x[u].w, sh, sl);
      }
      const float4 l = split4(x[u]);
      *reinterpret_cast<float4*>(hi + e0 + u * 512) = x[u];
      *reinterpret_cast<float4*>(lo + e0 + u * 512) = l;
    }
  }
}

// Byte offset of element (row n, column k) in a K-major 128B-swizzled operand
// whose rows are 128 bytes (32 FP32 values along K).
__device__ __forceinline__ uint32_t sw_off(int n, int k) {
  return (uint32_t)n * 128u + ((uint32_t)(((k >> 2) ^ (n & 7))) << 4) + (uint32_t)(k & 3) * 4u;
}

// FP64 sum of the 128 split threads' compensated pairs (named barrier 1 among
// them); valid in split thread 0.
__device__ __forceinline__ double split_sum(float sh, float sl, double* red4, int t) {
  double v = warp_sum((double)sh + (double)sl);
  if ((t & 31) == 0) red4[t >> 5] = v;
  asm volatile("bar.sync 1, 128;" ::: "memory");
  return t == 0 ? red4[0] + red4[1] + red4[2] + red4[3] : 0.0;
}

// ---------------------------------------------------------------------------
// Pass 1: W = B^T Q (3xTF32), ||W||^2
//
// Three rings decouple the stages. Raw slots receive the tensor by TMA and are
// released as soon as the split threads hold their column in registers, so a raw
// slot recycles after one TMA round trip and many bytes stay in flight. The A
// operand stages live in tensor memory: each split thread stores the hi and lo
// planes of its column (row m of A) into its own lane, and the MMAs read A from
// there -- no shared-memory operand traffic, and an MMA with A in tensor memory
// issues in ~46 cycles against ~75 from shared memory (measured). Beside each A
// stage, a shared-memory slot holds the stage's rows of the split basis (the B
// operand), released with it. Ring positions are kept as counters: a 64-bit
// division per stage cost more than the stage's MMAs.
// ---------------------------------------------------------------------------
// The raw stage is row-major without swizzle: one box [32 rows][128 columns]
// (wide), or four boxes [32 rows][32 columns] (narrow views, Q % 128 != 0). Thread
// t = tile column m reads its 32 values; a warp reads 32 consecutive floats of a
// row per load (conflict-free).
__device__ __forceinline__ void t32_read_col(const unsigned char* raw, int t, bool wide, float (&v)[32]) {
  const float* base = reinterpret_cast<const float*>(raw) + (wide ? t : (t >> 5) * 1024 + (t & 31));
  const int pitch = wide ? 128 : 32;
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = base[k * pitch];
}

// Column m of the stage split into hi and lo (32 values each, as raw 32-bit words
// for the tensor-memory stores).
__device__ __forceinline__ void t32_split_col(const float (&v)[32], uint32_t (&hi)[32], uint32_t (&lo)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float h = to_tf32(v[k]);
    hi[k] = __float_as_uint(h);
    lo[k] = __float_as_uint(to_tf32(v[k] - h));
  }
}

template <int RP>
__global__ void __launch_bounds__(kT32Threads, 1)
    t32_wpass_kernel(const __grid_constant__ CUtensorMap bmap, T32Args a, int nr, int no, int nq) {
  if (a.st != nullptr && a.st->done) return;   // uniform early exit, before any barrier
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  constexpr uint32_t kQB = 2 * RP * 128;            // split basis of one stage
  unsigned char* raw = base;                                      // nr x 16 KiB
  unsigned char* qsr = raw + (size_t)nr * kStage1;                // no x kQB
  uint64_t* bars = reinterpret_cast<uint64_t*>(qsr + (size_t)nq * kQB);
  uint64_t* rfull = bars;                     // raw stage landed (tx)
  uint64_t* rempty = rfull + kMaxStages;      // raw stage read by the split threads (128)
  uint64_t* ofull = rempty + kMaxStages;      // A operands stored in tensor memory (128)
  uint64_t* oempty = ofull + kMaxStages;      // MMAs done with the A stage and its basis slot (commit)
  uint64_t* qfull = oempty + kMaxStages;      // basis chunk landed (tx)
  uint64_t* dfull = qfull + kMaxStages;       // [kNB] group products ready (commit)
  uint64_t* dfree = dfull + kMaxDB;           // [kNB] group products read out (128 arrivals)
  uint64_t* alldone = dfree + kMaxDB;         // every MMA done (commit)
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(alldone + 1);
  __shared__ double red[32];
  __shared__ int s_fail;
  volatile int* vfail = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T32_TRACE_DECL
  const long long nt =
      a.ntiles > blockIdx.x ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long nst = nt * a.nkc;   // stages of this CTA
  if (tid == 0) {
    for (int k = 0; k < kMaxStages; ++k) {
      mbar_init(su32(&rfull[k]), 1);
      mbar_init(su32(&rempty[k]), 128);
      mbar_init(su32(&ofull[k]), 128);
      mbar_init(su32(&oempty[k]), 1);
      mbar_init(su32(&qfull[k]), 1);
    }
    for (int b = 0; b < kMaxDB; ++b) {
      mbar_init(su32(&dfull[b]), 1);
      mbar_init(su32(&dfree[b]), 128);
    }
    mbar_init(su32(alldone), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Tensor memory (all 512 columns): the A operand stages first, 64 columns each
  // (hi plane | lo plane: lane m = tile column m, column = row i of the stage), then
  // nb buffers of kDS columns, one per accumulation group of a.flush K-steps in
  // flight, each [B_hi Q_hi | B_hi Q_lo + B_lo Q_hi] started fresh.
  constexpr int kDS = (2 * RP + 31) / 32 * 32;
  constexpr uint32_t kCols = 512;
  const uint32_t acols = (uint32_t)no * 64u;
  const int nb = (int)((kCols - acols) / kDS) < kMaxDB ? (int)((kCols - acols) / kDS) : kMaxDB;
  if (warp == 0) tmem_alloc(su32(tmem_holder), kCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;
  float wsh = 0.f, wsl = 0.f;   // ||W||^2 (epilogue threads)

  if (warp == 8) {
    // ---------------- producer: raw stages and basis chunks ----------------
    long long s = 0;
    bool ok = true;
    // ring positions kept as counters (a 64-bit division per stage costs more than
    // the stage's MMAs)
    int rr = 0;
    uint32_t rph = 0;
    const int kcs = (int)(blockIdx.x % (unsigned)a.nkc);
    const bool wide = a.Q % 128 == 0;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      const long long t = blockIdx.x + lt * gridDim.x;
      // the tile's four 32-column blocks: (p, q) of each, once per tile (past the
      // last column: p out of range, zero fill)
      int pb[4], qb[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const long long j = t * 128 + 32 * b;
        pb[b] = (int)a.P;
        qb[b] = 0;
        if (j < a.J) {
          const long long p = j / a.Q;
          pb[b] = (int)p;
          qb[b] = (int)(j - p * a.Q);
        }
      }
      for (int kc0 = 0; kc0 < a.nkc && ok; ++kc0, ++s) {
        // every CTA starts its tiles at a different 32-row stage, so the CTAs do not
        // all fetch the same chunk of the split basis from L2 at the same time
        int kc = kc0 + kcs;
        if (kc >= a.nkc) kc -= a.nkc;
        const int r = rr;
        ok = TWAIT(0, mbar_wait_b(su32(&rempty[r]), rph ^ 1u, vfail));
        if (!ok) break;
        if (++rr == nr) {
          rr = 0;
          rph ^= 1u;
        }
        if (lane == 0) {
          unsigned char* st = raw + (size_t)r * kStage1;
          mbar_expect_tx(su32(&rfull[r]), (uint32_t)kStage1);
          if (wide) {
            tma_load_3d(su32(st), &bmap, su32(&rfull[r]), qb[0], kc * kKC, pb[0]);
          } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              tma_load_3d(su32(st + b * kBox1), &bmap, su32(&rfull[r]), qb[b], kc * kKC, pb[b]);
          }
        }
        __syncwarp();
      }
    }
    // every copy issued must have landed before the shared memory is released
    if (lane == 0) {
      for (int sl = 0; sl < nr && sl < s; ++sl)
        mbar_drain(su32(&rfull[sl]), (uint32_t)(((s / nr + (sl < s % nr ? 1 : 0)) - 1) & 1));

    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // ---------------- split: column m = t to registers, raw slot released, K-major hi / lo ----
    const int t = tid - 128;
    const bool wide = a.Q % 128 == 0;
    bool ok = true;
    long long nq_issued = 0;
    int r = 0, o = 0, kc0 = 0;
    uint32_t rph = 0, oph = 0;
    const int kcs = (int)(blockIdx.x % (unsigned)a.nkc);
    for (long long s = 0; s < nst && ok; ++s) {
      ok = TWAIT(1, mbar_wait_b(su32(&rfull[r]), rph, vfail));
      if (!ok) break;
      float v[32];
      t32_read_col(raw + (size_t)r * kStage1, t, wide, v);
      mbar_arrive(su32(&rempty[r]));
      ok = TWAIT(2, mbar_wait_b(su32(&oempty[o]), oph ^ 1u, vfail));
      if (!ok) break;
      fence_after();
      if (t == 0) {
        // the stage's rows of the split basis into the A stage's basis slot
        int kc = kc0 + kcs;
        if (kc >= a.nkc) kc -= a.nkc;
        mbar_expect_tx(su32(&qfull[o]), kQB);
        bulk_load(su32(qsr + (size_t)o * kQB), a.QS + (size_t)kc * (kQB / 4), kQB, su32(&qfull[o]));
      }
      // hi and lo of column t into lane t of A stage o
      uint32_t hi[32], lo[32];
      t32_split_col(v, hi, lo);
      const uint32_t ta = tmem + (uint32_t)o * 64u + ((uint32_t)((warp & 3) * 32) << 16);
      tmem_st32(ta, hi);
      tmem_st32(ta + 32u, lo);
      tmem_wait_st();
      fence_before();
      mbar_arrive(su32(&ofull[o]));
      ++nq_issued;
      if (++r == nr) {
        r = 0;
        rph ^= 1u;
      }
      if (++o == no) {
        o = 0;
        oph ^= 1u;
      }
      if (++kc0 == a.nkc) kc0 = 0;
    }
    // every basis copy issued must have landed before the shared memory is released
    if (t == 0)
      for (int sl = 0; sl < no && sl < nq_issued; ++sl)
        mbar_drain(su32(&qfull[sl]),
                   (uint32_t)(((nq_issued / no + (sl < nq_issued % no ? 1 : 0)) - 1) & 1));
  } else if (warp == 9) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t kIdAll = idesc(kFmtTF32, 128, 2 * RP, 0, 0);
    constexpr uint32_t kIdHi = idesc(kFmtTF32, 128, RP, 0, 0);
    const int F = a.flush;
    long long gseq = 0;   // accumulation groups
    bool ok = true;
    int o = 0, b = 0, bround = 0;
    uint32_t oph = 0;
    for (long long s = 0; s < nst && ok; ++s) {
      const int q = o;
      ok = TWAIT(3, mbar_wait_b(su32(&ofull[o]), oph, vfail));
      if (ok) ok = TWAIT(3, mbar_wait_b(su32(&qfull[q]), oph, vfail));
      if (!ok) break;
      fence_after();
      const uint32_t aop = tmem + (uint32_t)o * 64u;   // A stage: hi at +0, lo at +32
      const uint32_t qs = su32(qsr + (size_t)q * kQB);
      // groups of F K-steps, each into a fresh buffer (the epilogue adds the groups
      // up in registers with rounding to nearest); lane 0 issues a group's MMAs back
      // to back (a fence or commit between MMAs costs issue cycles)
      for (int g = 0; g < (kKC / 8) / F && ok; ++g, ++gseq) {
        if (bround >= 1) {
          ok = TWAIT(4, mbar_wait_b(su32(&dfree[b]), (uint32_t)((bround - 1) & 1), vfail));
          if (!ok) break;
          fence_after();
        }
        if (lane == 0) {
          const uint32_t d = tmem + acols + (uint32_t)(b * kDS);
          for (int k = 0; k < F; ++k) {
            const int ks = g * F + k;
            // B: K-major split basis, rows [Q_hi (RP) | Q_lo (RP)]; A from tensor
            // memory, 8 rows i (columns) per step
            const uint64_t bq = desc_sw128(qs + ks * 32, 16, 1024);
            mma_tf32_ts(d, aop + (uint32_t)(ks * 8), bq, kIdAll, k ? 1u : 0u);   // [B_hi Q_hi | B_hi Q_lo]
            mma_tf32_ts(d + RP, aop + 32u + (uint32_t)(ks * 8), bq, kIdHi, 1u);  // + B_lo Q_hi
          }
          mma_commit(su32(&dfull[b]));
        }
        __syncwarp();
        if (++b == nb) {
          b = 0;
          ++bround;
        }
      }
      // operand slot and basis slot released together
      if (lane == 0) mma_commit(su32(&oempty[o]));
      __syncwarp();
      if (++o == no) {
        o = 0;
        oph ^= 1u;
      }
    }
    if (lane == 0) mma_commit(su32(alldone));
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 0-3, lane = tile column ----------------
    bool ok = true;
    const int m = warp * 32 + lane;
    const int ngr = (kKC / 8) / a.flush;   // groups per stage
    int b = 0;
    uint32_t bph = 0;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      const long long t = blockIdx.x + lt * gridDim.x;
      float big[RP], small[RP];   // sum of B_hi Q_hi; of the two correction terms
#pragma unroll
      for (int k = 0; k < RP; ++k) big[k] = small[k] = 0.f;
      for (int kc = 0; kc < a.nkc && ok; ++kc) {
        for (int g = 0; g < ngr && ok; ++g) {
          ok = TWAIT(5, mbar_wait_b(su32(&dfull[b]), bph, vfail));
          if (!ok) break;
          fence_after();
#pragma unroll
          for (int cb = 0; cb < kDS; cb += 64) {
            uint32_t r0[32], r1[32];
            const uint32_t ta = tmem + acols + (uint32_t)(b * kDS + cb) + ((uint32_t)(warp * 32) << 16);
            tmem_ld32_nw(ta, r0);
            if (cb + 32 < kDS) tmem_ld32_nw(ta + 32u, r1);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 64; ++k) {
              const int c = cb + k;
              if (c >= kDS) break;
              const float x = __uint_as_float(k < 32 ? r0[k] : r1[k - 32]);
              if (c < RP) big[c] += x;
              else if (c < 2 * RP) small[c - RP] += x;
            }
          }
          fence_before();
          mbar_arrive(su32(&dfree[b]));
          if (++b == nb) {
            b = 0;
            bph ^= 1u;
          }
        }
      }
      if (!ok) break;
      const long long j = t * 128 + m;
      if (j < a.J) {
        const long long p = j / a.Q, q = j - p * a.Q;
        float* wp = a.W + (size_t)p * a.R * a.Q + q;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          if (r < a.R) {
            const float w = big[r] + small[r];
            wp[(size_t)r * a.Q] = w;
            acc_sq(w, wsh, wsl);
          }
        }
      }
    }
  }
  T32_TRACE_FLUSH(0)
  const double tot = block_sum((double)wsh + (double)wsl, red);
  if (tid == 0) {
    a.spart[blockIdx.x] = tot;
    if (*vfail) atomicExch(a.err, 5);   // TALS_ETIMEOUT
  }
  // nothing may still write the shared or tensor memory released below
  if (*vfail && tid == 288) mbar_drain(su32(alldone), 0u);
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}


// ---------------------------------------------------------------------------
// Pass 2: Y = B W and the residual ||B - Q W^T||^2 (3xTF32); init mode: Y0 = B S
// and ||B||^2.
//
// One CTA per (128-row chunk c, share of the 32-column blocks): grid (nch, ncol).
// The chunk's rows of the split basis Q_c stay in shared memory; each stage
// brings one block of B (128 rows x 32 columns) and, by TMA as well, the block's
// W (R x 32). Per stage:
//   P = Q_c W_blk^T (M = 128, N = 32, K = R)       -> tensor memory
//   split warps: residual sum (B - P)^2 of the stage, then B -> hi / lo
//   Y_c += B_blk W_blk (M = 128, N = R, K = 32)    -> tensor memory per K-step,
//                                                    summed in registers
// The residual is the stop rule's e_k^2 (Eq. 5.01) without cancellation: every
// tensor-core result carries a relative error of order 1e-7 (the products of
// each K = 8 step are aligned and truncated), so ||B||^2 - ||W||^2 would carry
// noise of order 1e-8 ||B||^2, while an error dP in P moves the residual only
// by 2 <B - P, dP> + ||dP||^2, both far below FP32 resolution of e^2 (the
// residual is orthogonal to P up to the error of W). The chunk's W blocks are
// read by all nch chunk CTAs of a column share at about the same time, so W
// mostly comes from L2.
// Warp roles: warps 0-3 prepare the W block (split for the Y product, transposed
// and split for the residual product) and write Y at the end; warps 4-7 take the
// residual and split B (lane = row of the chunk = tensor-memory lane); warp 8
// issues TMA; warp 9 issues the MMAs.
// ---------------------------------------------------------------------------
// Pass 2, warps 10-11 (t = 0..63): prepare the W block of stage lt once it has landed -- split
// for the Y product (hi in place, lo RP rows further on; init: the sketch block
// S, Sec. 4) and, with the residual, transposed and split for the P product.
template <int RP>
__device__ __forceinline__ bool t32_prep_w(const T32Args& a, unsigned char* ring, uint32_t kSB, int ns,
                                           long long lt, long long col, long long ncol, uint64_t* full,
                                           uint64_t* wrdy, int t, volatile int* vfail, bool resid) {
  constexpr uint32_t kW2 = 2u * RP * 128u;
  const int slot = (int)((uint32_t)lt % (uint32_t)ns);   // 32-bit: stages per CTA < 2^32
  const uint32_t ph = ((uint32_t)lt / (uint32_t)ns) & 1u;
  if (!mbar_wait_b(su32(&full[slot]), ph, vfail)) return false;
  const long long j0 = (col + lt * ncol) * 32;
  unsigned char* w2 = ring + (size_t)slot * kSB + kStage2;
  unsigned char* w3 = w2 + kW2;
  for (int e = t; e < 32 * a.R; e += 64) {
    const int r = e >> 5, q = e & 31;
    const float x = a.init ? sketch_entry(a.sketch, (uint64_t)(j0 + q), a.R, r)
                           : *reinterpret_cast<const float*>(w2 + sw_off(r, q));
    const float h = to_tf32(x), l = to_tf32(x - h);
    *reinterpret_cast<float*>(w2 + sw_off(r, q)) = h;
    *reinterpret_cast<float*>(w2 + sw_off(RP + r, q)) = l;
    if (resid) {
      const uint32_t kb = (uint32_t)(r >> 5) * (64u * 128u);
      *reinterpret_cast<float*>(w3 + kb + sw_off(q, r & 31)) = h;
      *reinterpret_cast<float*>(w3 + kb + sw_off(32 + q, r & 31)) = l;
    }
  }
  fence_async_smem();
  mbar_arrive(su32(&wrdy[slot]));
  return true;
}

template <int RP>
__global__ void __launch_bounds__(kT32Threads2, 1)
    t32_ypass_kernel(const __grid_constant__ CUtensorMap bmap, const __grid_constant__ CUtensorMap wmap,
                     T32Args a, int ns) {
  if (a.st != nullptr && a.st->done) return;   // uniform early exit, before any barrier
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  constexpr int KB = (RP + 31) / 32;                  // 32-wide blocks of the rank (K of P)
  constexpr uint32_t kQP = 128u * KB * 128u;          // one plane of Q_c: K-major, 128 rows
  constexpr uint32_t kW2 = 2u * RP * 128u;            // W block, Y product: rows [W_hi | W_lo]
  constexpr uint32_t kW3 = 64u * KB * 128u;           // W block, P product: rows [q hi | q lo]
  constexpr uint32_t kSB = kStage2 + kW2 + kW3;       // stage: B | W2 | W3
  unsigned char* qhi = base;
  unsigned char* qlo = qhi + kQP;
  unsigned char* ring = qlo + kQP;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)ns * kSB);
  uint64_t* full = bars;                      // B (and W) landed (tx)
  uint64_t* wrdy = full + kMaxStages;         // W block prepared (128 arrivals)
  uint64_t* afull = wrdy + kMaxStages;        // [nA] B split into an A stage of tensor memory (128)
  uint64_t* aempty = afull + kMaxDB;          // [nA] MMAs done with the A stage (commit)
  uint64_t* empty = aempty + kMaxDB;          // MMAs done with the stage (commit)
  uint64_t* pready = empty + kMaxStages;      // [2] P in tensor memory (commit)
  uint64_t* pfree = pready + 2;               // [2] P read out (128 arrivals)
  uint64_t* yfull = pfree + 2;                // [kYB] K-step products of Y ready (commit)
  uint64_t* yfree = yfull + kMaxDB;           // [kYB] K-step products read out (128 arrivals)
  uint64_t* qready = yfree + kMaxDB;          // Q_c operands written (128 arrivals)
  uint64_t* ydone = qready + 1;               // every MMA done (commit)
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(ydone + 1);
  __shared__ double red4[4];
  __shared__ int s_fail;
  volatile int* vfail = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T32_TRACE_DECL
  const int chunk = blockIdx.x;
  const long long ncol = gridDim.y, col = blockIdx.y;
  const long long nt = a.ntiles > col ? (a.ntiles - col + ncol - 1) / ncol : 0;
  const bool resid = !a.init;
  if (tid == 0) {
    for (int k = 0; k < kMaxStages; ++k) {
      mbar_init(su32(&full[k]), 1);
      mbar_init(su32(&wrdy[k]), 64);
      mbar_init(su32(&empty[k]), 1);
    }
    for (int k = 0; k < kMaxDB; ++k) {
      mbar_init(su32(&afull[k]), 128);
      mbar_init(su32(&aempty[k]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&pready[b]), 1);
      mbar_init(su32(&pfree[b]), 128);
    }
    for (int b = 0; b < kMaxDB; ++b) {
      mbar_init(su32(&yfull[b]), 1);
      mbar_init(su32(&yfree[b]), 128);
    }
    mbar_init(su32(qready), 128);
    mbar_init(su32(ydone), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // W blocks: rows beyond R (and the K columns beyond R of the P operand) are read
  // by the MMAs and never written: zero every stage's W regions once
  for (int sl = 0; sl < ns; ++sl) {
    uint4* w = reinterpret_cast<uint4*>(ring + (size_t)sl * kSB + kStage2);
    for (int e = tid; e < (int)((kW2 + kW3) / 16); e += kT32Threads2) w[e] = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_async_smem();
  // Tensor memory: kYB buffers of kYS columns for the accumulation groups (a.flush
  // K-steps) of the Y product in flight, each [B_hi W_hi | B_hi W_lo + B_lo W_hi]
  // started fresh (the tensor cores round each result toward zero; accumulated in
  // tensor memory over a whole pass, that bias varies from row to row and tilts the
  // weakest directions of the basis), summed in registers by warps 0-3; P buffers
  // at 384 and 448.
  // The A operand of the Y product (the stage's B split into hi | lo: lane = row,
  // column = block column) lives in tensor memory too, in nA stages of 64 columns
  // just below the P buffers.
  constexpr int kYS = (2 * RP + 31) / 32 * 32;
  constexpr int nA = (RP <= 32 || RP == 64) ? 2 : 3;
  constexpr uint32_t kPCol = 384;
  constexpr uint32_t kACol = kPCol - 64u * nA;
  constexpr int kYB = (int)kACol / kYS < kMaxDB ? (int)kACol / kYS : kMaxDB;
  constexpr uint32_t kCols = 512;
  if (warp == 0) tmem_alloc(su32(tmem_holder), kCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 8) {
    // ---------------- producer ----------------
    long long seq = 0;
    bool ok = true;
    for (long long lt = 0; lt < nt && ok; ++lt, ++seq) {
      const long long j = (col + lt * ncol) * 32;
      const long long p = j / a.Q, q = j - p * a.Q;
      const int slot = (int)((uint32_t)seq % (uint32_t)ns);
      const uint32_t ph = ((uint32_t)seq / (uint32_t)ns) & 1u;
      ok = TWAIT(0, mbar_wait_b(su32(&empty[slot]), ph ^ 1u, vfail));
      if (!ok) break;
      if (lane == 0) {
        unsigned char* st = ring + (size_t)slot * kSB;
        mbar_expect_tx(su32(&full[slot]), (uint32_t)kStage2 + (resid ? (uint32_t)a.R * 128u : 0u));
        tma_load_3d(su32(st), &bmap, su32(&full[slot]), (int)q, chunk * kRows2, (int)p);
        if (resid) tma_load_3d(su32(st + kStage2), &wmap, su32(&full[slot]), (int)q, 0, (int)p);
      }
      __syncwarp();
    }
    if (lane == 0)
      for (int sl = 0; sl < ns && sl < seq; ++sl) {
        const long long nfill = seq / ns + (sl < seq % ns ? 1 : 0);
        mbar_drain(su32(&full[sl]), (uint32_t)((nfill - 1) & 1));
      }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------- Q_c prologue, then the Y drains (t = row of the chunk) ----------------
    const int t = tid;
    if (resid) {
      // Q_c: rows chunk*128 + t of the basis, split, K-major with 32-wide K blocks
      const long long i = (long long)chunk * kRows2 + t;
      for (int r = 0; r < 32 * KB; ++r) {
        const float x = (i < a.I && r < a.R) ? a.L[i * a.R + r] : 0.f;
        const float h = to_tf32(x);
        const uint32_t off = (uint32_t)(r >> 5) * 16384u + sw_off(t, r & 31);
        *reinterpret_cast<float*>(qhi + off) = h;
        *reinterpret_cast<float*>(qlo + off) = to_tf32(x - h);
      }
      fence_async_smem();
      mbar_arrive(su32(qready));
    }
    bool ok = true;
    float big[RP], small[RP];   // Y of this row: B_hi W_hi; the two correction terms
#pragma unroll
    for (int k = 0; k < RP; ++k) big[k] = small[k] = 0.f;
    const int ngr = 4 / a.flush;   // accumulation groups per stage
    long long gseq = 0;
    for (long long lt = 0; lt < nt && ok; ++lt) {
      for (int g = 0; g < ngr && ok; ++g, ++gseq) {
        const int b = (int)((uint32_t)gseq % (uint32_t)kYB);
        ok = TWAIT(2, mbar_wait_b(su32(&yfull[b]), ((uint32_t)gseq / (uint32_t)kYB) & 1u, vfail));
        if (!ok) break;
        fence_after();
#pragma unroll
        for (int cb = 0; cb < kYS; cb += 64) {
          uint32_t r0[32], r1[32];
          const uint32_t ta = tmem + (uint32_t)(b * kYS + cb) + ((uint32_t)(warp * 32) << 16);
          tmem_ld32_nw(ta, r0);
          if (cb + 32 < kYS) tmem_ld32_nw(ta + 32u, r1);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 64; ++k) {
            const int c = cb + k;
            if (c >= kYS) break;
            const float x = __uint_as_float(k < 32 ? r0[k] : r1[k - 32]);
            if (c < RP) big[c] += x;
            else if (c < 2 * RP) small[c - RP] += x;
          }
        }
        fence_before();
        mbar_arrive(su32(&yfree[b]));
      }
    }
    // final Y of the chunk: lane = row
    if (ok && nt > 0) {
      const long long i = (long long)chunk * kRows2 + warp * 32 + lane;
      if (i < a.I) {
        float* yp = a.Ypart + ((size_t)col * a.I + i) * a.R;
#pragma unroll
        for (int r = 0; r < RP; ++r)
          if (r < a.R) yp[r] = big[r] + small[r];
      }
    }
  } else if (warp >= 10) {
    // ---------------- W preparation, running ahead by what the ring holds ----------------
    const int t = tid - 320;
    bool ok = true;
    for (long long lt = 0; lt < nt && ok; ++lt)
      ok = TWAIT(1, t32_prep_w<RP>(a, ring, kSB, ns, lt, col, ncol, full, wrdy, t, vfail, resid));
  } else if (warp < 8) {
    // ---------------- residual and split: lane = row of the chunk ----------------
    const int t = tid - 128;   // row of the chunk; tensor-memory lane quadrant warp % 4
    long long seq = 0;
    bool ok = true;
    float sh = 0.f, sl = 0.f;   // residual sum (init: ||B||^2)
    int ai = 0;
    uint32_t aph = 0;
    for (long long lt = 0; lt < nt && ok; ++lt, ++seq) {
      const int slot = (int)((uint32_t)seq % (uint32_t)ns);
      const uint32_t ph = ((uint32_t)seq / (uint32_t)ns) & 1u;
      ok = TWAIT(3, mbar_wait_b(su32(&full[slot]), ph, vfail));
      if (!ok) break;
      float pv[32];
      if (resid) {
        const int pb = (int)(seq & 1);
        ok = TWAIT(4, mbar_wait_b(su32(&pready[pb]), (uint32_t)((seq >> 1) & 1), vfail));
        if (!ok) break;
        fence_after();
        uint32_t p0[32], p1[32];
        const uint32_t tp = tmem + kPCol + (uint32_t)(pb * 64) + ((uint32_t)((warp & 3) * 32) << 16);
        tmem_ld32_nw(tp, p0);
        tmem_ld32_nw(tp + 32u, p1);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 32; ++k) pv[k] = __uint_as_float(p0[k]) + __uint_as_float(p1[k]);
        fence_before();
        mbar_arrive(su32(&pfree[pb]));
      }
      unsigned char* st = ring + (size_t)slot * kSB;
      unsigned char* row = st + t * 128;
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        // chunk c4 of the row holds columns 4 c4 .. 4 c4 + 3
        const uint32_t off = (uint32_t)((c4 ^ (t & 7)) << 4);
        float4 x = *reinterpret_cast<const float4*>(row + off);
        if (resid) {
          acc_sq(x.x - pv[4 * c4], sh, sl);
          acc_sq(x.y - pv[4 * c4 + 1], sh, sl);
          acc_sq(x.z - pv[4 * c4 + 2], sh, sl);
          acc_sq(x.w - pv[4 * c4 + 3], sh, sl);
        } else {
          acc_sq(x.x, sh, sl);
          acc_sq(x.y, sh, sl);
          acc_sq(x.z, sh, sl);
          acc_sq(x.w, sh, sl);
        }
        const float4 l = split4(x);
        hi[4 * c4] = __float_as_uint(x.x);
        hi[4 * c4 + 1] = __float_as_uint(x.y);
        hi[4 * c4 + 2] = __float_as_uint(x.z);
        hi[4 * c4 + 3] = __float_as_uint(x.w);
        lo[4 * c4] = __float_as_uint(l.x);
        lo[4 * c4 + 1] = __float_as_uint(l.y);
        lo[4 * c4 + 2] = __float_as_uint(l.z);
        lo[4 * c4 + 3] = __float_as_uint(l.w);
      }
      // the row's hi and lo into its lane of A stage ai, once the MMAs are done with it
      ok = TWAIT(9, mbar_wait_b(su32(&aempty[ai]), aph ^ 1u, vfail));
      if (!ok) break;
      fence_after();
      const uint32_t ta = tmem + kACol + (uint32_t)ai * 64u + ((uint32_t)((warp & 3) * 32) << 16);
      tmem_st32(ta, hi);
      tmem_st32(ta + 32u, lo);
      tmem_wait_st();
      fence_before();
      mbar_arrive(su32(&afull[ai]));
      if (++ai == nA) {
        ai = 0;
        aph ^= 1u;
      }
    }
    const double tot = split_sum(sh, sl, red4, t);
    if (t == 0) a.spart[(size_t)col * gridDim.x + chunk] = tot;
  } else {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t kIdY2 = idesc(kFmtTF32, 128, 2 * RP, 0, 0);
    constexpr uint32_t kIdY1 = idesc(kFmtTF32, 128, RP, 0, 0);
    constexpr uint32_t kIdP2 = idesc(kFmtTF32, 128, 64, 0, 0);
    constexpr uint32_t kIdP1 = idesc(kFmtTF32, 128, 32, 0, 0);
    bool ok = !resid || mbar_wait_b(su32(qready), 0u, vfail);
    const int F = a.flush;
    // stage lt's P product (after its W block is prepared)
    auto issue_p = [&](long long lt) -> bool {
      const int slot = (int)((uint32_t)lt % (uint32_t)ns);
      if (!TWAIT(5, mbar_wait_b(su32(&wrdy[slot]), ((uint32_t)lt / (uint32_t)ns) & 1u, vfail))) return false;
      fence_after();
      if (!resid) return true;
      // P = Q_c W^T: [Q_hi W_hi^T | Q_hi W_lo^T] (N = 64) and Q_lo W_hi^T into the first half
      const int pb = (int)(lt & 1);
      if (lt >= 2 && !TWAIT(6, mbar_wait_b(su32(&pfree[pb]), (uint32_t)(((lt >> 1) - 1) & 1), vfail)))
        return false;
      fence_after();
      if (lane == 0) {
        const uint32_t w3 = su32(ring + (size_t)slot * kSB) + kStage2 + kW2;
        const uint32_t d = tmem + kPCol + (uint32_t)(pb * 64);
#pragma unroll
        for (int ks = 0; ks < RP / 8; ++ks) {
          const uint32_t kq = (uint32_t)(ks >> 2) * 16384u + (uint32_t)(ks & 3) * 32u;
          const uint32_t kw = (uint32_t)(ks >> 2) * (64u * 128u) + (uint32_t)(ks & 3) * 32u;
          const uint64_t ah = desc_sw128(su32(qhi) + kq, 16, 1024);
          const uint64_t al = desc_sw128(su32(qlo) + kq, 16, 1024);
          const uint64_t bw = desc_sw128(w3 + kw, 16, 1024);
          mma_tf32(d, ah, bw, kIdP2, ks ? 1u : 0u);
          mma_tf32(d, al, bw, kIdP1, 1u);
        }
        mma_commit(su32(&pready[pb]));
      }
      __syncwarp();
      return true;
    };
    long long gseq = 0;
    int ai = 0;
    uint32_t aph = 0;
    // stage lt's Y product (after its residual and split), in groups of F K-steps
    auto issue_y = [&](long long lt) -> bool {
      const int slot = (int)((uint32_t)lt % (uint32_t)ns);
      if (!TWAIT(7, mbar_wait_b(su32(&afull[ai]), aph, vfail))) return false;
      fence_after();
      const uint32_t st = su32(ring + (size_t)slot * kSB);
      const uint32_t w2 = st + kStage2;
      const uint32_t aop = tmem + kACol + (uint32_t)ai * 64u;   // A stage: hi at +0, lo at +32
      for (int g = 0; g < 4 / F; ++g, ++gseq) {
        const int b = (int)((uint32_t)gseq % (uint32_t)kYB);
        if (gseq >= kYB) {
          if (!TWAIT(8, mbar_wait_b(su32(&yfree[b]), ((uint32_t)gseq / (uint32_t)kYB - 1u) & 1u, vfail))) return false;
          fence_after();
        }
        if (lane == 0) {
          const uint32_t d = tmem + (uint32_t)(b * kYS);
          for (int k = 0; k < F; ++k) {
            const int ks = g * F + k;
            const uint64_t bw = desc_sw128(w2 + ks * 32, 16, 1024);
            mma_tf32_ts(d, aop + (uint32_t)(ks * 8), bw, kIdY2, k ? 1u : 0u);        // [B_hi W_hi | B_hi W_lo]
            mma_tf32_ts(d + RP, aop + 32u + (uint32_t)(ks * 8), bw, kIdY1, 1u);      // + B_lo W_hi
          }
          mma_commit(su32(&yfull[b]));
        }
        __syncwarp();
      }
      if (lane == 0) {
        mma_commit(su32(&empty[slot]));
        mma_commit(su32(&aempty[ai]));
      }
      __syncwarp();
      if (++ai == nA) {
        ai = 0;
        aph ^= 1u;
      }
      return true;
    };
    // software pipeline: the next stage's P product goes ahead of this stage's Y
    // product, so the split warps' residual of stage lt + 1 does not wait for it
    if (ok && nt > 0) ok = issue_p(0);
    for (long long lt = 0; lt < nt && ok; ++lt) {
      if (lt + 1 < nt) ok = issue_p(lt + 1);
      if (ok) ok = issue_y(lt);
    }
    if (lane == 0) mma_commit(su32(ydone));
    __syncwarp();
  }
  T32_TRACE_FLUSH(1)
  if (tid == 0 && *vfail) atomicExch(a.err, 5);   // TALS_ETIMEOUT
  if (*vfail && tid == 288) mbar_drain(su32(ydone), 0u);
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// Split basis for pass 1: QS[kc] = rows [hi(Q[32kc + k][r]) for r < RP | lo(...)]
// of 32 values along k, 128B-swizzled (the K-major B operand layout), zero
// beyond I and R.
__global__ void t32_split_basis_kernel(const float* __restrict__ L, int I, int R, int RP, int nkc,
                                       float* __restrict__ QS) {
  const long long per = (long long)2 * RP * 32;
  const long long total = (long long)nkc * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int kc = (int)(e / per);
    const int rem = (int)(e - kc * per);
    const int n = rem >> 5, k = rem & 31;
    const int i = kc * 32 + k;
    float v = 0.f;
    if (i < I) {
      if (n < R) {
        v = to_tf32(L[(size_t)i * R + n]);
      } else if (n >= RP && n - RP < R) {
        const float x = L[(size_t)i * R + (n - RP)];
        v = to_tf32(x - to_tf32(x));
      }
    }
    QS[(size_t)kc * per + (sw_off(n, k) >> 2)] = v;
  }
}

struct Ring1 { int nr, no, nq; };

template <int RP>
size_t smem1(const Ring1& g) {
  return 1024 + (size_t)g.nr * kStage1 + (size_t)g.no * (2 * RP * 128) +
         (5 * kMaxStages + 2 * kMaxDB + 1) * 8 + 16;
}

template <int RP>
size_t smem2(int ns) {
  constexpr size_t KB = (RP + 31) / 32;
  const size_t stage = (size_t)kStage2 + 2 * RP * 128 + 64 * KB * 128;
  return 1024 + 2 * (128 * KB * 128) + (size_t)ns * stage + (3 * kMaxStages + 6 + 4 * kMaxDB) * 8 + 16;
}

// K-steps (of 8) per accumulation group: four, i.e. one group per 32-row stage.
// A group's products are summed by the tensor cores (truncating) and the groups
// by the registers (rounding to nearest); four keeps the truncation bias of W and
// Y below 1e-7 relative while the drains keep up with the MMAs.
constexpr int kFlush = 4;

int rp_of(int R) { return R <= 16 ? 16 : R <= 32 ? 32 : R <= 48 ? 48 : 64; }

// Pass 1 rings: three operand slots (each with its basis slot), as many raw slots
// (up to kMaxStages) as fit.
Ring1 ring1(int RP) {
  const size_t static_smem = 2048;
  for (int nq = 3; nq >= 3; --nq)
    for (int nr = kMaxStages; nr >= 3; --nr) {
      const Ring1 g{nr, 3, nq};
      const size_t s = RP == 16 ? smem1<16>(g) : RP == 32 ? smem1<32>(g) : RP == 48 ? smem1<48>(g) : smem1<64>(g);
      if (s + static_smem <= (size_t)kSmemCap) return g;
    }
  return Ring1{0, 0, 0};
}

int stages2(int RP) {
  const size_t static_smem = 2048;
  for (int ns = kMaxStages; ns >= 2; --ns) {
    size_t s = RP == 16 ? smem2<16>(ns) : RP == 32 ? smem2<32>(ns) : RP == 48 ? smem2<48>(ns) : smem2<64>(ns);
    if (s + static_smem <= (size_t)kSmemCap) return ns;
  }
  return 0;
}

// 3-D FP32 map of the view (Q, I, P) or of W (Q, R, P), boxes (box_cols, rows, 1),
// 128B swizzle (box_cols 32) or none.
bool make_map(const void* X, long long Q, long long rows, long long P, int box_rows, CUtensorMap* map,
              int box_cols = 32, bool swizzle = true) {
  EncodeTiledFn fn = tma_encode_fn();
  if (!fn) return false;
  if ((uintptr_t)X % 16 != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Q, (cuuint64_t)rows, (cuuint64_t)P};
  cuuint64_t strides[2] = {(cuuint64_t)Q * 4, (cuuint64_t)rows * Q * 4};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(X), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool t32_supported(const ModeView& v, int R) {
  if (R < 1 || R > 64 || v.Q % 32 != 0 || v.I < 1 || v.I > 1024) return false;
  if (v.P > 0x7fffffffLL || v.Q > 0x7fffffffLL || v.I > 0x7fffffffLL) return false;
  const int RP = rp_of(R);
  return ring1(RP).nr >= 3 && stages2(RP) >= 2;
}

size_t t32_basis_floats(long long I, int R) {
  return (size_t)((I + kKC - 1) / kKC) * 2 * rp_of(R) * 32;
}

int t32_grid(const ModeView& v, int pass, int sms) {
  if (pass == 1) return (int)std::max<long long>(1, std::min<long long>(sms, (v.J() + 127) / 128));
  // pass 2: column shares per 128-row chunk (about one CTA per SM in all)
  const long long nch = (v.I + kRows2 - 1) / kRows2;
  return (int)std::max<long long>(1, std::min<long long>(std::max<long long>(1, sms / nch), v.J() / 32));
}

int t32_chunks(const ModeView& v) { return (int)((v.I + kRows2 - 1) / kRows2); }

#ifdef T32_TRACE
extern "C" int tals_t32_trace(unsigned long long* out) {
  if (cudaMemcpyFromSymbol(out, g_t32_trace, sizeof(g_t32_trace)) != cudaSuccess) return 1;
  static unsigned long long zero[2][12][12];
  return cudaMemcpyToSymbol(g_t32_trace, zero, sizeof(zero)) == cudaSuccess ? 0 : 1;
}
#endif

cudaError_t launch_t32_split_basis(const float* L, long long I, int R, float* QS, cudaStream_t s) {
  const int RP = rp_of(R);
  const int nkc = (int)((I + kKC - 1) / kKC);
  const long long total = (long long)nkc * 2 * RP * 32;
  const int blocks = (int)std::min<long long>(1024, (total + 255) / 256);
  t32_split_basis_kernel<<<blocks, 256, 0, s>>>(L, (int)I, R, RP, nkc, QS);
  return cudaGetLastError();
}

cudaError_t launch_t32_wpass(const float* X, const ModeView& v, int R, const float* QS, float* W,
                             double* spart, int* err, int grid, cudaStream_t s, const ModeState* st) {
  if (!t32_supported(v, R) || !W || !QS) return cudaErrorInvalidValue;
  CUtensorMap bmap;
  if (!make_map(X, v.Q, v.I, v.P, kKC, &bmap, v.Q % 128 == 0 ? 128 : 32, false)) return cudaErrorInvalidValue;
  const int RP = rp_of(R);
  T32Args a;
  std::memset(&a, 0, sizeof(a));
  a.I = (int)v.I;
  a.R = R;
  a.RP = RP;
  a.P = v.P;
  a.Q = v.Q;
  a.J = v.J();
  a.nkc = (int)((v.I + kKC - 1) / kKC);
  a.nch = (int)((v.I + kRows2 - 1) / kRows2);
  a.ntiles = (v.J() + 127) / 128;
  a.QS = QS;
  a.W = W;
  a.spart = spart;
  a.err = err;
  a.st = st;
  a.flush = kFlush;
  grid = (int)std::max<long long>(1, std::min<long long>(grid, a.ntiles));
  Ring1 g = ring1(RP);
  void* fn = nullptr;
  size_t smem = 0;
  switch (RP) {
    case 16: fn = (void*)&t32_wpass_kernel<16>; smem = smem1<16>(g); break;
    case 32: fn = (void*)&t32_wpass_kernel<32>; smem = smem1<32>(g); break;
    case 48: fn = (void*)&t32_wpass_kernel<48>; smem = smem1<48>(g); break;
    default: fn = (void*)&t32_wpass_kernel<64>; smem = smem1<64>(g); break;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&bmap, &a, (void*)&g.nr, (void*)&g.no, (void*)&g.nq};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kT32Threads), args, smem, s);
}

cudaError_t launch_t32_ypass(const float* X, const ModeView& v, int R, const float* L, const float* W,
                             float* Ypart, double* spart, int* err, int ncol, cudaStream_t s, int init,
                             uint64_t sketch, const ModeState* st) {
  if (!t32_supported(v, R) || (!init && (!W || !L))) return cudaErrorInvalidValue;
  CUtensorMap bmap, wmap;
  if (!make_map(X, v.Q, v.I, v.P, kRows2, &bmap)) return cudaErrorInvalidValue;
  std::memset(&wmap, 0, sizeof(wmap));
  if (!init && !make_map(W, v.Q, R, v.P, R, &wmap)) return cudaErrorInvalidValue;
  const int RP = rp_of(R);
  T32Args a;
  std::memset(&a, 0, sizeof(a));
  a.I = (int)v.I;
  a.R = R;
  a.RP = RP;
  a.P = v.P;
  a.Q = v.Q;
  a.J = v.J();
  a.nkc = (int)((v.I + kKC - 1) / kKC);
  a.nch = t32_chunks(v);
  a.ntiles = v.J() / 32;
  a.L = L;
  a.Ypart = Ypart;
  a.spart = spart;
  a.err = err;
  a.init = init;
  a.sketch = sketch;
  a.st = st;
  a.flush = kFlush;
  ncol = (int)std::max<long long>(1, std::min<long long>(ncol, a.ntiles));
  int ns = stages2(RP);
  void* fn = nullptr;
  size_t smem = 0;
  switch (RP) {
    case 16: fn = (void*)&t32_ypass_kernel<16>; smem = smem2<16>(ns); break;
    case 32: fn = (void*)&t32_ypass_kernel<32>; smem = smem2<32>(ns); break;
    case 48: fn = (void*)&t32_ypass_kernel<48>; smem = smem2<48>(ns); break;
    default: fn = (void*)&t32_ypass_kernel<64>; smem = smem2<64>(ns); break;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&bmap, &wmap, &a, (void*)&ns};
  return cudaLaunchKernel(fn, dim3(a.nch, ncol), dim3(kT32Threads2), args, smem, s);
}

}  // namespace tals
