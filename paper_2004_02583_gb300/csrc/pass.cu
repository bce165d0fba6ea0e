// Grid-level launch of the fused ALS pass (see pass_impl.cuh for the device code).
#include <algorithm>

#include "pass_impl.cuh"

namespace tals {

template <typename T, int RC, int RPT, int RW, int NT, int JT, bool TR>
__global__ void __launch_bounds__(NT, 1) pass_kernel(PassArgs<T> a) {
  if (a.st != nullptr) {   // uniform early exits, before any barrier
    if (a.st->done) return;
    // split sweeps (split.cu): the fused pass yields to W alone, and the Y-only
    // pass runs only for a split sweep whose test did not stop the mode
    if (a.mode == PASS_SWEEP && a.st->split) return;
    if (a.mode == PASS_GIVEN && !a.st->split) return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* yp = a.Ypart != nullptr ? a.Ypart + (size_t)blockIdx.x * a.I * a.R : nullptr;
  const double tot =
      pass_cta<T, RC, RPT, RW, NT, JT, TR>(a, blockIdx.x, gridDim.x, blockIdx.y, smem_raw, yp);
  if (threadIdx.x == 0) a.spart[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// ---------------------------------------------------------------------------
// Host side: instantiation table and launch
// ---------------------------------------------------------------------------

namespace {

struct Inst {
  int rc, rpt, rw, nt, jt;
};

// Candidate instantiations per dtype. 512-thread shapes keep <= 128 registers
// per thread (16 warps per SM for latency hiding); 256-thread shapes serve
// larger per-thread tiles.
// Wider tiles (32 or 64 unfolding columns) keep the work per tile up for short
// modes, where a 16-column tile is only a few thousand elements.
const Inst kInstF32[] = {{32, 1, 16, 512, 16}, {32, 2, 16, 512, 16}, {32, 4, 16, 256, 16},
                         {16, 1, 16, 512, 16}, {16, 2, 16, 512, 16}, {16, 4, 16, 256, 16},
                         {8, 1, 8, 512, 16},   {8, 2, 8, 512, 16},   {8, 4, 8, 512, 16},
                         {8, 8, 8, 256, 16},
                         {32, 2, 8, 256, 64},  {16, 2, 4, 256, 64},  {16, 2, 8, 128, 64},
                         {8, 2, 4, 128, 64},   {32, 2, 16, 256, 32}, {16, 2, 8, 256, 32}};
const Inst kInstF64[] = {{16, 1, 8, 256, 16}, {16, 2, 8, 256, 16}, {16, 4, 8, 256, 16},
                         {8, 1, 8, 256, 16},  {8, 2, 8, 256, 16},  {8, 4, 8, 256, 16}};

template <typename T, int RC, int RPT, int RW, int NT, int JT, bool TR = false>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&pass_kernel<T, RC, RPT, RW, NT, JT, TR>);
}

// Instantiations with the transposed tile (views with Q = 1, FP32; an even
// number of ranks per step-1 lane).
const Inst kInstF32Tr[] = {{32, 4, 16, 256, 16}, {32, 2, 16, 512, 16}, {16, 1, 16, 512, 16},
                           {16, 4, 16, 256, 16}, {16, 2, 8, 128, 64},  {8, 2, 4, 128, 64},
                           {16, 2, 8, 256, 32},  {32, 2, 16, 256, 32}};

template <typename T>
void* lookup(const Inst& in, bool tr) {
#define TALS_CASE(RC, RPT, RW, NT, JT)                                               \
  if (in.rc == RC && in.rpt == RPT && in.rw == RW && in.nt == NT && in.jt == JT)     \
    return kernel_ptr<T, RC, RPT, RW, NT, JT>();
#define TALS_CASE_TR(RC, RPT, RW, NT, JT)                                            \
  if (in.rc == RC && in.rpt == RPT && in.rw == RW && in.nt == NT && in.jt == JT)     \
    return kernel_ptr<T, RC, RPT, RW, NT, JT, true>();
  if constexpr (sizeof(T) == 4) {
    if (tr) {
      TALS_CASE_TR(32, 4, 16, 256, 16) TALS_CASE_TR(32, 2, 16, 512, 16) TALS_CASE_TR(16, 1, 16, 512, 16)
      TALS_CASE_TR(16, 4, 16, 256, 16) TALS_CASE_TR(16, 2, 8, 128, 64) TALS_CASE_TR(8, 2, 4, 128, 64)
      TALS_CASE_TR(16, 2, 8, 256, 32) TALS_CASE_TR(32, 2, 16, 256, 32)
      return nullptr;
    }
    TALS_CASE(32, 1, 16, 512, 16) TALS_CASE(32, 2, 16, 512, 16) TALS_CASE(32, 4, 16, 256, 16)
    TALS_CASE(16, 1, 16, 512, 16) TALS_CASE(16, 2, 16, 512, 16) TALS_CASE(16, 4, 16, 256, 16)
    TALS_CASE(8, 1, 8, 512, 16) TALS_CASE(8, 2, 8, 512, 16) TALS_CASE(8, 4, 8, 512, 16)
    TALS_CASE(8, 8, 8, 256, 16)
    TALS_CASE(32, 2, 8, 256, 64) TALS_CASE(16, 2, 4, 256, 64) TALS_CASE(16, 2, 8, 128, 64)
    TALS_CASE(8, 2, 4, 128, 64) TALS_CASE(32, 2, 16, 256, 32) TALS_CASE(16, 2, 8, 256, 32)
  } else {
    TALS_CASE(16, 1, 8, 256, 16) TALS_CASE(16, 2, 8, 256, 16) TALS_CASE(16, 4, 8, 256, 16)
    TALS_CASE(8, 1, 8, 256, 16) TALS_CASE(8, 2, 8, 256, 16) TALS_CASE(8, 4, 8, 256, 16)
  }
#undef TALS_CASE
#undef TALS_CASE_TR
  return nullptr;
}

}  // namespace

namespace {

PassConfig pass_config_from(int dtype, const ModeView& v, int R, int num_sms, bool tr) {
  PassConfig cfg;
  const bool f32 = dtype == 1;
  const Inst* tab = tr ? kInstF32Tr : (f32 ? kInstF32 : kInstF64);
  const int ntab = tr ? (int)(sizeof(kInstF32Tr) / sizeof(Inst))
                      : (f32 ? (int)(sizeof(kInstF32) / sizeof(Inst)) : (int)(sizeof(kInstF64) / sizeof(Inst)));
  const size_t smem_max = 227 * 1024;
  // Score every fitting (instantiation, buffering): rank chunks re-read the
  // tensor (mostly from L2) and a single buffer exposes load latency; prefer
  // the smallest RPT (fewest idle rows) among equals.
  double best = 1e30;
  for (int nbuf = 2; nbuf >= 1; --nbuf) {
    for (int k = 0; k < ntab; ++k) {
      const Inst& in = tab[k];
      const int nrg = in.rc / in.rw;
      const int rowt = in.nt / nrg;
      if ((long long)rowt * in.rpt < v.I) continue;
      size_t sm = f32 ? pass_smem_bytes<float>(v.I, in.rc, rowt * in.rpt, nbuf, in.nt, in.jt, tr)
                      : pass_smem_bytes<double>(v.I, in.rc, rowt * in.rpt, nbuf, in.nt, in.jt);
      if (sm > smem_max) continue;
      const int chunks = (R + in.rc - 1) / in.rc;
      const double waste = (double)(in.rc * chunks - R) / (double)(in.rc * chunks);
      const double idle = (double)((long long)rowt * in.rpt - v.I) / (double)((long long)rowt * in.rpt);
      // fewer rank chunks and less padding first; then fewer idle rows; among
      // equals the larger per-thread tile (more FMAs per shared-memory load:
      // 4 rows x 16 ranks at 256 threads beats 2 x 16 at 512 when no row idles)
      // short tiles (I x columns well under 8K elements) are dominated by their
      // per-tile barriers and cross-warp reduction
      const double small_tile = std::max(0.0, 1.0 - (double)v.I * in.jt / 8192.0);
      const double score = chunks * (nbuf == 1 ? 1.35 : 1.0) * (1.0 + waste) +
                           (idle > 0.0 ? 0.01 + 0.5 * idle : 0.0) + 0.3 * small_tile -
                           1e-3 * in.rpt * in.rw / 16.0;
      if (score < best) {
        best = score;
        cfg.rc = in.rc;
        cfg.rpt = in.rpt;
        cfg.rw = in.rw;
        cfg.nt = in.nt;
        cfg.jt = in.jt;
        cfg.smem = sm;
        cfg.nbuf = nbuf;
        cfg.tr = tr;
        cfg.ok = true;
      }
    }
  }
  if (!cfg.ok) return cfg;
  cfg.grid_y = (R + cfg.rc - 1) / cfg.rc;
  const long long ntiles = (v.J() + cfg.jt - 1) / cfg.jt;
  int per_sm = (int)std::max<size_t>(1, (228 * 1024) / (cfg.smem + 1024));
  per_sm = std::min(per_sm, 2);
  long long gx = std::max<long long>(1, (long long)num_sms * per_sm / cfg.grid_y);
  gx = std::min(gx, ntiles);
  cfg.grid_x = (int)gx;
  return cfg;
}

}  // namespace

PassConfig pass_config(int dtype, const ModeView& v, int R, int num_sms) {
  // views with Q = 1 (the last mode): columns are contiguous rows, staged as a
  // transposed tile with 16-byte copies (FP32, I a multiple of 4); where no
  // transposed instantiation fits (I above 1024), the untransposed tile, whose
  // columns are then copied element by element
  if (dtype == 1 && v.Q == 1 && v.I % 4 == 0) {
    const PassConfig cfg = pass_config_from(dtype, v, R, num_sms, true);
    if (cfg.ok) return cfg;
  }
  return pass_config_from(dtype, v, R, num_sms, false);
}

cudaError_t launch_pass(int dtype, const PassConfig& cfg, int mode, const void* X,
                        const ModeView& v, int R, const void* Lq, void* Ypart, double* spart,
                        void* Wout, uint64_t sketch_state, const ModeState* st, int w_from_k,
                        cudaStream_t s, const void* Win, int resid) {
  if (!cfg.ok) return cudaErrorInvalidConfiguration;
  if (resid && cfg.grid_y != 1) return cudaErrorInvalidValue;
  const Inst in{cfg.rc, cfg.rpt, cfg.rw, cfg.nt, cfg.jt};
  if (cfg.tr && (dtype != 1 || v.Q != 1 || v.I % 4 != 0)) return cudaErrorInvalidValue;
  void* fn = dtype == 1 ? lookup<float>(in, cfg.tr) : lookup<double>(in, false);
  if (fn == nullptr) return cudaErrorInvalidDeviceFunction;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cfg.smem);
  if (e != cudaSuccess) return e;
  dim3 grid(cfg.grid_x, cfg.grid_y);
  const long long ntiles = (v.J() + cfg.jt - 1) / cfg.jt;
  const size_t esz = dtype == 1 ? 4 : 8;
  // 16-byte tile copies: rows of Q elements (of I elements for the transposed tile) stay aligned
  const int vec_ok = ((uintptr_t)X % 16 == 0) && (((cfg.tr ? v.I : v.Q) * esz) % 16 == 0);
  if (dtype == 1) {
    PassArgs<float> a{(const float*)X, v.P, v.I, v.Q, v.J(), R, mode, (const float*)Lq,
                      (const float*)Win, (float*)Ypart, spart, (float*)Wout, sketch_state, st,
                      w_from_k, ntiles, cfg.nbuf, vec_ok, resid};
    void* args[] = {&a};
    return cudaLaunchKernel(fn, grid, dim3(cfg.nt), args, cfg.smem, s);
  } else {
    PassArgs<double> a{(const double*)X, v.P, v.I, v.Q, v.J(), R, mode, (const double*)Lq,
                       (const double*)Win, (double*)Ypart, spart, (double*)Wout, sketch_state, st,
                       w_from_k, ntiles, cfg.nbuf, vec_ok, resid};
    void* args[] = {&a};
    return cudaLaunchKernel(fn, grid, dim3(cfg.nt), args, cfg.smem, s);
  }
}

}  // namespace tals
