// Mixed-precision form of the per-mode ALS: bulk sweeps on the tensor cores
// over a BF16 copy of the tensor, then finishing sweeps in FP32 on the original
// tensor until the Eq. 5.01 stop rule fires.
//
// The bulk sweeps drive the subspace to within BF16 resolution at half the
// bytes per sweep and tensor-core speed; the iterate stays the literal Alg. 3
// iterate of the (rounded) data, so the FP32 sweeps that follow start from it
// and contract the remaining error by sigma_{R+1}^2 / sigma_R^2 per sweep
// (Thm. 2). The stop rule is only evaluated on FP32 sweeps (at least two, so
// both compared errors are FP32), and the truncation W of Alg. 5 always comes
// from an FP32 sweep. Grams, Cholesky, QR and norms stay FP64 throughout.
// Modes whose shape the tensor-core pass does not cover (and the small later
// modes of st-HOSVD) run the plain FP32 path.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace tals {

struct MixedState {
  void* shadow = nullptr;       // BF16 copy of A
  size_t shadow_elems = 0;
  int* err = nullptr;           // tensor-core pass error flag
  double* sq = nullptr;         // per-block ||A||^2 partials of the conversion
  int sq_n = 0;
  const void* converted = nullptr;
};

tals_status mixed_alloc(tals_ctx* c) {
  if (c->mixed) return TALS_OK;
  c->mixed = new MixedState();
  size_t n = 1;
  for (int m = 0; m < c->N; ++m) n *= (size_t)c->dims[m];
  cudaError_t e = cudaMallocAsync(&c->mixed->shadow, n * 2, c->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&c->mixed->err, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->mixed->err, 0, sizeof(int), c->stream);
  c->mixed->sq_n = to_bf16_blocks(n, c->sms);
  if (e == cudaSuccess)
    e = cudaMallocAsync((void**)&c->mixed->sq, (size_t)c->mixed->sq_n * sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "BF16 shadow allocation");
  c->mixed->shadow_elems = n;
  return TALS_OK;
}

void mixed_free(tals_ctx* c) {
  if (!c->mixed) return;
  if (c->mixed->shadow) cudaFreeAsync(c->mixed->shadow, c->stream);
  if (c->mixed->err) cudaFreeAsync(c->mixed->err, c->stream);
  if (c->mixed->sq) cudaFreeAsync(c->mixed->sq, c->stream);
  delete c->mixed;
  c->mixed = nullptr;
}

// Whether mode job j runs its bulk sweeps on the tensor cores.
bool mixed_tc_mode(const tals_ctx* c, const ModeJob& j) {
  return c->mixed && j.X == c->A && c->dtype == TALS_F32 && tc_supported(j.v, j.R) &&
         c->opts.bulk_sweeps > 0;
}

// One CTA per SM, within the capacity of the per-CTA partial buffers (0: no room).
int mixed_grid(const tals_ctx* c, const ModeJob& j) {
  int grid = std::min<int>(c->sms, (int)((j.v.J() + 127) / 128));
  grid = (int)std::min<size_t>((size_t)grid, c->ypart_elems / ((size_t)j.v.I * j.R));
  grid = (int)std::min<size_t>((size_t)grid, c->spart_n);
  return std::max(grid, 0);
}

// BF16 copy and ||A||^2 in one read, then the Sec. 4 initial guess on the tensor
// cores: Y0 = B S over the BF16 copy (the sketch in BF16 too: any full-rank
// start serves, Thm. 2), then L0 = Q(Y0).
tals_status mixed_init_launch(tals_ctx* c, ModeJob& j, bool set_norm_a, int grid) {
  cudaStream_t s = c->stream;
  cudaError_t e = launch_to_bf16((const float*)c->A, c->mixed->shadow, c->mixed->shadow_elems, c->sms,
                                 s, c->mixed->sq);
  if (e != cudaSuccess) return cuda_fail(e, "BF16 conversion");
  e = launch_state_init(j.st, c->opts.eta, c->opts.max_sweeps, j.resid || j.t32, s, c->opts.bulk_sweeps,
                        j.t32, j.split_ok, j.prod);
  if (e == cudaSuccess)
    e = launch_tc_pass(c->mixed->shadow, j.v, j.R, nullptr, (float*)c->Ypart, c->spart,
                       c->mixed->err, grid, s, 1, sketch_state(c->opts.seed, j.n));
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core init pass");
  return mode_init_tail(c, j, set_norm_a, grid, c->mixed->sq, c->mixed->sq_n);
}

// One bulk sweep: the fused pass on the tensor cores, then the FP64 tail with
// the bulk-phase test (op 2).
tals_status mixed_bulk_sweep_launch(tals_ctx* c, ModeJob& j, int grid) {
  cudaError_t e = launch_tc_pass(c->mixed->shadow, j.v, j.R, (const float*)c->Lt, (float*)c->Ypart,
                                 c->spart, c->mixed->err, grid, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core pass");
  return mode_sweep_tail(c, j, grid, grid, 2);
}

tals_status tc_check(tals_ctx* c) {
  int err[2] = {0, 0};
  cudaError_t e = cudaSuccess;
  if (c->mixed)
    e = cudaMemcpyAsync(&err[0], c->mixed->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && c->t32_err)
    e = cudaMemcpyAsync(&err[1], c->t32_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core status");
  if (err[0] || err[1])
    return fail(TALS_ETIMEOUT, "a tensor-core pass gave up waiting (code %d)", err[0] ? err[0] : err[1]);
  return TALS_OK;
}

tals_status mixed_check(tals_ctx* c) { return tc_check(c); }

tals_status run_mode_mixed(tals_ctx* c, ModeJob& j, bool set_norm_a) {
  tals_status st = mode_setup(c, j);
  if (st != TALS_OK) return st;
  if (!mixed_tc_mode(c, j)) {
    if ((st = mode_init_launch(c, j, set_norm_a)) != TALS_OK) return st;
    if ((st = mode_loop_host(c, j, c->opts.max_sweeps)) != TALS_OK) return st;
    return tc_check(c);
  }
  const int grid = mixed_grid(c, j);
  if (grid < 1) return fail(TALS_ENOTSUP, "no room for the tensor-core partials");
  if ((st = mixed_init_launch(c, j, set_norm_a, grid)) != TALS_OK) return st;
  for (int k = 0; k < c->opts.max_sweeps; ++k) {
    if ((st = read_states(c)) != TALS_OK) return st;
    const ModeState& ms = c->st_host[j.n];
    if (ms.done) break;
    st = ms.bulk_mode ? mixed_bulk_sweep_launch(c, j, grid) : mode_sweep_launch(c, j);
    if (st != TALS_OK) return st;
  }
  if ((st = mixed_check(c)) != TALS_OK) return st;
  return read_states(c);
}

tals_status time_tc_pass(tals_ctx* c, const ModeJob& j, int iters, double* ms, double* bytes,
                         double* flops) {
  cudaStream_t s = c->stream;
  int grid = std::min<int>(c->sms, (int)((j.v.J() + 127) / 128));
  grid = (int)std::min<size_t>((size_t)grid, c->ypart_elems / ((size_t)j.v.I * j.R));
  grid = (int)std::min<size_t>((size_t)grid, c->spart_n);
  cudaError_t e = launch_to_bf16((const float*)c->A, c->mixed->shadow, c->mixed->shadow_elems,
                                 c->sms, s);
  if (e == cudaSuccess)
    e = launch_tc_pass(c->mixed->shadow, j.v, j.R, (const float*)c->Lt, (float*)c->Ypart, c->spart,
                       c->mixed->err, grid, s);   // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (int i = 0; i < iters && e == cudaSuccess; ++i)
    e = launch_tc_pass(c->mixed->shadow, j.v, j.R, (const float*)c->Lt, (float*)c->Ypart, c->spart,
                       c->mixed->err, grid, s);
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "timed tensor-core pass");
  const double T = (double)j.v.P * j.v.I * j.v.Q;
  if (ms) *ms = t / iters;
  if (bytes) *bytes = T * 2.0;   // one read of the BF16 copy
  if (flops) *flops = 4.0 * j.R * T;
  return TALS_OK;
}

}  // namespace tals

using namespace tals;

extern "C" tals_status tals_sweep_pass(const void* A, int ndim, const int64_t* dims, int mode,
                                       const void* Q, int R, int engine, double* Y_out,
                                       double* wnorm2, void* stream) {
  if (!A || !dims || !Q || !Y_out || ndim < 1 || ndim > TALS_MAX_NDIM || mode < 0 || mode >= ndim ||
      R < 1 || engine < 0 || engine > 5)
    return fail(TALS_EINVAL, "bad arguments");
  long long d[TALS_MAX_NDIM];
  size_t n = 1;
  for (int m = 0; m < ndim; ++m) {
    d[m] = dims[m];
    n *= (size_t)dims[m];
  }
  ModeView v = view_of(d, ndim, mode);
  if (R > v.I) return fail(TALS_EINVAL, "R exceeds I");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  void* ypart = nullptr;
  double* spart = nullptr;
  void* shadow = nullptr;
  int* err = nullptr;
  void* wbuf = nullptr;
  void* qs = nullptr;
  int sp_off = 0;   // where the ||W||^2 partials start in spart
  int gx = 0, nsp = 0;
  RowPlan rp = row_plan(v.I, R, sms);
  if (engine == 0) {
    PassConfig pc = pass_config(TALS_F32, v, R, sms);
    if (!pc.ok) return fail(TALS_ENOTSUP, "shape outside the pass kernel limits");
    gx = pc.grid_x;
    nsp = pc.grid_x * pc.grid_y;
    e = cudaMallocAsync(&ypart, (size_t)gx * v.I * R * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&spart, nsp * sizeof(double), s);
    if (e == cudaSuccess)
      e = launch_pass(TALS_F32, pc, PASS_SWEEP, A, v, R, Q, ypart, spart, nullptr, 0, nullptr, 0, s);
  } else if (engine == 5) {
    // the two-product form: W = B^T Q by the register-tiled mode product, then
    // Y = B W over column ranges with the ||W||^2 partials
    const size_t wn = (size_t)v.J() * R;
    if (!adjoint_rows_ok(v, R, A, A) ||
        !mode_gemm_gated_ok((const float*)A, v.P, v.I, v.Q, (const float*)Q, 1, R, R, (float*)A))
      return fail(TALS_ENOTSUP, "shape outside the two-product form's limits");
    gx = adjoint_rows_splits(v, R, sms);
    nsp = gx;
    e = cudaMallocAsync(&ypart, (size_t)gx * v.I * R * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&spart, nsp * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&wbuf, wn * 4, s);
    if (e == cudaSuccess)
      e = launch_mode_gemm((const float*)A, v.P, v.I, v.Q, (const float*)Q, 1, R, R, (float*)wbuf, s);
    if (e == cudaSuccess)
      e = launch_adjoint_rows((const float*)A, v, (const float*)wbuf, R, gx, (float*)ypart, spart, nullptr, s);
  } else if (engine >= 2) {
    if (!t32_supported(v, R)) return fail(TALS_ENOTSUP, "shape outside the split-TF32 pass limits");
    // engine 3 / 4 (diagnostics): one of the two passes replaced by the CUDA-core
    // pass (3: tensor-core W, CUDA-core Y; 4: CUDA-core W, tensor-core Y)
    const PassConfig pc = pass_config(TALS_F32, v, R, sms);
    if (engine > 2 && !pc.ok) return fail(TALS_ENOTSUP, "shape outside the pass kernel limits");
    const int g1 = engine == 4 ? pc.grid_x * pc.grid_y : t32_grid(v, 1, sms);
    const int ncol = t32_grid(v, 2, sms);
    const int np = std::max(ncol * t32_chunks(v), pc.ok ? pc.grid_x * pc.grid_y : 0);
    gx = engine == 3 ? pc.grid_x : ncol;
    nsp = g1;
    e = cudaMallocAsync(&ypart, (size_t)std::max(gx, ncol) * v.I * R * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&spart, (size_t)(np + g1) * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&wbuf, (size_t)v.J() * R * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&qs, t32_basis_floats(v.I, R) * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_t32_split_basis((const float*)Q, v.I, R, (float*)qs, s);
    // the W pass's ||W||^2 partials go after the Y pass's partials: spart + np
    if (e == cudaSuccess) {
      if (engine == 4)
        e = launch_pass(TALS_F32, pc, PASS_PROJECT, A, v, R, Q, nullptr, spart + np, wbuf, 0, nullptr, 0, s);
      else
        e = launch_t32_wpass((const float*)A, v, R, (const float*)qs, (float*)wbuf, spart + np, err, g1, s);
    }
    if (e == cudaSuccess) {
      if (engine == 3)
        e = launch_pass(TALS_F32, pc, PASS_GIVEN, A, v, R, nullptr, ypart, spart, nullptr, 0, nullptr, 0,
                        s, wbuf);
      else
        e = launch_t32_ypass((const float*)A, v, R, (const float*)Q, (const float*)wbuf, (float*)ypart,
                             spart, err, ncol, s);
    }
    sp_off = np;
  } else {
    if (!tc_supported(v, R)) return fail(TALS_ENOTSUP, "shape outside the tensor-core pass limits");
    gx = std::min<int>(sms, (int)((v.J() + 127) / 128));
    nsp = gx;
    e = cudaMallocAsync(&ypart, (size_t)gx * v.I * R * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&spart, nsp * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&shadow, n * 2, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_to_bf16((const float*)A, shadow, n, sms, s);
    if (e == cudaSuccess) e = launch_tc_pass(shadow, v, R, (const float*)Q, (float*)ypart, spart, err, gx, s);
  }
  if (e == cudaSuccess)
    e = launch_reduce_rows(TALS_F32, ypart, gx, v.I, R, Y_out, 0, nullptr, nullptr, rp, nullptr, 0,
                           0, nullptr, nullptr, s);
  std::vector<double> sp(nsp);
  int herr = 0;
  if (e == cudaSuccess && nsp > 0)
    e = cudaMemcpyAsync(sp.data(), spart + sp_off, nsp * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && err) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* p : {(void*)ypart, (void*)spart, shadow, (void*)err, wbuf, qs})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "sweep pass");
  if (herr) return fail(TALS_ETIMEOUT, "tensor-core pass gave up waiting");
  double t = 0.0;
  for (double x : sp) t += x;
  if (wnorm2) *wnorm2 = t;
  return TALS_OK;
}
