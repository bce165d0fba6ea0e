// C ABI of the tals library: contexts, validation, the per-mode ALS driver
// (Alg. 3 with the Sec. 4 initial guess and the Eq. 5.01 stop rule), and the
// st-HOSVD-ALS (Alg. 5) and t-HOSVD-ALS (Alg. 4) drivers.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tals.h"
#include "common.cuh"
#include "kernels.h"
#include "internal.h"

using namespace tals;

namespace {
thread_local std::string g_err;
}

namespace tals {

tals_status fail(tals_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

tals_status cuda_fail(cudaError_t e, const char* what) {
  return fail(TALS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

ModeView view_of(const long long* dims, int N, int n) {
  ModeView v;
  v.P = 1;
  v.Q = 1;
  for (int m = 0; m < n; ++m) v.P *= dims[m];
  for (int m = n + 1; m < N; ++m) v.Q *= dims[m];
  v.I = dims[n];
  return v;
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace tals

// ---------------------------------------------------------------------------
// Workspace planning
// ---------------------------------------------------------------------------
namespace {

struct Need {
  size_t ypart = 0, spart = 0, gpart = 0, ir = 0, tbuf = 0, qs = 0, unf = 0;
  void add_mode(int dtype, const ModeView& v, int R, int sms, bool sweep) {
    if (bigr_rank(R)) {
      // large ranks (bigr.cu): Y and its column-range partials in Ypart, W in a
      // scratch tensor buffer, ||.||^2 partials over the fixed grid; no Gram
      // partials (the R x R products are GEMMs)
      ir = std::max(ir, (size_t)v.I * (size_t)R);
      spart = std::max(spart, (size_t)kSumsqParts);
      if (sweep) {
        ypart = std::max(ypart, (size_t)(twopass_splits(v, R, sms) + 1) * (size_t)v.I * (size_t)R);
        tbuf = std::max(tbuf, (size_t)(v.J() * R));
        // general views: the written-out unfolding and its R x J product
        if (v.P > 1 && v.Q > 1) unf = std::max(unf, (size_t)(v.P * v.I * v.Q) + (size_t)(v.J() * R));
      } else {
        PassConfig pc = pass_config(dtype, v, R, sms);
        if (pc.ok) spart = std::max(spart, (size_t)pc.grid_x * pc.grid_y);
      }
      return;
    }
    PassConfig pc = pass_config(dtype, v, R, sms);
    RowPlan rp = row_plan(v.I, R, sms);
    gpart = std::max(gpart, (size_t)rp.blocks * (size_t)R * (size_t)R);
    ir = std::max(ir, (size_t)v.I * (size_t)R);
    if (!pc.ok) {
      // beyond the fused pass: the two-pass sweep (Y and its column-split partials
      // in Ypart, W in a scratch tensor buffer) or the tiled mode product, both
      // with ||.||^2 partials over a fixed grid
      spart = std::max(spart, (size_t)kSumsqParts);
      if (sweep) {
        ypart = std::max(ypart, (size_t)(twopass_splits(v, R, sms) + 1) * (size_t)v.I * (size_t)R);
        tbuf = std::max(tbuf, (size_t)(v.J() * R));
      }
      return;
    }
    if (sweep) ypart = std::max(ypart, (size_t)pc.grid_x * (size_t)v.I * (size_t)R);
    spart = std::max(spart, (size_t)pc.grid_x * pc.grid_y);
    if (sweep && dtype == TALS_F32) {
      // split sweeps: the W statistics' partials after the pass's, W in a scratch buffer
      spart = std::max(spart, (size_t)pc.grid_x * pc.grid_y + 2 * (size_t)split_stat_blocks(v, sms));
      tbuf = std::max(tbuf, (size_t)(v.J() * R));
      if (v.Q == 1) {
        // thin last modes as a GEMM pair: the row-range Y partials, ||W||^2 partials
        ypart = std::max(ypart, (size_t)thin_splits(v) * (size_t)v.I * (size_t)R);
        spart = std::max(spart, (size_t)kSumsqParts);
      }
      if (R <= 64 && v.Q % 16 == 0) {
        // the two-product form: the split-K Y product's partials and ||W||^2 partials
        const size_t S = (size_t)adjoint_rows_splits(v, R, sms);
        ypart = std::max(ypart, S * (size_t)v.I * (size_t)R);
        spart = std::max(spart, S + 2 * (size_t)split_stat_blocks(v, sms));
      }
    }
    if (sweep && dtype == TALS_F32 && t32_supported(v, R)) {
      // split-precision passes: per-CTA Y partials, W written every sweep (into a
      // scratch tensor buffer where the mode has no destination), the split basis
      ypart = std::max(ypart, (size_t)t32_grid(v, 2, sms) * (size_t)v.I * (size_t)R);
      spart = std::max(spart, (size_t)t32_grid(v, 1, sms) +
                                  (size_t)t32_grid(v, 2, sms) * (size_t)t32_chunks(v));
      tbuf = std::max(tbuf, (size_t)(v.J() * R));
      qs = std::max(qs, t32_basis_floats(v.I, R));
    }
  }
};

std::vector<int> default_order(const int* ranks, int N) {
  std::vector<int> o(N);
  for (int i = 0; i < N; ++i) o[i] = i;
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return ranks[a] < ranks[b]; });
  return o;
}

}  // namespace

namespace tals {

tals_status ctx_plan_and_alloc(tals_ctx* c) {
  const int N = c->N;
  Need need;
  // st-HOSVD shapes (in the context's order)
  {
    long long d[TALS_MAX_NDIM];
    for (int m = 0; m < N; ++m) d[m] = c->dims[m];
    for (int idx = 0; idx < N; ++idx) {
      const int n = c->order[idx];
      ModeView v = view_of(d, N, n);
      need.add_mode(c->dtype, v, c->ranks[n], c->sms, true);
      if (idx < N - 1) need.tbuf = std::max(need.tbuf, (size_t)(v.J() * c->ranks[n]));
      d[n] = c->ranks[n];
    }
  }
  // t-HOSVD shapes: every mode on A, then projections on shrinking tensors
  {
    long long d[TALS_MAX_NDIM];
    for (int m = 0; m < N; ++m) d[m] = c->dims[m];
    for (int n = 0; n < N; ++n) {
      ModeView v = view_of(d, N, n);
      need.add_mode(c->dtype, v, c->ranks[n], c->sms, true);
    }
    ModeView v = view_of(d, N, N - 1);
    need.tbuf = std::max(need.tbuf, (size_t)(v.J() * c->ranks[N - 1]));
    d[N - 1] = c->ranks[N - 1];
    for (int m = 0; m < N - 1; ++m) {
      ModeView w = view_of(d, N, m);
      need.add_mode(c->dtype, w, c->ranks[m], c->sms, false);
      need.tbuf = std::max(need.tbuf, (size_t)(w.J() * c->ranks[m]));
      d[m] = c->ranks[m];
    }
  }
  // HOOI shapes (Sec. 6.3): the ALS of mode n on A x_{m != n} U_m^T and the mode
  // products forming it (smaller views of the same modes; a view outside the pass
  // limits only makes tals_hooi return TALS_ENOTSUP)
  {
    std::vector<ViewR> sw, pr;
    hooi_views(N, c->dims, c->ranks, &sw, &pr, nullptr);
    for (const ViewR& x : sw) need.add_mode(c->dtype, x.v, x.R, c->sms, true);
    for (const ViewR& x : pr) need.add_mode(c->dtype, x.v, x.R, c->sms, false);
  }
  const size_t esz = c->esz;
  cudaStream_t s = c->stream;
  auto al = [&](void** p, size_t bytes) -> cudaError_t {
    return cudaMallocAsync(p, std::max<size_t>(bytes, 256), s);
  };
  cudaError_t e;
#define TALS_AL(ptr, bytes)                                                        \
  if ((e = al((void**)&(ptr), (bytes))) != cudaSuccess) {                          \
    return cuda_fail(e, "workspace allocation");                                   \
  }
  TALS_AL(c->tbuf[0], need.tbuf * esz);
  TALS_AL(c->tbuf[1], need.tbuf * esz);
  TALS_AL(c->Ypart, need.ypart * esz);
  TALS_AL(c->spart, need.spart * sizeof(double));
  TALS_AL(c->Gpart, need.gpart * sizeof(double));
  TALS_AL(c->GpartL, need.gpart * sizeof(double));
  int rmax = 1;
  for (int m = 0; m < N; ++m) rmax = std::max(rmax, c->ranks[m]);
  TALS_AL(c->Gfin, (size_t)rmax * rmax * (sizeof(double) + sizeof(float)));   // + FP32 copy
  TALS_AL(c->F, ((size_t)3 * rmax * rmax + rmax) * sizeof(double));   // [C | Ff | Fb | dinv]
  TALS_AL(c->GfinL, (size_t)rmax * rmax * sizeof(double));
  TALS_AL(c->Y64, need.ir * sizeof(double));
  TALS_AL(c->L64, need.ir * sizeof(double));
  TALS_AL(c->Z64, need.ir * sizeof(double));
  TALS_AL(c->Lt, need.ir * esz);
  if ((e = cudaMemsetAsync(c->Lt, 0, need.ir * esz, s)) != cudaSuccess)
    return cuda_fail(e, "workspace clear");
  TALS_AL(c->st, (size_t)TALS_MAX_NDIM * sizeof(ModeState));
  if (bigr_ws_doubles(rmax) > 0) TALS_AL(c->bw, bigr_ws_doubles(rmax) * sizeof(double));
  if (need.unf > 0) TALS_AL(c->ubuf, need.unf * esz);
  c->ubuf_elems = need.unf;
  TALS_AL(c->norm_a2, 8 * sizeof(double));
  if (need.qs > 0) {
    TALS_AL(c->QS, need.qs * sizeof(float));
    TALS_AL(c->t32_err, sizeof(int));
    if ((e = cudaMemsetAsync(c->t32_err, 0, sizeof(int), s)) != cudaSuccess)
      return cuda_fail(e, "workspace clear");
  }
#undef TALS_AL
  if ((e = cudaMallocHost((void**)&c->st_host, TALS_MAX_NDIM * sizeof(ModeState))) != cudaSuccess)
    return cuda_fail(e, "pinned state buffer");
  if ((e = cudaMallocHost((void**)&c->host_d, (need.spart + 16) * sizeof(double))) != cudaSuccess)
    return cuda_fail(e, "pinned scratch");
  c->host_d_n = need.spart + 16;
  c->need_ir = need.ir;
  c->ypart_elems = need.ypart;
  c->tbuf_elems = need.tbuf;
  c->spart_n = need.spart;
  return TALS_OK;
}

// ---------------------------------------------------------------------------
// Per-mode ALS (Alg. 3) on a given tensor view
// ---------------------------------------------------------------------------

// fp32_engine 0 (auto) puts the full-size FP32 modes of rank above 32 on the
// split-precision tensor-core passes: measured at 512^3, W + Y pass 0.221 + 0.447 ms
// (R = 48) and 0.235 + 0.498 ms (R = 64) against 0.951 ms for the CUDA-core fused
// pass, which runs two rank chunks there; at R <= 32 the fused pass is faster
// (0.489 ms against 0.210 + 0.407 ms at R = 32).
constexpr int kT32AutoMinRank = 33;
// fp32_engine 0 (auto) runs the full-size FP32 modes of rank up to 32 whose view
// has at least this many elements on the two-product form: W by the register-tiled
// mode product, Y = B W by the split-K adjoint (adjoint.cu).
constexpr int kProdAutoMaxRank = 32;
constexpr long long kProdAutoMinElems = 64LL << 20;
// Thin last modes run as a GEMM pair (bigr.cu) from this many elements on.
constexpr long long kThinMinElems = 16LL << 20;

tals_status mode_setup(tals_ctx* c, ModeJob& j) {
  j.st = c->st + j.n;
  // FP32: on tensors up to a quarter of the input (and at least 16M elements) the
  // sweeps measure e_k from the residual ||B - Q W^T||^2 directly; ||B||^2 - ||W||^2
  // cancels too many FP32 digits there (small e on small tensors). Costs one more
  // rank-R product per element on those small tensors only.
  long long tot = 1;
  for (int m = 0; m < c->N; ++m) tot *= c->dims[m];
  const long long mine = j.v.P * j.v.I * j.v.Q;
  const bool small_t = mine <= std::max(tot / 4, 16LL << 20);
  if (bigr_rank(j.R)) {
    // large rank: GEMM products, W in the destination or a scratch tensor buffer
    void* w = j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    const size_t ir = (size_t)j.v.I * j.R;
    j.splits = twopass_splits(j.v, j.R, c->sms);
    if (w == j.X || (size_t)(j.splits + 1) * ir > c->ypart_elems || ir > c->need_ir || c->blas == nullptr ||
        c->spart_n < (size_t)kSumsqParts || (j.Wdest == nullptr && (size_t)(j.v.J() * j.R) > c->tbuf_elems))
      return fail(TALS_ENOTSUP, "mode %d (I=%lld, R=%d) exceeds the context's workspace", j.n, j.v.I, j.R);
    j.bigr = 1;
    j.Wt = w;
    j.resid_kernel = c->dtype == TALS_F32 && small_t;
    // general views on the written-out unfolding (plain GEMMs), where it fits
    j.unf = j.v.P > 1 && j.v.Q > 1 &&
            (size_t)(j.v.P * j.v.I * j.v.Q) + (size_t)(j.v.J() * j.R) <= c->ubuf_elems;
    return TALS_OK;
  }
  j.pc = pass_config(c->dtype, j.v, j.R, c->sms);
  j.rp = row_plan(j.v.I, j.R, c->sms);
  j.twopass = 0;
  if (!j.pc.ok) {
    // I_n beyond the fused pass: two tiled products per sweep, W in the destination
    // or a scratch tensor buffer other than the input
    void* w = j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    const size_t ir = (size_t)j.v.I * j.R;
    j.splits = twopass_splits(j.v, j.R, c->sms);
    if (w == j.X || (size_t)(j.splits + 1) * ir > c->ypart_elems || ir > c->need_ir ||
        c->spart_n < (size_t)kSumsqParts)
      return fail(TALS_ENOTSUP, "mode %d (I=%lld, R=%d) exceeds the context's workspace", j.n, j.v.I, j.R);
    j.twopass = 1;
    j.t32 = 0;
    j.resid = 0;
    j.resid_kernel = (c->dtype == TALS_F32) && small_t;
    j.Wt = w;
    return TALS_OK;
  }
  j.resid = (c->dtype == TALS_F32) && j.pc.grid_y == 1 && small_t;
  // the same tensors with the rank split across CTAs cannot form the residual
  // inside the pass: the sweep writes W and a residual kernel takes it
  j.resid_kernel = (c->dtype == TALS_F32) && j.pc.grid_y > 1 && j.Wdest != nullptr && small_t;
  // a Q = 1 view without the transposed tile, in a context that holds cuBLAS (one
  // with a large-rank mode, whose loops are host-driven): the sweep as a GEMM pair
  // (bigr.cu), the fused pass's per-tile overhead avoided
  j.thin = 0;
  if (c->blas != nullptr && c->dtype == TALS_F32 && c->opts.fp32_engine == 0 && j.v.Q == 1 && !j.pc.tr &&
      !j.resid && !j.resid_kernel && mine >= kThinMinElems) {
    void* w = j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    const bool room = j.Wdest != nullptr || (size_t)(j.v.J() * j.R) <= c->tbuf_elems;
    if (w != j.X && room && (size_t)thin_splits(j.v) * j.v.I * j.R <= c->ypart_elems &&
        c->spart_n >= (size_t)kSumsqParts) {
      j.thin = 1;
      j.Wt = w;
    }
  }
  // the full-size FP32 modes: products on the split-precision tensor-core passes,
  // W written every sweep (the Y pass reads it) to the destination or a scratch
  // buffer that no other part of the mode uses
  // (engine 2: every mode whose view qualifies, its error then from the final
  // explicit residual instead of the per-sweep one)
  j.t32 = 0;
  const int eng = c->opts.fp32_engine;
  const bool want = !j.thin && (eng == 2 || (eng == 0 && j.R >= kT32AutoMinRank && !j.resid && !j.resid_kernel));
  if (c->dtype == TALS_F32 && want && c->QS != nullptr && t32_supported(j.v, j.R) &&
      (uintptr_t)j.X % 16 == 0) {
    void* w = j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    if ((uintptr_t)w % 16 == 0 && w != j.X) {
      j.t32 = 1;
      j.resid = 0;
      j.resid_kernel = 0;
      j.Wt = w;
      j.g1 = t32_grid(j.v, 1, c->sms);
      j.g2 = t32_grid(j.v, 2, c->sms);
    }
  }
  // Full-size FP32 modes of rank <= 32 (engine 3: every mode whose view qualifies)
  // on two products per sweep, W = B x_n Q_k^T (register-tiled mode product) into
  // the destination or a scratch buffer, then Y = B W (split-K adjoint, which also
  // sums ||W||^2): two reads of B, each product at a higher FMA rate than the
  // fused pass reaches with both
  j.prod = 0;
  if (c->dtype == TALS_F32 && !j.resid && !j.resid_kernel && !j.t32 && !j.thin &&
      (eng == 3 || (eng == 0 && j.R <= kProdAutoMaxRank && mine >= kProdAutoMinElems))) {
    void* w = j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    const bool room = j.Wdest != nullptr || (size_t)(j.v.J() * j.R) <= c->tbuf_elems;
    const size_t ir = (size_t)j.v.I * j.R;
    const long long S = std::min<long long>(adjoint_rows_splits(j.v, j.R, c->sms),
                                            (long long)std::min<size_t>(c->ypart_elems / ir, c->spart_n));
    if (w != j.X && room && S >= 1 && adjoint_rows_ok(j.v, j.R, j.X, w) &&
        mode_gemm_gated_ok((const float*)j.X, j.v.P, j.v.I, j.v.Q, (const float*)c->Lt, 1, j.R, j.R,
                           (float*)w)) {
      j.prod = 1;
      j.Wt = w;
      j.ys = (int)S;
    }
  }
  // FP32 modes whose error comes from ||B||^2 - ||W||^2: a sweep predicted to be
  // the last forms W alone (the register-tiled mode product into the destination
  // or a scratch buffer), takes the test, and forms Y only if needed
  j.split_ok = 0;
  if (c->dtype == TALS_F32 && !j.resid && !j.resid_kernel && !j.t32 && !j.thin) {
    void* w = j.prod ? j.Wt : j.Wdest;
    if (w == nullptr) w = (j.X == c->tbuf[1]) ? c->tbuf[0] : c->tbuf[1];
    const int nb = split_stat_blocks(j.v, c->sms);
    const bool room = j.Wdest != nullptr || (size_t)(j.v.J() * j.R) <= c->tbuf_elems;
    const size_t wpo = j.prod ? (size_t)j.ys : (size_t)j.pc.grid_x * j.pc.grid_y;
    if (w != j.X && room && wpo + 2 * (size_t)nb <= c->spart_n &&
        mode_gemm_gated_ok((const float*)j.X, j.v.P, j.v.I, j.v.Q, (const float*)c->Lt, 1, j.R, j.R,
                           (float*)w)) {
      j.split_ok = 1;
      j.Wt = w;
      j.nbw = nb;
      j.wpo = wpo;
    }
  }
  return TALS_OK;
}

uint64_t sketch_state(uint64_t seed, int mode) {
  return seed ^ ((uint64_t)mode << 56);
}

tals_status mode_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a) {
  return mode_init_launch_bulk(c, j, set_norm_a, 0);
}

tals_status mode_init_launch_bulk(tals_ctx* c, const ModeJob& j, bool set_norm_a, int bulk_max) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const long long I = j.v.I;
  cudaError_t e;
#define TALS_CK(x)                                   \
  if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x);
  TALS_CK(launch_state_init(j.st, c->opts.eta, c->opts.max_sweeps,
                            j.resid || j.resid_kernel || j.t32, s, bulk_max, j.t32, j.split_ok, j.prod));
  if (j.bigr) return bigr_init_launch(c, j, set_norm_a);
  if (j.thin) return thin_init_launch(c, j, set_norm_a);
  if (j.twopass) return twopass_init_launch(c, j, set_norm_a);
  if (j.t32) {
    // Sec. 4 on the tensor cores: Y0 = B_(n) S (split-precision) and ||B_(n)||^2
    TALS_CK(launch_t32_ypass((const float*)j.X, j.v, R, nullptr, nullptr, (float*)c->Ypart, c->spart,
                             c->t32_err, j.g2, s, 1, sketch_state(c->opts.seed, j.n), nullptr));
    return mode_init_tail(c, j, set_norm_a, j.g2, c->spart, j.g2 * t32_chunks(j.v));
  }
  // Sec. 4: Y0 = B_(n) S and ||B_(n)||^2 in one pass
  TALS_CK(launch_pass(c->dtype, j.pc, PASS_INIT, j.X, j.v, R, nullptr, c->Ypart, c->spart, nullptr,
                      sketch_state(c->opts.seed, j.n), j.st, 1 << 30, s));
#undef TALS_CK
  return mode_init_tail(c, j, set_norm_a, j.pc.grid_x, c->spart, j.pc.grid_x * j.pc.grid_y);
}

// Y0 partials are in Ypart (gx of them), the ||B||^2 partials in sp (nsp):
// reduce, then L0 = Q of QR(Y0).
tals_status mode_init_tail(tals_ctx* c, const ModeJob& j, bool set_norm_a, int gx, const double* sp,
                           int nsp) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const long long I = j.v.I;
  cudaError_t e;
#define TALS_CK(x)                                   \
  if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x);
  TALS_CK(launch_reduce_rows(c->dtype, c->Ypart, gx, I, R, c->Y64, 1, nullptr, c->Gpart, j.rp, sp,
                             nsp, 0, j.st, set_norm_a ? c->norm_a2 : nullptr, s));
  // L0 = Q of QR(Y0) by CholeskyQR2 (two rounds; Y0 can be ill-conditioned)
  TALS_CK(launch_gram_sum(c->Gpart, j.rp.blocks, R, c->Gfin, j.st, s));
  TALS_CK(launch_small(c->Gfin, 1, R, 0, c->F, j.st, c->norm_a2, j.cond, j.has_cond, s));
  TALS_CK(launch_row_solve(c->dtype, c->Y64, I, R, c->F, 0, c->Z64, nullptr, c->Gpart, j.rp, j.st, s));
  TALS_CK(launch_gram_sum(c->Gpart, j.rp.blocks, R, c->Gfin, j.st, s));
  TALS_CK(launch_small(c->Gfin, 1, R, 0, c->F, j.st, c->norm_a2, j.cond, j.has_cond, s));
  TALS_CK(launch_row_solve(c->dtype, c->Z64, I, R, c->F, 0, c->L64, c->Lt, c->GpartL, j.rp, j.st, s,
                           1));
  TALS_CK(launch_gram_sum(c->GpartL, j.rp.blocks, R, c->GfinL, j.st, s));
  return TALS_OK;
}

tals_status mode_sweep_launch(tals_ctx* c, const ModeJob& j) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const long long I = j.v.I;
  cudaError_t e;
  if (j.bigr) return bigr_sweep_launch(c, j);
  if (j.thin) return thin_sweep_launch(c, j);
  if (j.twopass) return twopass_sweep_launch(c, j);
  if (j.t32) {
    // split-precision passes: W = B^T Q_k (written), then Y = B W with the residual
    // ||B - Q_k W^T||^2 -- e_k of the stop rule -- from the same read of B
    const int np = j.g2 * t32_chunks(j.v);
    TALS_CK(launch_t32_split_basis((const float*)c->Lt, I, R, c->QS, s));
    TALS_CK(launch_t32_wpass((const float*)j.X, j.v, R, c->QS, (float*)j.Wt, c->spart + np, c->t32_err,
                             j.g1, s, j.st));
    TALS_CK(launch_state_sum(c->spart + np, j.g1, j.st, s));
    TALS_CK(launch_t32_ypass((const float*)j.X, j.v, R, (const float*)c->Lt, (const float*)j.Wt,
                             (float*)c->Ypart, c->spart, c->t32_err, j.g2, s, 0, 0, j.st));
    return mode_sweep_tail(c, j, j.g2, np, 1);
  }
  if (j.prod) {
    // W = B^T Q_k (Alg. 3 R-update) by the mode product; on a split sweep its
    // statistics and the Eq. 5.01 step (both exit at once otherwise); then Y = B W
    // (Alg. 3 L-update) and the ||W||^2 partials unless the test stopped the mode
    TALS_CK(launch_mode_gemm_gated((const float*)j.X, j.v.P, I, j.v.Q, (const float*)c->Lt, 1, R, R,
                                   (float*)j.Wt, j.st, s, 1));
    if (j.split_ok) {
      double* wpart = c->spart + j.wpo;
      TALS_CK(launch_split_stats((const float*)j.Wt, j.v, R, c->GfinL, j.st, wpart, j.nbw, s));
      TALS_CK(launch_split_test(wpart, j.nbw, j.st, c->norm_a2, j.cond, j.has_cond, s));
    }
    TALS_CK(launch_adjoint_rows((const float*)j.X, j.v, (const float*)j.Wt, R, j.ys, (float*)c->Ypart,
                                c->spart, j.st, s));
    return mode_sweep_tail(c, j, j.ys, j.ys, 1);
  }
  // one read of B: W = B^T Q_k (LS optimum for Q_k, Alg. 3 R-update), Y = B W
  // (the pass exits at once on a split sweep)
  TALS_CK(launch_pass(c->dtype, j.pc, PASS_SWEEP, j.X, j.v, R, c->Lt, c->Ypart, c->spart,
                      j.Wdest, 0, j.st, j.resid_kernel ? 0 : 1, s, nullptr, j.resid));
  if (j.split_ok) {
    // a split sweep (each kernel exits at once otherwise): W alone, its statistics
    // and the Eq. 5.01 step, then Y = B W only if the mode goes on
    double* wpart = c->spart + j.wpo;
    TALS_CK(launch_mode_gemm_gated((const float*)j.X, j.v.P, I, j.v.Q, (const float*)c->Lt, 1, R, R,
                                   (float*)j.Wt, j.st, s));
    TALS_CK(launch_split_stats((const float*)j.Wt, j.v, R, c->GfinL, j.st, wpart, j.nbw, s));
    TALS_CK(launch_split_test(wpart, j.nbw, j.st, c->norm_a2, j.cond, j.has_cond, s));
    TALS_CK(launch_pass(c->dtype, j.pc, PASS_GIVEN, j.X, j.v, R, nullptr, c->Ypart, c->spart, nullptr, 0, j.st,
                        0, s, j.Wt));
  }
  return mode_sweep_tail(c, j, j.pc.grid_x, j.pc.grid_x * j.pc.grid_y, 1);
}

tals_status mode_sweep_tail(tals_ctx* c, const ModeJob& j, int gx, int nsp, int test_op) {
  cudaStream_t s = c->stream;
  const int R = j.R;
  const long long I = j.v.I;
  cudaError_t e;
  // Y (FP64), X = Q_k^T Y partials, ||W||^2
  TALS_CK(launch_reduce_rows(c->dtype, c->Ypart, gx, I, R, c->Y64, 2, c->L64, c->Gpart,
                             j.rp, c->spart, nsp, 1, j.st, nullptr, s));
  // e_k^2 = ||B - Q W^T||^2 from this sweep's W (written by the pass) into sW;
  // the Y partials are consumed, so their buffer holds the residual partials
  if (j.resid_kernel && test_op == 1)
    TALS_CK(launch_mode_residual((const float*)j.X, j.v, R, (const float*)(j.twopass ? j.Wt : j.Wdest),
                                 (const float*)c->Lt, (double*)c->Ypart, (long long)(c->ypart_elems / 2),
                                 j.st, s));
  TALS_CK(launch_gram_sum(c->Gpart, j.rp.blocks, R, c->Gfin, j.st, s, c->dtype == TALS_F32));
  // e_k, Eq. 5.01, and chol(X) if the sweep continues
  // FP32 data: chol(X) in FP32 -- X^-1 only preconditions Z = Y X^-1 (span(Z) =
  // span(Y) for any invertible factor, applied exactly in FP64 by the row
  // solves); the factor of Z^T Z, which sets the orthonormality of Q, stays FP64
  const int f32 = c->dtype == TALS_F32;
  TALS_CK(launch_small(c->Gfin, 1, R, test_op, c->F, j.st, c->norm_a2, j.cond, j.has_cond, s,
                       c->GfinL, f32));
  // L_{k+1} = Y X^{-1} (Alg. 3 L-update in the Q_k basis), then its Q factor
  TALS_CK(launch_row_solve(c->dtype, c->Y64, I, R, c->F, 1, c->Z64, nullptr, c->Gpart, j.rp, j.st, s));
  TALS_CK(launch_gram_sum(c->Gpart, j.rp.blocks, R, c->Gfin, j.st, s));
  TALS_CK(launch_small(c->Gfin, 1, R, 0, c->F, j.st, c->norm_a2, j.cond, j.has_cond, s));
  TALS_CK(launch_row_solve(c->dtype, c->Z64, I, R, c->F, 0, c->L64, c->Lt, c->GpartL, j.rp, j.st, s,
                           1));
  TALS_CK(launch_gram_sum(c->GpartL, j.rp.blocks, R, c->GfinL, j.st, s));
#undef TALS_CK
  return TALS_OK;
}

tals_status read_states(tals_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->st_host, c->st, TALS_MAX_NDIM * sizeof(ModeState),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state readback");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return TALS_OK;
}

// Run the sweep loop of a mode until its state says done (host-driven).
tals_status mode_loop_host(tals_ctx* c, const ModeJob& j, int max_iters) {
  int launched = 0;
  tals_status st;
  // the stop rule can fire first after the second sweep: launch two before checking
  const int first = std::min(2, max_iters);
  for (; launched < first; ++launched)
    if ((st = mode_sweep_launch(c, j)) != TALS_OK) return st;
  while (true) {
    if ((st = read_states(c)) != TALS_OK) return st;
    const ModeState& ms = c->st_host[j.n];
    if (ms.done || launched >= max_iters) break;
    if ((st = mode_sweep_launch(c, j)) != TALS_OK) return st;
    ++launched;
  }
  return TALS_OK;
}

double t_hosvd_rel_err(const tals_ctx* c, double na2, double g2) {
  if (!(na2 > 0)) return 0.0;
  const int N = c->N;
  // rounded-basis terms of every mode (first-order corrections of ||G||^2)
  for (int n = 0; n < N; ++n) g2 -= c->st_host[n].corr;
  const ModeState& last = c->st_host[N - 1];
  double err2 = na2 - g2;
  if (last.tc_resid) {
    // e_N^2 (explicit residual) + ||W_N||^2 (of the stored W_N) - ||G||^2 (a mode
    // measured by its residual carries no rounded-basis term)
    err2 = last.e_cur * last.e_cur + last.sw_tc - g2;
  }
  return std::sqrt(std::max(err2, 0.0) / na2);
}

tals_status run_mode(tals_ctx* c, ModeJob& j, bool set_norm_a) {
  tals_status st = mode_setup(c, j);
  if (st != TALS_OK) return st;
  if ((st = mode_init_launch(c, j, set_norm_a)) != TALS_OK) return st;
  if ((st = mode_loop_host(c, j, c->opts.max_sweeps)) != TALS_OK) return st;
  return tc_check(c);
}

tals_status mode_status(tals_ctx* c, int n) {
  const ModeState& ms = c->st_host[n];
  if (ms.status != 0)
    return fail((tals_status)ms.status,
                "mode %d: Gram matrix not positive definite at %s (truncation above the "
                "numerical rank, Remark 3)",
                n, ms.fail_stage == 1 ? "the R-update" : "the QR step");
  return TALS_OK;
}

}  // namespace tals

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void tals_default_opts(tals_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eta = 1e-4;
  o->max_sweeps = 50;
  o->seed = 0;
  o->has_order = 0;
  o->precision = TALS_PREC_NATIVE;
  o->bulk_sweeps = 8;
  o->use_graph = 1;
}

const char* tals_last_error(void) { return g_err.c_str(); }

const char* tals_version(void) { return "tals 0.1 (sm_103a)"; }

tals_status tals_selftest_wait_timeout(double seconds, void* stream) {
  if (!(seconds > 0.0) || seconds > 10.0) return fail(TALS_EINVAL, "seconds must be in (0, 10]");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device clock");
  int* err = nullptr;
  if ((e = cudaMallocAsync(&err, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "status buffer");
  int host = -1;
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_wait_timeout_probe(err, (long long)(seconds * khz * 1e3), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  if (host == TALS_ETIMEOUT) return fail(TALS_ETIMEOUT, "bounded wait gave up as intended");
  return TALS_OK;
}

static tals_status validate(int dtype, int ndim, const int64_t* dims, const int* ranks) {
  if (dtype != TALS_F32 && dtype != TALS_F64) return fail(TALS_EINVAL, "unsupported dtype %d", dtype);
  if (ndim < 2 || ndim > TALS_MAX_NDIM) return fail(TALS_EINVAL, "ndim %d outside [2, 8]", ndim);
  if (!dims || !ranks) return fail(TALS_EINVAL, "dims/ranks must not be NULL");
  for (int n = 0; n < ndim; ++n) {
    if (dims[n] < 1) return fail(TALS_EINVAL, "dims[%d] = %lld < 1", n, (long long)dims[n]);
    if (ranks[n] < 1 || ranks[n] > dims[n])
      return fail(TALS_EINVAL, "ranks[%d] = %d outside [1, I_n = %lld]", n, ranks[n],
                  (long long)dims[n]);
    long long other = 1;
    for (int m = 0; m < ndim; ++m)
      if (m != n) other *= ranks[m];
    if (ranks[n] > other)
      return fail(TALS_EINVAL, "ranks[%d] = %d exceeds the product of the other ranks (%lld)", n,
                  ranks[n], other);
    if (ranks[n] > kBigRankMax)
      return fail(TALS_ENOTSUP, "ranks[%d] = %d above the largest supported rank %d", n, ranks[n], kBigRankMax);
  }
  return TALS_OK;
}

static tals_status ctx_create(tals_ctx** out, const void* A, bool owned, int dtype, int ndim,
                              const int64_t* dims, const int* ranks, const tals_opts* opts,
                              void* stream) {
  if (!out) return fail(TALS_EINVAL, "ctx must not be NULL");
  *out = nullptr;
  tals_status st = validate(dtype, ndim, dims, ranks);
  if (st != TALS_OK) return st;
  if (!owned && !A) return fail(TALS_EINVAL, "A must not be NULL");
  tals_ctx* c = new tals_ctx();
  c->dtype = dtype;
  c->esz = dtype == TALS_F32 ? 4 : 8;
  c->N = ndim;
  for (int n = 0; n < ndim; ++n) {
    c->dims[n] = dims[n];
    c->ranks[n] = ranks[n];
  }
  if (opts) c->opts = *opts; else tals_default_opts(&c->opts);
  if (c->opts.max_sweeps < 1) {
    delete c;
    return fail(TALS_EINVAL, "max_sweeps must be >= 1");
  }
  if (c->opts.precision == TALS_PREC_MIXED_BF16 && dtype != TALS_F32) {
    delete c;
    return fail(TALS_EINVAL, "mixed BF16 precision needs an FP32 tensor");
  }
  std::vector<int> ord;
  if (c->opts.has_order) {
    std::vector<int> seen(ndim, 0);
    for (int i = 0; i < ndim; ++i) {
      const int n = c->opts.order[i];
      if (n < 0 || n >= ndim || seen[n]) {
        delete c;
        return fail(TALS_EINVAL, "order is not a permutation of 0..%d", ndim - 1);
      }
      seen[n] = 1;
      ord.push_back(n);
    }
  } else {
    ord = default_order(ranks, ndim);
  }
  for (int i = 0; i < ndim; ++i) c->order[i] = ord[i];
  c->stream = (cudaStream_t)stream;
  c->sms = device_sms();
  if (c->sms <= 0) {
    delete c;
    return fail(TALS_ECUDA, "no CUDA device available");
  }
  for (int n = 0; n < ndim; ++n) c->has_bigr = c->has_bigr || bigr_rank(ranks[n]);
  // a rank above 64: those modes read their stop flag on the host every sweep
  if (c->has_bigr) c->opts.use_graph = 0;
  st = ctx_plan_and_alloc(c);
  if (st == TALS_OK && c->has_bigr) st = bigr_open(c);
  if (st == TALS_OK && owned) {
    size_t n = 1;
    for (int m = 0; m < ndim; ++m) n *= (size_t)dims[m];
    cudaError_t e = cudaMallocAsync(&c->A_owned, n * c->esz, c->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "tensor allocation");
    c->A = c->A_owned;
  } else {
    c->A = A;
  }
  if (st == TALS_OK && c->opts.precision == TALS_PREC_MIXED_BF16) st = mixed_alloc(c);
  if (st != TALS_OK) {
    tals_destroy(c);
    return st;
  }
  *out = c;
  return TALS_OK;
}

tals_status tucker_als_init(tals_ctx** ctx, const void* A, int dtype, int ndim,
                            const int64_t* dims, const int* ranks, const tals_opts* opts,
                            void* stream) {
  return ctx_create(ctx, A, false, dtype, ndim, dims, ranks, opts, stream);
}

tals_status tucker_als_init_owned(tals_ctx** ctx, int dtype, int ndim, const int64_t* dims,
                                  const int* ranks, const tals_opts* opts, void* stream) {
  return ctx_create(ctx, nullptr, true, dtype, ndim, dims, ranks, opts, stream);
}

tals_status tucker_als_init_strided(tals_ctx** ctx, const void* A, int dtype, int ndim, const int64_t* dims,
                                    const int64_t* strides, const int* ranks, const tals_opts* opts,
                                    void* stream) {
  if (!ctx) return fail(TALS_EINVAL, "ctx must not be NULL");
  *ctx = nullptr;
  if (!A || !dims || !strides) return fail(TALS_EINVAL, "A, dims and strides must not be NULL");
  if (ndim < 2 || ndim > TALS_MAX_NDIM) return fail(TALS_EINVAL, "ndim %d outside [2, 8]", ndim);
  if (!strides_valid(ndim, dims, strides))
    return fail(TALS_EINVAL, "strides must be non-negative and describe a tensor whose elements do not overlap");
  tals_status st = ctx_create(ctx, nullptr, true, dtype, ndim, dims, ranks, opts, stream);
  if (st != TALS_OK) return st;
  tals_ctx* c = *ctx;
  const cudaError_t e = launch_gather(dtype, A, ndim, dims, strides, c->A_owned, c->sms, c->stream);
  if (e != cudaSuccess) {
    tals_destroy(c);
    *ctx = nullptr;
    return cuda_fail(e, "strided gather");
  }
  return TALS_OK;
}

void* tals_ctx_tensor(tals_ctx* ctx) { return ctx ? const_cast<void*>(ctx->A) : nullptr; }

void tals_destroy(tals_ctx* c) {
  if (!c) return;
  cudaStream_t s = c->stream;
  graphs_destroy(c);
  mixed_free(c);
  if (c->upload) cudaStreamSynchronize(c->upload);
  bigr_close(c);
  void* bufs[] = {c->GpartL, c->GfinL, c->tbuf[0], c->tbuf[1], c->Ypart, c->spart, c->Gpart, c->Gfin, c->F,
                  c->Y64,     c->L64,     c->Z64,   c->Lt,    c->st,    c->norm_a2, c->A_owned,
                  c->A_owned2, c->hostio_G, c->pipe_G[0], c->pipe_G[1], c->bw, c->ubuf};
  for (void* p : bufs)
    if (p) cudaFreeAsync(p, s);
  for (int m = 0; m < TALS_MAX_NDIM; ++m)
    for (void* p : {c->hostio_U[m], c->pipe_U[0][m], c->pipe_U[1][m]})
      if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_loaded[i]) cudaEventDestroy(c->ev_loaded[i]);
    if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
  }
  if (c->upload) cudaStreamDestroy(c->upload);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->host_d) cudaFreeHost(c->host_d);
  delete c;
}

// Copy the current orthonormal factor Q (dtype) of a finished mode to U_out.
static tals_status emit_factor(tals_ctx* c, const ModeJob& j, void* U_out) {
  if (!U_out) return TALS_OK;
  cudaError_t e = launch_copy(U_out, c->Lt, (size_t)j.v.I * j.R * c->esz, c->stream);
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "factor copy");
}

static void fill_mode_stats(tals_ctx* c, int n, tals_stats* st) {
  if (!st) return;
  const ModeState& ms = c->st_host[n];
  st->err_per_mode[n] = ms.e_cur;
  st->sweeps[n] = ms.k;
  st->bulk_sweeps[n] = ms.bulk;
  st->tc_sweeps[n] = ms.tc_resid ? ms.k - ms.bulk : 0;
  st->split_capable[n] = ms.split_ok;
  st->split_sweeps[n] = ms.nsplit;
  st->two_product[n] = ms.prod;
  st->converged[n] = ms.converged;
  if (ms.status && !st->status) st->status = ms.status;
}

tals_status st_hosvd(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* stats) {
  if (!c || !G_out) return fail(TALS_EINVAL, "ctx and G_out must not be NULL");
  if (c->opts.use_graph) return st_hosvd_graph(c, G_out, U_out, stats);
  const int N = c->N;
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < N; ++m) d[m] = c->dims[m];
  const void* cur = c->A;
  tals_stats local;
  std::memset(&local, 0, sizeof(local));
  tals_status st;
  for (int idx = 0; idx < N; ++idx) {
    const int n = c->order[idx];
    ModeJob j;
    j.n = n;
    j.v = view_of(d, N, n);
    j.R = c->ranks[n];
    j.X = cur;
    j.Wdest = (idx == N - 1) ? G_out : c->tbuf[idx & 1];
    if (c->opts.precision == TALS_PREC_MIXED_BF16)
      st = run_mode_mixed(c, j, idx == 0);
    else
      st = run_mode(c, j, idx == 0);
    if (st != TALS_OK) return st;
    if ((st = read_states(c)) != TALS_OK) return st;
    if ((st = mode_status(c, n)) != TALS_OK) return st;
    if (U_out && (st = emit_factor(c, j, U_out[n])) != TALS_OK) return st;
    fill_mode_stats(c, n, &local);
    cur = j.Wdest;
    d[n] = c->ranks[n];
  }
  double na2 = 0.0;
  cudaError_t e = cudaMemcpyAsync(&c->host_d[0], c->norm_a2, sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "readback");
  na2 = c->host_d[0];
  double err2 = 0.0;
  for (int n = 0; n < N; ++n) err2 += local.err_per_mode[n] * local.err_per_mode[n];
  local.norm_a = std::sqrt(na2);
  local.rel_err = na2 > 0 ? std::sqrt(err2 / na2) : 0.0;
  for (int i = 0; i < N; ++i) local.order[i] = c->order[i];
  if (stats) *stats = local;
  return TALS_OK;
}

tals_status t_hosvd(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* stats) {
  if (!c || !G_out) return fail(TALS_EINVAL, "ctx and G_out must not be NULL");
  if (!U_out) return fail(TALS_EINVAL, "t_hosvd needs U_out (the projections read the factors)");
  for (int n = 0; n < c->N; ++n)
    if (!U_out[n]) return fail(TALS_EINVAL, "U_out[%d] is NULL", n);
  if (c->opts.use_graph) return t_hosvd_graph(c, G_out, U_out, stats);
  const int N = c->N;
  tals_stats local;
  std::memset(&local, 0, sizeof(local));
  tals_status st;
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < N; ++m) d[m] = c->dims[m];
  for (int n = 0; n < N; ++n) {
    ModeJob j;
    j.n = n;
    j.v = view_of(d, N, n);
    j.R = c->ranks[n];
    j.X = c->A;
    j.Wdest = (n == N - 1) ? c->tbuf[0] : nullptr;   // A x_n U^T of the last mode
    if (c->opts.precision == TALS_PREC_MIXED_BF16)
      st = run_mode_mixed(c, j, n == 0);
    else
      st = run_mode(c, j, n == 0);
    if (st != TALS_OK) return st;
    if ((st = read_states(c)) != TALS_OK) return st;
    if ((st = mode_status(c, n)) != TALS_OK) return st;
    if ((st = emit_factor(c, j, U_out[n])) != TALS_OK) return st;
    fill_mode_stats(c, n, &local);
  }
  // core: G = (A x_N U_N^T) x_1 U_1^T ... x_{N-1} U_{N-1}^T on shrinking tensors
  d[N - 1] = c->ranks[N - 1];
  const void* cur = c->tbuf[0];
  int nsp = 0;
  for (int m = 0; m < N - 1; ++m) {
    ModeView v = view_of(d, N, m);
    void* dest = (m == N - 2) ? G_out : c->tbuf[(m + 1) & 1];
    if ((st = project_mode(c, cur, v, c->ranks[m], U_out[m], dest, &nsp)) != TALS_OK) return st;
    cur = dest;
    d[m] = c->ranks[m];
  }
  cudaError_t e = cudaMemcpyAsync(c->host_d, c->spart, nsp * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->host_d + nsp, c->norm_a2, sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "readback");
  double g2 = 0.0;
  for (int i = 0; i < nsp; ++i) g2 += c->host_d[i];
  const double na2 = c->host_d[nsp];
  local.norm_a = std::sqrt(na2);
  local.rel_err = t_hosvd_rel_err(c, na2, g2);
  for (int i = 0; i < N; ++i) local.order[i] = i;
  if (stats) *stats = local;
  return TALS_OK;
}

tals_status st_hosvd_host(tals_ctx* c, const void* A_host, void* G_host, void* const* U_host,
                          tals_stats* stats) {
  if (!c || !A_host || !G_host) return fail(TALS_EINVAL, "NULL argument");
  if (!c->A_owned) return fail(TALS_EINVAL, "st_hosvd_host needs a context from tucker_als_init_owned");
  size_t nA = 1, nG = 1;
  for (int m = 0; m < c->N; ++m) {
    nA *= (size_t)c->dims[m];
    nG *= (size_t)c->ranks[m];
  }
  cudaError_t e = cudaMemcpyAsync(c->A_owned, A_host, nA * c->esz, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor upload");
  if (!c->hostio_G) {
    if ((e = cudaMallocAsync(&c->hostio_G, nG * c->esz, c->stream)) != cudaSuccess)
      return cuda_fail(e, "core buffer");
    for (int m = 0; m < c->N; ++m)
      if ((e = cudaMallocAsync(&c->hostio_U[m], (size_t)c->dims[m] * c->ranks[m] * c->esz,
                               c->stream)) != cudaSuccess)
        return cuda_fail(e, "factor buffer");
  }
  tals_status st = st_hosvd(c, c->hostio_G, c->hostio_U, stats);
  if (st != TALS_OK) return st;
  e = cudaMemcpyAsync(G_host, c->hostio_G, nG * c->esz, cudaMemcpyDeviceToHost, c->stream);
  for (int m = 0; m < c->N && e == cudaSuccess; ++m)
    if (U_host && U_host[m])
      e = cudaMemcpyAsync(U_host[m], c->hostio_U[m], (size_t)c->dims[m] * c->ranks[m] * c->esz,
                          cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "result download");
}

tals_status st_hosvd_host_many(tals_ctx* c, int count, const void* const* A_host,
                               void* const* G_host, void* const* U_host, tals_stats* stats) {
  if (!c || count < 1 || !A_host || !G_host) return fail(TALS_EINVAL, "NULL argument or count < 1");
  if (!c->A_owned) return fail(TALS_EINVAL, "st_hosvd_host_many needs a context from tucker_als_init_owned");
  const int N = c->N;
  for (int t = 0; t < count; ++t)
    if (!A_host[t] || !G_host[t]) return fail(TALS_EINVAL, "NULL host buffer for tensor %d", t);
  if (!c->opts.use_graph) {
    // the host-driven loop waits inside every decomposition: nothing to overlap
    for (int t = 0; t < count; ++t) {
      tals_status st = st_hosvd_host(c, A_host[t], G_host[t], U_host ? U_host + (size_t)t * N : nullptr,
                                     stats ? stats + t : nullptr);
      if (st != TALS_OK) return st;
    }
    return TALS_OK;
  }
  size_t nA = 1, nG = 1;
  for (int m = 0; m < N; ++m) {
    nA *= (size_t)c->dims[m];
    nG *= (size_t)c->ranks[m];
  }
  cudaError_t e = cudaSuccess;
  if (!c->A_owned2 && (e = cudaMallocAsync(&c->A_owned2, nA * c->esz, c->stream)) != cudaSuccess)
    return cuda_fail(e, "second tensor buffer");
  if (!c->upload) {
    if ((e = cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "upload stream");
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&c->ev_loaded[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pipeline events");
  }
  for (int i = 0; i < 2; ++i)
    if (!c->pipe_G[i]) {
      if ((e = cudaMallocAsync(&c->pipe_G[i], nG * c->esz, c->stream)) != cudaSuccess)
        return cuda_fail(e, "core buffer");
      for (int m = 0; m < N; ++m)
        if ((e = cudaMallocAsync(&c->pipe_U[i][m], (size_t)c->dims[m] * c->ranks[m] * c->esz,
                                 c->stream)) != cudaSuccess)
          return cuda_fail(e, "factor buffer");
    }
  void* bufs[2] = {c->A_owned, c->A_owned2};
  // uploads wait for everything already queued on the context's stream
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(c->ev_free[i], c->stream);
  auto upload = [&](int t, int slot) {
    cudaError_t u = cudaStreamWaitEvent(c->upload, c->ev_free[slot], 0);
    if (u == cudaSuccess)
      u = cudaMemcpyAsync(bufs[slot], A_host[t], nA * c->esz, cudaMemcpyHostToDevice, c->upload);
    if (u == cudaSuccess) u = cudaEventRecord(c->ev_loaded[slot], c->upload);
    return u;
  };
  if (e == cudaSuccess) e = upload(0, 0);
  if (e != cudaSuccess) return cuda_fail(e, "tensor upload");
  tals_status result = TALS_OK;
  for (int t = 0; t < count && result == TALS_OK; ++t) {
    const int slot = t & 1;
    if ((e = cudaStreamWaitEvent(c->stream, c->ev_loaded[slot], 0)) != cudaSuccess) {
      result = cuda_fail(e, "upload wait");
      break;
    }
    c->A = bufs[slot];
    if ((result = st_hosvd_graph_launch(c, c->pipe_G[slot], c->pipe_U[slot])) != TALS_OK) break;
    e = cudaEventRecord(c->ev_free[slot], c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(G_host[t], c->pipe_G[slot], nG * c->esz, cudaMemcpyDeviceToHost, c->stream);
    for (int m = 0; m < N && e == cudaSuccess; ++m)
      if (U_host && U_host[(size_t)t * N + m])
        e = cudaMemcpyAsync(U_host[(size_t)t * N + m], c->pipe_U[slot][m],
                            (size_t)c->dims[m] * c->ranks[m] * c->esz, cudaMemcpyDeviceToHost, c->stream);
    // tensor t+1 crosses the link while tensor t is decomposed; queued after the
    // decomposition's launch, so that a host thread held inside a large copy call
    // still finds the decomposition already running
    if (e == cudaSuccess && t + 1 < count && (e = upload(t + 1, slot ^ 1)) != cudaSuccess) {
      result = cuda_fail(e, "tensor upload");
      break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      result = cuda_fail(e, "result download");
      break;
    }
    result = st_hosvd_graph_collect(c, c->pipe_G[slot], c->pipe_U[slot], stats ? stats + t : nullptr);
  }
  c->A = c->A_owned;
  cudaStreamSynchronize(c->upload);   // no upload left in flight into a buffer reused later
  return result;
}

tals_status als_mode_sweep(tals_ctx* c, int mode, int max_iters, double* err_out,
                           int* converged_out) {
  if (!c || mode < 0 || mode >= c->N) return fail(TALS_EINVAL, "bad context or mode");
  if (max_iters < 0) return fail(TALS_EINVAL, "max_iters < 0");
  DriveState& ds = c->drive[mode];
  tals_status st;
  if (ds.finished) return fail(TALS_EINVAL, "mode %d already finished", mode);
  if (!ds.inited) {
    if (!c->cur) {
      c->cur = c->A;
      for (int m = 0; m < c->N; ++m) c->cur_dims[m] = c->dims[m];
    }
    ds.job.n = mode;
    ds.job.v = view_of(c->cur_dims, c->N, mode);
    ds.job.R = c->ranks[mode];
    ds.job.X = c->cur;
    ds.job.Wdest = c->tbuf[c->cur_buf];
    if ((st = mode_setup(c, ds.job)) != TALS_OK) return st;
    if ((st = mode_init_launch(c, ds.job, !c->norm_set)) != TALS_OK) return st;
    c->norm_set = true;
    ds.inited = true;
  }
  for (int k = 0; k < max_iters; ++k) {
    if ((st = read_states(c)) != TALS_OK) return st;
    if (c->st_host[mode].done) break;
    // before the stop rule fires no further sweep may overwrite W while it is
    // still needed, so W is written on every sweep once k >= 1
    if ((st = mode_sweep_launch(c, ds.job)) != TALS_OK) return st;
  }
  if ((st = read_states(c)) != TALS_OK) return st;
  if (ds.job.t32 && (st = tc_check(c)) != TALS_OK) return st;
  if ((st = mode_status(c, mode)) != TALS_OK) return st;
  if (err_out) *err_out = c->st_host[mode].e_cur;
  if (converged_out) *converged_out = c->st_host[mode].converged;
  return TALS_OK;
}

tals_status als_mode_finish(tals_ctx* c, int mode, void* U_out, int truncate) {
  if (!c || mode < 0 || mode >= c->N) return fail(TALS_EINVAL, "bad context or mode");
  DriveState& ds = c->drive[mode];
  if (!ds.inited) return fail(TALS_EINVAL, "mode %d has not been swept", mode);
  if (c->st_host[mode].k < 1) return fail(TALS_EINVAL, "mode %d needs at least one sweep", mode);
  tals_status st = emit_factor(c, ds.job, U_out);
  if (st != TALS_OK) return st;
  // the last sweep wrote W = B^T Q into tbuf[cur_buf] only if k >= 1 at its start
  // or it was the budgeted last; re-project when W is stale
  const ModeState& ms = c->st_host[mode];
  if (truncate) {
    // W of the last sweep is B x_n Q^T only when that sweep ended the mode; a
    // mode interrupted by the caller is truncated with its latest iterate
    if (!ms.done) {
      // the fused pass in projection mode, or the tiled mode product for the
      // modes beyond it (long modes, large ranks)
      cudaError_t e = ds.job.pc.ok ? launch_pass(c->dtype, ds.job.pc, PASS_PROJECT, ds.job.X, ds.job.v, ds.job.R,
                                                 c->Lt, nullptr, c->spart, ds.job.Wdest, 0, nullptr, 0, c->stream)
                                   : launch_mode_project_any(c->dtype, ds.job.X, ds.job.v, c->Lt, ds.job.R,
                                                             ds.job.Wdest, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "projection pass");
    }
    c->cur = ds.job.Wdest;
    c->cur_dims[mode] = c->ranks[mode];
    c->cur_buf ^= 1;
  }
  ds.finished = true;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "synchronize");
}

tals_status tals_pass_plan(int dtype, int64_t P, int64_t I, int64_t Q, int R, int num_sms,
                           int* plan_out) {
  if (dtype != TALS_F32 && dtype != TALS_F64) return fail(TALS_EINVAL, "unsupported dtype %d", dtype);
  if (P < 1 || I < 1 || Q < 1 || R < 1 || num_sms < 1 || !plan_out)
    return fail(TALS_EINVAL, "P, I, Q, R and num_sms must be >= 1, plan_out not NULL");
  const PassConfig pc = pass_config(dtype, ModeView{P, I, Q}, R, num_sms);
  if (!pc.ok) return fail(TALS_ENOTSUP, "no pass configuration fits I = %lld, R = %d", (long long)I, R);
  const int plan[10] = {pc.rc, pc.rpt, pc.rw, pc.nt, pc.jt, pc.nbuf, pc.tr ? 1 : 0, (int)pc.smem,
                        pc.grid_x, pc.grid_y};
  std::copy(plan, plan + 10, plan_out);
  return TALS_OK;
}

tals_status tals_time_sweep(tals_ctx* c, int mode, int engine, int iters, double* ms_out,
                            double* bytes_out, double* flops) {
  if (!c || mode < 0 || mode >= c->N || iters < 1 || engine < 0 || engine > 3 || !ms_out || !bytes_out)
    return fail(TALS_EINVAL, "bad arguments");
  ModeJob j;
  j.n = mode;
  j.v = view_of(c->dims, c->N, mode);
  j.R = c->ranks[mode];
  j.X = c->A;
  tals_status st = mode_setup(c, j);
  if (st != TALS_OK) return st;
  const double T = (double)j.v.P * j.v.I * j.v.Q;
  const double JR = (double)j.v.J() * j.R;
  ms_out[0] = ms_out[1] = bytes_out[0] = bytes_out[1] = 0.0;
  if (flops) *flops = 4.0 * j.R * T;
  if (j.bigr) return bigr_time_products(c, j, iters, ms_out, bytes_out);
  if (engine == 1) {
    if (!(c->mixed && c->dtype == TALS_F32 && tc_supported(j.v, j.R)))
      return fail(TALS_ENOTSUP, "the BF16 tensor-core pass needs a mixed-precision context and its shapes");
    return time_tc_pass(c, j, iters, &ms_out[0], &bytes_out[0], nullptr);
  }
  if (engine == 2 && !(c->dtype == TALS_F32 && c->QS && t32_supported(j.v, j.R) &&
                       (uintptr_t)j.X % 16 == 0))
    return fail(TALS_ENOTSUP, "view outside the split-precision pass limits");
  if (engine == 3 &&
      !(c->dtype == TALS_F32 && adjoint_rows_ok(j.v, j.R, j.X, c->tbuf[1]) &&
        mode_gemm_gated_ok((const float*)j.X, j.v.P, j.v.I, j.v.Q, (const float*)c->Lt, 1, j.R, j.R,
                           (float*)c->tbuf[1]) &&
        (size_t)(j.v.J() * j.R) <= c->tbuf_elems && c->tbuf[1] != c->A))
    return fail(TALS_ENOTSUP, "view outside the two-product form's limits");
  const int ys = engine == 3 ? (int)std::min<long long>(adjoint_rows_splits(j.v, j.R, c->sms),
                                                        (long long)(c->ypart_elems / ((size_t)j.v.I * j.R)))
                             : 0;
  cudaStream_t s = c->stream;
  float* W = (float*)c->tbuf[1];
  cudaEvent_t ev[3];
  for (auto& x : ev) cudaEventCreate(&x);
  double acc[2] = {0.0, 0.0};
  cudaError_t e = cudaSuccess;
  const int g1 = t32_grid(j.v, 1, c->sms), g2 = t32_grid(j.v, 2, c->sms);
  const int np = g2 * t32_chunks(j.v);
  if (engine == 2) e = launch_t32_split_basis((const float*)c->Lt, j.v.I, j.R, c->QS, s);
  for (int it = -1; it < iters && e == cudaSuccess; ++it) {   // it = -1: warm-up
    cudaEventRecord(ev[0], s);
    if (engine == 0) {
      e = launch_pass(c->dtype, j.pc, PASS_SWEEP, j.X, j.v, j.R, c->Lt, c->Ypart, c->spart, c->tbuf[0],
                      0, nullptr, 0, s);
      cudaEventRecord(ev[1], s);
    } else if (engine == 3) {
      e = launch_mode_gemm((const float*)j.X, j.v.P, j.v.I, j.v.Q, (const float*)c->Lt, 1, j.R, j.R, W, s);
      cudaEventRecord(ev[1], s);
      if (e == cudaSuccess)
        e = launch_adjoint_rows((const float*)j.X, j.v, W, j.R, ys, (float*)c->Ypart, c->spart, nullptr, s);
      cudaEventRecord(ev[2], s);
    } else {
      e = launch_t32_wpass((const float*)j.X, j.v, j.R, c->QS, W, c->spart + np, c->t32_err, g1, s);
      cudaEventRecord(ev[1], s);
      if (e == cudaSuccess)
        e = launch_t32_ypass((const float*)j.X, j.v, j.R, (const float*)c->Lt, W, (float*)c->Ypart,
                             c->spart, c->t32_err, g2, s);
      cudaEventRecord(ev[2], s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(engine == 0 ? ev[1] : ev[2]);
    float t0 = 0.f, t1 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess && engine >= 2) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
    if (it >= 0) {
      acc[0] += t0;
      acc[1] += t1;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "timed sweep");
  if ((st = tc_check(c)) != TALS_OK) return st;
  ms_out[0] = acc[0] / iters;
  bytes_out[0] = T * c->esz + JR * c->esz;   // tensor read + W written
  if (engine >= 2) {
    ms_out[1] = acc[1] / iters;
    bytes_out[1] = T * 4.0 + JR * 4.0;       // tensor read + W read (once; its other chunk
                                             // or row-tile CTAs find it in L2)
  }
  return TALS_OK;
}

tals_status tals_time_pass(tals_ctx* c, int mode, int iters, double* ms, double* bytes,
                           double* flops) {
  if (!c || mode < 0 || mode >= c->N || iters < 1) return fail(TALS_EINVAL, "bad arguments");
  ModeJob j;
  j.n = mode;
  j.v = view_of(c->dims, c->N, mode);
  j.R = c->ranks[mode];
  j.X = c->A;
  tals_status st = mode_setup(c, j);
  if (st != TALS_OK) return st;
  if (c->mixed && c->dtype == TALS_F32 && tc_supported(j.v, j.R))
    return time_tc_pass(c, j, iters, ms, bytes, flops);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = launch_pass(c->dtype, j.pc, PASS_SWEEP, j.X, j.v, j.R, c->Lt, c->Ypart, c->spart,
                              c->tbuf[0], 0, nullptr, 0, c->stream);   // warm-up
  cudaEventRecord(e0, c->stream);
  for (int i = 0; i < iters && e == cudaSuccess; ++i)
    e = launch_pass(c->dtype, j.pc, PASS_SWEEP, j.X, j.v, j.R, c->Lt, c->Ypart, c->spart,
                    c->tbuf[0], 0, nullptr, 0, c->stream);
  cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "timed pass");
  const double T = (double)j.v.P * j.v.I * j.v.Q;
  if (ms) *ms = t / iters;
  if (bytes) *bytes = T * c->esz + (double)j.v.J() * j.R * c->esz;
  if (flops) *flops = 4.0 * j.R * T;
  return TALS_OK;
}

}  // extern "C"
