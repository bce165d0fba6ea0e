// Library-internal declarations shared by the host-side translation units.
#pragma once

#include <cstdarg>
#include <cstddef>
#include <vector>

#include "../../include/tals.h"
#include "kernels.h"

namespace tals {

struct ModeJob {
  int n = 0;
  ModeView v{};
  int R = 0;
  const void* X = nullptr;       // tensor the mode reads
  void* Wdest = nullptr;         // where the final sweep writes B x_n Q^T (P x R x Q), or null
  PassConfig pc;
  RowPlan rp{};
  ModeState* st = nullptr;
  unsigned long long cond = 0;   // CUDA graph conditional handle of the sweep loop
  int has_cond = 0;
  int resid = 0;                 // sweeps measure the error from the explicit residual
  int resid_kernel = 0;          // rank split across CTAs: e_k from a residual kernel per sweep
  int t32 = 0;                   // FP32 sweeps on the split-precision (3xTF32) tensor-core passes
  void* Wt = nullptr;            // where those passes (or the two-pass form) write W every
                                 // sweep (Wdest or scratch)
  int g1 = 0, g2 = 0;            // their grids (W pass CTAs; Y pass column shares per chunk)
  int twopass = 0;               // I_n beyond the fused pass: two tiled products per sweep
  int splits = 1;                // column splits of the two-pass form's Y product
  int split_ok = 0;              // sweeps predicted to be the last run split (split.cu), W in Wt
  int nbw = 0;                   // CTAs of their W statistics
  size_t wpo = 0;                // offset of those statistics' partials in spart
  int prod = 0;                  // FP32 sweeps as two products (mode product W, split-K Y)
  int ys = 0;                    // column splits of that Y product
  int bigr = 0;                  // R above kBigRankMin: bigr.cu (GEMM products, blocked FP64 algebra)
  int thin = 0;                  // Q = 1 view without the fused pass's transposed tile, as a GEMM pair
  int unf = 0;                   // large rank on a general view: products on the written-out unfolding
};

struct DriveState {
  bool inited = false;
  bool finished = false;
  ModeJob job;
};

struct GraphCache;
struct MixedState;

tals_status fail(tals_status code, const char* fmt, ...);
tals_status cuda_fail(cudaError_t e, const char* what);
ModeView view_of(const long long* dims, int N, int n);
tals_status mode_setup(tals_ctx* c, ModeJob& j);
tals_status mode_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a);
tals_status mode_sweep_launch(tals_ctx* c, const ModeJob& j);
// The sweep chain after the pass: reduce, TEST (op), CholeskyQR update.
tals_status mode_sweep_tail(tals_ctx* c, const ModeJob& j, int gx, int nsp, int test_op);
tals_status mode_init_launch_bulk(tals_ctx* c, const ModeJob& j, bool set_norm_a, int bulk_max);
uint64_t sketch_state(uint64_t seed, int mode);
tals_status mode_init_tail(tals_ctx* c, const ModeJob& j, bool set_norm_a, int gx, const double* sp,
                           int nsp);
tals_status read_states(tals_ctx* c);
tals_status run_mode(tals_ctx* c, ModeJob& j, bool set_norm_a);
tals_status mode_loop_host(tals_ctx* c, const ModeJob& j, int max_iters);
// TALS_ESINGULAR with a message when mode n's state reports a failed factorisation.
tals_status mode_status(tals_ctx* c, int n);
// Error flags of the tensor-core passes (BF16 and split-precision).
tals_status tc_check(tals_ctx* c);
// t-HOSVD relative error from ||A||^2 (na2), ||G||^2 (g2) and the mode states (read
// back): ||A - G x U||^2 = ||A||^2 - ||G||^2 corrected by each mode's rounded-basis
// term; when the last mode ran on the tensor cores, the equivalent
// e_N^2 + ||A x_N U_N^T||^2 - ||G||^2 with e_N its explicit residual and the norm
// of the stored A x_N U_N^T, which does not rest on ||A||^2 - ||W||^2 of
// tensor-core products.
double t_hosvd_rel_err(const tals_ctx* c, double na2, double g2);

// twopass.cu: the mode's init and sweep for views beyond the fused pass
tals_status twopass_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a);
tals_status twopass_sweep_launch(tals_ctx* c, const ModeJob& j);
// out = X x_n U^T (fused pass in projection mode, else the tiled mode product);
// *nsp partial sums of ||out||^2 left in c->spart.
tals_status project_mode(tals_ctx* c, const void* X, const ModeView& v, int R, const void* U, void* out, int* nsp);
// strided.cu: element strides that describe a tensor without aliasing (non-negative,
// each axis of size above 1 stepping over the extent of the next smaller one), and
// the gather of such a tensor into the dense row-major layout.
bool strides_valid(int ndim, const int64_t* dims, const int64_t* strides);
cudaError_t launch_gather(int dtype, const void* src, int ndim, const int64_t* dims, const int64_t* strides,
                          void* dst, int sms, cudaStream_t s);
// bigr.cu: modes of rank above kBigRankMin (largest rank kBigRankMax). Their loop
// is host-driven: a sweep reads the stop flag before its L-update.
constexpr int kBigRankMin = 64;
constexpr int kBigRankMax = 1024;
bool bigr_rank(int R);
size_t bigr_ws_doubles(int rmax);
tals_status bigr_open(tals_ctx* c);
void bigr_close(tals_ctx* c);
tals_status bigr_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a);
tals_status bigr_sweep_launch(tals_ctx* c, const ModeJob& j);
// Mean durations (ms) and algorithmic bytes of a large-rank mode's two products
// (W = B^T Q, then Y = B W with its FP64 range sums), timed on the current basis.
tals_status bigr_time_products(tals_ctx* c, const ModeJob& j, int iters, double* ms, double* bytes);
// Thin last modes (bigr.cu): FP32 views with Q = 1 whose I_n rules out the fused
// pass's transposed tile, in contexts holding a cuBLAS handle: W = X Q and the
// row-range partials of Y = X^T W as GEMMs, then the fused path's tail over those
// partials. thin_splits: the number of row ranges (Y partials).
int thin_splits(const ModeView& v);
tals_status thin_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a);
tals_status thin_sweep_launch(tals_ctx* c, const ModeJob& j);

// hooi.cu: HOOI refinement (Sec. 6.3) and singular vectors (Sec. 5)
struct ViewR {
  ModeView v;
  int R;
};
// Modes other than skip (-1: all) in the order of a projection chain.
std::vector<int> hooi_chain(int N, const long long* dims, const int* ranks, int skip);
// The views HOOI runs on: the ALS of mode n on Y = A x_{m != n} U_m^T (sweeps), the
// mode products forming every Y and the initial core (products), and the largest
// product output (inter_elems).
void hooi_views(int N, const long long* dims, const int* ranks, std::vector<ViewR>* sweeps,
                std::vector<ViewR>* products, size_t* inter_elems);
tals_status hooi_run(tals_ctx* c, void* const* U, void* G_out, double tol, int max_iters, double inner_eta,
                     int inner_sweeps, double* resid_out, tals_hooi_stats* hs);
tals_status singular_vectors_run(tals_ctx* c, int mode, const void* Qhat, void* U_out, double* sigma_out);

// graph.cu: whole decompositions as one CUDA graph per context and output set
tals_status st_hosvd_graph(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* st);
// The cached st-HOSVD graph for (c->A, G_out, U_out), launched on c->stream without
// waiting; collect reads its status and statistics once the stream is synchronized.
tals_status st_hosvd_graph_launch(tals_ctx* c, void* G_out, void* const* U_out);
tals_status st_hosvd_graph_collect(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* stats);
tals_status t_hosvd_graph(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* st);
void graphs_destroy(tals_ctx* c);

// mixed.cu: BF16 shadow + tcgen05 bulk sweeps
tals_status mixed_alloc(tals_ctx* c);
void mixed_free(tals_ctx* c);
bool mixed_tc_mode(const tals_ctx* c, const ModeJob& j);
int mixed_grid(const tals_ctx* c, const ModeJob& j);
tals_status mixed_init_launch(tals_ctx* c, ModeJob& j, bool set_norm_a, int grid);
tals_status mixed_bulk_sweep_launch(tals_ctx* c, ModeJob& j, int grid);
tals_status mixed_check(tals_ctx* c);
tals_status run_mode_mixed(tals_ctx* c, ModeJob& j, bool set_norm_a);
tals_status time_tc_pass(tals_ctx* c, const ModeJob& j, int iters, double* ms, double* bytes,
                         double* flops);

}  // namespace tals

struct tals_ctx {
  int dtype = 0;
  size_t esz = 4;
  int N = 0;
  long long dims[TALS_MAX_NDIM] = {};
  int ranks[TALS_MAX_NDIM] = {};
  int order[TALS_MAX_NDIM] = {};
  tals_opts opts{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap[2] = {nullptr, nullptr};   // private streams used only for graph capture
  int sms = 0;
  const void* A = nullptr;
  void* A_owned = nullptr;
  // workspace
  void* tbuf[2] = {nullptr, nullptr};
  void* Ypart = nullptr;
  double* spart = nullptr;
  double* Gpart = nullptr;
  double* Gfin = nullptr;
  double* GpartL = nullptr;   // Gram partials of the stored (rounded) basis
  double* GfinL = nullptr;
  double* F = nullptr;
  double* Y64 = nullptr;
  double* L64 = nullptr;
  double* Z64 = nullptr;
  void* Lt = nullptr;
  tals::ModeState* st = nullptr;
  double* norm_a2 = nullptr;
  tals::ModeState* st_host = nullptr;   // pinned
  double* host_d = nullptr;             // pinned scratch
  size_t host_d_n = 0;
  size_t need_ir = 0;
  size_t ypart_elems = 0;     // capacity of Ypart (elements)
  size_t tbuf_elems = 0;      // capacity of each tbuf (elements)
  size_t spart_n = 0;         // capacity of spart
  // als_mode_sweep / als_mode_finish drive state
  tals::DriveState drive[TALS_MAX_NDIM];
  const void* cur = nullptr;
  long long cur_dims[TALS_MAX_NDIM] = {};
  int cur_buf = 0;
  bool norm_set = false;
  // st_hosvd_host device buffers
  void* hostio_G = nullptr;
  void* hostio_U[TALS_MAX_NDIM] = {};
  // st_hosvd_host_many: a second input buffer, the upload stream, and per slot
  // the upload / release events and the device outputs
  void* A_owned2 = nullptr;
  cudaStream_t upload = nullptr;
  cudaEvent_t ev_loaded[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  void* pipe_G[2] = {nullptr, nullptr};
  void* pipe_U[2][TALS_MAX_NDIM] = {};
  tals::GraphCache* graphs = nullptr;
  tals::MixedState* mixed = nullptr;
  float* QS = nullptr;        // split basis of the split-precision W pass
  int* t32_err = nullptr;     // error flag of the split-precision passes
  void* blas = nullptr;       // cuBLAS handle of the large-rank modes (bigr.cu)
  double* bw = nullptr;       // their R x R scratch (bigr_ws_doubles)
  bool has_bigr = false;      // some rank above kBigRankMin: host-driven mode loops
  void* ubuf = nullptr;       // a large-rank general view's unfolding and its R x J product
  size_t ubuf_elems = 0;
  const void* ubuf_src = nullptr;   // the tensor and mode whose unfolding ubuf holds
  int ubuf_mode = -1;
};
