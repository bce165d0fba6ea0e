// Host-side launchers of the tals kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tals {

enum PassMode { PASS_INIT = 0, PASS_SWEEP = 1, PASS_PROJECT = 2, PASS_GIVEN = 3 };

// View of a row-major tensor for mode n: P (product of earlier sizes) x I_n x Q
// (product of later sizes). Column j = p*Q + q of the unfolding B_(n).
struct ModeView {
  long long P, I, Q;
  __host__ __device__ long long J() const { return P * Q; }
};

struct PassConfig {
  int rc = 0;        // r-chunk width of the instantiation
  int rpt = 0;       // rows per thread of the Y accumulation
  int rw = 0;        // r-columns per thread of the Y accumulation
  int grid_x = 0;    // CTAs along the tiles
  int grid_y = 0;    // r-chunks
  size_t smem = 0;   // dynamic shared memory
  int nbuf = 2;      // tile buffers (2: cp.async double buffering)
  int nt = 256;      // threads per CTA
  int jt = 16;       // unfolding columns per tile
  bool tr = false;   // transposed tile (Q = 1 views, FP32)
  bool ok = false;
};

// Pick the instantiation and launch shape for a pass over `v` with rank R.
PassConfig pass_config(int dtype, const ModeView& v, int R, int num_sms);

// One read of the tensor:
//   INIT:    Y += B_(n) S (S the seeded sketch), ||B||^2 partials
//   SWEEP:   W = B_(n)^T Lq, Y += B_(n) W, ||W||^2 partials, optional W output
//   PROJECT: W = B_(n)^T Lq, ||W||^2 partials, W output
//   GIVEN:   Y += B_(n) W with W read from Win (P x R x Q layout)
// Ypart: [grid_x][I][R] (dtype), spart: [grid_y*grid_x] doubles.
// W output layout: P x R x Q (the tensor B x_n Lq^T). Written when Wout != 0
// and (st == 0 or st->k >= w_from_k or st->k + 1 >= st->max_sweeps).
cudaError_t launch_pass(int dtype, const PassConfig& cfg, int mode, const void* X,
                        const ModeView& v, int R, const void* Lq, void* Ypart,
                        double* spart, void* Wout, uint64_t sketch_state,
                        const ModeState* st, int w_from_k, cudaStream_t s,
                        const void* Win = nullptr, int resid = 0);

// Y64[i][r] = sum_b Ypart[b][i][r] (FP64, fixed order); Gram partials per row
// block: gram_mode 1 = Y64^T Y64, 2 = L64^T Y64; scalar: sum of spart[0..nsp)
// stored into st->normM2 (which = 0, also into *norm_a2 if non-null) or st->sW (which = 1).
struct RowPlan { int rows_per_block; int blocks; };
RowPlan row_plan(long long I, int R, int num_sms);
cudaError_t launch_reduce_rows(int dtype, const void* Ypart, int gx, long long I, int R,
                               double* Y64, int gram_mode, const double* L64, double* Gpart,
                               const RowPlan& rp, const double* spart, int nsp, int which,
                               ModeState* st, double* norm_a2, cudaStream_t s,
                               void* YT = nullptr);

// Out[c][r] = In[r][c] for a rows x cols row-major matrix (dtype).
cudaError_t launch_transpose(int dtype, const void* In, long long rows, long long cols, void* Out,
                             cudaStream_t s);

// Gfin[o] = sum_b Gpart[b][o] over nb partials of R x R (deterministic order).
// write32: also an FP32 copy of the R x R result right after it (Gfin + R*R, as floats).
cudaError_t launch_gram_sum(const double* Gpart, int nb, int R, double* Gfin,
                            const ModeState* st, cudaStream_t s, int write32 = 0);

// Single-CTA FP64 kernel: sums nb Gram partials, then
//   op 0 (QR):   lower Cholesky factor F of the Gram (fails -> ESINGULAR)
//   op 1 (TEST): e_k = sqrt(normM2 - sW), Eq. 5.01 stop rule, k++, and if the
//                sweep continues, F = chol(Gram).
// When has_cond, thread 0 sets the CUDA graph conditional `cond` to 0 once the
// mode is done (stop rule, sweep budget or failure), ending the device-side loop.
// f32: factor in FP32 (a preconditioning factor; any pivot failure falls back to FP64).
cudaError_t launch_small(const double* Gpart, int nb, int R, int op, double* F,
                         ModeState* st, const double* norm_a2, unsigned long long cond,
                         int has_cond, cudaStream_t s, const double* GL = nullptr, int f32 = 0);

// F (small kernel output, 3 R^2 + R doubles): the lower Cholesky factor C, then
// its copies with rows scaled by 1 / C[r][r] and with columns scaled by
// 1 / C[c][c], then the R values 1 / C[r][r]. The row solves read the last three.
// Row-wise solves against the R x R lower factor F (FP64):
//   op 0 (LT):  Out = In F^-T          (Q factor of CholeskyQR)
//   op 1 (SPD): Out = In (F F^T)^-1
// optional: OutT (dtype copy of Out), Gpart (per-block Out^T Out partials).
cudaError_t launch_row_solve(int dtype, const double* In, long long I, int R, const double* F,
                             int op, double* Out, void* OutT, double* Gpart, const RowPlan& rp,
                             const ModeState* st, cudaStream_t s, int gram_rounded = 0);

// Copy `bytes` (a multiple of 4; both pointers 4-byte aligned, else
// cudaErrorInvalidValue) from src to dst, both in device memory, by a kernel.
cudaError_t launch_copy(void* dst, const void* src, size_t bytes, cudaStream_t s);

// Initialise a ModeState (k = 0, flags cleared) on the device. resid: the
// sweeps accumulate ||B - Q W^T||^2 directly (see PassArgs::resid).
// tc: the mode's products run on the split-precision tensor-core passes;
// split_ok: sweeps may run split; prod: sweeps run as two products (adjoint.cu).
cudaError_t launch_state_init(ModeState* st, double eta, int max_sweeps, int resid, cudaStream_t s,
                              int bulk_max = 0, int tc = 0, int split_ok = 0, int prod = 0);

// Tensor-core (tcgen05, BF16) sweep pass; see tc_pass.cu.
bool tc_supported(const ModeView& v, int R);
cudaError_t launch_tc_pass(const void* Xb, const ModeView& v, int R, const float* L, float* Ypart,
                           double* spart, int* err, int grid, cudaStream_t s, int init = 0,
                           uint64_t sketch = 0);
// Split-precision (3xTF32) sweep on tcgen05; see tf32_pass.cu. Views with Q % 32 == 0,
// I <= 1024, R <= 64.
bool t32_supported(const ModeView& v, int R);
// Floats of the split basis buffer of launch_t32_split_basis.
size_t t32_basis_floats(long long I, int R);
// CTAs of pass 1 (W), or column shares per 128-row chunk of pass 2 (Y), for a view
// on `sms` SMs; pass 2 runs t32_chunks(v) x t32_grid(v, 2, sms) CTAs.
int t32_grid(const ModeView& v, int pass, int sms);
int t32_chunks(const ModeView& v);
cudaError_t launch_t32_split_basis(const float* L, long long I, int R, float* QS, cudaStream_t s);
// Pass 1: W (P x R x Q) = B_(n)^T Q from the split basis QS, ||W||^2 per CTA in spart.
cudaError_t launch_t32_wpass(const float* X, const ModeView& v, int R, const float* QS, float* W,
                             double* spart, int* err, int grid, cudaStream_t s,
                             const ModeState* st = nullptr);
// Pass 2: Ypart[share] (I x R) = B_(n) W over each column share, and
// spart[share * chunks + chunk] = ||B - L W^T||^2 partials (L the FP32 basis W was
// formed with); init: W = the sketch S (L and W unused) and spart = ||B||^2 partials.
cudaError_t launch_t32_ypass(const float* X, const ModeView& v, int R, const float* L, const float* W,
                             float* Ypart, double* spart, int* err, int ncol, cudaStream_t s,
                             int init = 0, uint64_t sketch = 0, const ModeState* st = nullptr);
// st->sw_tc = sum of n partials (unless the mode is done).
cudaError_t launch_state_sum(const double* part, int n, ModeState* st, cudaStream_t s);
// out[p, a, q] = sum_b M[a*sa + b*sb] X[p, b, q] (FP32; cudaErrorNotSupported for
// views other than Q == 1, Q % 4 == 0 with 16-byte aligned X and out, or Q >= 64).
cudaError_t launch_mode_gemm(const float* X, long long P, long long Bin, long long Q, const float* M,
                             long long sa, long long sb, long long Aout, float* out, cudaStream_t s);
// st->sW = ||B_(n) - Q W^T||^2 of a sweep (FP32 data); part: scratch for up to
// cap FP64 partial sums.
cudaError_t launch_mode_residual(const float* X, const ModeView& v, int R, const float* W,
                                 const float* L, double* part, long long cap, ModeState* st,
                                 cudaStream_t s);
// launch_mode_gemm in loss form: out = 2 (M X - tgt) (the gradient of
// ||M X - tgt||^2 with respect to M X; tgt in out's layout, 16-byte aligned) and
// part[0 .. *nparts) the per-CTA sums of (M X - tgt)^2 (cudaErrorNotSupported where
// the register-tiled plan does not take the view or needs more than cap partials).
cudaError_t launch_mode_gemm_loss(const float* X, long long P, long long Bin, long long Q, const float* M,
                                  long long sa, long long sb, long long Aout, float* out, const float* tgt,
                                  double* part, long long cap, long long* nparts, cudaStream_t s);
// The register-tiled mode product of launch_mode_gemm, its CTAs exiting at once
// unless gate's sweep is split and not done (every = 1: unless the mode is done)
// (cudaErrorNotSupported where the register-tiled plan does not take the view;
// mode_gemm_gated_ok tells beforehand).
bool mode_gemm_gated_ok(const float* X, long long P, long long Bin, long long Q, const float* M, long long sa,
                        long long sb, long long Aout, float* out);
cudaError_t launch_mode_gemm_gated(const float* X, long long P, long long Bin, long long Q, const float* M,
                                   long long sa, long long sb, long long Aout, float* out, const ModeState* gate,
                                   cudaStream_t s, int every = 0);
// split.cu: the split sweep's statistics of W (||W||^2 and the rounded-basis term,
// two FP64 partials per CTA; nb = split_stat_blocks CTAs) and its Eq. 5.01 step.
int split_stat_blocks(const ModeView& v, int sms);
cudaError_t launch_split_stats(const float* W, const ModeView& v, int R, const double* GL, const ModeState* st,
                               double* part, int nb, cudaStream_t s);
cudaError_t launch_split_test(const double* part, int nb, ModeState* st, const double* norm_a2,
                              unsigned long long cond, int has_cond, cudaStream_t s);
// adjoint.cu: Ypart[s] (I x R) = B_(n) W over the s-th of S column ranges (FP32,
// R <= 64, Q % 16 == 0, 16-byte aligned X and W; adjoint_rows_ok tells), and, when
// wsq is set, wsq[s] = ||W||^2 over that range. CTAs exit at once when gate is
// set and its mode is done.
bool adjoint_rows_ok(const ModeView& v, int R, const void* X, const void* W);
int adjoint_rows_splits(const ModeView& v, int R, int sms);
cudaError_t launch_adjoint_rows(const float* X, const ModeView& v, const float* W, int R, int S, float* part,
                                double* wsq, const ModeState* gate, cudaStream_t s);
// Partial sums launch_mode_resid_gemm writes for this view (0: not covered).
long long mode_resid_gemm_parts(const float* X, long long P, long long Bin, long long Q, const float* M,
                                long long sa, long long sb, long long Aout, const float* B);
cudaError_t launch_mode_resid_gemm(const float* X, long long P, long long Bin, long long Q,
                                   const float* M, long long sa, long long sb, long long Aout,
                                   const float* B, double* part, cudaStream_t s);
// Any-view mode product out[p, a, q] = sum_b M[a*sa + b*sb] X[p, b, q]
// (T = float or double); the fallback of the paths above.
template <typename T>
cudaError_t launch_mode_gemm_any(const T* X, long long P, long long Bin, long long Q, const T* M, long long sa,
                                 long long sb, long long Aout, T* out, cudaStream_t s);
// Ubar (I x R) = X_(n) V_(n)^T for X viewed P x I x Q and V viewed P x R x Q, in
// S column splits (part: S * I * R elements of scratch).
int factor_adjoint_splits(long long P, long long I, long long Q, int R, int sms);
template <typename T>
cudaError_t launch_factor_adjoint_any(const T* X, long long P, long long I, long long Q, const T* V, int R,
                                      int S, T* part, T* Ubar, cudaStream_t s);
// twopass.cu: the two-pass sweep's building blocks.
// ||x||^2 as kSumsqParts FP64 partial sums (fixed grid), or summed into *out.
constexpr int kSumsqParts = 512;
cudaError_t launch_sumsq_parts(int dtype, const void* x, size_t n, double* part, cudaStream_t s);
cudaError_t launch_sumsq(int dtype, const void* x, size_t n, double* part, double* out, cudaStream_t s);
// S[p, r, q] = entry (p Q + q, r) of the Sec. 4 sketch drawn from `state`.
cudaError_t launch_sketch_prq(int dtype, void* S, const ModeView& v, int R, uint64_t state, int sms,
                              cudaStream_t s);
// out = X x_n U^T (P x R x Q) for any view: FP32 register-tiled GEMM where it
// applies, else plain shared-memory tiles (FP32 or FP64).
cudaError_t launch_mode_project_any(int dtype, const void* X, const ModeView& v, const void* U, int R, void* out,
                                    cudaStream_t s);
// Y (I x R) = X_(n) W_(n)^T for W viewed P x R x Q, in S column splits of at most
// 2048 columns (FP32 sums stay short; at most 4096 splits), the splits added in
// FP64 in a fixed order (part: S I R elements of scratch).
int twopass_splits(const ModeView& v, int R, int sms);
cudaError_t launch_mode_adjoint_any(int dtype, const void* X, const ModeView& v, const void* W, int R, int S,
                                    void* part, void* Y, cudaStream_t s);
// The column-split partials of launch_factor_adjoint_any without their sum:
// part[s][i][r] over the s-th of S equal column ranges (rounded up to 32).
template <typename T>
cudaError_t launch_factor_adjoint_parts(const T* X, long long P, long long I, long long Q, const T* V, int R,
                                        int S, T* part, cudaStream_t s);
// One CTA whose bounded mbarrier wait runs out after limit_cycles; *err = 5
// (TALS_ETIMEOUT) afterwards. Exercises the failure path without a fault.
cudaError_t launch_wait_timeout_probe(int* err, long long limit_cycles, cudaStream_t s);
cudaError_t launch_to_bf16(const float* x, void* y, size_t n, int sms, cudaStream_t s,
                           double* sq = nullptr);
int to_bf16_blocks(size_t n, int sms);

}  // namespace tals
