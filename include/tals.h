/*
 * tals.h -- C ABI of the GB300 (sm_103a) library for ALS-based truncated HOSVD.
 *
 * Method: Xiao, Yang, Li, "Efficient Alternating Least Squares Algorithms for
 * Low Multilinear Rank Approximation of Tensors" (arXiv 2004.02583).
 *   - Alg. 3  matrix ALS  R_k = (A^T L_k)(L_k^T L_k)^-1,  L_{k+1} = (A R_k)(R_k^T R_k)^-1
 *   - Alg. 4  t-HOSVD-ALS (ALS per mode on A_(n), QR of L, core projection)
 *   - Alg. 5  st-HOSVD-ALS (ALS on B_(n), QR, B_(n) <- R^ R^T, G <- last B)
 *   - Sec. 4  initial guess  L_0 = Q of QR(A_(n) S), S uniform on [0,1)
 *   - Eq. 5.01 stop rule  | e_k - e_{k+1} | <= eta ||A||_F,  at most 50 sweeps (Sec. 6)
 *   - Sec. 2  mode-n unfolding, mode-n product, Tucker model
 *
 * Conventions shared by every entry point
 *   Tensors are dense, contiguous, row-major (C order): element (i_1..i_N) of a
 *   tensor with sizes (I_1..I_N) sits at offset ((i_1*I_2 + i_2)*I_3 + ...) + i_N
 *   (tucker_als_init_strided takes an input tensor in any strided layout).
 *   The mode-n unfolding column index j is the row-major linear index over the
 *   remaining modes in logical order (the paper writes the Fortran order; the
 *   two differ only by a column permutation, which no result depends on except
 *   the seeded random initial sketch S).
 *   Factor matrices U^(n) are I_n x R_n row-major: U[i*R_n + r].
 *   dtype: TALS_F64 (double) or TALS_F32 (float); one dtype per call for the
 *   tensor, the core and the factors.
 *   All data pointers are DEVICE pointers unless an entry point says "host".
 *   The library never writes the input tensor and never keeps a pointer to a
 *   caller buffer beyond the call (tucker_als_init keeps A until tals_destroy:
 *   the caller keeps A alive and unmodified until then).
 *   `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream. All device work of a call is enqueued on that stream. Calls that
 *   return statistics synchronise the stream once at their end.
 *   Errors: every call returns a tals_status; TALS_EINVAL for bad arguments
 *   (checked on the host before any launch), TALS_ECUDA for a CUDA runtime
 *   error, TALS_ESINGULAR when an R x R Gram matrix is not numerically positive
 *   definite (the truncation exceeds the numerical rank, Remark 3), TALS_ENOTSUP
 *   for shapes outside the kernels' limits. Contexts (tucker_als_init*): R_n <= 1024
 *   (checked on the host). Modes of rank up to 64 run the sweeps described
 *   below with their R x R algebra in single-CTA kernels; a mode of rank above 64
 *   (the dense test of Sec. 6.4, ranks (500, 500, 5)) forms its products as
 *   GEMMs (W = B^T Q, then Y = B W over column ranges of at most 2048 added in
 *   FP64) and its R x R algebra (Grams, Cholesky factors, triangular solves,
 *   CholeskyQR) as blocked FP64 GEMM algorithms; such a context runs every mode
 *   loop host-driven (use_graph is ignored: the host reads the stop flag after
 *   each sweep's test), and tals_hooi / tals_singular_vectors refuse it
 *   (TALS_ENOTSUP). A mode view whose I_n fits the fused sweep pass's
 *   shared-memory tile (up to 1920 in FP32 and 852 in FP64 at the smallest tile
 *   shapes, less for some ranks) reads the tensor once per sweep; a longer mode
 *   runs the same sweep as two tiled products (W = B^T Q, then Y = B W), reading
 *   it twice. The Tucker operators (reconstruct, project and their adjoints) take
 *   any sizes and ranks.
 *   tals_last_error() returns a
 *   thread-local message for the last failure. Not converging within
 *   max_sweeps is TALS_OK with converged[n] = 0.
 */
#ifndef TALS_H
#define TALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TALS_MAX_NDIM 8

typedef enum {
  TALS_OK = 0,
  TALS_EINVAL = 1,
  TALS_ENOMEM = 2,
  TALS_ECUDA = 3,
  TALS_ESINGULAR = 4,
  TALS_ETIMEOUT = 5,
  TALS_ENOTSUP = 6
} tals_status;

typedef enum { TALS_F64 = 0, TALS_F32 = 1 } tals_dtype;

/* Arithmetic of the unfolding products.
 *   TALS_PREC_NATIVE      products in the tensor dtype on CUDA cores (FP32 or FP64).
 *   TALS_PREC_MIXED_BF16  F32 tensors only: bulk sweeps read a BF16 shadow copy of
 *                         the tensor and run on tcgen05 tensor cores (BF16 operands,
 *                         FP32 accumulation); finishing sweeps run in FP32 on the
 *                         original tensor until the stop rule fires.
 * In every mode the Grams, Cholesky factorisations, QR and norms are FP64. */
typedef enum { TALS_PREC_NATIVE = 0, TALS_PREC_MIXED_BF16 = 1 } tals_precision;

typedef struct {
  double eta;            /* Eq. 5.01 tolerance; default 1e-4 (Sec. 6). eta < 0: never stop early */
  int max_sweeps;        /* ALS iterations (R-updates) per mode; default 50 (Sec. 6) */
  uint64_t seed;         /* seed of the initial sketch S (Sec. 4) */
  int has_order;         /* 1: use order[] for st-HOSVD; 0: ascending R_n, ties by n (Prop. 1) */
  int order[TALS_MAX_NDIM];
  int precision;         /* tals_precision */
  int bulk_sweeps;       /* mixed precision: most BF16 sweeps per mode (default 8) */
  int use_graph;         /* 1 (default): run each mode's sweep loop as one CUDA graph whose
                            device-side while-node evaluates the stop rule; 0: host loop */
  int fp32_engine;       /* FP32 products: 0 (default, auto) the faster engine per mode -- the
                            split-precision tensor-core passes for the modes of rank above 32
                            that read the full-size tensor, the two-product form (engine 3)
                            for the modes of rank up to 32 whose view has at least 2^26
                            elements (each where it measured faster than the fused pass),
                            the fused CUDA-core pass elsewhere; 1 the fused CUDA-core pass
                            for every mode; 2 split-precision 3xTF32 on the tcgen05 tensor
                            cores for every mode whose view qualifies (two passes per sweep;
                            views with Q % 32 == 0, I <= 1024, R <= 64), the stop rule's e_k
                            and the reported error taken from the explicit residual
                            ||B_(n) - Q W^T|| formed in the second pass; 3 the two-product
                            form on CUDA cores (exact FP32 arithmetic) for every mode whose
                            view qualifies (R <= 64, Q % 16 == 0, 16-byte aligned data):
                            W = B x_n Q^T by the register-tiled mode product, then
                            Y = B_(n) W split over column ranges -- two reads of B per
                            sweep. */
} tals_opts;

typedef struct {
  double rel_err;                       /* ||A - G x U||_F / ||A||_F (see st_hosvd/t_hosvd) */
  double norm_a;                        /* ||A||_F */
  double err_per_mode[TALS_MAX_NDIM];   /* e_n = ||B_(n) - L R^T||_F at the returned pair */
  int sweeps[TALS_MAX_NDIM];            /* R-updates performed on mode n (all precisions) */
  int bulk_sweeps[TALS_MAX_NDIM];       /* of which BF16 bulk sweeps */
  int tc_sweeps[TALS_MAX_NDIM];         /* of which FP32 sweeps on the split-precision (3xTF32)
                                           tensor-core passes */
  int converged[TALS_MAX_NDIM];         /* 1 if Eq. 5.01 fired before max_sweeps */
  int order[TALS_MAX_NDIM];             /* processing order used */
  int status;                           /* worst per-mode status */
  int split_capable[TALS_MAX_NDIM];     /* 1 if mode n's FP32 sweeps could run split: a sweep
                                           predicted to be the last forms W alone, takes the
                                           Eq. 5.01 test, and forms Y only if the loop goes on */
  int split_sweeps[TALS_MAX_NDIM];      /* sweeps of mode n that ran split */
  int two_product[TALS_MAX_NDIM];       /* 1 if mode n's FP32 sweeps ran as two products (the
                                           mode product W, then the split-K Y = B_(n) W) */
} tals_stats;

typedef struct tals_ctx tals_ctx;

/* Fills *o with the defaults above. */
void tals_default_opts(tals_opts* o);

/* Create a context for tensor A (device, dtype, ndim <= 8, dims[ndim] >= 1) with
 * truncation ranks[ndim]. Validates on the host: 1 <= R_n <= I_n and
 * R_n <= prod_{m != n} R_m (so every sequential truncation is feasible).
 * Allocates all workspace on `stream` (stream-ordered) and builds nothing else;
 * the context owns its workspace and frees it in tals_destroy. A must stay
 * alive and unmodified for the lifetime of the context. */
tals_status tucker_als_init(tals_ctx** ctx, const void* A, int dtype, int ndim,
                            const int64_t* dims, const int* ranks, const tals_opts* opts,
                            void* stream);

/* The user-drivable unit of Alg. 3: run up to max_iters ALS sweeps on the mode-n
 * unfolding of the context's current tensor (A for t-HOSVD, the partially
 * truncated B for st-HOSVD). The first call on a mode draws S and forms the
 * initial guess (Sec. 4); later calls continue from the stored iterate. Each
 * sweep reads the tensor once: with Q_k the orthonormal basis of L_k it forms
 * W = B_(n)^T Q_k and Y = B_(n) W in one pass (Eq. 2.2), e_k from
 * ||B_(n)||^2 - ||W||^2, and L_{k+1} = Y (Q_k^T Y)^-1 re-orthonormalised by
 * CholeskyQR, which leaves the iterates of Alg. 3 unchanged up to an R x R
 * triangular factor. Returns the current e_k in *err_out and whether the stop
 * rule (Eq. 5.01) has fired in *converged_out (either may be NULL). Synchronises
 * the stream. */
tals_status als_mode_sweep(tals_ctx* ctx, int mode, int max_iters, double* err_out,
                           int* converged_out);

/* Finish a mode driven by als_mode_sweep: write U^(n) (I_n x R_n, device) and, if
 * truncate != 0, replace the context's current tensor by B x_n U^(n)T taken from
 * the last sweep's W (Alg. 5, B_(n) <- R^ R^T; no extra pass over B). */
tals_status als_mode_finish(tals_ctx* ctx, int mode, void* U_out, int truncate);

/* st-HOSVD-ALS (Alg. 5) of the context's tensor. G_out: device buffer of
 * prod R_n elements (row-major R_1 x ... x R_N). U_out[n]: device buffers of
 * I_n x R_n. st (host, may be NULL) receives the statistics; rel_err is
 * sqrt(sum_n e_n^2) / ||A|| (the st-HOSVD error is the sum of the mode-wise
 * truncation errors, Lemma 2). May be called repeatedly on one context. */
tals_status st_hosvd(tals_ctx* ctx, void* G_out, void* const* U_out, tals_stats* st);

/* t-HOSVD-ALS (Alg. 4): every mode on A, then G = A x_1 U1^T ... x_N UN^T. The first
 * projection is the last mode's W (no extra pass), the rest run on shrinking
 * tensors. rel_err = sqrt(||A||^2 - ||G||^2) / ||A||. */
tals_status t_hosvd(tals_ctx* ctx, void* G_out, void* const* U_out, tals_stats* st);

/* Same as st_hosvd, with HOST buffers: copies A (host, dtype, dims as in the
 * context) to the device, runs st-HOSVD-ALS and copies G and U^(n) back to the
 * host buffers. The context's own device copy of A is used as the tensor; the
 * context must have been created with A == NULL (see tucker_als_init_owned). */
tals_status st_hosvd_host(tals_ctx* ctx, const void* A_host, void* G_host,
                          void* const* U_host, tals_stats* st);

/* st_hosvd_host over `count` tensors, pipelined: while tensor t is decomposed on
 * the context's stream, tensor t+1 is copied to a second device buffer on an
 * upload stream, so the host-to-device copies overlap the decompositions. Every
 * tensor is copied in full and every result copied back, in order.
 * A_host[t]: host tensor t (dims of the context; pinned memory for the copy to
 * run asynchronously); G_host[t]: host core; U_host: NULL or count*N host
 * factor pointers (U_host[t*N + n], I_n x R_n, any entry may be NULL); stats:
 * NULL or `count` entries. The caller owns every host buffer and keeps them
 * alive until the call returns (it returns after the last result is on the
 * host). Context: from tucker_als_init_owned; the first call allocates a second
 * tensor buffer and per-slot outputs (freed by tals_destroy). Without CUDA
 * graphs (opts.use_graph = 0) the tensors run one after another as
 * st_hosvd_host. Errors: TALS_EINVAL for NULL arguments or count < 1; the
 * first failing tensor's status otherwise (later tensors are not run). */
tals_status st_hosvd_host_many(tals_ctx* ctx, int count, const void* const* A_host,
                               void* const* G_host, void* const* U_host, tals_stats* stats);

/* Self-test of the failure path of the bounded device waits (failure detection
 * without a fault): one CTA waits on an mbarrier that nothing arrives at, using
 * the tensor-core pass's own bounded-wait helper with a limit of `seconds`
 * (0 < seconds <= 10) of SM clock cycles; the wait gives up, the kernel records
 * the timeout and returns, and the device stays usable. Returns TALS_ETIMEOUT
 * when the failure path works (TALS_OK would mean the wait completed), TALS_EINVAL
 * for a bad limit, TALS_ECUDA on a CUDA error. stream: a cudaStream_t or NULL. */
tals_status tals_selftest_wait_timeout(double seconds, void* stream);

/* Like tucker_als_init but the context allocates and owns a device buffer for A
 * (to be filled by st_hosvd_host or by copying into tals_ctx_tensor()). */
tals_status tucker_als_init_owned(tals_ctx** ctx, int dtype, int ndim, const int64_t* dims,
                                  const int* ranks, const tals_opts* opts, void* stream);

/* Like tucker_als_init for a tensor in any strided layout (the unfoldings of
 * Sec. 3 taken from the tensor as it is laid out): element (i_1..i_N) is at
 * A + sum_k i_k * strides[k], strides in elements, in any order (a permuted or
 * sliced view). The context gathers A into a dense row-major buffer it owns
 * (as tucker_als_init_owned), stream-ordered on `stream` during this call; the
 * decompositions then read that copy, so later changes of A are not seen, and the
 * caller keeps A alive and unchanged until the stream has run the gather.
 * Errors (checked on the host before any device work): TALS_EINVAL for NULL
 * pointers, ndim outside [2, 8], a negative stride, a zero stride on an axis of
 * size above 1, or strides under which two elements share an address (each axis
 * of size above 1 must step over the whole extent of the next smaller-strided
 * one); otherwise as tucker_als_init. */
tals_status tucker_als_init_strided(tals_ctx** ctx, const void* A, int dtype, int ndim, const int64_t* dims,
                                    const int64_t* strides, const int* ranks, const tals_opts* opts,
                                    void* stream);

/* Device pointer of the tensor the context reads (A, or its owned buffer). */
void* tals_ctx_tensor(tals_ctx* ctx);

/* Tucker reconstruction (Sec. 2): B = G x_1 U1 x_2 U2 ... x_N UN.
 * G: device, prod R_n elements; U[n]: device I_n x R_n; B_out: device prod I_n.
 * Intermediate mode products are formed in stream-ordered scratch. */
tals_status reconstruct(const void* G, void* const* U, int dtype, int ndim,
                        const int64_t* dims, const int* ranks, void* B_out, void* stream);

/* Reconstruction loss of the Tucker model (Sec. 2): f = ||G x_1 U1 ... x_N UN - A||_F^2
 * with its gradient with respect to the reconstruction, D_out = 2 (B - A) (device,
 * dims, same layout as A), formed without writing B: in FP32 the last mode product of
 * the reconstruction computes B - A, writes D_out and sums the squares from the same
 * registers; otherwise (FP64, or a last view the register-tiled product does not
 * take) B is written to D_out and turned into the gradient by one elementwise pass.
 * The gradients with respect to G and U follow from reconstruct_backward with
 * B_bar = D_out (scaled by the caller's output gradient). loss_out: a DEVICE double
 * (FP64 sum of FP32 squares, compensated per thread). D_out must not alias A.
 * Stream-ordered scratch; not synchronised. Errors as for reconstruct. */
tals_status reconstruction_loss(const void* G, void* const* U, const void* A, int dtype, int ndim,
                                const int64_t* dims, const int* ranks, void* D_out, double* loss_out,
                                void* stream);

/* Core projection G = A x_1 U1^T ... x_N UN^T (Alg. 1/4 core step). */
tals_status project(const void* A, void* const* U, int dtype, int ndim, const int64_t* dims,
                    const int* ranks, void* G_out, void* stream);

/* Adjoint of reconstruct: given B_bar (device, prod I_n), write
 * G_bar = B_bar x_1 U1^T ... x_N UN^T and U_bar[n] = (B_bar x_{m!=n} Um^T)_(n) G_(n)^T.
 * The partial contractions are recomputed per mode, never stored for all n.
 * Any U_bar[n] may be NULL (skipped). */
tals_status reconstruct_backward(const void* G, void* const* U, const void* B_bar, int dtype,
                                 int ndim, const int64_t* dims, const int* ranks,
                                 void* G_bar, void* const* U_bar, void* stream);

/* Adjoint of project: given G_bar, write A_bar = G_bar x_1 U1 ... x_N UN (may be
 * NULL) and U_bar[n] = (A x_{m!=n} Um^T)_(n) G_bar_(n)^T (any may be NULL). */
tals_status project_backward(const void* A, void* const* U, const void* G_bar, int dtype,
                             int ndim, const int64_t* dims, const int* ranks, void* A_bar,
                             void* const* U_bar, void* stream);

/* Host only, no CUDA call: the order in which project (expand = 0) or
 * reconstruct (expand = 1) apply their ndim mode products. A mode product costs
 * min(I_n, R_n) multiply-adds per element of its larger side (the input of a
 * contraction, the output of an expansion); the order written to order_out
 * (host, ndim entries: the modes in the order applied) is the exact minimum of
 * the summed cost over all ndim! orders, found by dynamic programming over the
 * subsets of applied modes (ties keep the lower mode first), and *madds_out
 * (host, may be NULL) receives that minimum. dims and ranks: host, ndim entries.
 * TALS_EINVAL for ndim outside 1..TALS_MAX_NDIM, a NULL dims, ranks or
 * order_out, or a size or rank below 1. */
tals_status tals_mode_product_order(int ndim, const int64_t* dims, const int* ranks, int expand,
                                    int* order_out, double* madds_out);

/* Batched st-HOSVD-ALS over `count` independent third-order FP32 tensors of
 * uneven sizes. A_ptrs/G_ptrs/U_ptrs are HOST arrays of DEVICE pointers
 * (U_ptrs has 3*count entries: tensor t's factors at 3t, 3t+1, 3t+2); dims and
 * ranks are host arrays of 3*count entries. One persistent kernel (captured in
 * a CUDA graph on first use) processes all tensors; each CTA takes whole
 * tensors from an atomic queue, so no CTA ever waits on another. stats (host,
 * may be NULL) receives count entries. Limits: I_n <= 128, R_n <= 16. */
tals_status tals_batched_st_hosvd(int count, void* const* A_ptrs, const int64_t* dims,
                                  const int* ranks, const tals_opts* opts, void* const* G_ptrs,
                                  void* const* U_ptrs, tals_stats* stats, void* stream);

/* Measurement hook (no counterpart in the paper): launch the sweep pass of `mode`
 * (one read of the context's tensor A viewed as its mode-`mode` unfolding, with
 * the context's current factor buffer and W written) `iters` times on the
 * context's stream between two CUDA events recorded on that stream. Returns the
 * mean duration in *ms, and the pass's algorithmic bytes (tensor read + W write)
 * and flops (4 R_n prod(I)) per launch. Synchronises the stream. */
tals_status tals_time_pass(tals_ctx* ctx, int mode, int iters, double* ms, double* bytes,
                           double* flops);

/* Measurement hook (no counterpart in the paper): time the product passes of one
 * sweep of `mode` on the context's tensor A, `iters` times after one warm-up, with
 * CUDA events recorded on the context's stream around each launch. engine 0: the
 * fused FP32 CUDA-core pass; 1: the fused BF16 tensor-core pass (mixed-precision
 * contexts only); 2: the two split-precision 3xTF32 tensor-core passes; 3: the
 * two-product form (FP32 mode product W, then the split-K product Y = B_(n) W).
 * ms_out[0], bytes_out[0]: mean duration and algorithmic bytes of the first (or
 * only) pass; ms_out[1], bytes_out[1]: the second pass of engines 2 and 3, else 0 (both
 * host arrays of 2). *flops: FP32-equivalent flops of the sweep (4 R_n prod(I)).
 * TALS_ENOTSUP when the mode's view is outside the engine's limits. Synchronises
 * the stream. */
tals_status tals_time_sweep(tals_ctx* ctx, int mode, int engine, int iters, double* ms_out,
                            double* bytes_out, double* flops);

/* Host only, no CUDA call (diagnostics): the configuration of the fused sweep pass
 * for a mode view P x I x Q (I the mode's size, P and Q the products of the sizes
 * before and after it) at rank R on a GPU with num_sms SMs. plan_out (host, 10
 * ints): rank chunk, rows per thread, ranks per thread, threads per CTA, columns
 * per tile, tile buffers, transposed tile (0/1), dynamic shared memory in bytes,
 * CTAs along the tiles, rank chunks. TALS_EINVAL for a bad dtype, a size, rank
 * or SM count below 1 or a NULL plan_out; TALS_ENOTSUP when no configuration
 * fits in shared memory (above the limits of I_n stated with the error codes). */
tals_status tals_pass_plan(int dtype, int64_t P, int64_t I, int64_t Q, int R, int num_sms,
                           int* plan_out);

/* Diagnostics (one sweep of products, Eq. 2.2): for the FP32 tensor A (device,
 * dims[ndim]) viewed as its mode-`mode` unfolding B and the FP32 basis Q (device,
 * I_mode x R, row-major), write Y = B B^T Q (device, FP64, I_mode x R) and
 * *wnorm2 = ||B^T Q||^2.
 * engine 0: CUDA-core FP32 pass. engine 1: tensor-core pass (tcgen05, BF16 operands,
 * FP32 accumulation) on a BF16 copy of A; needs I_mode % 128 == 0, I_mode <= 512,
 * prod of the later sizes % 128 == 0 and R <= 64. engine 2: the two split-precision
 * (3xTF32) tensor-core passes on A itself; needs prod of the later sizes % 32 == 0,
 * I_mode <= 1024, R <= 64 and a 16-byte aligned A. engines 3 and 4 (diagnostics):
 * one of engine 2's passes replaced by the CUDA-core pass (3: tensor-core W; 4:
 * tensor-core Y). engine 5: the two-product form on CUDA cores (W = B^T Q by the
 * register-tiled mode product, then Y = B W split over column ranges); needs
 * R <= 64, prod of the later sizes % 16 == 0 and a 16-byte aligned A. Shapes outside
 * an engine's limits return TALS_ENOTSUP. Uses stream-ordered scratch and
 * synchronises the stream. */
tals_status tals_sweep_pass(const void* A, int ndim, const int64_t* dims, int mode, const void* Q,
                            int R, int engine, double* Y_out, double* wnorm2, void* stream);

/* The paper has no counterpart to this entry point; it serves callers that cannot
 * allocate device memory at call time -- for example code running while a memory
 * pool or a framework's caching allocator owns the device memory, or a
 * latency-critical loop that cannot pay for an allocation. It computes exactly
 * what tals_sweep_pass with engine 0 computes (FP32 tensor A, FP32 basis Q,
 * Y_out = B B^T Q as FP64 I_mode x R, device), except that the sum ||B^T Q||^2 is
 * written to *wnorm2_out, a DEVICE double, and nothing is synchronised.
 * It allocates nothing: its scratch (the per-CTA partial sums) is one fixed array
 * of 4 MiB + 8 KiB in device global memory, defined in the library and held by
 * every GPU that loads the library until the process exits. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and keeps it
 * for the life of the process, so make the first call on each device before any
 * stream capture; a cudaDeviceReset of that device invalidates the kept address
 * (do not call this entry point on a device after resetting it). Limit: I_mode x R <= 2^20
 * (larger shapes return TALS_EINVAL); the pass uses fewer CTAs when their partials
 * would not fit. All calls share the one array: calls whose work overlaps on the
 * GPU (two streams, or two host threads) race and must be serialised by the
 * caller. Nothing in the array carries over from one call to the next. */
tals_status tals_sweep_pass_noalloc(const void* A, int ndim, const int64_t* dims, int mode,
                                    const void* Q, int R, double* Y_out, double* wnorm2_out,
                                    void* stream);

/* Statistics of tals_hooi. */
typedef struct {
  int iters;                          /* HOOI cycles performed (k) */
  int converged;                      /* 1: |r_{k-1} - r_k| < tol fired before max_iters */
  double resid0;                      /* r_0 = ||A - G0 x U0|| / ||A|| of the initial guess */
  double resid;                       /* r_k after the last cycle */
  int inner_sweeps[TALS_MAX_NDIM];    /* ALS R-updates of mode n, summed over the cycles */
} tals_hooi_stats;

/* HOOI (higher-order orthogonal iteration) refinement of a Tucker approximation of
 * the context's tensor A, started from the factors in U_io -- Sec. 6.3 runs it from
 * the t-/st-HOSVD(-ALS) results (e.g. the U_out of st_hosvd or t_hosvd).
 * Cycle k (k = 1 .. max_iters), modes n = 0 .. N-1 in turn:
 *   Y = A x_{m != n} U_m^T  (the factors already updated in this cycle);
 *   U_n = an orthonormal basis of the dominant R_n-dim left subspace of Y_(n),
 *         found by the ALS of Alg. 3 on Y_(n) started from L_0 = U_n (instead of
 *         the Sec. 4 sketch), with the Eq. 5.01 stop rule at tolerance inner_eta
 *         (relative to ||A||; negative: never stop early) and at most inner_sweeps
 *         R-updates per mode and cycle;
 * then G = Y x_N U_N^T and r_k = sqrt(||A||^2 - ||G||^2) / ||A||. Stops after the
 * first cycle with |r_{k-1} - r_k| < tol (r_0: the initial guess), or after
 * max_iters cycles. The identity for r_k assumes orthonormal U (true of every
 * factor it writes); in FP32 it cancels, so r_k is resolved only to about
 * sqrt(1e-7) -- use FP64 contexts for tolerances like Sec. 6.3's 1e-12.
 * U_io: N device buffers (I_n x R_n, dtype), read as the initial guess (orthonormal
 * columns) and overwritten with the refined factors. G_out: device buffer of
 * prod R_n (dtype) for the final core, or NULL. resid_out: host array of
 * max_iters + 1 doubles (r_0 .. r_k), or NULL. stats: host, or NULL.
 * Uses the context's workspace and stream-ordered scratch (two tensors of the
 * largest partial projection); synchronises the stream once per cycle.
 * TALS_EINVAL for NULL U_io entries, max_iters < 1, inner_sweeps < 1, tol < 0 or
 * a zero tensor; TALS_ENOTSUP if a partial projection is outside the pass limits;
 * TALS_ESINGULAR as for the ALS. */
tals_status tals_hooi(tals_ctx* ctx, void* const* U_io, void* G_out, double tol, int max_iters,
                      double inner_eta, int inner_sweeps, double* resid_out, tals_hooi_stats* stats);

/* Singular vectors from a t-HOSVD-ALS basis (Sec. 5, after Alg. 4): for the
 * context's tensor A and Qhat (device, I_n x R_n, dtype, orthonormal columns --
 * U^(n) as t_hosvd returns it), the SVD Qhat^T A_(n) = U S V^T gives
 * U_out = Qhat U (device, I_n x R_n, dtype) and sigma_out = S (host, R_n doubles,
 * descending). Formed through the R_n x R_n Gram M = Qhat^T A_(n) A_(n)^T Qhat --
 * one read of A by the fused sweep pass with Qhat as its basis -- and the
 * eigendecomposition M = V diag(S^2) V^T by cyclic Jacobi rotations in FP64
 * (U = V); S_r = sqrt(max(lambda_r, 0)), so singular values far below S_1 carry
 * an absolute error of about 1e-16 S_1^2 / S_r (FP64 data). The sign of each column
 * of U_out makes its entry of largest magnitude positive (the first on ties).
 * Qhat and U_out must not alias. TALS_EINVAL for bad arguments; TALS_ENOTSUP if
 * the Jacobi sweeps do not converge (not expected for a symmetric M).
 * Synchronises the stream. */
tals_status tals_singular_vectors(tals_ctx* ctx, int mode, const void* Qhat, void* U_out,
                                  double* sigma_out);

/* Free a context (its workspace, graphs and owned buffers). NULL is allowed. */
void tals_destroy(tals_ctx* ctx);

/* Thread-local message describing the last non-OK status. */
const char* tals_last_error(void);

/* Library version string. */
const char* tals_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TALS_H */
