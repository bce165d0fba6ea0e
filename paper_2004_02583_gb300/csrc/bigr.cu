// Modes of rank R_n > 64 -- the dense parallel test of Sec. 6.4 (5000 x 5000 x 50
// at ranks (500, 500, 5)) -- through the ALS of Alg. 3 with the same iterates as
// the fused path: two reads of B per sweep for the products, and the R x R
// algebra as blocked FP64 linear algebra spread over the GPU instead of the
// single-CTA factorizations the small ranks use.
//
//   W = B_(n)^T Q_k, written as the tensor B x_n Q_k^T (P x R x Q layout): one
//       GEMM for P = 1 or Q = 1 views, the tiled mode product otherwise;
//   Y = B_(n) W over column ranges of at most 2048 (FP32 partial sums stay
//       short), the ranges added in FP64;
//   X = Q_k^T Y (= W^T W, the Gram of the R-update), and the Eq. 5.01 step on
//       e_k^2 = ||B||^2 - ||W||^2 + tr((Q'^T Q' - I) X) (Q' the stored basis); the
//       host reads the stop flag, so these modes run the host-driven loop;
//   L_{k+1} = Y X^{-1}: Cholesky X = F F^T, then two triangular solves on the
//       I_n x R rows; Q_{k+1} from CholeskyQR of L_{k+1} (two rounds for the
//       initial guess Y_0 = B_(n) S of Sec. 4, whose columns are far from
//       orthogonal).
// The Cholesky factor is formed 64 columns at a time: one CTA factors the
// diagonal block and inverts it in FP64, GEMMs form the panel below it (A_21
// F_11^{-T}) and update the trailing matrix (A_22 - F_21 F_21^T). The solves use
// the same inverted diagonal blocks with GEMM updates (forward for Y F^{-T},
// backward for T F^{-1}). All GEMMs are plain cuBLAS DGEMM / SGEMM calls in
// pedantic math mode (no reduced-precision arithmetic).
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace tals {

namespace {

constexpr int kNb = 64;            // Cholesky block
constexpr int kChunk = 2048;       // longest FP32 partial sum of the Y product
constexpr int kBlkThreads = 256;
constexpr size_t kCholSmem = 2 * (size_t)kNb * (kNb + 1) * sizeof(double);   // the block and its inverse

// ---------------------------------------------------------------------------
// Device kernels
// ---------------------------------------------------------------------------

// A = (X + X^T) / 2 and md = max_i A[i][i] (the pivot threshold's scale).
__global__ void symm_kernel(const double* __restrict__ X, int R, double* __restrict__ A, double* __restrict__ md) {
  const long long n = (long long)R * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / R), j = (int)(e % R);
    A[e] = 0.5 * (X[e] + X[(long long)j * R + i]);
  }
  if (blockIdx.x == 0) {
    __shared__ double red[kBlkThreads];
    double m = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) m = fmax(m, X[(long long)i * R + i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) *md = red[0];
  }
}

// One CTA: the Cholesky factor of the kb x kb diagonal block of A at (k0, k0)
// (lower, A_kk = F_kk F_kk^T; right-looking, one barrier-separated step per
// column) into F, and its inverse (forward substitution on the identity) into D
// (kb x kb, row stride kb). A pivot at or below 64 eps max_i A[i][i] (or not a
// number) marks the mode singular (Remark 3) and continues with pivot 1.
__global__ void __launch_bounds__(kBlkThreads) chol_block_kernel(const double* __restrict__ A, int R, int k0,
                                                                 int kb, double* __restrict__ F,
                                                                 double* __restrict__ D,
                                                                 const double* __restrict__ md, ModeState* st,
                                                                 int stage) {
  extern __shared__ double chol_dyn[];
  double(*S)[kNb + 1] = reinterpret_cast<double(*)[kNb + 1]>(chol_dyn);
  double(*V)[kNb + 1] = reinterpret_cast<double(*)[kNb + 1]>(chol_dyn + kNb * (kNb + 1));
  __shared__ double dinv[kNb];
  __shared__ short tri_i[kNb * (kNb - 1) / 2], tri_j[kNb * (kNb - 1) / 2];
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += kBlkThreads) {
    const int i = e / kb, j = e % kb;
    S[i][j] = A[(long long)(k0 + i) * R + k0 + j];
    V[i][j] = i == j ? 1.0 : 0.0;
  }
  // (i', j') of the dense index a = i'(i'+1)/2 + j' over a lower triangle
  for (int a = tid; a < kNb * (kNb - 1) / 2; a += kBlkThreads) {
    int ip = (int)((sqrtf(8.f * (float)a + 1.f) - 1.f) * 0.5f);
    while (ip * (ip + 1) / 2 > a) --ip;
    while ((ip + 1) * (ip + 2) / 2 <= a) ++ip;
    tri_i[a] = (short)ip;
    tri_j[a] = (short)(a - ip * (ip + 1) / 2);
  }
  if (tid == 0) bad = 0;
  const double tiny = 64.0 * 2.220446049250313e-16 * *md;
  __syncthreads();
  for (int k = 0; k < kb; ++k) {
    if (tid == 0) {
      double d = S[k][k];
      if (!(d > tiny) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      const double s = sqrt(d);
      S[k][k] = s;
      dinv[k] = 1.0 / s;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < kb; i += kBlkThreads) S[i][k] *= dinv[k];
    __syncthreads();
    // trailing block: k < j <= i < kb
    const int m = kb - k - 1;
    const int na = m * (m + 1) / 2;
    for (int a = tid; a < na; a += kBlkThreads) {
      const int i = k + 1 + tri_i[a], j = k + 1 + tri_j[a];
      S[i][j] = fma(-S[i][k], S[j][k], S[i][j]);
    }
    __syncthreads();
  }
  // V = S^{-1}: S V = I, row l finished (scaled by 1 / S[l][l]) then eliminated
  // from the rows below
  for (int l = 0; l < kb; ++l) {
    for (int j = tid; j <= l; j += kBlkThreads) V[l][j] *= dinv[l];
    __syncthreads();
    const int w = l + 1, n = (kb - l - 1) * w;
    for (int a = tid; a < n; a += kBlkThreads) {
      const int i = l + 1 + a / w, j = a % w;
      V[i][j] = fma(-S[i][l], V[l][j], V[i][j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += kBlkThreads) {
    const int i = e / kb, j = e % kb;
    F[(long long)(k0 + i) * R + k0 + j] = j <= i ? S[i][j] : 0.0;
    D[e] = j <= i ? V[i][j] : 0.0;
  }
  if (tid == 0 && bad && st != nullptr) {
    st->status = 4;   // TALS_ESINGULAR: Gram not numerically SPD (Remark 3)
    st->fail_stage = stage;
    st->done = 1;
  }
}

// Y64[e] = sum over s of part[s * n + e], in FP64, s in order.
template <typename T>
__global__ void sum_to_f64_kernel(const T* __restrict__ part, int S, long long n, double* __restrict__ Y) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += (double)part[(long long)s * n + e];
    Y[e] = v;
  }
}

// U[i][p Q + q] = X[p][i][q]: the mode-n unfolding written out (I x P Q).
template <typename T>
__global__ void unfold_kernel(const T* __restrict__ X, long long P, long long I, long long Q, T* __restrict__ U) {
  const long long J = P * Q, n = I * J;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const long long i = o / J, jj = o - i * J;
    const long long p = jj / Q, q = jj - p * Q;
    U[o] = X[(p * I + i) * Q + q];
  }
}

// W[p][r][q] = Wr[r][p Q + q]: an R x P Q product back in the P x R x Q layout.
template <typename T>
__global__ void fold_kernel(const T* __restrict__ Wr, long long P, long long R, long long Q, T* __restrict__ W) {
  const long long n = P * R * Q;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const long long q = o % Q, pr = o / Q;
    const long long r = pr % R, p = pr / R;
    W[o] = Wr[r * (P * Q) + p * Q + q];
  }
}

// The stored basis: Lt = L64 rounded to the tensor's type and, for FP32, its
// rounding error D = Lt - L64 (exact in FP32 to its own rounding: |D| is near
// 2^-24 |L64|).
template <typename T>
__global__ void store_basis_kernel(const double* __restrict__ L64, long long n, T* __restrict__ Lt,
                                   float* __restrict__ D) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const T q = (T)L64[e];
    Lt[e] = q;
    if (D != nullptr) D[e] = (float)((double)q - L64[e]);
  }
}

// GL = I + H + H^T (H = D^T Lt, R x R FP32; null: GL = I).
__global__ void basis_gram_kernel(const float* __restrict__ H, int R, double* __restrict__ GL) {
  const long long n = (long long)R * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / R), j = (int)(e % R);
    double g = i == j ? 1.0 : 0.0;
    if (H != nullptr) g += (double)H[e] + (double)H[(long long)j * R + i];
    GL[e] = g;
  }
}

__device__ double block_sum_256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = kBlkThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double t = red[0];
  __syncthreads();
  return t;
}

// ||B_(n)||^2 of the initial pass (and ||A||^2 for the first mode).
__global__ void __launch_bounds__(kBlkThreads) bigr_norm_kernel(ModeState* st, const double* __restrict__ spart,
                                                                int nsp, double* norm_a2) {
  __shared__ double red[kBlkThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < nsp; i += kBlkThreads) a += spart[i];
  const double t = block_sum_256(a, red);
  if (threadIdx.x == 0) {
    st->normM2 = t;
    if (norm_a2 != nullptr) *norm_a2 = t;
  }
}

// The Eq. 5.01 step: ||W||^2 from its partials, the rounded-basis term
// tr((GL - I) X), e_k^2 = ||B||^2 - ||W||^2 + that term; or, for a mode that
// measures the residual (st->resid), e_k^2 = the sW the residual kernel wrote.
__global__ void __launch_bounds__(kBlkThreads) bigr_test_kernel(ModeState* st, const double* __restrict__ spart,
                                                                int nsp, const double* __restrict__ X,
                                                                const double* __restrict__ GL, int R,
                                                                const double* __restrict__ norm_a2) {
  __shared__ double red[kBlkThreads];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nsp; i += kBlkThreads) a += spart[i];
  const long long n = (long long)R * R;
  for (long long o = threadIdx.x; o < n; o += kBlkThreads) {
    const long long r = o / R, q = o % R;
    c += (GL[o] - (r == q ? 1.0 : 0.0)) * X[o];
  }
  const double sW = block_sum_256(a, red);
  const double corr = block_sum_256(c, red);
  if (threadIdx.x == 0) {
    double e2;
    if (st->resid) {
      st->corr = 0.0;
      e2 = st->sW;
    } else {
      st->sW = sW;
      st->corr = corr;
      e2 = st->normM2 - sW + corr;
    }
    als_stop_step(st, sqrt(e2 > 0.0 ? e2 : 0.0), sqrt(*norm_a2));
  }
}

unsigned grid_of(long long n, int sms) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * sms));
}

// ---------------------------------------------------------------------------
// Row-major GEMM wrappers: C (M x N) = alpha op(A) op(B) + beta C, every matrix
// row-major with the given row strides. cuBLAS is column-major: the row-major C
// is the column-major C^T = op(B)^T op(A)^T.
// ---------------------------------------------------------------------------
cublasStatus_t gemm_rm(cublasHandle_t h, bool tA, bool tB, long long M, long long N, long long K, double alpha,
                       const double* A, long long lda, const double* B, long long ldb, double beta, double* C,
                       long long ldc) {
  return cublasDgemm(h, tB ? CUBLAS_OP_T : CUBLAS_OP_N, tA ? CUBLAS_OP_T : CUBLAS_OP_N, (int)N, (int)M, (int)K,
                     &alpha, B, (int)ldb, A, (int)lda, &beta, C, (int)ldc);
}
cublasStatus_t gemm_rm(cublasHandle_t h, bool tA, bool tB, long long M, long long N, long long K, float alpha,
                       const float* A, long long lda, const float* B, long long ldb, float beta, float* C,
                       long long ldc) {
  return cublasSgemm(h, tB ? CUBLAS_OP_T : CUBLAS_OP_N, tA ? CUBLAS_OP_T : CUBLAS_OP_N, (int)N, (int)M, (int)K,
                     &alpha, B, (int)ldb, A, (int)lda, &beta, C, (int)ldc);
}
cublasStatus_t gemm_rm_batched(cublasHandle_t h, bool tA, bool tB, long long M, long long N, long long K,
                               const double* A, long long lda, long long sA, const double* B, long long ldb,
                               long long sB, double* C, long long ldc, long long sC, int count) {
  const double one = 1.0, zero = 0.0;
  return cublasDgemmStridedBatched(h, tB ? CUBLAS_OP_T : CUBLAS_OP_N, tA ? CUBLAS_OP_T : CUBLAS_OP_N, (int)N,
                                   (int)M, (int)K, &one, B, (int)ldb, sB, A, (int)lda, sA, &zero, C, (int)ldc, sC,
                                   count);
}
cublasStatus_t gemm_rm_batched(cublasHandle_t h, bool tA, bool tB, long long M, long long N, long long K,
                               const float* A, long long lda, long long sA, const float* B, long long ldb,
                               long long sB, float* C, long long ldc, long long sC, int count) {
  const float one = 1.f, zero = 0.f;
  return cublasSgemmStridedBatched(h, tB ? CUBLAS_OP_T : CUBLAS_OP_N, tA ? CUBLAS_OP_T : CUBLAS_OP_N, (int)N,
                                   (int)M, (int)K, &one, B, (int)ldb, sB, A, (int)lda, sA, &zero, C, (int)ldc, sC,
                                   count);
}

// The mode's workspace slices (FP64, in the context's large-rank scratch).
struct BigWs {
  double* A;    // R x R working copy of the Gram being factored
  double* F;    // R x R Cholesky factor (lower)
  double* D;    // inverted diagonal blocks, 64 x 64 slots
  double* md;   // max diagonal entry
};

BigWs big_ws(tals_ctx* c, int R) {
  BigWs w;
  w.A = c->bw;
  w.F = w.A + (size_t)R * R;
  w.D = w.F + (size_t)R * R;
  w.md = w.D + (size_t)((R + kNb - 1) / kNb) * kNb * kNb;
  return w;
}

#define TALS_CK(x) \
  if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x);
#define TALS_BL(x)                                                                   \
  do {                                                                               \
    const cublasStatus_t bs_ = (x);                                                  \
    if (bs_ != CUBLAS_STATUS_SUCCESS) return fail(TALS_ECUDA, "%s: cuBLAS status %d", #x, (int)bs_); \
  } while (0)

// F F^T = G (G R x R, FP64): F and the inverted diagonal blocks in ws.
tals_status big_chol(tals_ctx* c, const ModeJob& j, const double* G, int stage) {
  const int R = j.R;
  cublasHandle_t h = (cublasHandle_t)c->blas;
  cudaStream_t s = c->stream;
  const BigWs w = big_ws(c, R);
  cudaError_t e;
  // the attribute belongs to the current device: set on every call
  TALS_CK(cudaFuncSetAttribute(chol_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem));
  symm_kernel<<<grid_of((long long)R * R, c->sms), kBlkThreads, 0, s>>>(G, R, w.A, w.md);
  TALS_CK(cudaGetLastError());
  const int nb = (R + kNb - 1) / kNb;
  for (int b = 0; b < nb; ++b) {
    const int c0 = b * kNb, cb = std::min(kNb, R - c0), c1 = c0 + cb, rest = R - c1;
    double* Db = w.D + (size_t)b * kNb * kNb;
    chol_block_kernel<<<1, kBlkThreads, kCholSmem, s>>>(w.A, R, c0, cb, w.F, Db, w.md, j.st, stage);
    TALS_CK(cudaGetLastError());
    if (rest > 0) {
      // panel F_21 = A_21 F_11^{-T}; trailing A_22 -= F_21 F_21^T
      TALS_BL(gemm_rm(h, false, true, rest, cb, cb, 1.0, w.A + (size_t)c1 * R + c0, R, Db, cb, 0.0,
                      w.F + (size_t)c1 * R + c0, R));
      TALS_BL(gemm_rm(h, false, true, rest, rest, cb, -1.0, w.F + (size_t)c1 * R + c0, R,
                      w.F + (size_t)c1 * R + c0, R, 1.0, w.A + (size_t)c1 * R + c1, R));
    }
  }
  // the strictly upper blocks of F are never read: the solves use its lower
  // blocks and the inverted diagonal blocks only
  return TALS_OK;
}

// T = Y F^{-T} (Y I x R, destroyed: its column blocks hold the updated right-hand
// sides), by column blocks in ascending order.
tals_status big_solve_fwd(tals_ctx* c, const ModeJob& j, double* Y, double* T) {
  const int R = j.R;
  const long long I = j.v.I;
  cublasHandle_t h = (cublasHandle_t)c->blas;
  const BigWs w = big_ws(c, R);
  const int nb = (R + kNb - 1) / kNb;
  for (int b = 0; b < nb; ++b) {
    const int c0 = b * kNb, cb = std::min(kNb, R - c0);
    if (c0 > 0)
      TALS_BL(gemm_rm(h, false, true, I, cb, c0, -1.0, T, R, w.F + (size_t)c0 * R, R, 1.0, Y + c0, R));
    TALS_BL(gemm_rm(h, false, true, I, cb, cb, 1.0, Y + c0, R, w.D + (size_t)b * kNb * kNb, cb, 0.0, T + c0, R));
  }
  return TALS_OK;
}

// Z = T F^{-1} (T destroyed), by column blocks in descending order.
tals_status big_solve_bwd(tals_ctx* c, const ModeJob& j, double* T, double* Z) {
  const int R = j.R;
  const long long I = j.v.I;
  cublasHandle_t h = (cublasHandle_t)c->blas;
  const BigWs w = big_ws(c, R);
  const int nb = (R + kNb - 1) / kNb;
  for (int b = nb - 1; b >= 0; --b) {
    const int c0 = b * kNb, cb = std::min(kNb, R - c0), c1 = c0 + cb;
    if (c1 < R)
      TALS_BL(gemm_rm(h, false, false, I, cb, R - c1, -1.0, Z + c1, R, w.F + (size_t)c1 * R + c0, R, 1.0, T + c0,
                      R));
    TALS_BL(gemm_rm(h, false, false, I, cb, cb, 1.0, T + c0, R, w.D + (size_t)b * kNb * kNb, cb, 0.0, Z + c0, R));
  }
  return TALS_OK;
}

// G = M^T M (M I x R, FP64).
tals_status big_gram(tals_ctx* c, const ModeJob& j, const double* M, double* G) {
  TALS_BL(gemm_rm((cublasHandle_t)c->blas, true, false, j.R, j.R, j.v.I, 1.0, M, j.R, M, j.R, 0.0, G, j.R));
  return TALS_OK;
}

// Q R = M (M I x R, FP64, destroyed) by one CholeskyQR round: Q into out.
tals_status big_cholqr(tals_ctx* c, const ModeJob& j, double* M, double* out, int stage) {
  tals_status st;
  if ((st = big_gram(c, j, M, c->Gfin)) != TALS_OK) return st;
  if ((st = big_chol(c, j, c->Gfin, stage)) != TALS_OK) return st;
  return big_solve_fwd(c, j, M, out);
}

// L64 holds the new basis (orthonormal to FP64 rounding): store its rounding Lt
// and the Gram GL = Lt^T Lt of the stored basis (GfinL, the rounded-basis term of
// the next test). With Lt = L64 + D, GL = I + D^T L64 + L64^T D + D^T D +
// (L64^T L64 - I); the last two terms are at FP64 rounding level, and D^T L64 =
// D^T Lt - D^T D, so GL = I + H + H^T with H = D^T Lt to that level: one FP32 GEMM
// (D is ~2^-24 |L|, so H's FP32 rounding is far below the term itself) instead of
// an FP64 Gram. FP64 tensors: Lt = L64, GL = I.
tals_status big_store_basis(tals_ctx* c, const ModeJob& j) {
  const int R = j.R;
  const long long n = j.v.I * R;
  cudaError_t e;
  float* H = reinterpret_cast<float*>(c->F);   // R x R FP32 (F holds 3 R^2 + R doubles)
  if (c->dtype == TALS_F32) {
    float* D = reinterpret_cast<float*>(c->Z64);
    store_basis_kernel<float><<<grid_of(n, c->sms), 256, 0, c->stream>>>(c->L64, n, (float*)c->Lt, D);
    TALS_CK(cudaGetLastError());
    TALS_BL(gemm_rm((cublasHandle_t)c->blas, true, false, R, R, j.v.I, 1.f, D, R, (const float*)c->Lt, R, 0.f, H,
                    R));
  } else {
    store_basis_kernel<double><<<grid_of(n, c->sms), 256, 0, c->stream>>>(c->L64, n, (double*)c->Lt, nullptr);
    TALS_CK(cudaGetLastError());
    H = nullptr;
  }
  basis_gram_kernel<<<grid_of((long long)R * R, c->sms), 256, 0, c->stream>>>(H, R, c->GfinL);
  TALS_CK(cudaGetLastError());
  return TALS_OK;
}

// Y64 = B_(n) V for V in the P x R x Q layout (the sketch or W), the column
// ranges' FP32 (or FP64) partial sums in Ypart, added in FP64.
template <typename T>
tals_status big_adjoint(tals_ctx* c, const ModeJob& j, const T* X, const T* V) {
  cublasHandle_t h = (cublasHandle_t)c->blas;
  cudaStream_t s = c->stream;
  const ModeView& v = j.v;
  const int R = j.R;
  const long long I = v.I, n = I * R;
  T* part = (T*)c->Ypart;
  cudaError_t e;
  int S = 0;
  if (v.P == 1 || v.Q == 1) {
    // the unfolding is a plain matrix: X (I x Q) for P = 1, X^T (I x P) for Q = 1
    const long long K = v.P == 1 ? v.Q : v.P;
    // ranges of 2048 columns, longer where more would not fit the j.splits partials
    const long long chunk = std::max<long long>(kChunk, (K + j.splits - 1) / j.splits);
    S = (int)((K + chunk - 1) / chunk);
    const int full = (int)(K / chunk);
    const long long tail = K - (long long)full * chunk;
    if (v.P == 1) {
      // part_s = X[:, range s] V[:, range s]^T
      if (full > 0)
        TALS_BL(gemm_rm_batched(h, false, true, I, R, chunk, X, K, chunk, V, K, chunk, part, R, n, full));
      if (tail > 0)
        TALS_BL(gemm_rm(h, false, true, I, R, tail, T(1), X + (size_t)full * chunk, K,
                        V + (size_t)full * chunk, K, T(0), part + (size_t)full * n, R));
    } else {
      // part_s = X[range s, :]^T V[range s, :] (X P x I, V P x R)
      if (full > 0)
        TALS_BL(gemm_rm_batched(h, true, false, I, R, chunk, X, I, chunk * I, V, R, chunk * R, part, R, n, full));
      if (tail > 0)
        TALS_BL(gemm_rm(h, true, false, I, R, tail, T(1), X + (size_t)full * chunk * I, I,
                        V + (size_t)full * chunk * R, R, T(0), part + (size_t)full * n, R));
    }
  } else {
    S = j.splits;
    TALS_CK(launch_factor_adjoint_parts(X, v.P, I, v.Q, V, R, S, part, s));
  }
  sum_to_f64_kernel<T><<<grid_of(n, c->sms), 256, 0, s>>>(part, S, n, c->Y64);
  TALS_CK(cudaGetLastError());
  return TALS_OK;
}

// W = B x_n Q^T (P x R x Q) for the stored basis Lt (I x R).
template <typename T>
tals_status big_project(tals_ctx* c, const ModeJob& j, const T* X, const T* Lt, T* W) {
  cublasHandle_t h = (cublasHandle_t)c->blas;
  const ModeView& v = j.v;
  const int R = j.R;
  cudaError_t e;
  if (v.P == 1) {
    TALS_BL(gemm_rm(h, true, false, R, v.Q, v.I, T(1), Lt, R, X, v.Q, T(0), W, v.Q));   // Q^T X
  } else if (v.Q == 1) {
    TALS_BL(gemm_rm(h, false, false, v.P, R, v.I, T(1), X, v.I, Lt, R, T(0), W, R));    // X Q
  } else {
    TALS_CK(launch_mode_project_any(c->dtype, X, v, Lt, R, W, c->stream));
  }
  return TALS_OK;
}

// General views (P > 1 and Q > 1): the products run on the unfolding written out
// once per mode (I x P Q in the context's unfolding buffer, followed by room for
// an R x P Q product), i.e. as the P = 1 view {1, I, P Q} with plain GEMMs; the
// mode's W is folded back to the P x R x Q layout when the stop rule ends it.
ModeJob unfolded_job(const tals_ctx* c, const ModeJob& j) {
  ModeJob u = j;
  u.v = ModeView{1, j.v.I, j.v.P * j.v.Q};
  u.X = c->ubuf;
  u.Wt = (char*)c->ubuf + (size_t)(j.v.P * j.v.I * j.v.Q) * c->esz;
  return u;
}

// The unfolding of j's tensor in the buffer: written unless it already holds it
// (force: always, at the start of a mode -- the tensor may have new contents).
tals_status ensure_unfolded(tals_ctx* c, const ModeJob& j, bool force) {
  if (!force && c->ubuf_src == j.X && c->ubuf_mode == j.n) return TALS_OK;
  const long long n = j.v.P * j.v.I * j.v.Q;
  cudaError_t e;
  if (c->dtype == TALS_F32)
    unfold_kernel<float><<<grid_of(n, c->sms), 256, 0, c->stream>>>((const float*)j.X, j.v.P, j.v.I, j.v.Q,
                                                                     (float*)c->ubuf);
  else
    unfold_kernel<double><<<grid_of(n, c->sms), 256, 0, c->stream>>>((const double*)j.X, j.v.P, j.v.I, j.v.Q,
                                                                      (double*)c->ubuf);
  TALS_CK(cudaGetLastError());
  c->ubuf_src = j.X;
  c->ubuf_mode = j.n;
  return TALS_OK;
}

tals_status fold_result(tals_ctx* c, const ModeJob& j, const ModeJob& u) {
  const long long n = j.v.P * j.R * j.v.Q;
  cudaError_t e;
  if (c->dtype == TALS_F32)
    fold_kernel<float><<<grid_of(n, c->sms), 256, 0, c->stream>>>((const float*)u.Wt, j.v.P, j.R, j.v.Q,
                                                                   (float*)j.Wt);
  else
    fold_kernel<double><<<grid_of(n, c->sms), 256, 0, c->stream>>>((const double*)u.Wt, j.v.P, j.R, j.v.Q,
                                                                    (double*)j.Wt);
  TALS_CK(cudaGetLastError());
  return TALS_OK;
}

template <typename T>
tals_status big_init_t(tals_ctx* c, const ModeJob& j0, bool set_norm_a) {
  cudaStream_t s = c->stream;
  const int R = j0.R;
  cudaError_t e;
  tals_status st;
  if (j0.unf && (st = ensure_unfolded(c, j0, true)) != TALS_OK) return st;
  const ModeJob j = j0.unf ? unfolded_job(c, j0) : j0;
  // Sec. 4: Y0 = B_(n) S with S written out in the P x R x Q layout (the same
  // counter-based entries the fused pass draws: column j = p Q + q either way), and
  // ||B_(n)||^2
  TALS_CK(launch_sketch_prq(c->dtype, j.Wt, j.v, R, sketch_state(c->opts.seed, j.n), c->sms, s));
  if ((st = big_adjoint<T>(c, j, (const T*)j.X, (const T*)j.Wt)) != TALS_OK) return st;
  TALS_CK(launch_sumsq_parts(c->dtype, j.X, (size_t)(j.v.P * j.v.I * j.v.Q), c->spart, s));
  bigr_norm_kernel<<<1, kBlkThreads, 0, s>>>(j.st, c->spart, kSumsqParts, set_norm_a ? c->norm_a2 : nullptr);
  TALS_CK(cudaGetLastError());
  // L0 = Q of QR(Y0), CholeskyQR2
  if ((st = big_cholqr(c, j, c->Y64, c->Z64, 2)) != TALS_OK) return st;
  if ((st = big_cholqr(c, j, c->Z64, c->L64, 2)) != TALS_OK) return st;
  return big_store_basis(c, j);
}

template <typename T>
tals_status big_sweep_t(tals_ctx* c, const ModeJob& j0) {
  cudaStream_t s = c->stream;
  const int R = j0.R;
  cudaError_t e;
  tals_status st;
  if ((st = read_states(c)) != TALS_OK) return st;
  if (c->st_host[j0.n].done) return TALS_OK;
  if (j0.unf && (st = ensure_unfolded(c, j0, false)) != TALS_OK) return st;
  const ModeJob j = j0.unf ? unfolded_job(c, j0) : j0;
  // R-update W = B^T Q_k (as B x_n Q_k^T), ||W||^2, then Y = B W and X = Q_k^T Y
  if ((st = big_project<T>(c, j, (const T*)j.X, (const T*)c->Lt, (T*)j.Wt)) != TALS_OK) return st;
  if (j.resid_kernel) {
    // FP32 on a small tensor: e_k^2 = ||B - Q' W^T||^2 directly into the state (the
    // Y partials' buffer serves as the residual's scratch before Y is formed)
    if constexpr (sizeof(T) == 4)
      TALS_CK(launch_mode_residual((const float*)j.X, j.v, R, (const float*)j.Wt, (const float*)c->Lt,
                                   (double*)c->Ypart, (long long)(c->ypart_elems / 2), j.st, s));
  } else {
    TALS_CK(launch_sumsq_parts(c->dtype, j.Wt, (size_t)(j.v.P * j.v.Q) * R, c->spart, s));
  }
  if ((st = big_adjoint<T>(c, j, (const T*)j.X, (const T*)j.Wt)) != TALS_OK) return st;
  TALS_BL(gemm_rm((cublasHandle_t)c->blas, true, false, R, R, j.v.I, 1.0, c->L64, R, c->Y64, R, 0.0, c->Gfin, R));
  bigr_test_kernel<<<1, kBlkThreads, 0, s>>>(j.st, c->spart, kSumsqParts, c->Gfin, c->GfinL, R, c->norm_a2);
  TALS_CK(cudaGetLastError());
  if ((st = read_states(c)) != TALS_OK) return st;
  if (c->st_host[j.n].done) {
    // Q_k and this sweep's W are the mode's result
    return j0.unf ? fold_result(c, j0, j) : TALS_OK;
  }
  // L-update: L_{k+1} = Y X^{-1} = (Y F^{-T}) F^{-1}, then its Q factor
  if ((st = big_chol(c, j, c->Gfin, 1)) != TALS_OK) return st;
  if ((st = big_solve_fwd(c, j, c->Y64, c->Z64)) != TALS_OK) return st;
  if ((st = big_solve_bwd(c, j, c->Z64, c->Y64)) != TALS_OK) return st;
  if ((st = big_cholqr(c, j, c->Y64, c->L64, 2)) != TALS_OK) return st;
  return big_store_basis(c, j);
}

}  // namespace

bool bigr_rank(int R) { return R > kBigRankMin; }

size_t bigr_ws_doubles(int rmax) {
  if (rmax <= kBigRankMin) return 0;
  return 2 * (size_t)rmax * rmax + (size_t)((rmax + kNb - 1) / kNb) * kNb * kNb + 8;
}

tals_status bigr_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a) {
  return c->dtype == TALS_F32 ? big_init_t<float>(c, j, set_norm_a) : big_init_t<double>(c, j, set_norm_a);
}

tals_status bigr_sweep_launch(tals_ctx* c, const ModeJob& j) {
  return c->dtype == TALS_F32 ? big_sweep_t<float>(c, j) : big_sweep_t<double>(c, j);
}

tals_status bigr_time_products(tals_ctx* c, const ModeJob& j0, int iters, double* ms, double* bytes) {
  cudaStream_t s = c->stream;
  if (j0.unf) {
    const tals_status us = ensure_unfolded(c, j0, true);
    if (us != TALS_OK) return us;
  }
  const ModeJob j = j0.unf ? unfolded_job(c, j0) : j0;
  cudaEvent_t ev[3];
  for (auto& x : ev) cudaEventCreate(&x);
  double acc[2] = {0.0, 0.0};
  tals_status st = TALS_OK;
  cudaError_t e = cudaSuccess;
  for (int it = -1; it < iters && st == TALS_OK && e == cudaSuccess; ++it) {   // it = -1: warm-up
    cudaEventRecord(ev[0], s);
    st = c->dtype == TALS_F32 ? big_project<float>(c, j, (const float*)j.X, (const float*)c->Lt, (float*)j.Wt)
                              : big_project<double>(c, j, (const double*)j.X, (const double*)c->Lt, (double*)j.Wt);
    cudaEventRecord(ev[1], s);
    if (st == TALS_OK)
      st = c->dtype == TALS_F32 ? big_adjoint<float>(c, j, (const float*)j.X, (const float*)j.Wt)
                                : big_adjoint<double>(c, j, (const double*)j.X, (const double*)j.Wt);
    cudaEventRecord(ev[2], s);
    e = cudaEventSynchronize(ev[2]);
    float t0 = 0.f, t1 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
    if (it >= 0) {
      acc[0] += t0;
      acc[1] += t1;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (st != TALS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "timed products");
  const double T = (double)j.v.P * j.v.I * j.v.Q, JR = (double)j.v.J() * j.R;
  ms[0] = acc[0] / iters;
  ms[1] = acc[1] / iters;
  bytes[0] = (T + JR) * c->esz;   // tensor read + W written
  bytes[1] = (T + JR) * c->esz;   // tensor read + W read
  return TALS_OK;
}

// ---------------------------------------------------------------------------
// Thin last modes: a Q = 1 view (B_(n) = X^T for X the P x I row-major tensor)
// whose I_n is not a multiple of 4 has no transposed tile in the fused pass, whose
// untransposed tiles of I_n rows are then dominated by per-tile overhead (the
// rank-5 third mode of Sec. 6.4's dense test, I_n = 50: 12.5 ms per sweep on the
// 4.7 GiB tensor). Where the context holds a cuBLAS handle the sweep is two GEMMs
// instead: W = X Q_k (P x R, the R-update written as B x_n Q_k^T) and the Y
// partials X[range]^T W[range] over row ranges of at most max(2048, P / 1024) rows
// (each an FP32 sum no longer than the fused pass's own per-CTA sums), followed by
// the fused path's reduction, stop test and L-update over those partials; the
// initial guess likewise with the sketch S written out in place of W.
// ---------------------------------------------------------------------------
namespace {

long long thin_chunk(const ModeView& v) { return std::max<long long>(kChunk, (v.P + 1023) / 1024); }

// Ypart[s] = X[range s]^T V[range s] (I x R), V P x R.
tals_status thin_y_parts(tals_ctx* c, const ModeJob& j, const float* X, const float* V) {
  cublasHandle_t h = (cublasHandle_t)c->blas;
  const long long I = j.v.I, P = j.v.P, R = j.R, n = I * R;
  const long long chunk = thin_chunk(j.v);
  const int full = (int)(P / chunk);
  const long long tail = P - (long long)full * chunk;
  float* part = (float*)c->Ypart;
  if (full > 0)
    TALS_BL(gemm_rm_batched(h, true, false, I, R, chunk, X, I, chunk * I, V, R, chunk * R, part, R, n, full));
  if (tail > 0)
    TALS_BL(gemm_rm(h, true, false, I, R, tail, 1.f, X + (size_t)full * chunk * I, I, V + (size_t)full * chunk * R,
                    R, 0.f, part + (size_t)full * n, R));
  return TALS_OK;
}

}  // namespace

int thin_splits(const ModeView& v) {
  const long long chunk = thin_chunk(v);
  return (int)((v.P + chunk - 1) / chunk);
}

tals_status thin_init_launch(tals_ctx* c, const ModeJob& j, bool set_norm_a) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  tals_status st;
  // Sec. 4: Y0 = B_(n) S (S written out as P x R with the fused pass's entries), ||B||^2
  TALS_CK(launch_sketch_prq(c->dtype, j.Wt, j.v, j.R, sketch_state(c->opts.seed, j.n), c->sms, s));
  if ((st = thin_y_parts(c, j, (const float*)j.X, (const float*)j.Wt)) != TALS_OK) return st;
  TALS_CK(launch_sumsq_parts(c->dtype, j.X, (size_t)(j.v.P * j.v.I), c->spart, s));
  return mode_init_tail(c, j, set_norm_a, thin_splits(j.v), c->spart, kSumsqParts);
}

tals_status thin_sweep_launch(tals_ctx* c, const ModeJob& j) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  tals_status st;
  // W = B^T Q_k = X Q_k (P x R), ||W||^2, the Y partials; then the fused path's tail
  TALS_BL(gemm_rm((cublasHandle_t)c->blas, false, false, j.v.P, j.R, j.v.I, 1.f, (const float*)j.X, j.v.I,
                  (const float*)c->Lt, j.R, 0.f, (float*)j.Wt, j.R));
  TALS_CK(launch_sumsq_parts(c->dtype, j.Wt, (size_t)j.v.P * j.R, c->spart, s));
  if ((st = thin_y_parts(c, j, (const float*)j.X, (const float*)j.Wt)) != TALS_OK) return st;
  return mode_sweep_tail(c, j, thin_splits(j.v), kSumsqParts, 1);
}

tals_status bigr_open(tals_ctx* c) {
  if (c->blas != nullptr) return TALS_OK;
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return fail(TALS_ECUDA, "cuBLAS handle creation failed");
  if (cublasSetStream(h, c->stream) != CUBLAS_STATUS_SUCCESS ||
      cublasSetMathMode(h, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS) {
    cublasDestroy(h);
    return fail(TALS_ECUDA, "cuBLAS handle setup failed");
  }
  c->blas = h;
  return TALS_OK;
}

void bigr_close(tals_ctx* c) {
  if (c->blas != nullptr) cublasDestroy((cublasHandle_t)c->blas);
  c->blas = nullptr;
}

#undef TALS_BL
#undef TALS_CK

}  // namespace tals
