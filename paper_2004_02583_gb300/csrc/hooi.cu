// HOOI refinement (Sec. 6.3) and singular-vector recovery (Sec. 5, after Alg. 4).
//
// HOOI cycles over the modes; mode n is replaced by the dominant R_n-dimensional
// left subspace of Y_(n), Y = A x_{m != n} U_m^T (the factors already updated in
// the cycle). Y is formed by the fused pass in projection mode, one mode product
// at a time, the most compressing mode first; the subspace of Y_(n) is found by
// the paper's own ALS (Alg. 3) on Y, warm-started from the current U_n instead of
// the Sec. 4 sketch, so that the ALS machinery (fused sweep pass, FP64 Grams,
// CholeskyQR, the Eq. 5.01 stop rule) is the inner solver and no SVD is needed.
// The last mode's final sweep writes G = Y x_N U_N^T, as in st-HOSVD. The
// relative residual r_k = sqrt(||A||^2 - ||G||^2) / ||A|| (orthonormal U) is
// read back after every cycle for the stop test |r_{k-1} - r_k| < tol.
//
// Singular vectors: the SVD Qhat^T A_(n) = U S V^T through the R x R Gram
// M = Qhat^T A_(n) A_(n)^T Qhat (one fused sweep pass with Qhat as the basis,
// which forms exactly this product), its eigendecomposition M = V diag(S^2) V^T
// by cyclic Jacobi in FP64 on one CTA, U^(n) = Qhat V, and the column signs fixed
// so that each column's entry of largest magnitude is positive.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace tals {

namespace {

constexpr int kJacThreads = 256;
constexpr int kJacMaxSweeps = 40;
constexpr int kMaxR = 64;
constexpr size_t kJacSmem = 2 * kMaxR * (kMaxR + 1) * sizeof(double);

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition M = V diag(lam) V^T (R <= 64, FP64) by the cyclic
// Jacobi method (Golub and Van Loan, Matrix Computations, Sec. 8.5) with the
// round-robin ordering: each round rotates R/2 disjoint index pairs at once
// (positions 0..n'-1, n' = R rounded up to even, position 0 fixed and the others
// shifted by one per round; an index R is a placeholder that pairs with nothing).
// The rotation of pair (p, q) zeroes a_pq: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c, and
// A <- J^T A J, V <- V J with J_pp = J_qq = c, J_pq = s, J_qp = -s. A pair whose
// a_pq is below 1e-16 sqrt(|a_pp a_qq|) or 1e-17 ||A||_F is not rotated; the
// method has converged after a sweep that rotates no pair (at most
// kJacMaxSweeps). Output: lam descending, V's columns in the same order,
// info = sweeps that rotated (negative: not converged).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kJacThreads) jacobi_eig_kernel(const double* __restrict__ M, int R,
                                                                  double* __restrict__ Vout,
                                                                  double* __restrict__ lam,
                                                                  int* __restrict__ info) {
  constexpr int LD = kMaxR + 1;
  extern __shared__ double jac_dyn[];   // a and v, kJacSmem bytes
  double* a = jac_dyn;
  double* v = jac_dyn + kMaxR * LD;
  __shared__ double cs[kMaxR / 2], sn[kMaxR / 2];
  __shared__ int pp[kMaxR / 2], qq[kMaxR / 2];
  __shared__ double red_off[kJacThreads];
  __shared__ int s_rot;
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += kJacThreads) {
    const int i = e / R, j = e % R;
    a[i * LD + j] = 0.5 * (M[i * R + j] + M[j * R + i]);
    v[i * LD + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = (R + 1) & ~1;   // even count of positions
  const int half = np / 2;
  // ||A||_F (invariant under the rotations) for the absolute skip threshold
  double fro = 0.0;
  for (int e = tid; e < R * R; e += kJacThreads) {
    const double x = 0.5 * (M[(e / R) * R + e % R] + M[(e % R) * R + e / R]);
    fro = fma(x, x, fro);
  }
  red_off[tid] = fro;
  __syncthreads();
  for (int w = kJacThreads / 2; w > 0; w >>= 1) {
    if (tid < w) red_off[tid] += red_off[tid + w];
    __syncthreads();
  }
  const double skip_abs = 1e-17 * sqrt(red_off[0]);
  int sweeps = 0;
  bool conv = false;
  for (int sw = 0; sw < kJacMaxSweeps; ++sw) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      if (tid < half) {
        auto pos = [&](int i) { return i == 0 ? 0 : ((i - 1 + round) % (np - 1)) + 1; };
        int p = pos(tid), q = pos(np - 1 - tid);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        bool rot = false;
        if (q < R) {
          const double apq = a[p * LD + q], app = a[p * LD + p], aqq = a[q * LD + q];
          // negligible against the diagonal pair or against ||A||: no rotation
          rot = fabs(apq) > skip_abs && fabs(apq) > 1e-16 * sqrt(fabs(app) * fabs(aqq));
          if (rot) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            s_rot = 1;
          }
        }
        pp[tid] = p;
        qq[tid] = rot ? q : p;   // p == q: the pair rotates nothing
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // columns: A J and V J (pairs touch disjoint columns)
      for (int e = tid; e < R * half; e += kJacThreads) {
        const int i = e / half, k = e % half;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], s = sn[k];
        const double x = a[i * LD + p], y = a[i * LD + q];
        a[i * LD + p] = c * x - s * y;
        a[i * LD + q] = s * x + c * y;
        const double vx = v[i * LD + p], vy = v[i * LD + q];
        v[i * LD + p] = c * vx - s * vy;
        v[i * LD + q] = s * vx + c * vy;
      }
      __syncthreads();
      // rows: J^T (A J) (pairs touch disjoint rows)
      for (int e = tid; e < R * half; e += kJacThreads) {
        const int j = e / half, k = e % half;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], s = sn[k];
        const double x = a[p * LD + j], y = a[q * LD + j];
        a[p * LD + j] = c * x - s * y;
        a[q * LD + j] = s * x + c * y;
      }
      __syncthreads();
    }
    const int any = s_rot;   // every thread reads before thread 0 clears it
    __syncthreads();
    if (!any) {
      conv = true;
      break;
    }
    ++sweeps;
  }
  // descending order: rank of each eigenvalue (ties by index)
  for (int i = tid; i < R; i += kJacThreads) {
    const double li = a[i * LD + i];
    int rank = 0;
    for (int j = 0; j < R; ++j) {
      const double lj = a[j * LD + j];
      rank += (lj > li || (lj == li && j < i)) ? 1 : 0;
    }
    lam[rank] = li;
    for (int r = 0; r < R; ++r) Vout[r * R + rank] = v[r * LD + i];
  }
  if (tid == 0) *info = conv ? sweeps : -sweeps - 1;
}

// Z (I x R, FP64) = L (I x R, FP64) V (R x R, FP64); one thread per entry.
__global__ void __launch_bounds__(256) rotate_basis_kernel(const double* __restrict__ L, long long I, int R,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ Z) {
  __shared__ double vs[kMaxR * kMaxR];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) vs[e] = V[e];
  __syncthreads();
  const long long tot = I * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / R;
    const int c = (int)(e % R);
    const double* li = L + i * R;
    double acc = 0.0;
    for (int r = 0; r < R; ++r) acc = fma(li[r], vs[r * R + c], acc);
    Z[e] = acc;
  }
}

// sgn[c] = the sign of column c's entry of largest magnitude (first on ties);
// one block per column.
__global__ void __launch_bounds__(256) column_sign_kernel(const double* __restrict__ Z, long long I, int R,
                                                          double* __restrict__ sgn) {
  __shared__ double bv[256];
  __shared__ long long bi[256];
  const int c = blockIdx.x;
  double best = -1.0;
  long long at = I;
  for (long long i = threadIdx.x; i < I; i += blockDim.x) {
    const double m = fabs(Z[i * R + c]);
    if (m > best) {   // increasing i per thread: the first maximum is kept
      best = m;
      at = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = at;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double ov = bv[threadIdx.x + w];
      const long long oi = bi[threadIdx.x + w];
      if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ov;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sgn[c] = (bi[0] < I && Z[bi[0] * R + c] < 0.0) ? -1.0 : 1.0;
}

template <typename T>
__global__ void __launch_bounds__(256) write_signed_kernel(const double* __restrict__ Z, long long I, int R,
                                                           const double* __restrict__ sgn,
                                                           T* __restrict__ U) {
  const long long tot = I * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    U[e] = (T)(sgn[e % R] * Z[e]);
}

cudaError_t launch_jacobi(const double* M, int R, double* V, double* lam, int* info, cudaStream_t s) {
  // the attribute belongs to the current device: set on every call
  cudaError_t e = cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacSmem);
  if (e != cudaSuccess) return e;
  jacobi_eig_kernel<<<1, kJacThreads, kJacSmem, s>>>(M, R, V, lam, info);
  return cudaGetLastError();
}

unsigned grid_for(long long n, int sms) {
  const long long want = (n + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(want, (long long)sms * 8));
}

}  // namespace

}  // namespace tals

namespace tals {

// Modes other than `skip` (-1: all) in the order of a projection chain: ascending
// R_m / I_m (the most compressing product first, so the later products read the
// smallest tensors), ties by m.
std::vector<int> hooi_chain(int N, const long long* dims, const int* ranks, int skip) {
  std::vector<int> o;
  for (int m = 0; m < N; ++m)
    if (m != skip) o.push_back(m);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
    return (double)ranks[a] * (double)dims[b] < (double)ranks[b] * (double)dims[a];
  });
  return o;
}

void hooi_views(int N, const long long* dims, const int* ranks, std::vector<ViewR>* sweeps,
                std::vector<ViewR>* products, size_t* inter_elems) {
  size_t inter = 1;
  for (int skip = -1; skip < N; ++skip) {
    long long d[TALS_MAX_NDIM];
    for (int m = 0; m < N; ++m) d[m] = dims[m];
    for (int m : hooi_chain(N, dims, ranks, skip)) {
      const ModeView v = view_of(d, N, m);
      if (products) products->push_back({v, ranks[m]});
      inter = std::max(inter, (size_t)(v.P * v.Q) * (size_t)ranks[m]);
      d[m] = ranks[m];
    }
    if (skip >= 0 && sweeps) sweeps->push_back({view_of(d, N, skip), ranks[skip]});
  }
  if (inter_elems) *inter_elems = inter;
}

namespace {

struct DevScratch {
  cudaStream_t s;
  std::vector<void*> p;
  explicit DevScratch(cudaStream_t st) : s(st) {}
  void* get(size_t bytes, cudaError_t* e) {
    void* q = nullptr;
    *e = cudaMallocAsync(&q, std::max<size_t>(bytes, 256), s);
    if (*e == cudaSuccess) p.push_back(q);
    return q;
  }
  ~DevScratch() {
    for (void* q : p) cudaFreeAsync(q, s);
  }
};

// Y = X x_m U_m^T for m in ms (in that order), sizes d updated. Each product goes
// to the buffer of bufs[0..1] that does not hold its input, the last one to
// `last` when given. *nsp: ||Y||^2 partial sums the last product left in c->spart.
tals_status project_chain(tals_ctx* c, const void* X, long long* d, const std::vector<int>& ms,
                          void* const* U, void* const* bufs, void* last, const void** out, int* nsp) {
  const void* cur = X;
  *nsp = 0;
  for (size_t k = 0; k < ms.size(); ++k) {
    const int m = ms[k];
    const ModeView v = view_of(d, c->N, m);
    void* dest = (k + 1 == ms.size() && last) ? last : (cur == bufs[0] ? bufs[1] : bufs[0]);
    tals_status st = project_mode(c, cur, v, c->ranks[m], U[m], dest, nsp);
    if (st != TALS_OK) return st;
    d[m] = c->ranks[m];
    cur = dest;
  }
  *out = cur;
  return TALS_OK;
}

// ||x||^2 (n elements of the context's dtype) to the host.
tals_status host_sumsq(tals_ctx* c, const void* x, size_t n, double* part, double* dev_out, double* out) {
  cudaError_t e = launch_sumsq(c->dtype, x, n, part, dev_out, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->host_d, dev_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "norm");
  *out = c->host_d[0];
  return TALS_OK;
}

}  // namespace

tals_status hooi_run(tals_ctx* c, void* const* U, void* G_out, double tol, int max_iters, double inner_eta,
                     int inner_sweeps, double* resid_out, tals_hooi_stats* hs) {
  const int N = c->N;
  cudaStream_t s = c->stream;
  const size_t esz = c->esz;
  size_t total = 1, gsize = 1;
  for (int m = 0; m < N; ++m) {
    total *= (size_t)c->dims[m];
    gsize *= (size_t)c->ranks[m];
  }
  size_t inter = 1;
  hooi_views(N, c->dims, c->ranks, nullptr, nullptr, &inter);
  DevScratch sc(s);
  cudaError_t e;
  void* bufs[2];
  bufs[0] = sc.get(inter * esz, &e);
  if (e == cudaSuccess) bufs[1] = sc.get(inter * esz, &e);
  void* G = G_out;
  if (e == cudaSuccess && !G) G = sc.get(gsize * esz, &e);
  double* part = e == cudaSuccess ? (double*)sc.get(kSumsqParts * sizeof(double), &e) : nullptr;
  double* dsc = e == cudaSuccess ? (double*)sc.get(4 * sizeof(double), &e) : nullptr;
  if (e != cudaSuccess) return cuda_fail(e, "HOOI scratch");
  tals_hooi_stats st;
  std::memset(&st, 0, sizeof(st));
  tals_status rs;
  // ||A||^2 (also the norm of Eq. 5.01's stop rule for the inner ALS)
  double na2 = 0.0, g2 = 0.0;
  if ((rs = host_sumsq(c, c->A, total, part, c->norm_a2, &na2)) != TALS_OK) return rs;
  if (!(na2 > 0)) return fail(TALS_EINVAL, "HOOI: the tensor is zero");
  // r_0 from the initial guess
  {
    long long d[TALS_MAX_NDIM];
    for (int m = 0; m < N; ++m) d[m] = c->dims[m];
    const void* out = nullptr;
    int nsp = 0;
    if ((rs = project_chain(c, c->A, d, hooi_chain(N, c->dims, c->ranks, -1), U, bufs, G, &out, &nsp)) != TALS_OK)
      return rs;
    if ((rs = host_sumsq(c, G, gsize, part, dsc, &g2)) != TALS_OK) return rs;
  }
  double r_prev = std::sqrt(std::max(na2 - g2, 0.0) / na2);
  st.resid0 = st.resid = r_prev;
  if (resid_out) resid_out[0] = r_prev;
  for (int k = 1; k <= max_iters; ++k) {
    for (int n = 0; n < N; ++n) {
      long long d[TALS_MAX_NDIM];
      for (int m = 0; m < N; ++m) d[m] = c->dims[m];
      const void* Y = c->A;
      int nsp = 0;
      const std::vector<int> ms = hooi_chain(N, c->dims, c->ranks, n);
      if (ms.empty()) {   // one mode: Y is A itself, ||A||^2 as the one partial
        if ((e = launch_copy(c->spart, c->norm_a2, sizeof(double), s)) != cudaSuccess)
          return cuda_fail(e, "HOOI norm copy");
        nsp = 1;
      } else if ((rs = project_chain(c, c->A, d, ms, U, bufs, nullptr, &Y, &nsp)) != TALS_OK) {
        return rs;
      }
      // the ALS of Alg. 3 on Y_(n), started from L_0 = U_n
      ModeJob j;
      j.n = n;
      j.v = view_of(d, N, n);
      j.R = c->ranks[n];
      j.X = Y;
      j.Wdest = (n == N - 1) ? G : nullptr;
      if ((rs = mode_setup(c, j)) != TALS_OK) return rs;
      const size_t ir = (size_t)j.v.I * j.R;
      const size_t yp = (size_t)(j.t32 ? j.g2 : j.prod ? j.ys : j.pc.grid_x) * ir;
      if (yp > c->ypart_elems || ir > c->need_ir)
        return fail(TALS_ENOTSUP, "HOOI: mode %d exceeds the context's workspace", n);
      if ((e = launch_state_init(j.st, inner_eta, inner_sweeps, j.resid || j.resid_kernel || j.t32, s, 0,
                                 j.t32, j.split_ok, j.prod)) != cudaSuccess)
        return cuda_fail(e, "HOOI state");
      if ((e = launch_copy(c->Ypart, U[n], ir * esz, s)) != cudaSuccess) return cuda_fail(e, "HOOI warm start");
      if ((rs = mode_init_tail(c, j, false, 1, c->spart, nsp)) != TALS_OK) return rs;
      if ((rs = mode_loop_host(c, j, inner_sweeps)) != TALS_OK) return rs;
      if ((rs = tc_check(c)) != TALS_OK) return rs;
      if ((rs = read_states(c)) != TALS_OK) return rs;
      if ((rs = mode_status(c, n)) != TALS_OK) return rs;
      st.inner_sweeps[n] += c->st_host[n].k;
      if ((e = launch_copy(U[n], c->Lt, ir * esz, s)) != cudaSuccess) return cuda_fail(e, "HOOI factor");
    }
    if ((rs = host_sumsq(c, G, gsize, part, dsc, &g2)) != TALS_OK) return rs;
    const double r = std::sqrt(std::max(na2 - g2, 0.0) / na2);
    if (resid_out) resid_out[k] = r;
    st.iters = k;
    st.resid = r;
    if (std::fabs(r_prev - r) < tol) {
      st.converged = 1;
      break;
    }
    r_prev = r;
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "HOOI");
  if (hs) *hs = st;
  return TALS_OK;
}

tals_status singular_vectors_run(tals_ctx* c, int mode, const void* Qhat, void* U_out, double* sigma_out) {
  cudaStream_t s = c->stream;
  const int R = c->ranks[mode];
  ModeJob j;
  j.n = mode;
  j.v = view_of(c->dims, c->N, mode);
  j.R = R;
  j.X = c->A;
  j.Wdest = nullptr;
  tals_status rs = mode_setup(c, j);
  if (rs != TALS_OK) return rs;
  j.t32 = 0;   // one plain product pass
  j.resid = 0;
  j.resid_kernel = 0;
  const long long I = j.v.I;
  cudaError_t e;
#define TALS_CK(x) \
  if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x);
  TALS_CK(launch_state_init(j.st, -1.0, 2, 0, s));
  // L64 = Qhat in FP64 and the pass's basis Lt = Qhat, exactly as given
  TALS_CK(launch_reduce_rows(c->dtype, Qhat, 1, I, R, c->L64, 1, nullptr, c->Gpart, j.rp, nullptr, 0, 0, j.st,
                             nullptr, s));
  TALS_CK(launch_copy(c->Lt, Qhat, (size_t)I * R * c->esz, s));
  // W = A_(n)^T Qhat, Y = A_(n) W; M = Qhat^T Y = (Qhat^T A_(n)) (Qhat^T A_(n))^T
  int gx = 1, nsp = 0;
  if (j.twopass) {
    const size_t ir = (size_t)I * R;
    TALS_CK(launch_mode_project_any(c->dtype, c->A, j.v, c->Lt, R, j.Wt, s));
    TALS_CK(launch_mode_adjoint_any(c->dtype, c->A, j.v, j.Wt, R, j.splits, (char*)c->Ypart + ir * c->esz,
                                    c->Ypart, s));
  } else {
    TALS_CK(launch_pass(c->dtype, j.pc, PASS_SWEEP, c->A, j.v, R, c->Lt, c->Ypart, c->spart, nullptr, 0, j.st, 1,
                        s));
    gx = j.pc.grid_x;
    nsp = j.pc.grid_x * j.pc.grid_y;
  }
  TALS_CK(launch_reduce_rows(c->dtype, c->Ypart, gx, I, R, c->Y64, 2, c->L64, c->Gpart, j.rp, c->spart, nsp, 1,
                             j.st, nullptr, s));
  TALS_CK(launch_gram_sum(c->Gpart, j.rp.blocks, R, c->Gfin, j.st, s));
  // M = V diag(lam) V^T; scratch in F (3 R^2 + R doubles): V, lam, info, signs
  double* V = c->F;
  double* lam = c->F + (size_t)R * R;
  int* info = reinterpret_cast<int*>(c->F + (size_t)R * R + R);
  double* sgn = c->F + (size_t)R * R + R + 1;
  TALS_CK(launch_jacobi(c->Gfin, R, V, lam, info, s));
  const unsigned g = grid_for(I * R, c->sms);
  rotate_basis_kernel<<<g, 256, 0, s>>>(c->L64, I, R, V, c->Z64);
  TALS_CK(cudaGetLastError());
  column_sign_kernel<<<R, 256, 0, s>>>(c->Z64, I, R, sgn);
  TALS_CK(cudaGetLastError());
  if (c->dtype == TALS_F32)
    write_signed_kernel<float><<<g, 256, 0, s>>>(c->Z64, I, R, sgn, (float*)U_out);
  else
    write_signed_kernel<double><<<g, 256, 0, s>>>(c->Z64, I, R, sgn, (double*)U_out);
  TALS_CK(cudaGetLastError());
  std::vector<double> h((size_t)R + 1);
  TALS_CK(cudaMemcpyAsync(h.data(), lam, ((size_t)R + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  TALS_CK(cudaStreamSynchronize(s));
#undef TALS_CK
  int inf = 0;
  std::memcpy(&inf, &h[R], sizeof(int));
  if (inf < 0) return fail(TALS_ENOTSUP, "singular vectors: the Jacobi sweeps did not converge");
  if (sigma_out)
    for (int r = 0; r < R; ++r) sigma_out[r] = std::sqrt(std::max(h[r], 0.0));
  return TALS_OK;
}

}  // namespace tals

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

tals_status tals_hooi(tals_ctx* c, void* const* U_io, void* G_out, double tol, int max_iters,
                      double inner_eta, int inner_sweeps, double* resid_out, tals_hooi_stats* stats) {
  using namespace tals;
  if (!c || !U_io) return fail(TALS_EINVAL, "ctx and U_io must not be NULL");
  for (int n = 0; n < c->N; ++n)
    if (!U_io[n]) return fail(TALS_EINVAL, "U_io[%d] is NULL", n);
  if (max_iters < 1) return fail(TALS_EINVAL, "max_iters must be >= 1");
  if (inner_sweeps < 1) return fail(TALS_EINVAL, "inner_sweeps must be >= 1");
  if (!(tol >= 0.0)) return fail(TALS_EINVAL, "tol must be >= 0");
  if (c->has_bigr) return fail(TALS_ENOTSUP, "HOOI takes ranks up to %d", kBigRankMin);
  return hooi_run(c, U_io, G_out, tol, max_iters, inner_eta, inner_sweeps, resid_out, stats);
}

tals_status tals_singular_vectors(tals_ctx* c, int mode, const void* Qhat, void* U_out, double* sigma_out) {
  using namespace tals;
  if (!c || !Qhat || !U_out) return fail(TALS_EINVAL, "ctx, Qhat and U_out must not be NULL");
  if (mode < 0 || mode >= c->N) return fail(TALS_EINVAL, "mode %d outside [0, %d)", mode, c->N);
  if (U_out == Qhat) return fail(TALS_EINVAL, "U_out must not alias Qhat");
  if (c->ranks[mode] > kBigRankMin) return fail(TALS_ENOTSUP, "singular vectors take ranks up to %d", kBigRankMin);
  return singular_vectors_run(c, mode, Qhat, U_out, sigma_out);
}

}  // extern "C"
