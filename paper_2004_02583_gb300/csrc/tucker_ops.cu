// Tucker-model operators and their adjoints (Sec. 2 mode products and Tucker
// model; the core step of Alg. 1/4):
//   project      G = A x_1 U1^T ... x_N UN^T
//   reconstruct  B = G x_1 U1 ... x_N UN
//   project_backward / reconstruct_backward: the vector-Jacobian products.
// Every mode product is one pass of the same tiled kernel that the ALS sweep
// uses (PROJECT mode: X x_n L^T with L = U_n, or L = U_n^T to expand a mode).
// The factor adjoints U_bar_n = (X x_{m!=n} Um^T)_(n) V_(n)^T need, for every n,
// X projected on all other modes. Those partial contractions are recomputed
// with a leave-one-out tree: split the modes in halves, project X on one half
// and recurse into the other, so the full-size X is read twice for any N and no
// partial is stored for all n at once.
#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"

namespace tals {

namespace {

struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  void* get(size_t bytes, cudaError_t* e) {
    void* p = nullptr;
    *e = cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s);
    if (*e == cudaSuccess) ptrs.push_back(p);
    return p;
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFreeAsync(q, s);
        q = nullptr;
      }
  }
  ~Scratch() {
    for (void* p : ptrs)
      if (p) cudaFreeAsync(p, s);
  }
};

struct OpCtx {
  int dtype;
  size_t esz;
  int N;
  long long dims[TALS_MAX_NDIM];
  int ranks[TALS_MAX_NDIM];
  void* const* U;
  cudaStream_t s;
  int sms;
  Scratch* sc;
};

size_t numel(const long long* d, int N) {
  size_t n = 1;
  for (int m = 0; m < N; ++m) n *= (size_t)d[m];
  return n;
}

// out = X x_n L^T, where X has sizes d and L is d[n] x R_out (row-major).
tals_status apply_mode(OpCtx& o, const void* X, const long long* d, int n, const void* L,
                       int R_out, void* out) {
  ModeView v = view_of(d, o.N, n);
  if (o.dtype == TALS_F32 && (v.Q >= 64 || v.Q == 1 || v.Q % 4 == 0)) {
    // register-tiled mode product: M = L^T, element (a, b) = L[b * R_out + a]
    cudaError_t e = launch_mode_gemm((const float*)X, v.P, v.I, v.Q, (const float*)L, 1, R_out, R_out,
                                     (float*)out, o.s);
    if (e == cudaSuccess) return TALS_OK;
    if (e != cudaErrorNotSupported) return cuda_fail(e, "mode product");
  }
  PassConfig pc = pass_config(o.dtype, v, R_out, o.sms);
  if (!pc.ok) {
    // any-view tiled product: M = L^T
    cudaError_t e = o.dtype == TALS_F32
                        ? launch_mode_gemm_any((const float*)X, v.P, v.I, v.Q, (const float*)L, 1, R_out, R_out,
                                               (float*)out, o.s)
                        : launch_mode_gemm_any((const double*)X, v.P, v.I, v.Q, (const double*)L, 1, R_out,
                                               R_out, (double*)out, o.s);
    if (e != cudaSuccess) return fail(TALS_ENOTSUP, "mode product of mode %d (size %lld -> %d): %s", n, v.I,
                                      R_out, cudaGetErrorString(e));
    return TALS_OK;
  }
  cudaError_t e;
  double* sp = (double*)o.sc->get((size_t)pc.grid_x * pc.grid_y * sizeof(double), &e);
  if (e != cudaSuccess) return cuda_fail(e, "scratch");
  e = launch_pass(o.dtype, pc, PASS_PROJECT, X, v, R_out, L, nullptr, sp, out, 0, nullptr, 0, o.s);
  if (e != cudaSuccess) return cuda_fail(e, "mode product");
  return TALS_OK;
}

// X x_m Um^T for every m in `modes` (in that order); returns the new tensor
// (scratch) and updates d. Never frees X.
tals_status project_modes(OpCtx& o, const void* X, long long* d, const std::vector<int>& modes,
                          const void** out) {
  const void* cur = X;
  void* prev_owned = nullptr;
  for (int m : modes) {
    long long nd[TALS_MAX_NDIM];
    std::copy(d, d + o.N, nd);
    nd[m] = o.ranks[m];
    cudaError_t e;
    void* dst = o.sc->get(numel(nd, o.N) * o.esz, &e);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    tals_status st = apply_mode(o, cur, d, m, o.U[m], o.ranks[m], dst);
    if (st != TALS_OK) return st;
    if (prev_owned) o.sc->release(prev_owned);
    prev_owned = dst;
    cur = dst;
    d[m] = o.ranks[m];
  }
  *out = cur;
  return TALS_OK;
}

// U_bar_n = (P)_(n) V_(n)^T where P has sizes d (mode n full, others at rank).
tals_status factor_adjoint(OpCtx& o, const void* P, const long long* d, int n, const void* V,
                           void* Ubar) {
  ModeView v = view_of(d, o.N, n);
  const int R = o.ranks[n];
  PassConfig pc = pass_config(o.dtype, v, R, o.sms);
  if (!pc.ok) {
    // any-view form in column splits
    const int S = factor_adjoint_splits(v.P, v.I, v.Q, R, o.sms);
    cudaError_t e;
    void* part = o.sc->get((size_t)S * v.I * R * o.esz, &e);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    e = o.dtype == TALS_F32
            ? launch_factor_adjoint_any((const float*)P, v.P, v.I, v.Q, (const float*)V, R, S, (float*)part,
                                        (float*)Ubar, o.s)
            : launch_factor_adjoint_any((const double*)P, v.P, v.I, v.Q, (const double*)V, R, S, (double*)part,
                                        (double*)Ubar, o.s);
    if (e != cudaSuccess) return fail(TALS_ENOTSUP, "factor adjoint of mode %d: %s", n, cudaGetErrorString(e));
    o.sc->release(part);
    return TALS_OK;
  }
  RowPlan rp = row_plan(v.I, R, o.sms);
  cudaError_t e;
  void* yp = o.sc->get((size_t)pc.grid_x * v.I * R * o.esz, &e);
  if (e != cudaSuccess) return cuda_fail(e, "scratch");
  double* sp = (double*)o.sc->get((size_t)pc.grid_x * pc.grid_y * sizeof(double), &e);
  if (e != cudaSuccess) return cuda_fail(e, "scratch");
  e = launch_pass(o.dtype, pc, PASS_GIVEN, P, v, R, nullptr, yp, sp, nullptr, 0, nullptr, 0, o.s, V);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint pass");
  e = launch_reduce_rows(o.dtype, yp, pc.grid_x, v.I, R, nullptr, 0, nullptr, nullptr, rp, nullptr,
                         0, 0, nullptr, nullptr, o.s, Ubar);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint reduction");
  o.sc->release(yp);
  return TALS_OK;
}

// Leave-one-out tree over `targets` (all still full in X, as are the modes in `full`).
tals_status loo(OpCtx& o, const void* X, const long long* d, std::vector<int> full,
                std::vector<int> targets, const void* V, void* const* Ubar, void* Gproj,
                bool* gproj_done) {
  if (targets.size() == 1) {
    const int n = targets[0];
    std::vector<int> others;
    for (int m : full)
      if (m != n) others.push_back(m);
    long long dd[TALS_MAX_NDIM];
    std::copy(d, d + o.N, dd);
    const void* P = nullptr;
    tals_status st = project_modes(o, X, dd, others, &P);
    if (st != TALS_OK) return st;
    if (Ubar && Ubar[n] && (st = factor_adjoint(o, P, dd, n, V, Ubar[n])) != TALS_OK) return st;
    if (Gproj && !*gproj_done) {
      if ((st = apply_mode(o, P, dd, n, o.U[n], o.ranks[n], Gproj)) != TALS_OK) return st;
      *gproj_done = true;
    }
    if (P != X) o.sc->release(const_cast<void*>(P));
    return TALS_OK;
  }
  const size_t h = targets.size() / 2;
  std::vector<int> t1(targets.begin(), targets.begin() + h), t2(targets.begin() + h, targets.end());
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<int>& keep = pass == 0 ? t1 : t2;
    const std::vector<int>& drop = pass == 0 ? t2 : t1;
    long long dd[TALS_MAX_NDIM];
    std::copy(d, d + o.N, dd);
    const void* Xp = nullptr;
    tals_status st = project_modes(o, X, dd, drop, &Xp);
    if (st != TALS_OK) return st;
    std::vector<int> rest;
    for (int m : full)
      if (std::find(drop.begin(), drop.end(), m) == drop.end()) rest.push_back(m);
    st = loo(o, Xp, dd, rest, keep, V, Ubar, Gproj, gproj_done);
    if (Xp != X) o.sc->release(const_cast<void*>(Xp));
    if (st != TALS_OK) return st;
  }
  return TALS_OK;
}

tals_status validate_ops(int dtype, int ndim, const int64_t* dims, const int* ranks,
                         void* const* U) {
  if (dtype != TALS_F32 && dtype != TALS_F64) return fail(TALS_EINVAL, "unsupported dtype %d", dtype);
  if (ndim < 1 || ndim > TALS_MAX_NDIM) return fail(TALS_EINVAL, "ndim %d outside [1, 8]", ndim);
  if (!dims || !ranks || !U) return fail(TALS_EINVAL, "dims, ranks and U must not be NULL");
  for (int n = 0; n < ndim; ++n) {
    if (dims[n] < 1 || ranks[n] < 1 || ranks[n] > dims[n])
      return fail(TALS_EINVAL, "mode %d: need 1 <= R_n <= I_n", n);
    if (!U[n]) return fail(TALS_EINVAL, "U[%d] is NULL", n);
  }
  return TALS_OK;
}

OpCtx make_ctx(int dtype, int ndim, const int64_t* dims, const int* ranks, void* const* U,
               void* stream, Scratch* sc) {
  OpCtx o;
  o.dtype = dtype;
  o.esz = dtype == TALS_F32 ? 4 : 8;
  o.N = ndim;
  for (int n = 0; n < ndim; ++n) {
    o.dims[n] = dims[n];
    o.ranks[n] = ranks[n];
  }
  o.U = U;
  o.s = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
  o.sc = sc;
  return o;
}

// Order in which a chain of mode products keeps intermediates smallest.
// Order of the mode products of a projection (expand = false: I_m -> R_m from
// the full tensor) or a reconstruction (expand = true: R_m -> I_m from the
// core) with the fewest multiply-adds: a mode product costs (elements of the
// larger of its input and output) x (the smaller of I_m, R_m), and the
// minimum over all orders is found exactly by dynamic programming over the
// subsets of modes already applied (N <= 8: at most 256 subsets). Ties keep
// the lower mode first.
std::vector<int> product_order(int N, const long long* dims, const int* ranks, bool expand,
                               double* cost) {
  const int full = (1 << N) - 1;
  // elements of the tensor once the modes in `done` are applied
  auto size_of = [&](int done) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) {
      const bool applied = (done >> m) & 1;
      const double at_rank = (double)ranks[m], at_full = (double)dims[m];
      v *= expand ? (applied ? at_full : at_rank) : (applied ? at_rank : at_full);
    }
    return v;
  };
  std::vector<double> best(full + 1, 1e300);
  std::vector<int> last(full + 1, -1);
  best[0] = 0.0;
  for (int done = 1; done <= full; ++done)
    for (int m = 0; m < N; ++m) {
      if (!((done >> m) & 1)) continue;
      const int prev = done & ~(1 << m);
      const double big = expand ? size_of(done) : size_of(prev);
      const double c = best[prev] + big * (double)std::min<long long>(ranks[m], dims[m]);
      if (c < best[done] * (1.0 - 1e-12)) {
        best[done] = c;
        last[done] = m;
      }
    }
  std::vector<int> ord(N);
  for (int done = full, k = N - 1; k >= 0; --k) {
    ord[k] = last[done];
    done &= ~(1 << last[done]);
  }
  if (cost) *cost = best[full];
  return ord;
}

std::vector<int> shrink_order(const OpCtx& o, bool expand) {
  return product_order(o.N, o.dims, o.ranks, expand, nullptr);
}

tals_status do_project(OpCtx& o, const void* A, void* G_out) {
  std::vector<int> ord = shrink_order(o, false);
  long long d[TALS_MAX_NDIM];
  std::copy(o.dims, o.dims + o.N, d);
  const void* cur = A;
  void* owned = nullptr;
  for (size_t k = 0; k < ord.size(); ++k) {
    const int m = ord[k];
    long long nd[TALS_MAX_NDIM];
    std::copy(d, d + o.N, nd);
    nd[m] = o.ranks[m];
    void* dst = G_out;
    cudaError_t e = cudaSuccess;
    if (k + 1 < ord.size()) dst = o.sc->get(numel(nd, o.N) * o.esz, &e);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    tals_status st = apply_mode(o, cur, d, m, o.U[m], o.ranks[m], dst);
    if (st != TALS_OK) return st;
    if (owned) o.sc->release(owned);
    owned = (dst == G_out) ? nullptr : dst;
    cur = dst;
    d[m] = o.ranks[m];
  }
  return TALS_OK;
}

// B = G x_1 U1 ... x_N UN into B_out. With tgt (FP32, the loss form of the last
// register-tiled expansion): B_out = 2 (B - tgt) and part[0 .. *nparts) the sums of
// (B - tgt)^2; *nparts stays 0 where that form does not apply (B_out then holds B).
tals_status do_reconstruct(OpCtx& o, const void* G, void* B_out, const void* tgt = nullptr,
                           double* part = nullptr, long long cap = 0, long long* nparts = nullptr) {
  std::vector<int> ord = shrink_order(o, true);
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < o.N; ++m) d[m] = o.ranks[m];
  const void* cur = G;
  void* owned = nullptr;
  cudaError_t e;
  for (size_t k = 0; k < ord.size(); ++k) {
    const int m = ord[k];
    long long nd[TALS_MAX_NDIM];
    std::copy(d, d + o.N, nd);
    nd[m] = o.dims[m];
    {
      // register-tiled expansion with M = U_m (element (i, r) = U[i * R + r])
      ModeView v = view_of(d, o.N, m);
      if (o.dtype == TALS_F32 && (v.Q >= 64 || v.Q == 1 || v.Q % 4 == 0)) {
        void* dst = B_out;
        if (k + 1 < ord.size()) dst = o.sc->get(numel(nd, o.N) * o.esz, &e);
        if (e != cudaSuccess) return cuda_fail(e, "scratch");
        e = cudaErrorNotSupported;
        if (tgt != nullptr && k + 1 == ord.size())
          e = launch_mode_gemm_loss((const float*)cur, v.P, v.I, v.Q, (const float*)o.U[m], o.ranks[m], 1,
                                    o.dims[m], (float*)dst, (const float*)tgt, part, cap, nparts, o.s);
        if (e == cudaErrorNotSupported)
          e = launch_mode_gemm((const float*)cur, v.P, v.I, v.Q, (const float*)o.U[m], o.ranks[m], 1,
                               o.dims[m], (float*)dst, o.s);
        if (e == cudaSuccess) {
          if (owned) o.sc->release(owned);
          owned = (dst == B_out) ? nullptr : dst;
          cur = dst;
          d[m] = o.dims[m];
          continue;
        }
        if (e != cudaErrorNotSupported) return cuda_fail(e, "expansion");
        if (dst != B_out) o.sc->release(dst);
      }
    }
    // expand mode m: X x_m U_m = X x_m (U_m^T)^T with L = U_m^T (R_m x I_m)
    void* Lt = o.sc->get((size_t)o.dims[m] * o.ranks[m] * o.esz, &e);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    e = launch_transpose(o.dtype, o.U[m], o.dims[m], o.ranks[m], Lt, o.s);
    if (e != cudaSuccess) return cuda_fail(e, "transpose");
    void* dst = B_out;
    if (k + 1 < ord.size()) dst = o.sc->get(numel(nd, o.N) * o.esz, &e);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    tals_status st = apply_mode(o, cur, d, m, Lt, (int)o.dims[m], dst);
    if (st != TALS_OK) return st;
    o.sc->release(Lt);
    if (owned) o.sc->release(owned);
    owned = (dst == B_out) ? nullptr : dst;
    cur = dst;
    d[m] = o.dims[m];
  }
  return TALS_OK;
}

constexpr int kLossThreads = 256;
constexpr int kLossBlocks = 1024;

// D = 2 (D - A) in place (D holds B) and per-block sums of (B - A)^2 in FP64.
template <typename T>
__global__ void __launch_bounds__(kLossThreads) loss_kernel(T* __restrict__ D, const T* __restrict__ A, long long n,
                                                            double* __restrict__ part) {
  __shared__ double red[kLossThreads];
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * kLossThreads + threadIdx.x; e < n;
       e += (long long)gridDim.x * kLossThreads) {
    const T d = D[e] - A[e];
    D[e] = (T)2 * d;
    acc = fma((double)d, (double)d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// *out = sum of the n partials, in a fixed order.
__global__ void __launch_bounds__(kLossThreads) loss_sum_kernel(const double* __restrict__ part, long long n,
                                                                double* __restrict__ out) {
  __shared__ double red[kLossThreads];
  double acc = 0.0;
  for (long long k = threadIdx.x; k < n; k += kLossThreads) acc += part[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

tals_status finish(cudaStream_t s) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "tucker op");
}

}  // namespace

}  // namespace tals

using namespace tals;

extern "C" {

tals_status tals_mode_product_order(int ndim, const int64_t* dims, const int* ranks, int expand,
                                    int* order_out, double* madds_out) {
  if (ndim < 1 || ndim > TALS_MAX_NDIM) return fail(TALS_EINVAL, "ndim must be in 1..%d", TALS_MAX_NDIM);
  if (!dims || !ranks || !order_out) return fail(TALS_EINVAL, "NULL argument");
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < ndim; ++m) {
    if (dims[m] < 1 || ranks[m] < 1) return fail(TALS_EINVAL, "sizes and ranks must be >= 1");
    d[m] = dims[m];
  }
  const std::vector<int> ord = product_order(ndim, d, ranks, expand != 0, madds_out);
  std::copy(ord.begin(), ord.end(), order_out);
  return TALS_OK;
}

tals_status project(const void* A, void* const* U, int dtype, int ndim, const int64_t* dims,
                    const int* ranks, void* G_out, void* stream) {
  tals_status st = validate_ops(dtype, ndim, dims, ranks, U);
  if (st != TALS_OK) return st;
  if (!A || !G_out) return fail(TALS_EINVAL, "A and G_out must not be NULL");
  Scratch sc((cudaStream_t)stream);
  OpCtx o = make_ctx(dtype, ndim, dims, ranks, U, stream, &sc);
  if ((st = do_project(o, A, G_out)) != TALS_OK) return st;
  return finish(o.s);
}

tals_status reconstruct(const void* G, void* const* U, int dtype, int ndim, const int64_t* dims,
                        const int* ranks, void* B_out, void* stream) {
  tals_status st = validate_ops(dtype, ndim, dims, ranks, U);
  if (st != TALS_OK) return st;
  if (!G || !B_out) return fail(TALS_EINVAL, "G and B_out must not be NULL");
  Scratch sc((cudaStream_t)stream);
  OpCtx o = make_ctx(dtype, ndim, dims, ranks, U, stream, &sc);
  if ((st = do_reconstruct(o, G, B_out)) != TALS_OK) return st;
  return finish(o.s);
}

tals_status reconstruction_loss(const void* G, void* const* U, const void* A, int dtype, int ndim,
                                const int64_t* dims, const int* ranks, void* D_out, double* loss_out,
                                void* stream) {
  tals_status st = validate_ops(dtype, ndim, dims, ranks, U);
  if (st != TALS_OK) return st;
  if (!G || !A || !D_out || !loss_out) return fail(TALS_EINVAL, "G, A, D_out and loss_out must not be NULL");
  if (D_out == A) return fail(TALS_EINVAL, "D_out must not alias A");
  Scratch sc((cudaStream_t)stream);
  OpCtx o = make_ctx(dtype, ndim, dims, ranks, U, stream, &sc);
  cudaError_t e;
  const long long cap = 1 << 16;
  double* part = (double*)sc.get((size_t)cap * sizeof(double), &e);
  if (e != cudaSuccess) return cuda_fail(e, "scratch");
  long long np = 0;
  if ((st = do_reconstruct(o, G, D_out, dtype == TALS_F32 ? A : nullptr, part, cap, &np)) != TALS_OK) return st;
  if (np == 0) {
    // the loss form did not apply: D_out holds B
    const long long n = (long long)numel(o.dims, ndim);
    np = std::min<long long>(kLossBlocks, std::max<long long>(1, (n + kLossThreads - 1) / kLossThreads));
    if (dtype == TALS_F32)
      loss_kernel<float><<<(unsigned)np, kLossThreads, 0, o.s>>>((float*)D_out, (const float*)A, n, part);
    else
      loss_kernel<double><<<(unsigned)np, kLossThreads, 0, o.s>>>((double*)D_out, (const double*)A, n, part);
  }
  loss_sum_kernel<<<1, kLossThreads, 0, o.s>>>(part, np, loss_out);
  return finish(o.s);
}

tals_status reconstruct_backward(const void* G, void* const* U, const void* B_bar, int dtype,
                                 int ndim, const int64_t* dims, const int* ranks, void* G_bar,
                                 void* const* U_bar, void* stream) {
  tals_status st = validate_ops(dtype, ndim, dims, ranks, U);
  if (st != TALS_OK) return st;
  if (!G || !B_bar) return fail(TALS_EINVAL, "G and B_bar must not be NULL");
  Scratch sc((cudaStream_t)stream);
  OpCtx o = make_ctx(dtype, ndim, dims, ranks, U, stream, &sc);
  std::vector<int> all(ndim);
  std::iota(all.begin(), all.end(), 0);
  bool gdone = false;
  // G_bar = B_bar x U^T; U_bar_n = (B_bar x_{m!=n} Um^T)_(n) G_(n)^T
  if ((st = loo(o, B_bar, o.dims, all, all, G, U_bar, G_bar, &gdone)) != TALS_OK) return st;
  return finish(o.s);
}

tals_status project_backward(const void* A, void* const* U, const void* G_bar, int dtype,
                             int ndim, const int64_t* dims, const int* ranks, void* A_bar,
                             void* const* U_bar, void* stream) {
  tals_status st = validate_ops(dtype, ndim, dims, ranks, U);
  if (st != TALS_OK) return st;
  if (!A || !G_bar) return fail(TALS_EINVAL, "A and G_bar must not be NULL");
  Scratch sc((cudaStream_t)stream);
  OpCtx o = make_ctx(dtype, ndim, dims, ranks, U, stream, &sc);
  // A_bar = G_bar x_1 U1 ... x_N UN
  if (A_bar && (st = do_reconstruct(o, G_bar, A_bar)) != TALS_OK) return st;
  if (U_bar) {
    std::vector<int> all(ndim);
    std::iota(all.begin(), all.end(), 0);
    bool gdone = true;
    if ((st = loo(o, A, o.dims, all, all, G_bar, U_bar, nullptr, &gdone)) != TALS_OK) return st;
  }
  return finish(o.s);
}

}  // extern "C"
