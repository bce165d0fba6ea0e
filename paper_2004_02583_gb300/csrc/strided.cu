// Strided input: a tensor whose element (i_1 .. i_N) sits at src + sum_k i_k s_k
// (element strides in any order) gathered into the dense row-major layout every
// other entry point reads. The method reads each mode-n unfolding from the
// tensor's layout (Sec. 3); the kernels here read P x I_n x Q views with unit
// stride along Q, so a tensor in another layout is written out once, when its
// context is created.
#include "internal.h"

namespace tals {

namespace {

struct StrideSpec {
  int ndim;
  long long dims[TALS_MAX_NDIM];
  long long strides[TALS_MAX_NDIM];
};

template <typename T>
__global__ void gather_kernel(const T* __restrict__ src, StrideSpec sp, long long n, T* __restrict__ dst) {
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    long long rem = o, off = 0;
    for (int k = sp.ndim - 1; k >= 0; --k) {
      const long long i = rem % sp.dims[k];
      rem /= sp.dims[k];
      off += i * sp.strides[k];
    }
    dst[o] = src[off];
  }
}

}  // namespace

bool strides_valid(int ndim, const int64_t* dims, const int64_t* strides) {
  if (ndim < 1 || ndim > TALS_MAX_NDIM || dims == nullptr || strides == nullptr) return false;
  // axes of size above 1, by stride: each must step over the whole extent of the
  // previous one, so that no two elements share an address
  int ax[TALS_MAX_NDIM];
  int m = 0;
  for (int k = 0; k < ndim; ++k) {
    if (dims[k] < 1 || strides[k] < 0) return false;
    if (dims[k] > 1) {
      if (strides[k] < 1) return false;
      ax[m++] = k;
    }
  }
  for (int a = 1; a < m; ++a)
    for (int b = a; b > 0 && strides[ax[b]] < strides[ax[b - 1]]; --b) {
      const int t = ax[b];
      ax[b] = ax[b - 1];
      ax[b - 1] = t;
    }
  for (int a = 1; a < m; ++a)
    if (strides[ax[a]] < strides[ax[a - 1]] * dims[ax[a - 1]]) return false;
  return true;
}

cudaError_t launch_gather(int dtype, const void* src, int ndim, const int64_t* dims, const int64_t* strides,
                          void* dst, int sms, cudaStream_t s) {
  StrideSpec sp{};
  sp.ndim = ndim;
  long long n = 1;
  for (int k = 0; k < ndim; ++k) {
    sp.dims[k] = dims[k];
    sp.strides[k] = strides[k];
    n *= dims[k];
  }
  const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * sms));
  if (dtype == TALS_F32)
    gather_kernel<float><<<g, 256, 0, s>>>((const float*)src, sp, n, (float*)dst);
  else
    gather_kernel<double><<<g, 256, 0, s>>>((const double*)src, sp, n, (double*)dst);
  return cudaGetLastError();
}

}  // namespace tals
