// A variant of the fused sweep pass (tals_sweep_pass, CUDA-core FP32 engine)
// that allocates no device memory.
//
// The regular entry points take their scratch (the per-CTA partial sums of Y
// and of ||W||^2) from stream-ordered allocations. Some callers cannot
// allocate at call time: code that runs while a memory pool owns all device
// memory, code whose allocator is a framework's caching pool that must not
// be bypassed, or latency-critical loops that cannot afford an allocation
// (and the synchronisation a plain cudaMalloc implies). This entry point takes
// its scratch from one fixed array in device global memory instead, declared
// at file scope below. Every GPU that loads the library holds that array until
// the process exits.
#include <mutex>

#include "internal.h"

namespace tals {

// Scratch layout: [kNoAllocSums doubles of per-CTA ||W||^2 partials]
//                 [kNoAllocPartials floats of per-CTA Y partials].
constexpr size_t kNoAllocSums = 1024;
constexpr size_t kNoAllocPartials = (size_t)1 << 20;   // 4 MiB of FP32 partials
constexpr size_t kNoAllocBytes = kNoAllocSums * sizeof(double) + kNoAllocPartials * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device. The first call on
// a device looks it up (the host-side name of the array is only a stand-in, not
// a device address).
tals_status scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "current device");
  if (dev < 0 || dev >= kMaxDevices) return fail(TALS_ENOTSUP, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "scratch symbol address");
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return TALS_OK;
}

// *out = sum of n partials, fixed order (one CTA).
__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) *out = t;
}

}  // namespace

}  // namespace tals

using namespace tals;

extern "C" tals_status tals_sweep_pass_noalloc(const void* A, int ndim, const int64_t* dims,
                                               int mode, const void* Q, int R, double* Y_out,
                                               double* wnorm2_out, void* stream) {
  if (!A || !dims || !Q || !Y_out || !wnorm2_out || ndim < 1 || ndim > TALS_MAX_NDIM ||
      mode < 0 || mode >= ndim || R < 1)
    return fail(TALS_EINVAL, "bad arguments");
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < ndim; ++m) {
    if (dims[m] < 1) return fail(TALS_EINVAL, "dims[%d] < 1", m);
    d[m] = dims[m];
  }
  const ModeView v = view_of(d, ndim, mode);
  if (R > v.I) return fail(TALS_EINVAL, "R exceeds I");
  const size_t ir = (size_t)v.I * (size_t)R;
  if (ir > kNoAllocPartials)
    return fail(TALS_EINVAL,
                "I_mode x R = %zu exceeds the no-allocation scratch limit of %zu (2^20) elements",
                ir, kNoAllocPartials);
  unsigned char* scratch = nullptr;
  tals_status st = scratch_on_current_device(&scratch);
  if (st != TALS_OK) return st;
  int dev = 0, sms = 0;
  cudaError_t qe = cudaGetDevice(&dev);
  if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (qe != cudaSuccess) return cuda_fail(qe, "device query");
  PassConfig pc = pass_config(TALS_F32, v, R, sms);
  if (!pc.ok) return fail(TALS_ENOTSUP, "shape outside the pass kernel limits");
  // fewer CTAs when their partials would not fit the fixed scratch
  const size_t max_gx_y = kNoAllocPartials / ir;
  const size_t max_gx_s = kNoAllocSums / (size_t)pc.grid_y;
  pc.grid_x = (int)std::min<size_t>((size_t)pc.grid_x, std::min(max_gx_y, max_gx_s));
  if (pc.grid_x < 1) return fail(TALS_EINVAL, "shape too large for the no-allocation scratch");
  double* spart = reinterpret_cast<double*>(scratch);
  float* ypart = reinterpret_cast<float*>(scratch + kNoAllocSums * sizeof(double));
  cudaStream_t s = (cudaStream_t)stream;
  // Every scratch word this call reads is written earlier by the same call (each
  // CTA writes its whole partial slot), so nothing needs clearing between calls.
  cudaError_t e = launch_pass(TALS_F32, pc, PASS_SWEEP, A, v, R, Q, ypart, spart, nullptr, 0,
                              nullptr, 0, s);
  if (e == cudaSuccess) {
    const RowPlan rp = row_plan(v.I, R, sms);
    e = launch_reduce_rows(TALS_F32, ypart, pc.grid_x, v.I, R, Y_out, 0, nullptr, nullptr, rp,
                           nullptr, 0, 0, nullptr, nullptr, s);
  }
  if (e == cudaSuccess) {
    sum_partials_kernel<<<1, 256, 0, s>>>(spart, pc.grid_x * pc.grid_y, wnorm2_out);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "no-allocation sweep pass");
}
