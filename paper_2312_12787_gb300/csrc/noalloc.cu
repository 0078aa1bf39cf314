// Refinement residual for callers that must not allocate device memory.
//
// bem_residual obtains the scratch it needs (x split into two complex FP32 blocks) from the problem's
// solver workspace, which it allocates on first use.  Some callers cannot let a library allocate at that
// point: an application whose device memory is fully handed to its own arena or caching allocator, a
// latency-bound loop in which a cudaMalloc would stall or synchronise the device, or a process running
// close to its memory limit where a new allocation could fail halfway through a computation.  For them,
// bem_residual_noalloc runs the same double-float residual kernels with their scratch in a fixed static
// device array of this file (2 x kNoAllocMaxEntries complex FP32 entries, 8 MiB), which every GPU that
// loads the library holds until the process exits.
//
// Set-up.  Under CUDA's lazy module loading the array (and the residual kernels, which live in another
// translation unit) only become resident on a device when first touched, and that costs device memory.  So
// the set-up, which looks up the array's device address with cudaGetSymbolAddress and loads the residual
// kernels, runs from calls that allocate anyway: the assembly of a mixed-precision problem (bem_assemble and
// the solve entry points) and the batched admission.  bem_residual_noalloc then only reads the cached
// address.  Should a device reach it without that set-up (not possible through the public interface, since
// it needs an assembled mixed-precision problem), the call performs the set-up itself.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kNoAllocMaxEntries = (size_t)1 << 19;   // n_rhs * 2N complex entries per call, at most

// x_hi and x_lo are packed back to back at the start of the array (n_rhs * 2N entries each).  Device code
// could name the array directly; host code only ever passes the device address obtained below.
static __device__ __align__(256) float2 g_noalloc_scratch[2 * kNoAllocMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device (and, at the same
// time, the residual kernels loaded on it).
bem_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bem::report_error(BEM_ECUDA, "cudaGetDevice failed in the no-allocation residual set-up");
  if (dev < 0 || dev >= kMaxDevices) return bem::report_error(BEM_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return bem::report_error(BEM_ECUDA, "cudaGetSymbolAddress of the static residual scratch failed");
    e = bem::residual_split_preload();
    if (e != cudaSuccess) return bem::report_error(BEM_ECUDA, "loading the residual kernels failed");
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return BEM_OK;
}

}  // namespace

namespace bem {
bem_status noalloc_setup() {
  void* ptr = nullptr;
  return scratch_address(&ptr);
}
}  // namespace bem

extern "C" BEM_API bem_status bem_residual_noalloc(bem_problem* p, int n_rhs, const bem_c64* x_dev,
                                                   const bem_c64* b_dev, bem_c64* r_dev, void* stream) {
  if (!p || !x_dev || !b_dev || !r_dev || n_rhs < 1) return bem::report_error(BEM_EINVAL, "invalid argument");
  if ((const void*)r_dev == (const void*)x_dev) return bem::report_error(BEM_EINVAL, "r_dev must not alias x_dev");
  const float2* hi = nullptr;
  const float2* lo = nullptr;
  int n2 = 0;
  if (!bem::problem_mixed_matrix(p, &hi, &lo, &n2))
    return bem::report_error(BEM_ESTATE,
                             "bem_residual_noalloc needs a mixed-precision problem assembled beforehand "
                             "(call bem_assemble first; this entry point never assembles or allocates)");
  if ((size_t)n_rhs * (size_t)n2 > kNoAllocMaxEntries)
    return bem::report_error(BEM_EINVAL,
                             "bem_residual_noalloc: n_rhs * 2N exceeds the static scratch limit of 524288 "
                             "complex entries; use bem_residual");
  void* scratch = nullptr;
  bem_status st = scratch_address(&scratch);
  if (st != BEM_OK) return st;
  // every entry of the scratch that the kernels read is written earlier in the same call, so nothing
  // left from a previous call needs clearing
  cudaError_t e = bem::launch_residual_split(hi, lo, (size_t)n2, n2, n_rhs, reinterpret_cast<const double2*>(x_dev),
                                             reinterpret_cast<const double2*>(b_dev), reinterpret_cast<double2*>(r_dev),
                                             scratch, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bem::report_error(BEM_ECUDA, cudaGetErrorString(e));
  return BEM_OK;
}
