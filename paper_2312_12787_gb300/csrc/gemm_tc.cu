// Multi-right-hand-side complex GEMM on the tcgen05 tensor cores (step a11).  Placeholder until the
// tensor-core kernel lands: reports the shape as unsupported so the solver uses the SIMT FP32 GEMM.
#include "internal.cuh"

namespace bem {

bool matvec_tc_supported(int, int) { return false; }
size_t matvec_tc_workspace_bytes(int, int) { return 0; }
cudaError_t launch_matvec_tc(const float2*, size_t, int, int, const float2*, float2*, void*, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace bem
