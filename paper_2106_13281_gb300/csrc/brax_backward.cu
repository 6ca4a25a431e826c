// Reverse-mode kernels (filled in by the adjoint implementation).
#include <cuda_runtime.h>

#include "../../include/brax.h"
#include "brax_kernels.h"

namespace brax {
__constant__ __align__(16) unsigned char c_pool[kPoolBytes];
cudaError_t upload_pool_backward(int off, const void* data, size_t bytes) {
  return cudaMemcpyToSymbol(c_pool, data, bytes, (size_t)off, cudaMemcpyHostToDevice);
}
cudaError_t launch_rollout_backward(const Launch&, int, int, size_t, int, bool, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace brax

extern "C" {
int brax_workspace_size(const brax_system*, int64_t, int32_t, int32_t, size_t* bytes) {
  if (bytes) *bytes = 0;
  return BRAX_ERR_INVALID_ARGUMENT;
}
int brax_rollout_backward(const brax_system*, int64_t, int32_t, int32_t, const float*, const float*, const float*,
                          const float*, const float*, float*, float*, void*, size_t, void*) {
  return BRAX_ERR_INVALID_ARGUMENT;
}
int brax_batch_workspace_size(const brax_batch*, int32_t, int32_t, size_t* bytes) {
  if (bytes) *bytes = 0;
  return BRAX_ERR_INVALID_ARGUMENT;
}
int brax_batch_rollout_backward(const brax_batch*, int32_t, int32_t, const float*, const float*, const float*,
                                const float*, const float*, float*, float*, void*, size_t, void*) {
  return BRAX_ERR_INVALID_ARGUMENT;
}
}
