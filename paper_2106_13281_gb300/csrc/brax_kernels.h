// Launchers of the device kernels (host side of the kernel translation units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "brax_device.cuh"

namespace brax {

// Launch-bounds variants (max threads per block, min blocks per SM):
// 0 = (384, 2), 1 = (576, 1), 2 = (1024, 1), 3 = (288, 3); the autotuner
// (brax_tune.cu) picks one per system.
cudaError_t launch_rollout(const Launch& L, int grid, int threads, size_t smem, int variant, bool general,
                           cudaStream_t st);
// Copy a parameter blob into the constant pool of each kernel translation unit.
cudaError_t upload_pool_forward(int off, const void* data, size_t bytes);
cudaError_t upload_pool_backward(int off, const void* data, size_t bytes);
int rollout_variant_max_threads(int variant);
// Resident blocks per SM of a one-environment kernel variant (0 if it cannot launch).
int rollout_blocks_per_sm(int variant, bool general, int threads, size_t smem);
// Two environments per thread (systems whose blob carries the paired section).
cudaError_t launch_rollout_pair(const Launch& L, int grid, int threads, size_t smem, int variant, cudaStream_t st);
int pair_variant_max_threads(int variant);
// Resident blocks per SM of a paired-kernel variant (0 if it cannot launch).
int pair_blocks_per_sm(int variant, int threads, size_t smem);
size_t pair_group_bytes(int B);
cudaError_t launch_rollout_backward(const Launch& L, int grid, int threads, size_t smem, int variant, bool general,
                                    cudaStream_t st);
size_t backward_smem_bytes(int B, int P, int groups);
// Resident blocks per SM of a reverse kernel variant (0 if it cannot launch).
int backward_blocks_per_sm(int variant, bool general, int threads, size_t smem);
int64_t backward_ws_floats_per_group(int B, int P, int K, int S);
cudaError_t launch_default_qp(const unsigned char* blob, int64_t N, const float* root_pos, const float* root_rot,
                              const float* angles, float* out, cudaStream_t st);

}  // namespace brax
