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
// flat: every plane of the system has the world z axis as its normal (SysP::flat).
cudaError_t launch_rollout_pair(const Launch& L, int grid, int threads, size_t smem, int variant, bool flat,
                                cudaStream_t st);
int pair_variant_max_threads(int variant);
// Resident blocks per SM of a paired-kernel variant (0 if it cannot launch).
int pair_blocks_per_sm(int variant, int threads, size_t smem);
size_t pair_group_bytes(int B, int A);
// iso: a hinge-only system whose bodies all have isotropic inertia (the
// two-barrier reverse substep); ignored when general.
cudaError_t launch_rollout_backward(const Launch& L, int grid, int threads, size_t smem, int variant, bool general,
                                    bool iso, cudaStream_t st);
size_t backward_smem_bytes(int B, int P, int groups);
// Largest block of a reverse-kernel variant (0..3 as the forward; 4: 112 registers, up to 576 threads).
int backward_variant_max_threads(int variant);
// Resident blocks per SM of a reverse kernel variant (0 if it cannot launch).
int backward_blocks_per_sm(int variant, bool general, bool iso, int threads, size_t smem);
int64_t backward_ws_floats_per_group(int B, int P, int K, int S);
// fast_atan2 (and its packed form, out_packed) elementwise, for its accuracy test.
cudaError_t launch_atan2_probe(const float* y, const float* x, float* out, float* out_packed, int64_t n,
                               cudaStream_t st);
cudaError_t launch_default_qp(const unsigned char* blob, int64_t N, const float* root_pos, const float* root_rot,
                              const float* angles, float* out, cudaStream_t st);

}  // namespace brax
