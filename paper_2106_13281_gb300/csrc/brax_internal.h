// Host-side definition of a system handle (shared by the C ABI translation
// units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/brax.h"

namespace brax {
// Scheduler scratch of chunked rollouts: kRing regions of (32 + units) int32,
// taken in turn by successive launches so that rollouts on different streams
// do not share one; replaced buffers are freed with the owner.
struct SchedScratch {
  static constexpr int kRing = 4;
  std::mutex mu;
  int32_t* d = nullptr;
  int64_t units = 0;
  int next = 0;
  std::vector<int32_t*> retired;
};
}  // namespace brax

struct brax_system {
  int B = 0, A = 0, D = 0, P = 0, n_planes = 0;
  bool general = false;  // 3-DOF joints or body-body pairs present
  bool iso = false;      // every body has isotropic inertia
  int device = 0;
  int pool_off = -1;     // offset of the blob in the constant parameter pool
  std::vector<unsigned char> blob;
  unsigned char* d_blob = nullptr;
  int32_t* d_status = nullptr;
  int groups = 1;   // groups of 32 environments per thread block
  int variant = 0;  // launch-bounds variant of the rollout kernel
  // Two environments per thread (hinge-only systems with at most two plane
  // points per body): used for brax_rollout / brax_step when pair_mode is 1.
  bool paired = false;
  int pair_mode = 0;
  int pair_groups = 1;   // groups of 64 environments per thread block
  int pair_variant = 0;  // launch-bounds variant of the paired kernel
  int bwd_variant = -1;  // launch-bounds variant of the reverse kernel (-1: smallest that fits)
  // Chunked schedule of rollouts (Sched in brax_device.cuh).  Mode 1
  // (default): used when the blocks do not fill a whole number of resident
  // waves; 0: never; 2: always, with chunks of sched_chunk steps.
  int sched_mode = 1;
  int sched_chunk = 0;
  int sched_first = 0;              // first item handed out (the wait test starts past chunk 0)
  int64_t sched_wait_ns = 2000000000;
  mutable brax::SchedScratch sched;
  // brax_rollout_streamed's copy stream and events (created on first use).
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  std::mutex stream_mu;
  // The last brax_rollout launch: blocks launched, chunks (0 = static) and
  // steps per chunk (reported by brax_system_last_rollout).
  mutable int64_t last_grid = 0;
  mutable int32_t last_chunks = 0, last_chunk_steps = 0;
};

struct brax_batch {
  std::vector<const brax_system*> sys;
  std::vector<int64_t> n_envs;
  int warps = 0;  // warps per thread block
  int sched_mode = 1, sched_chunk = 0;  // as brax_system's
  mutable brax::SchedScratch sched;     // chunked schedule of the batch's forward rollouts
};

extern "C" int brax_system_set_launch(brax_system* s, int32_t groups, int32_t variant);
extern "C" int brax_system_set_pair_launch(brax_system* s, int32_t mode, int32_t groups, int32_t variant);
// Chunked schedule of a system's rollouts: mode 0 off, 1 automatic, 2 always
// with chunks of chunk_steps steps; first_item > 0 and a short wait_ns serve
// the test of the bounded wait (items past chunk 0 wait for flags nothing sets).
extern "C" int brax_batch_set_schedule(brax_batch* b, int32_t mode, int32_t chunk_steps);
// The chunked-schedule plan for `slots` resident blocks (host arithmetic
// only, for tests): n_chunks = 0 means the static schedule.
extern "C" int brax_internal_plan_schedule(int32_t mode, int32_t chunk_steps, int64_t units, int32_t T, int64_t slots,
                                           int32_t min_chunk, int32_t* n_chunks, int32_t* steps);
// The launch of the system's last brax_rollout: blocks launched, chunks of
// the chunked schedule (0 = static schedule) and steps per chunk.
extern "C" int brax_system_last_rollout(const brax_system* s, int64_t* grid, int32_t* n_chunks, int32_t* chunk_steps);
// The kernels' fast_atan2 elementwise over n device floats (out) and its
// packed two-environment form with element i paired with n-1-i (out_packed):
// the probe of the arctangent's accuracy test.
extern "C" int brax_internal_atan2(const float* y, const float* x, float* out, float* out_packed, int64_t n,
                                   void* stream);
extern "C" int brax_system_set_schedule(brax_system* s, int32_t mode, int32_t chunk_steps, int32_t first_item,
                                        int64_t wait_ns);


namespace brax {
// Reverse-mode scratch bytes a system needs for (n_envs, K) (defined with the C ABI).
size_t backward_workspace_bytes(const brax_system* s, int64_t n_envs, int32_t K);
// Set the message brax_last_error() returns on this thread.
void set_last_error(const std::string& msg);
// brax_rollout_backward whose chunked schedule (if the launch takes one) uses
// the caller's scheduler region `sched` of `sched_bytes` bytes of device
// memory instead of the system's own scratch; when that region is null or
// smaller than (32 + blocks of 32 environments) int32 the launch takes the
// static schedule.  Allocates nothing.
int rollout_backward_fixed_sched(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                                 const float* actions, const float* checkpoints, const float* g_state_T,
                                 const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                                 size_t workspace_bytes, int32_t* sched, size_t sched_bytes, void* stream);
}  // namespace brax
