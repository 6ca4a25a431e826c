// Host-side definition of a system handle (shared by the C ABI translation
// units).
#pragma once
#include <string>
#include <vector>

#include "../../include/brax.h"

struct brax_system {
  int B = 0, A = 0, D = 0, P = 0, n_planes = 0;
  bool general = false;  // 3-DOF joints or body-body pairs present
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
};

struct brax_batch {
  std::vector<const brax_system*> sys;
  std::vector<int64_t> n_envs;
  int warps = 0;  // warps per thread block
};

extern "C" int brax_system_set_launch(brax_system* s, int32_t groups, int32_t variant);
extern "C" int brax_system_set_pair_launch(brax_system* s, int32_t mode, int32_t groups, int32_t variant);


namespace brax {
// Reverse-mode scratch bytes a system needs for (n_envs, K) (defined with the C ABI).
size_t backward_workspace_bytes(const brax_system* s, int64_t n_envs, int32_t K);
// Set the message brax_last_error() returns on this thread.
void set_last_error(const std::string& msg);
}  // namespace brax
