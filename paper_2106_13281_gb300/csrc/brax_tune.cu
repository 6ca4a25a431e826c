// Autotuner (brax_autotune in brax.h): times the caller's own workload sample
// under every launch configuration the kernels offer and keeps the fastest.
//
// Forward candidates: the one-environment kernel with 1..4 groups of 32
// environments per block under each launch-bounds variant that admits the
// block, and, for systems that have it, the two-environments kernel with
// 1..4 groups of 64.  Reverse candidates: checkpoint intervals K from
// {1, 2, 4, 5, 8, 10, 16, 20, 25, 50, 100} (K <= T, checkpoints + workspace
// within the memory budget) times the reverse kernel's launch-bounds
// variants; the figure compared is (forward with checkpoints + reverse) per
// step, timed on the first min(n_envs, 16384) environments.  Each candidate
// runs once untimed, then three times timed with CUDA events; the smallest
// time counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "brax_internal.h"
#include "brax_kernels.h"

namespace {

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Runs fn (which returns a brax status) once untimed and three times timed
// on st.  Returns the smallest time in ms, or a negative value when fn failed.
template <class F>
float time_best(F fn, cudaStream_t st, Events& ev) {
  if (fn() != BRAX_OK) return -1.f;
  float best = -1.f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(ev.a, st);
    if (fn() != BRAX_OK) return -1.f;
    cudaEventRecord(ev.b, st);
    if (cudaEventSynchronize(ev.b) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    if (best < 0.f || ms < best) best = ms;
  }
  return best;
}

struct DeviceBuffer {
  void* p = nullptr;
  cudaError_t alloc(size_t bytes) {
    if (p) cudaFree(p);
    p = nullptr;
    return bytes ? cudaMalloc(&p, bytes) : cudaSuccess;
  }
  ~DeviceBuffer() {
    if (p) cudaFree(p);
  }
};

int tune_fail(int code, const std::string& msg) {
  brax::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int brax_autotune(brax_system* s, int64_t n_envs, int32_t T, const float* state0, const float* actions,
                             int32_t flags, size_t mem_budget, void* stream, brax_tune_result* out) {
  if (!s || !out || n_envs < 1 || T < 1 || !state0 || (s->A > 0 && !actions) ||
      (flags & ~(BRAX_TUNE_FORWARD | BRAX_TUNE_REVERSE)) != 0)
    return tune_fail(BRAX_ERR_INVALID_ARGUMENT, "brax_autotune: bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::memset(out, 0, sizeof(*out));
  out->fwd_groups = s->pair_mode ? s->pair_groups : s->groups;
  out->fwd_kernel = s->pair_mode;
  out->fwd_variant = s->pair_mode ? s->pair_variant : s->variant;
  out->bwd_variant = -1;
  Events ev;
  DeviceBuffer stT;
  const size_t state_bytes = (size_t)n_envs * s->B * 13 * sizeof(float);
  if (stT.alloc(state_bytes) != cudaSuccess) return tune_fail(BRAX_ERR_OUT_OF_MEMORY, "brax_autotune: cudaMalloc");
  float* state_T = static_cast<float*>(stT.p);

  if (flags & BRAX_TUNE_FORWARD) {
    const int Tf = std::min(T, 50);
    struct Cand {
      int kernel, groups, variant;
    };
    std::vector<Cand> cands;
    for (int v : {3, 0, 1, 2})
      for (int g = 1; g <= 4 && 32 * s->B * g <= brax::rollout_variant_max_threads(v); ++g) cands.push_back({0, g, v});
    if (s->paired)
      for (int v : {0, 3, 1, 4, 2})
        for (int g = 1; g <= 4 && 32 * s->B * g <= brax::pair_variant_max_threads(v); ++g) cands.push_back({1, g, v});
    // the fastest one-environment configuration is kept in any case: it runs
    // the rollouts that write checkpoints
    float best[2] = {-1.f, -1.f};
    Cand pick[2] = {{0, s->groups, s->variant}, {1, s->pair_groups, s->pair_variant}};
    for (const Cand& c : cands) {
      const int rc = c.kernel ? brax_system_set_pair_launch(s, 1, c.groups, c.variant)
                              : (brax_system_set_pair_launch(s, 0, 1, 0), brax_system_set_launch(s, c.groups, c.variant));
      if (rc != BRAX_OK) continue;
      const float ms = time_best(
          [&] { return brax_rollout(s, n_envs, Tf, 1, state0, actions, state_T, nullptr, nullptr, nullptr, stream); },
          st, ev);
      cudaGetLastError();  // a configuration the device rejects is skipped
      ++out->n_candidates;
      float& b = best[c.kernel];
      if (ms >= 0.f && (b < 0.f || ms < b)) {
        b = ms;
        pick[c.kernel] = c;
      }
    }
    if (best[0] < 0.f && best[1] < 0.f) return tune_fail(BRAX_ERR_CUDA, "brax_autotune: no forward configuration ran");
    brax_system_set_launch(s, pick[0].groups, pick[0].variant);
    const int k = (best[1] >= 0.f && (best[0] < 0.f || best[1] < best[0])) ? 1 : 0;
    if (k == 1) brax_system_set_pair_launch(s, 1, pick[1].groups, pick[1].variant);
    else brax_system_set_pair_launch(s, 0, 1, 0);
    out->fwd_kernel = k;
    out->fwd_groups = pick[k].groups;
    out->fwd_variant = pick[k].variant;
    out->fwd_ms = best[k];
  }

  if (flags & BRAX_TUNE_REVERSE) {
    if (mem_budget == 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return tune_fail(BRAX_ERR_CUDA, "brax_autotune: cudaMemGetInfo");
      mem_budget = fr / 2;
    }
    const int Ks[] = {1, 2, 4, 5, 8, 10, 16, 20, 25, 50, 100};
    // candidates are timed on the first n_r environments over Tb steps; a K
    // qualifies when its checkpoints and workspace for the full (n_envs, T)
    // rollout fit the budget
    const int64_t n_r = std::min<int64_t>(n_envs, 16384);
    const size_t r_state_bytes = (size_t)n_r * s->B * 13 * sizeof(float);
    struct Plan {
      int K, Tb;
      size_t ck_bytes, ws_bytes;  // of the timing sample
    };
    std::vector<Plan> plans;
    for (int K : Ks) {
      if (K > T) break;
      const int Tb = std::min(T, std::max(2 * K, 20));
      size_t ws_full = 0, ws_r = 0;
      if (brax_workspace_size(s, n_envs, T, K, &ws_full) != BRAX_OK ||
          brax_workspace_size(s, n_r, Tb, K, &ws_r) != BRAX_OK)
        return BRAX_ERR_INVALID_ARGUMENT;
      const size_t ck_full = (size_t)((T + K - 1) / K) * state_bytes;
      if (ck_full + ws_full <= mem_budget) plans.push_back({K, Tb, (size_t)((Tb + K - 1) / K) * r_state_bytes, ws_r});
    }
    if (plans.empty()) return tune_fail(BRAX_ERR_OUT_OF_MEMORY, "brax_autotune: no checkpoint interval fits the budget");
    size_t ck_max = 0, ws_max = 0;
    int Tb_max = 0;
    for (const Plan& p : plans) {
      ck_max = std::max(ck_max, p.ck_bytes);
      ws_max = std::max(ws_max, p.ws_bytes);
      Tb_max = std::max(Tb_max, p.Tb);
    }
    DeviceBuffer ck, ws, gst, gs0, gact, sst, sact;
    const size_t row = (size_t)n_r * std::max(s->A, 1) * sizeof(float);
    if (ck.alloc(ck_max) != cudaSuccess || ws.alloc(ws_max) != cudaSuccess || gst.alloc(r_state_bytes) != cudaSuccess ||
        gs0.alloc(r_state_bytes) != cudaSuccess || gact.alloc((size_t)Tb_max * row) != cudaSuccess)
      return tune_fail(BRAX_ERR_OUT_OF_MEMORY, "brax_autotune: cudaMalloc");
    cudaMemsetAsync(gst.p, 0, r_state_bytes, st);
    const float* r_state0 = state0;
    const float* r_actions = actions;
    if (n_r < n_envs) {  // copy out the sample's states and action rows
      if (sst.alloc(r_state_bytes) != cudaSuccess || sact.alloc((size_t)Tb_max * row) != cudaSuccess)
        return tune_fail(BRAX_ERR_OUT_OF_MEMORY, "brax_autotune: cudaMalloc");
      cudaMemcpyAsync(sst.p, state0, r_state_bytes, cudaMemcpyDeviceToDevice, st);
      if (s->A > 0)
        cudaMemcpy2DAsync(sact.p, (size_t)n_r * s->A * sizeof(float), actions, (size_t)n_envs * s->A * sizeof(float),
                          (size_t)n_r * s->A * sizeof(float), Tb_max, cudaMemcpyDeviceToDevice, st);
      r_state0 = static_cast<const float*>(sst.p);
      if (s->A > 0) r_actions = static_cast<const float*>(sact.p);
    }
    const int threads = 32 * s->B;
    float best = -1.f;
    int bestK = plans[0].K, bestV = -1;
    const int saved = s->bwd_variant;
    for (const Plan& p : plans)
      for (int v : {3, 0, 1, 4, 2}) {
        if (threads > brax::backward_variant_max_threads(v)) continue;
        s->bwd_variant = v;
        const float ms = time_best(
            [&] {
              int rc = brax_rollout(s, n_r, p.Tb, p.K, r_state0, r_actions, state_T, static_cast<float*>(ck.p),
                                    nullptr, nullptr, stream);
              if (rc == BRAX_OK)
                rc = brax_rollout_backward(s, n_r, p.Tb, p.K, r_state0, r_actions, static_cast<float*>(ck.p),
                                           static_cast<float*>(gst.p), nullptr, static_cast<float*>(gact.p),
                                           static_cast<float*>(gs0.p), ws.p, ws_max, stream);
              return rc;
            },
            st, ev);
        cudaGetLastError();
        ++out->n_candidates;
        if (ms < 0.f) continue;
        const float per_step = ms / p.Tb;
        if (best < 0.f || per_step < best) {
          best = per_step;
          bestK = p.K;
          bestV = v;
        }
      }
    if (best < 0.f) {
      s->bwd_variant = saved;
      return tune_fail(BRAX_ERR_CUDA, "brax_autotune: no reverse configuration ran");
    }
    s->bwd_variant = bestV;
    out->K = bestK;
    out->bwd_variant = bestV;
    out->fwd_bwd_ms_per_step = best;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return tune_fail(BRAX_ERR_CUDA, std::string("brax_autotune: ") + cudaGetErrorString(e));
  return BRAX_OK;
}

extern "C" int brax_batch_autotune(brax_batch* b, int32_t T, int32_t K, const float* state0, const float* actions,
                                   int32_t flags, void* stream, int32_t* warps_out, float* ms_out) {
  if (!b || T < 1 || K < 1 || !state0 || (flags & ~(BRAX_TUNE_FORWARD | BRAX_TUNE_REVERSE)) != 0 || flags == 0)
    return tune_fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_autotune: bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int maxB = 0;
  for (const brax_system* s : b->sys) maxB = std::max(maxB, s->B);
  const bool rev = (flags & BRAX_TUNE_REVERSE) != 0;
  const int Ts = std::min(T, rev ? 20 : 10);
  const int Ke = std::min(K, Ts);
  int64_t st_n = 0, ck_n = 0, act_n = 0;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    st_n += b->n_envs[i] * b->sys[i]->B * 13;
    ck_n += (int64_t)((Ts + Ke - 1) / Ke) * b->n_envs[i] * b->sys[i]->B * 13;
    act_n += (int64_t)Ts * b->n_envs[i] * std::max(b->sys[i]->A, 1);
  }
  const int saved = b->warps;
  size_t ws_max = 0;
  std::vector<int> cands;
  for (int w = maxB; w <= 32; ++w) {
    b->warps = w;
    size_t ws = 0;
    if (rev && brax_batch_workspace_size(b, Ts, Ke, &ws) != BRAX_OK) continue;
    ws_max = std::max(ws_max, ws);
    cands.push_back(w);
  }
  DeviceBuffer stT, ck, ws, gst, gs0, gact;
  if (stT.alloc(st_n * sizeof(float)) != cudaSuccess ||
      (rev && (ck.alloc(ck_n * sizeof(float)) != cudaSuccess || ws.alloc(ws_max) != cudaSuccess ||
               gst.alloc(st_n * sizeof(float)) != cudaSuccess || gs0.alloc(st_n * sizeof(float)) != cudaSuccess ||
               gact.alloc(act_n * sizeof(float)) != cudaSuccess))) {
    b->warps = saved;
    return tune_fail(BRAX_ERR_OUT_OF_MEMORY, "brax_batch_autotune: cudaMalloc");
  }
  if (rev) cudaMemsetAsync(gst.p, 0, st_n * sizeof(float), st);
  Events ev;
  float best = -1.f;
  int pick = saved;
  for (int w : cands) {
    b->warps = w;
    const float ms = time_best(
        [&] {
          int rc = brax_batch_rollout(b, Ts, Ke, state0, actions, static_cast<float*>(stT.p),
                                      rev ? static_cast<float*>(ck.p) : nullptr, nullptr, stream);
          if (rc == BRAX_OK && rev)
            rc = brax_batch_rollout_backward(b, Ts, Ke, state0, actions, static_cast<float*>(ck.p),
                                             static_cast<float*>(gst.p), nullptr, static_cast<float*>(gact.p),
                                             static_cast<float*>(gs0.p), ws.p, ws_max, stream);
          return rc;
        },
        st, ev);
    cudaGetLastError();
    if (ms >= 0.f && (best < 0.f || ms < best)) {
      best = ms;
      pick = w;
    }
  }
  b->warps = pick;
  if (best < 0.f) return tune_fail(BRAX_ERR_CUDA, "brax_batch_autotune: no configuration ran");
  if (warps_out) *warps_out = pick;
  if (ms_out) *ms_out = best;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return tune_fail(BRAX_ERR_CUDA, std::string("brax_batch_autotune: ") + cudaGetErrorString(e));
  return BRAX_OK;
}
