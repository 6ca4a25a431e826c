// Forward kernels: persistent rollout (also used for a single step) and
// default_qp.
//
// Mapping: a thread block holds G groups of 32 environments of one system;
// in a group, warp b is body b and lane i is environment i.  A thread keeps
// its body's 13-float state in registers for the whole rollout; only the
// actions stream in from HBM (three loads per step at most, reused over the
// step's substeps).  Within a substep the warps of a group exchange the
// parent state, joint reactions and pair impulses through shared memory at
// two named barriers (see brax_physics.cuh).  Every warp is uniform in its
// body role, so the only divergence is data-dependent (limits, contacts).
#include "brax_kernels.h"
#include "brax_pair.cuh"
#include "brax_physics.cuh"

namespace brax {

__constant__ __align__(16) unsigned char c_pool[kPoolBytes];

// One substep of one (body, environment) thread; returns the number of
// contacts this thread counted (own plane contacts + owned pairs).
template <bool kGeneral>
__device__ __forceinline__ int substep_forward(const SysP& S, const BodyP* bodies, const PairP* pairs,
                                               const PlaneP* planes, const BodyP& bp, const HingeRegs& hr,
                                               const PointRegs* pr, int b, int B, int lane, GroupMem& gm, int bar,
                                               int nthr, bool tree, Body& s, const float* act) {
  kinematic(bp, S.h, s);
  const Frame f = make_frame(bp, s);
  if (!kGeneral && tree) {
    // Tree synchronisation: a child waits only for its parent's published
    // state, a parent only for its own children's reactions.
    const bool parent_of = bp.tree_slot >= 0;
    const int my_n = 32 * (1 + bp.n_children);
    if (parent_of) {
      publish<false>(gm, b, lane, s, f, bp);
      bar_arrive(2 + 2 * bp.tree_slot, my_n);
    }
    // the own contacts need only the own state: do them while the parent publishes
    Acc acc{mk3(0.f, 0.f, 0.f), mk3(0.f, 0.f, 0.f), 0};
    const int np = bp.n_points;
    plane_points_regs(S, bp, pr, planes, np < 2 ? np : 2, s, f, acc);
    for (int i = 2; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
    const int counted = acc.n;
    Wrench wr{mk3(0.f, 0.f, 0.f), mk3(0.f, 0.f, 0.f)};
    if (bp.flags & kHasParent) {
      const BodyP& pb = bodies[bp.parent];
      const int pid = 2 + 2 * pb.tree_slot, pn = 32 * (1 + pb.n_children);
      group_sync(pid, pn);
      const Pub pp = read_pub(gm, bp.parent, lane);
      wr = joint_forward<false>(hr, pp, s, f, act, gm.react4(b, 0) + lane);
      bar_arrive(pid + 1, pn);
    }
    if (parent_of) group_sync(3 + 2 * bp.tree_slot, my_n);
    integrate<false>(S, bp, gm, lane, s, f, wr, acc);
    return counted;
  }
  if (bp.flags & kPublish) {
    if (kGeneral && (bp.flags & kInPair)) publish<true>(gm, b, lane, s, f, bp);
    else publish<false>(gm, b, lane, s, f, bp);
  }
  group_sync(bar, nthr);
  Wrench wr{mk3(0.f, 0.f, 0.f), mk3(0.f, 0.f, 0.f)};
  if (bp.flags & kHasParent) {
    const Pub pp = read_pub(gm, bp.parent, lane);
    if (kGeneral) wr = joint_forward<true>(bp, pp, s, f, act, gm.react4(b, 0) + lane);
    else wr = joint_forward<false>(hr, pp, s, f, act, gm.react4(b, 0) + lane);
  }
  Acc acc{mk3(0.f, 0.f, 0.f), mk3(0.f, 0.f, 0.f), 0};
  const int np = bp.n_points;
  if (kGeneral) {
    for (int i = 0; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
  } else {
    plane_points_regs(S, bp, pr, planes, np < 2 ? np : 2, s, f, acc);
    for (int i = 2; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
  }
  int counted = acc.n;
  if (kGeneral)
    for (int k = b; k < S.P; k += B) counted += pair_forward(S, bodies, pairs[k], gm, k, lane);
  group_sync(bar, nthr);
  integrate<kGeneral>(S, bp, gm, lane, s, f, wr, acc);
  return counted;
}

// Persistent rollout.  Parameters are read from the constant pool with a
// warp-uniform body index (broadcast from lane 0 so the compiler can treat it
// as uniform); the state stays in registers for all T x substeps.  A block
// runs one unit (a block-sized set of environment groups of one segment):
// unit blockIdx.x for the whole rollout, or, under a chunked schedule
// (Sched), one chunk of the unit of the item it takes.
template <int MAXT, int MINB, bool kGeneral, bool kEnv>
__global__ void __launch_bounds__(MAXT, MINB) rollout_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const bool chunked = L.sc.n_chunks > 0;
  int unit = blockIdx.x, c = 0, t0 = 0, t1 = L.T;
  if (chunked) {
    const int n_units = L.sc.n_units, n_items = L.sc.n_chunks * n_units;
    if (threadIdx.x == 0) {
      int ticket;
      const int it = take_item(L.sc, n_items, &ticket);
      if (it == -2) {  // report the timeout to the system of the unit that was waited for
        const int u = ticket % n_units;
        int si = 0;
        while (si + 1 < L.n_segs && u >= L.seg[si].cta_end) ++si;
        atomicOr(L.seg[si].status, kStatusTimeout);
      }
      s_item = it;
    }
    group_sync(0, blockDim.x);
    const int it = s_item;
    if (it < 0 || it >= n_items) return;
    unit = it % n_units;
    c = it / n_units;
    t0 = c * L.sc.chunk_steps;
    t1 = min(L.T, t0 + L.sc.chunk_steps);
  }
  int si = 0;
  while (si + 1 < L.n_segs && unit >= L.seg[si].cta_end) ++si;
  const Seg& sg = L.seg[si];
  const unsigned char* blob = c_pool + sg.pool_off;
  const SysP& S = *reinterpret_cast<const SysP*>(blob);
  const BodyP* bodies = reinterpret_cast<const BodyP*>(blob + blob_bodies_off());
  const PairP* pairs = reinterpret_cast<const PairP*>(blob + blob_pairs_off(sg.B));
  const PlaneP* planes = reinterpret_cast<const PlaneP*>(blob + blob_planes_off(sg.B, sg.P));
  const int B = sg.B;
  const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
  const int lane = threadIdx.x & 31;
  const int g = warp / B, b = warp - g * B;
  if (g >= sg.groups) return;  // spare warps take no part in the group barriers
  const int64_t N = sg.n_envs;
  const int64_t env = ((int64_t)(unit - sg.cta_begin) * sg.groups + g) * 32 + lane;
  const bool valid = env < N;
  GroupMem gm = group_mem(reinterpret_cast<float*>(smem) + g * group_floats(B, sg.P), B, sg.P);
  const int bar = 1 + g, nthr = 32 * B;
  const BodyP& bp = bodies[b];
  // tree barriers need the block to be exactly one group (their ids are per block)
  const bool tree = !kGeneral && sg.groups == 1 && (int)blockDim.x == 32 * B && tree_barriers_fit(S.n_parents);
  if (b == 0) gm.cnt[lane] = 0;
  if (sg.ccount) group_sync(bar, nthr);

  Body s;
  if (valid) {  // chunk 0 starts from state0, a later chunk from what the previous one left in state_T
    load_body_l2((c == 0 ? sg.state0 : sg.state_T) + (env * B + b) * 13, s);
  } else {  // padding lanes step a resting body and write nothing
    s.x = ld3(bp.rest_pos);
    s.qw = bp.rest_rot[0];
    s.qx = bp.rest_rot[1];
    s.qy = bp.rest_rot[2];
    s.qz = bp.rest_rot[3];
    s.v = mk3(0.f, 0.f, 0.f);
    s.w = mk3(0.f, 0.f, 0.f);
  }
  const int K = L.K, A = sg.A;
  const int nsub = S.substeps;
  int ccount = 0;
  bool bad = false;
  float act[3] = {0.f, 0.f, 0.f};
  HingeRegs hr;
  PointRegs pr[2];
  if (!kGeneral) {
    if (bp.flags & kHasParent) hr = hinge_regs(bp);
    if (bp.n_points > 0) pr[0] = point_regs(bp.pt[0]);
    if (bp.n_points > 1) pr[1] = point_regs(bp.pt[1]);
  }
  for (int t = t0; t < t1; ++t) {
    if (sg.ckpt && valid && (t % K) == 0) store_body(sg.ckpt + (((int64_t)(t / K) * N + env) * B + b) * 13, s);
    if (valid && (bp.flags & kHasParent)) {
      const float* ap = sg.actions + ((int64_t)t * N + env) * A;
#pragma unroll
      for (int a = 0; a < 3; ++a) act[a] = bp.act[a] >= 0 ? __ldg(ap + bp.act[a]) : 0.f;
    }
    if (kEnv && b == 0) gm.react4(0, 0)[lane].x = s.x.x;  // the root's x before the step (its react slot is free)
    for (int k = 0; k < nsub; ++k)
      ccount += substep_forward<kGeneral>(S, bodies, pairs, planes, bp, hr, pr, b, B, lane, gm, bar, nthr, tree, s,
                                          act);
    if (sg.torso && b == 0 && valid) {
      float* tp = sg.torso + ((int64_t)t * N + env) * 3;
      tp[0] = s.x.x;
      tp[1] = s.x.y;
      tp[2] = s.x.z;
    }
    if (kEnv) {
      // environment layer (Sec. 4.2 gym-like env): observation, reward and
      // done of the step, then the auto reset; two group barriers.  A parent
      // leaves its final angular velocity where its children read its
      // published state (its rotation there is already the final one: only
      // velocities change after the kinematic integrator); a joint's child
      // leaves its actions' squared clamped values beside its reaction.
      if (bp.flags & kPublish) {
        gm.pub4(b, 3)[lane].w = s.w.x;
        st2(gm.pub4(b, 4) + lane, s.w.y, s.w.z);
      }
      if (bp.flags & kHasParent) {
        float c2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (bp.act[a] >= 0) {
            const float u = clamp1(act[a]);
            c2 = fmaf(u, u, c2);
          }
        gm.react4(b, 1)[lane].z = c2;
      }
      group_sync(bar, nthr);
      float* ob = sg.obs + ((int64_t)t * N + env) * sg.obs_dim;
      if (valid && (bp.flags & kHasParent)) {
        const Pub pp = read_pub(gm, bp.parent, lane);
        float ang[3], rate[3];
        joint_obs<kGeneral>(bp, pp.R, pp.w, qmat(s.qw, s.qx, s.qy, s.qz), s.w, ang, rate);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (a < bp.dof) {
            ob[11 + bp.dof_offset + a] = ang[a];
            ob[11 + S.D + bp.dof_offset + a] = rate[a];
          }
      }
      if (b == 0) {
        float ctrl = 0.f;
        for (int c = 1; c < B; ++c)
          if (bodies[c].flags & kHasParent) ctrl += gm.react4(c, 1)[lane].z;
        bool done = false;
        if (valid)
          done = root_env(sg, s, gm.react4(0, 0)[lane].x, ctrl, ob, sg.reward + (int64_t)t * N + env,
                          sg.done + (int64_t)t * N + env);
        gm.react4(0, 0)[lane].y = done ? 1.f : 0.f;
      }
      group_sync(bar, nthr);
      if (sg.auto_reset && valid && gm.react4(0, 0)[lane].y != 0.f)
        load_body(sg.reset_state + (env * B + b) * 13, s);
    }
    bad |= !body_finite(s);
  }
  if (valid) store_body(sg.state_T + (env * B + b) * 13, s);
  if (bad && valid) atomicOr(sg.status, kStatusNonfinite);
  if (sg.ccount) {
    atomicAdd(&gm.cnt[lane], ccount);
    group_sync(bar, nthr);
    if (b == 0 && valid) __stcg(sg.ccount + env, (c ? __ldcg(sg.ccount + env) : 0) + gm.cnt[lane]);
  }
  if (chunked) {  // the item is done: its stores are made visible, then the unit's flag says so
    __threadfence();
    group_sync(0, 32 * B * sg.groups);
    if (threadIdx.x == 0) store_release(L.sc.sched + 32 + unit, c + 1);
  }
}

// ------------------------------------------------------------------ two environments per thread
namespace p2 {
// Load environment A's and B's body into the pair state (a padding half
// steps the body's rest pose).
__device__ __forceinline__ void load_pair(const float* pa, const float* pb, const BodyP& bp, Body& s) {
  auto ld = [&](int i) {
    const float r = i < 3 ? bp.rest_pos[i] : (i < 7 ? bp.rest_rot[i - 3] : 0.f);
    return make_float2(pa ? __ldcg(pa + i) : r, pb ? __ldcg(pb + i) : r);
  };
  s.x = V{ld(0), ld(1), ld(2)};
  s.qw = ld(3);
  s.qx = ld(4);
  s.qy = ld(5);
  s.qz = ld(6);
  s.v = V{ld(7), ld(8), ld(9)};
  s.w = V{ld(10), ld(11), ld(12)};
}
// Store one half (0: A, 1: B) of the pair state.
__device__ __forceinline__ void store_half(float* p, const Body& s, int half) {
  auto h = [half](f2 v) { return half ? v.y : v.x; };
  p[0] = h(s.x.x);
  p[1] = h(s.x.y);
  p[2] = h(s.x.z);
  p[3] = h(s.qw);
  p[4] = h(s.qx);
  p[5] = h(s.qy);
  p[6] = h(s.qz);
  p[7] = h(s.v.x);
  p[8] = h(s.v.y);
  p[9] = h(s.v.z);
  p[10] = h(s.w.x);
  p[11] = h(s.w.y);
  p[12] = h(s.w.z);
}
// One environment (half 0: A, 1: B) of the pair state as a scalar body.
__device__ __forceinline__ brax::Body half_body(const Body& s, int h) {
  auto c = [h](f2 v) { return h ? v.y : v.x; };
  brax::Body o;
  o.x = mk3(c(s.x.x), c(s.x.y), c(s.x.z));
  o.qw = c(s.qw);
  o.qx = c(s.qx);
  o.qy = c(s.qy);
  o.qz = c(s.qz);
  o.v = mk3(c(s.v.x), c(s.v.y), c(s.v.z));
  o.w = mk3(c(s.w.x), c(s.w.y), c(s.w.z));
  return o;
}
// Replace one half of the pair state by the 13 floats at p.
__device__ __forceinline__ void load_half(const float* p, Body& s, int h) {
  auto set = [h](f2& v, float x) {
    if (h) v.y = x;
    else v.x = x;
  };
  set(s.x.x, p[0]);
  set(s.x.y, p[1]);
  set(s.x.z, p[2]);
  set(s.qw, p[3]);
  set(s.qx, p[4]);
  set(s.qy, p[5]);
  set(s.qz, p[6]);
  set(s.v.x, p[7]);
  set(s.v.y, p[8]);
  set(s.v.z, p[9]);
  set(s.w.x, p[10]);
  set(s.w.y, p[11]);
  set(s.w.z, p[12]);
}
__device__ __forceinline__ bool finite_pair(const Body& s) {
  const f2 t = add(add(add(s.x.x, s.x.y), add(s.x.z, s.qw)),
                   add(add(add(s.qx, s.qy), add(s.qz, s.v.x)), add(add(s.v.y, s.v.z), add(s.w.x, add(s.w.y, s.w.z)))));
  return fabsf(t.x) < INFINITY && fabsf(t.y) < INFINITY;
}
}  // namespace p2

// Persistent rollout of a hinge-only system, two environments per thread
// (brax_pair.cuh).  A block holds G groups of 64 environments (a unit): unit
// blockIdx.x for the whole rollout, or, under a chunked schedule (Sched), one
// chunk of the unit of the item it takes.
template <int MAXT, int MINB, bool kFlat, bool kEnv>
__global__ void __launch_bounds__(MAXT, MINB) rollout_pair_kernel(const __grid_constant__ Launch L) {
  using namespace p2;
  const Seg& sg = L.seg[0];
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const bool chunked = L.sc.n_chunks > 0;
  int unit = blockIdx.x, c = 0, t0 = 0, t1 = L.T;
  if (chunked) {
    const int n_units = L.sc.n_units, n_items = L.sc.n_chunks * n_units;
    if (threadIdx.x == 0) {
      int ticket;
      const int it = take_item(L.sc, n_items, &ticket);
      if (it == -2) atomicOr(sg.status, kStatusTimeout);
      s_item = it;
    }
    group_sync(0, blockDim.x);
    const int it = s_item;
    if (it < 0 || it >= n_items) return;
    unit = it % n_units;
    c = it / n_units;
    t0 = c * L.sc.chunk_steps;
    t1 = min(L.T, t0 + L.sc.chunk_steps);
  }
  const unsigned char* blob = c_pool + sg.pool_off;
  const SysP& S = *reinterpret_cast<const SysP*>(blob);
  const BodyP* bodies = reinterpret_cast<const BodyP*>(blob + blob_bodies_off());
  const SysP2& S2 = *reinterpret_cast<const SysP2*>(blob + S.pair_off);
  const BodyP2* bodies2 = reinterpret_cast<const BodyP2*>(blob + S.pair_off + sizeof(SysP2));
  const int B = sg.B;
  const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
  const int lane = threadIdx.x & 31;
  const int g = warp / B, b = warp - g * B;
  if (g >= sg.groups) return;  // spare warps take no part in the group barriers
  const int64_t N = sg.n_envs;
  const int64_t ea = ((int64_t)unit * sg.groups + g) * 64 + lane, eb = ea + 32;
  const bool va = ea < N, vb = eb < N;
  GroupMem2 gm = group_mem2(reinterpret_cast<float*>(smem) + g * group_floats2(B, sg.A), B);
  const int bar = 1 + g, nthr = 32 * B;
  const BodyP& bp = bodies[b];
  const BodyP2& q = bodies2[b];
  // The group's actions come as one tile per step, [64 environments][A]
  // (contiguous in the action array), brought into shared memory by a bulk
  // asynchronous copy issued one step ahead by one thread and double-buffered;
  // each body warp then reads its actuator's column.  A group whose tile is
  // not 16-byte sized and aligned (a ragged last group, A * N not a multiple
  // of 4) loads its actions directly, and a launch of no steps copies none.
  const int64_t e0 = ((int64_t)unit * sg.groups + g) * 64;
  const int64_t nv = N - e0 < 64 ? N - e0 : 64;
  const uint32_t tile_bytes = nv > 0 ? (uint32_t)(nv * sg.A * 4) : 0u;
  const bool use_tile = t1 > t0 && sg.A > 0 && nv > 0 && (tile_bytes & 15u) == 0 && ((N * sg.A) & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(sg.actions) & 15u) == 0;
  const bool issuer = use_tile && b == 0 && lane == 0;
  if (issuer) {
    mbar_init(gm.mbar, 1);
    mbar_init(gm.mbar + 1, 1);
    fence_mbar_init();
  }
  if (b == 0) {
    gm.cnt[lane] = 0;
    gm.cnt[32 + lane] = 0;
  }
  if (sg.ccount || use_tile) group_sync(bar, nthr);
  auto issue_tile = [&](int t) {  // the issuing thread: step t's tile into buffer (t - t0) & 1
    const int i = (t - t0) & 1;
    fence_proxy_async();  // this buffer's earlier reads (before the last barrier) precede the async write
    bulk_copy_g2s(gm.tile + i * 64 * sg.A, sg.actions + ((int64_t)t * N + e0) * sg.A, tile_bytes, gm.mbar + i);
  };
  if (issuer) {
    issue_tile(t0);
    if (t0 + 1 < t1) issue_tile(t0 + 1);
  }
  // checkpoint staging buffer of this group, [64 environments][B][13] floats,
  // after the groups' shared memory (sg.ck_stage)
  float* stage = sg.ck_stage ? reinterpret_cast<float*>(smem) + sg.groups * group_floats2(B, sg.A) + g * 64 * B * 13
                             : nullptr;
  bool staged = false;  // this thread issued a bulk store of a staged checkpoint
  p2::Body s;
  {  // chunk 0 starts from state0, a later chunk from what the previous one left in state_T
    const float* src = c == 0 ? sg.state0 : sg.state_T;
    load_pair(va ? src + (ea * B + b) * 13 : nullptr, vb ? src + (eb * B + b) * 13 : nullptr, bp, s);
  }
  const int K = L.K, A = sg.A;
  const int nsub = S.substeps;
  const bool has_parent = (bp.flags & kHasParent) != 0, publishes = (bp.flags & kPublish) != 0;
  const int act_idx = bp.act[0];
  const int np = bp.n_points;
  const bool average = S.average != 0;
  int cca = 0, ccb = 0;
  bool bad = false;
  for (int t = t0; t < t1; ++t) {
    if (sg.ckpt && (t % K) == 0) {
      float* ck = sg.ckpt + ((int64_t)(t / K) * N) * B * 13;
      // The group's environments are one contiguous block of the checkpoint
      // ([N][B][13]): every thread leaves its two states in the group's
      // staging buffer and one thread stores the block with one bulk
      // asynchronous copy, in place of 26 scattered 4-byte stores a thread.
      // A block not 16-byte sized and aligned is stored directly.
      float* dst = ck + e0 * B * 13;
      const uint32_t ck_bytes = (uint32_t)(nv * B * 13) * 4u;
      if (stage && nv > 0 && (ck_bytes & 15u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        store_half(stage + (lane * B + b) * 13, s, 0);
        store_half(stage + ((32 + lane) * B + b) * 13, s, 1);
        fence_proxy_async();  // the staged states, written by this thread, precede the bulk read
        group_sync(bar, nthr);
        if (b == 0 && lane == 0) {
          // the buffer is written again only after the next group barrier,
          // which this thread reaches once the copy has read it
          bulk_copy_s2g(dst, stage, ck_bytes);
          bulk_wait_read();
          staged = true;
        }
      } else {
        if (va) store_half(ck + (ea * B + b) * 13, s, 0);
        if (vb) store_half(ck + (eb * B + b) * 13, s, 1);
      }
    }
    f2 act = zero2();
    if (use_tile) {
      const int i = t - t0;
      if (issuer && i > 0 && t + 1 < t1) issue_tile(t + 1);  // every warp has left step t - 1's buffer
      if (has_parent && act_idx >= 0) {
        if (!mbar_wait(gm.mbar + (i & 1), (uint32_t)((i >> 1) & 1), L.sc.wait_ns > 0 ? L.sc.wait_ns : 2000000000LL))
          atomicOr(sg.status, kStatusTimeout);
        const float* tl = gm.tile + (i & 1) * 64 * A + act_idx;
        act = make_float2(va ? tl[lane * A] : 0.f, vb ? tl[(32 + lane) * A] : 0.f);
      }
    } else if (has_parent && act_idx >= 0) {
      const float* ap = sg.actions + (int64_t)t * N * A + act_idx;
      act = make_float2(va ? __ldg(ap + ea * A) : 0.f, vb ? __ldg(ap + eb * A) : 0.f);
    }
    if (kEnv && b == 0) gm.reactf(0, 10)[lane] = s.x.x;  // the root's x before the step (its react slot is free)
    for (int k = 0; k < nsub; ++k) {
      kinematic(S2, bp.flags, s);
      p2::Frame f;
      f.R = qmat(s.qw, s.qx, s.qy, s.qz, S2.one);
      // every body leaves its rotation in its pub slot (a publishing body for
      // its children, the others for themselves): after the joint the
      // rotation is read back instead of being kept live in registers
      if (publishes) publish(gm, b, lane, s, f);
      else {
        f2* pr = gm.pubf(b, 3) + lane;
#pragma unroll
        for (int i = 0; i < 9; ++i) pr[i * 32] = f.R.m[i];
      }
      group_sync(bar, nthr);
      if (has_parent) {
        const p2::Pub pp = read_pub(gm, bp.parent, lane);
        joint(q, act_idx >= 0, pp, s, f, act, gm.reactf(b, 0) + lane);
      }
      {
        const f2* pr = gm.pubf(b, 3) + lane;
#pragma unroll
        for (int i = 0; i < 9; ++i) f.R.m[i] = pr[i * 32];
      }
      p2::Acc acc{vzero(), vzero(), 0, 0};
      f.Ii = inv_inertia_world(f.R, q.inv_I);  // not needed by the joint: computed after it
      if (kFlat) plane_points_z(S2, q, bp.flags, np, s, f, acc);
      else plane_points(S2, q, bp.flags, np, s, f, acc);
      cca += acc.na;
      ccb += acc.nb;
      group_sync(bar, nthr);
      integrate(S2, average, bp, q, gm, b, lane, s, f, acc);
    }
    if (sg.torso && b == 0) {
      float* tp = sg.torso + (int64_t)t * N * 3;
      if (va) {
        tp[ea * 3 + 0] = s.x.x.x;
        tp[ea * 3 + 1] = s.x.y.x;
        tp[ea * 3 + 2] = s.x.z.x;
      }
      if (vb) {
        tp[eb * 3 + 0] = s.x.x.y;
        tp[eb * 3 + 1] = s.x.y.y;
        tp[eb * 3 + 2] = s.x.z.y;
      }
    }
    if (kEnv) {
      // environment layer (Sec. 4.2 gym-like env), as in rollout_kernel: a
      // parent leaves its final angular velocity in its pub slot, a joint's
      // child its squared clamped action in a free react field; then each
      // environment of the pair is observed, rewarded and reset in turn.
      if (publishes) {
        f2* p = gm.pubf(b, 15) + lane;
        p[0] = s.w.x;
        p[32] = s.w.y;
        p[64] = s.w.z;
      }
      if (has_parent) {
        f2 c2 = zero2();
        if (act_idx >= 0) {
          const float ua = clamp1(act.x), ub = clamp1(act.y);
          c2 = make_float2(ua * ua, ub * ub);
        }
        gm.reactf(b, 9)[lane] = c2;
      }
      group_sync(bar, nthr);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const bool vh = h ? vb : va;
        const int64_t eh = h ? eb : ea;
        auto c = [h](f2 v) { return h ? v.y : v.x; };
        const brax::Body sh = half_body(s, h);
        float* ob = sg.obs + ((int64_t)t * N + eh) * sg.obs_dim;
        if (vh && has_parent) {
          const f2* pp = gm.pubf(bp.parent, 0) + lane;
          M3 Rp;
#pragma unroll
          for (int i = 0; i < 9; ++i) Rp.m[i] = c(pp[(3 + i) * 32]);
          const V3 wp = mk3(c(pp[15 * 32]), c(pp[16 * 32]), c(pp[17 * 32]));
          float ang[3], rate[3];
          joint_obs<false>(bp, Rp, wp, brax::qmat(sh.qw, sh.qx, sh.qy, sh.qz), sh.w, ang, rate);
          ob[11 + bp.dof_offset] = ang[0];
          ob[11 + S.D + bp.dof_offset] = rate[0];
        }
        if (b == 0) {
          float ctrl = 0.f;
          for (int cb = 1; cb < B; ++cb)
            if (bodies[cb].flags & kHasParent) ctrl += c(gm.reactf(cb, 9)[lane]);
          bool done = false;
          if (vh)
            done = root_env(sg, sh, c(gm.reactf(0, 10)[lane]), ctrl, ob, sg.reward + (int64_t)t * N + eh,
                            sg.done + (int64_t)t * N + eh);
          reinterpret_cast<float*>(gm.reactf(0, 11) + lane)[h] = done ? 1.f : 0.f;
        }
      }
      group_sync(bar, nthr);
      if (sg.auto_reset) {
        const f2 fl = gm.reactf(0, 11)[lane];
        if (va && fl.x != 0.f) load_half(sg.reset_state + (ea * B + b) * 13, s, 0);
        if (vb && fl.y != 0.f) load_half(sg.reset_state + (eb * B + b) * 13, s, 1);
      }
    }
    bad |= !finite_pair(s);
  }
  if (staged) bulk_wait_all();  // the checkpoint stores are complete before the block ends
  if (issuer) {  // no bulk copy may outlive the block: wait (bounded) for the last one into each buffer
    const int n = t1 - t0;
    for (int i = (n >= 2 ? n - 2 : 0); i < n; ++i)
      if (!mbar_wait(gm.mbar + (i & 1), (uint32_t)((i >> 1) & 1), 2000000000LL)) atomicOr(sg.status, kStatusTimeout);
  }
  if (va) store_half(sg.state_T + (ea * B + b) * 13, s, 0);
  if (vb) store_half(sg.state_T + (eb * B + b) * 13, s, 1);
  if (bad && (va || vb)) atomicOr(sg.status, kStatusNonfinite);
  if (sg.ccount) {
    atomicAdd(&gm.cnt[lane], cca);
    atomicAdd(&gm.cnt[32 + lane], ccb);
    group_sync(bar, nthr);
    if (b == 0) {
      if (va) __stcg(sg.ccount + ea, (c ? __ldcg(sg.ccount + ea) : 0) + gm.cnt[lane]);
      if (vb) __stcg(sg.ccount + eb, (c ? __ldcg(sg.ccount + eb) : 0) + gm.cnt[32 + lane]);
    }
  }
  if (chunked) {  // the item is done: its stores are made visible, then the unit's flag says so
    __threadfence();
    group_sync(0, 32 * B * sg.groups);
    if (threadIdx.x == 0) store_release(L.sc.sched + 32 + unit, c + 1);
  }
}

// ------------------------------------------------------------------ default_qp
__device__ __forceinline__ void qmul4(const float* a, const float* b, float* o) {
  const float r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  const float r1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  const float r2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  const float r3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  o[0] = r0;
  o[1] = r1;
  o[2] = r2;
  o[3] = r3;
}
__device__ __forceinline__ void qrot(const float* q, const float* v, float* o) {
  const M3 R = qmat(q[0], q[1], q[2], q[3]);
  const V3 r = mulc(R, v);
  o[0] = r.x;
  o[1] = r.y;
  o[2] = r.z;
}

// One thread per environment walks the joint tree from its roots (Sec. 4.1
// default_qp): R_c = R_p F_p Rot(angles) F_c^-1 and the child's anchor on the
// parent's anchor.
__global__ void default_qp_kernel(const unsigned char* blob, int64_t N, const float* root_pos, const float* root_rot,
                                  const float* angles, float* out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const SysP& S = *reinterpret_cast<const SysP*>(blob);
  const BodyP* bodies = reinterpret_cast<const BodyP*>(blob + blob_bodies_off());
  const int B = S.B;
  float* o = out + n * B * 13;
  for (int b = 0; b < B; ++b) {
    float* ob = o + b * 13;
    for (int i = 0; i < 3; ++i) ob[i] = bodies[b].rest_pos[i];
    for (int i = 0; i < 4; ++i) ob[3 + i] = bodies[b].rest_rot[i];
    for (int i = 7; i < 13; ++i) ob[i] = 0.f;
  }
  if (root_pos)
    for (int i = 0; i < 3; ++i) o[i] = root_pos[n * 3 + i];
  if (root_rot)
    for (int i = 0; i < 4; ++i) o[3 + i] = root_rot[n * 4 + i];
  for (int k = 0; k < S.n_order; ++k) {
    const int c = S.joint_order[k];
    const BodyP& bc = bodies[c];
    const int p = bc.parent;
    float qp[4] = {o[p * 13 + 3], o[p * 13 + 4], o[p * 13 + 5], o[p * 13 + 6]};
    const float np_ = rsqrtf(qp[0] * qp[0] + qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3]);
    for (int i = 0; i < 4; ++i) qp[i] *= np_;
    float rel[4] = {1.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < bc.dof; ++a) {
      const float th = angles ? angles[n * S.D + bc.dof_offset + a] : 0.f;
      float sn, cs;
      sincosf(0.5f * th, &sn, &cs);
      float r[4] = {cs, 0.f, 0.f, 0.f};
      r[1 + a] = sn;
      qmul4(rel, r, rel);
    }
    const float fci[4] = {bc.frame_c[0], -bc.frame_c[1], -bc.frame_c[2], -bc.frame_c[3]};
    float qc[4];
    qmul4(qp, bc.frame_p, qc);
    qmul4(qc, rel, qc);
    qmul4(qc, fci, qc);
    const float nc = rsqrtf(qc[0] * qc[0] + qc[1] * qc[1] + qc[2] * qc[2] + qc[3] * qc[3]);
    for (int i = 0; i < 4; ++i) qc[i] *= nc;
    float rp[3], rc[3];
    qrot(qp, bc.off_p, rp);
    qrot(qc, bc.off_c, rc);
    for (int i = 0; i < 3; ++i) o[c * 13 + i] = o[p * 13 + i] + rp[i] - rc[i];
    for (int i = 0; i < 4; ++i) o[c * 13 + 3 + i] = qc[i];
  }
}

// ------------------------------------------------------------------ launchers
template <class KernelT>
static cudaError_t launch_k(KernelT k, const Launch& L, int grid, int threads, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(L);
  return cudaGetLastError();
}
template <class KernelT>
static int occupancy_k(KernelT k, int threads, size_t smem) {
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

// Launch-bounds variants (max threads per block, min blocks per SM):
//   0: (384, 2)  1: (576, 1)  2: (1024, 1)  3: (288, 3)
// A rollout with the environment layer (Seg::obs) runs the kernels compiled
// with it, in the (576, 1) launch, or (1024, 1) for larger blocks; the
// others are compiled without it, so plain rollouts carry none of its code.
template <bool G>
static cudaError_t launch_rollout_g(const Launch& L, int grid, int threads, size_t smem, int variant, cudaStream_t st) {
  if (L.seg[0].obs)
    return threads <= 576 ? launch_k(rollout_kernel<576, 1, G, true>, L, grid, threads, smem, st)
                          : launch_k(rollout_kernel<1024, 1, G, true>, L, grid, threads, smem, st);
  switch (variant) {
    case 0: return launch_k(rollout_kernel<384, 2, G, false>, L, grid, threads, smem, st);
    case 1: return launch_k(rollout_kernel<576, 1, G, false>, L, grid, threads, smem, st);
    case 3: return launch_k(rollout_kernel<288, 3, G, false>, L, grid, threads, smem, st);
    default: return launch_k(rollout_kernel<1024, 1, G, false>, L, grid, threads, smem, st);
  }
}
cudaError_t launch_rollout(const Launch& L, int grid, int threads, size_t smem, int variant, bool general,
                           cudaStream_t st) {
  return general ? launch_rollout_g<true>(L, grid, threads, smem, variant, st)
                 : launch_rollout_g<false>(L, grid, threads, smem, variant, st);
}

template <bool G>
static int rollout_blocks_per_sm_g(int variant, int threads, size_t smem) {
  switch (variant) {
    case 0: return occupancy_k(rollout_kernel<384, 2, G, false>, threads, smem);
    case 1: return occupancy_k(rollout_kernel<576, 1, G, false>, threads, smem);
    case 3: return occupancy_k(rollout_kernel<288, 3, G, false>, threads, smem);
    default: return occupancy_k(rollout_kernel<1024, 1, G, false>, threads, smem);
  }
}
int rollout_blocks_per_sm(int variant, bool general, int threads, size_t smem) {
  return general ? rollout_blocks_per_sm_g<true>(variant, threads, smem)
                 : rollout_blocks_per_sm_g<false>(variant, threads, smem);
}

// Two-environments-per-thread variants: 0: (288, 2)  1: (576, 1)  2: (1024, 1)  3: (288, 3)
// 4: (864, 1); flat: every plane's normal is the world z axis.  With the
// environment layer: (576, 1), or (1024, 1) for larger blocks.
template <bool kFlat>
static cudaError_t launch_rollout_pair_t(const Launch& L, int grid, int threads, size_t smem, int variant,
                                         cudaStream_t st) {
  if (L.seg[0].obs)
    return threads <= 576 ? launch_k(rollout_pair_kernel<576, 1, kFlat, true>, L, grid, threads, smem, st)
                          : launch_k(rollout_pair_kernel<1024, 1, kFlat, true>, L, grid, threads, smem, st);
  switch (variant) {
    case 0: return launch_k(rollout_pair_kernel<288, 2, kFlat, false>, L, grid, threads, smem, st);
    case 1: return launch_k(rollout_pair_kernel<576, 1, kFlat, false>, L, grid, threads, smem, st);
    case 3: return launch_k(rollout_pair_kernel<288, 3, kFlat, false>, L, grid, threads, smem, st);
    case 4: return launch_k(rollout_pair_kernel<864, 1, kFlat, false>, L, grid, threads, smem, st);
    default: return launch_k(rollout_pair_kernel<1024, 1, kFlat, false>, L, grid, threads, smem, st);
  }
}
cudaError_t launch_rollout_pair(const Launch& L, int grid, int threads, size_t smem, int variant, bool flat,
                                cudaStream_t st) {
  return flat ? launch_rollout_pair_t<true>(L, grid, threads, smem, variant, st)
              : launch_rollout_pair_t<false>(L, grid, threads, smem, variant, st);
}
int pair_blocks_per_sm(int variant, int threads, size_t smem) {
  switch (variant) {
    case 0: return occupancy_k(rollout_pair_kernel<288, 2, true, false>, threads, smem);
    case 1: return occupancy_k(rollout_pair_kernel<576, 1, true, false>, threads, smem);
    case 3: return occupancy_k(rollout_pair_kernel<288, 3, true, false>, threads, smem);
    case 4: return occupancy_k(rollout_pair_kernel<864, 1, true, false>, threads, smem);
    default: return occupancy_k(rollout_pair_kernel<1024, 1, true, false>, threads, smem);
  }
}
int pair_variant_max_threads(int variant) {
  static const int t[5] = {288, 576, 1024, 288, 864};
  return (variant >= 0 && variant < 5) ? t[variant] : 0;
}
size_t pair_group_bytes(int B, int A) { return (size_t)p2::group_floats2(B, A) * sizeof(float); }

int rollout_variant_max_threads(int variant) {
  static const int t[4] = {384, 576, 1024, 288};
  return (variant >= 0 && variant < 4) ? t[variant] : 0;
}

// The kernels' arctangent and its packed form, elementwise over arrays (for
// the accuracy test of fast_atan2; not on the rollout path).
__global__ void atan2_probe_kernel(const float* y, const float* x, float* out, float* out_packed, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = fast_atan2(y[i], x[i]);
  // the packed form pairs element i with element n-1-i
  const int64_t j = n - 1 - i;
  const float2 r = p2::atan2p(make_float2(y[i], y[j]), make_float2(x[i], x[j]));
  out_packed[i] = r.x;
  (void)r.y;
}
cudaError_t launch_atan2_probe(const float* y, const float* x, float* out, float* out_packed, int64_t n,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  atan2_probe_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(y, x, out, out_packed, n);
  return cudaGetLastError();
}

cudaError_t upload_pool_forward(int off, const void* data, size_t bytes) {
  return cudaMemcpyToSymbol(c_pool, data, bytes, (size_t)off, cudaMemcpyHostToDevice);
}

cudaError_t launch_default_qp(const unsigned char* blob, int64_t N, const float* root_pos, const float* root_rot,
                              const float* angles, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const int threads = 128;
  const int64_t grid = (N + threads - 1) / threads;
  default_qp_kernel<<<(unsigned)grid, threads, 0, st>>>(blob, N, root_pos, root_rot, angles, out);
  return cudaGetLastError();
}

}  // namespace brax
