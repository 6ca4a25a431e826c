// Reverse-mode rollout kernel and its C ABI (brax_workspace_size,
// brax_rollout_backward, the batch variants).
//
// Memory plan per group of 32 environments (workspace, caller-owned):
//   steps  [K][13][B][32]  states at the start of every step of one
//                          checkpoint segment (recomputed from the segment's
//                          checkpoint);
//   subs   [S][13][B][32]  states at the start of every substep of one step
//                          (recomputed from that step's state);
//   slots  [P][8][32]      body-body pair impulses of the current substep
//                          (systems with pairs only);
//   pairg  [P][2][18][32]  each pair's adjoints of its two bodies' x1, R,
//                          v, w, gathered by the bodies in a fixed order.
// The reverse of a substep recomputes its forward intermediates (two group
// barriers, as in the forward), then runs the adjoint in reverse order:
//   P  potential + collision integrators          -> gwr[b] (dL/dF, dL/dtau)
//   -- barrier --
//   J  joint (child side; parent adjoints -> gpub[b]), own plane contacts,
//      owned pairs (their adjoints of both bodies to pairg in the workspace)
//   -- barrier --
//   K  gather children's gpub and the own pairs' pairg (in the body's pair
//      order, so the sums do not depend on warp timing), frame and kinematic
//      integrator.
// Every thread of a group holds one (body, environment) and its 13-float
// adjoint in registers for the whole reverse sweep.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/brax.h"
#include "brax_adjoint.cuh"
#include "brax_internal.h"
#include "brax_kernels.h"

namespace brax {

__constant__ __align__(16) unsigned char c_pool[kPoolBytes];

// Backward shared memory of one group (floats), after the forward layout.
__host__ __device__ inline int bwd_extra_floats(int B, int P) {
  return B * 6 * 32 + B * 18 * 32 + (P > 0 ? B * 6 * 32 : 0);
}
__host__ __device__ inline int bwd_fwd_floats(int B, int P, bool slots_in_smem) {
  return B * kPubFields * 32 + B * kReactFields * 32 + (slots_in_smem ? P * kSlotFields * 32 : 0) + 32;
}
__host__ __device__ inline int bwd_group_floats(int B, int P) { return bwd_fwd_floats(B, P, false) + bwd_extra_floats(B, P); }
// Workspace of one group: step states [K][13][B][32], substep states
// [S][13][B][32], pair slots [P][kSlotFields][32], pair adjoints
// [P][2][18][32], and the state adjoint carried from one chunk of a chunked
// schedule to the next [13][B][32].
__host__ __device__ inline int64_t ws_pairg_off(int B, int P, int K, int S) {
  return (int64_t)(K + S) * 13 * B * 32 + (int64_t)P * kSlotFields * 32;
}
__host__ __device__ inline int64_t ws_carry_off(int B, int P, int K, int S) {
  return ws_pairg_off(B, P, K, S) + (int64_t)P * 2 * 18 * 32;
}
__host__ __device__ inline int64_t ws_group_floats(int B, int P, int K, int S) {
  return ws_carry_off(B, P, K, S) + (int64_t)13 * B * 32;
}

struct BwdMem {
  float* gwr;    // [B][6][32]  adjoint of a body's summed force, torque
  float* gpub;   // [B][18][32] a child's adjoints of its parent's x1, R, v, w
  float* gacc;   // [B][6][32]  adjoint of a body's contact velocity update (pairs)
  float* pairg;  // workspace [P][2][18][32]: a pair's adjoints of body a's and body b's x1, R, v, w
};

__device__ __forceinline__ void load_body_ws(const float* p, int stride, Body& s) {
  s.x = mk3(p[0], p[stride], p[2 * stride]);
  s.qw = p[3 * stride];
  s.qx = p[4 * stride];
  s.qy = p[5 * stride];
  s.qz = p[6 * stride];
  s.v = mk3(p[7 * stride], p[8 * stride], p[9 * stride]);
  s.w = mk3(p[10 * stride], p[11 * stride], p[12 * stride]);
}
// Drop one 128-byte line of the workspace from L2 without writing it back:
// the reverse sweep has read it for the last time before the next recompute
// overwrites it, so writing it back to DRAM would move dead data.
__device__ __forceinline__ void discard_line(const float* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
// Lane i < 13 drops field i's line of a lane-contiguous state (13 rows of
// 32 floats, `stride` floats apart).  Called once the warp has consumed the
// state (after a __syncwarp).
__device__ __forceinline__ void discard_state_ws(const float* row0, int stride, int lane) {
  if (lane < 13) discard_line(row0 + (int64_t)lane * stride);
}

__device__ __forceinline__ void store_body_ws(float* p, int stride, const Body& s) {
  p[0] = s.x.x;
  p[stride] = s.x.y;
  p[2 * stride] = s.x.z;
  p[3 * stride] = s.qw;
  p[4 * stride] = s.qx;
  p[5 * stride] = s.qy;
  p[6 * stride] = s.qz;
  p[7 * stride] = s.v.x;
  p[8 * stride] = s.v.y;
  p[9 * stride] = s.v.z;
  p[10 * stride] = s.w.x;
  p[11 * stride] = s.w.y;
  p[12 * stride] = s.w.z;
}

template <bool kGeneral, bool kIso = false>
__device__ __forceinline__ void fwd_substep(const SysP& S, const BodyP* bodies, const PairP* pairs,
                                            const PlaneP* planes, const BodyP& bp, const HingeRegs& hr,
                                            const PointRegs* pr, int b, int B, int lane, GroupMem& gm, int bar,
                                            int nthr, Body& s, const float* act) {
  kinematic(bp, S.h, s);
  const Frame f = make_frame(bp, s);
  if (bp.flags & kPublish) {
    if (kGeneral && (bp.flags & kInPair)) publish<true>(gm, b, lane, s, f, bp);
    else publish<false>(gm, b, lane, s, f, bp);
  }
  group_sync(bar, nthr);
  Wrench wr{zero3(), zero3()};
  if (bp.flags & kHasParent) {
    const Pub pp = read_pub(gm, bp.parent, lane);
    if (kGeneral) wr = joint_forward<true>(bp, pp, s, f, act, gm.react4(b, 0) + lane);
    else wr = joint_forward<false>(hr, pp, s, f, act, gm.react4(b, 0) + lane);
  }
  Acc acc{zero3(), zero3(), 0};
  const int np = bp.n_points;
  if (kGeneral) {
    for (int i = 0; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
    for (int k = b; k < S.P; k += B) pair_forward(S, bodies, pairs[k], gm, k, lane);
  } else {
    plane_points_regs(S, bp, pr, planes, np < 2 ? np : 2, s, f, acc);
    for (int i = 2; !kIso && i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
  }
  group_sync(bar, nthr);
  integrate<kGeneral>(S, bp, gm, lane, s, f, wr, acc);
}

// Reverse of one substep.  s_in: the substep's input state; g: adjoint of
// its output state (updated in place to the adjoint of the input state).
template <bool kGeneral>
__device__ __forceinline__ void bwd_substep(const SysP& S, const BodyP* bodies, const PairP* pairs,
                                            const PlaneP* planes, const BodyP& bp, const HingeRegs& hr,
                                            const PointRegs* pr, int b, int B, int lane, GroupMem& gm, BwdMem& bm,
                                            int bar, int nthr, const Body& s_in, GBody& g, const float* act,
                                            float* gact) {
  const float h = S.h;
  // ---- forward recompute: phase K
  Body s = s_in;
  kinematic(bp, h, s);
  const Frame f = make_frame(bp, s);
  if (bp.flags & kPublish) {
    if (kGeneral && (bp.flags & kInPair)) publish<true>(gm, b, lane, s, f, bp);
    else publish<false>(gm, b, lane, s, f, bp);
  }
  group_sync(bar, nthr);
  // ---- forward recompute: phase J
  Wrench wr{zero3(), zero3()};
  Pub pp;
  if (bp.flags & kHasParent) {
    pp = read_pub(gm, bp.parent, lane);
    if (kGeneral) wr = joint_forward<true>(bp, pp, s, f, act, gm.react4(b, 0) + lane);
    else wr = joint_forward<false>(hr, pp, s, f, act, gm.react4(b, 0) + lane);
  }
  Acc acc{zero3(), zero3(), 0};
  const int np = bp.n_points;
  if (kGeneral) {
    for (int i = 0; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
    for (int k = b; k < S.P; k += B) pair_forward(S, bodies, pairs[k], gm, k, lane);
  } else {
    plane_points_regs(S, bp, pr, planes, np < 2 ? np : 2, s, f, acc);
    for (int i = 2; i < np; ++i) plane_point(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, acc);
  }
  group_sync(bar, nthr);
  // ---- forward values of phase P
  int n_pair = 0;
  if (kGeneral)
    for (int i = 0; i < bp.n_bpairs; ++i)
      if (gm.slot4(bp.bpair[i] >> 1, 1)[lane].z != 0.f) ++n_pair;
  V3 Ft = wr.F, Tt = wr.tau;
  {
    Wrench sum{Ft, Tt};
    for (int c = 0; c < bp.n_children; ++c) add_reaction(gm, bp.children[c], lane, sum);
    Ft = sum.F;
    Tt = sum.tau;
  }
  // ---- reverse P: potential and collision integrators
  const int n = acc.n + n_pair;
  const float inv = n > 0 ? ((S.average && n > 1) ? __fdividef(1.f, (float)n) : 1.f) : 0.f;
  const V3 gdv = inv * g.v, gdw = inv * g.w;
  V3 gv2 = g.v, gw2 = g.w;
  if (bp.flags & kAnyFrozen) {
    gv2 = mask3(bp.flags, gv2);
    gw2 = mask3(bp.flags >> 3, gw2);
  }
  V3 gvm = gv2, gwm = gw2;
  const V3 gFt = (h * bp.inv_mass) * gv2;
  S6 gI;
  zero(gI);
  V3 gTt = zero3();
  S6 gIw;  // adjoint of I_w = R diag(I) R^T (the gyroscopic term)
  zero(gIw);
  if (kGeneral && S.variants) {
    // v1 = v + h (F/m + g - ld v);  w1 = w + h (Ii (T - w x I_w w) - ad w)
    gvm = fma3(-h * S.lin_damp, gv2, gvm);
    gwm = fma3(-h * S.ang_damp, gw2, gwm);
    V3 Te = Tt;
    V3 u = zero3();
    S6 Iw;
    if (S.gyro) {
      Iw = inv_inertia_world(f.R, bp.I);
      u = mul(Iw, s.w);
      Te = Tt - cross(s.w, u);
    }
    s6_mul_bwd(f.Ii, Te, h * gw2, gI, gTt);
    if (S.gyro) {  // c = w x u, u = I_w w, Te = T - c
      const V3 gc = -gTt;
      V3 gu = zero3();
      cross_bwd(s.w, u, gc, gwm, gu);
      s6_mul_bwd(Iw, s.w, gu, gIw, gwm);
    }
  } else {
    s6_mul_bwd(f.Ii, Tt, h * gw2, gI, gTt);
  }
  {
    float* o = bm.gwr + (b * 6) * 32 + lane;
    o[0] = gFt.x;
    o[32] = gFt.y;
    o[64] = gFt.z;
    o[96] = gTt.x;
    o[128] = gTt.y;
    o[160] = gTt.z;
  }
  if (kGeneral && (bp.flags & kInPair)) {
    float* o = bm.gacc + (b * 6) * 32 + lane;
    o[0] = gdv.x;
    o[32] = gdv.y;
    o[64] = gdv.z;
    o[96] = gdw.x;
    o[128] = gdw.y;
    o[160] = gdw.z;
  }
  group_sync(bar, nthr);
  // ---- reverse J
  V3 gx1 = g.x;
  M3 gR;
  zero(gR);
  if (bp.flags & kHasParent) {
    const float* pg = bm.gwr + (bp.parent * 6) * 32 + lane;
    const V3 gFp = mk3(pg[0], pg[32], pg[64]);
    const V3 gTp = mk3(pg[96], pg[128], pg[160]);
    V3 gxp = zero3(), gvp = zero3(), gwp = zero3();
    M3 gRp;
    zero(gRp);
    if (!kGeneral)
      joint_hinge_bwd(hr, pp, s, f, act, gFt, gTt, gFp, gTp, gx1, gR, gvm, gwm, gxp, gRp, gvp, gwp, gact);
    else if (bp.dof == 1)
      joint_hinge_bwd(bp, pp, s, f, act, gFt, gTt, gFp, gTp, gx1, gR, gvm, gwm, gxp, gRp, gvp, gwp, gact);
    else
      joint3_bwd(bp, pp, s, f, act, gFt, gTt, gFp, gTp, gx1, gR, gvm, gwm, gxp, gRp, gvp, gwp, gact);
    float* o = bm.gpub + (b * 18) * 32 + lane;
    o[0] = gxp.x;
    o[32] = gxp.y;
    o[64] = gxp.z;
#pragma unroll
    for (int i = 0; i < 9; ++i) o[(3 + i) * 32] = gRp.m[i];
    o[12 * 32] = gvp.x;
    o[13 * 32] = gvp.y;
    o[14 * 32] = gvp.z;
    o[15 * 32] = gwp.x;
    o[16 * 32] = gwp.y;
    o[17 * 32] = gwp.z;
  }
  if (n > 0) {
    if (kGeneral) {
      for (int i = 0; i < np; ++i)
        plane_point_bwd(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, gdv, gdw, gx1, gR, gI, gvm, gwm);
    } else {
      if (np > 0) plane_point_bwd(S, bp, pr[0], planes[bp.pt[0].plane], s, f, gdv, gdw, gx1, gR, gI, gvm, gwm);
      if (np > 1) plane_point_bwd(S, bp, pr[1], planes[bp.pt[1].plane], s, f, gdv, gdw, gx1, gR, gI, gvm, gwm);
      for (int i = 2; i < np; ++i)
        plane_point_bwd(S, bp, bp.pt[i], planes[bp.pt[i].plane], s, f, gdv, gdw, gx1, gR, gI, gvm, gwm);
    }
  }
  if (kGeneral) {
    for (int k = b; k < S.P; k += B) {
      const PairP& prk = pairs[k];
      if (gm.slot4(k, 1)[lane].z == 0.f) continue;
      GSide GA, GB;
      zero(GA);
      zero(GB);
      pair_bwd(S, bodies, prk, gm, bm.gacc, lane, GA, GB);
      for (int side = 0; side < 2; ++side) {
        const int body = side == 0 ? prk.ba : prk.bb;
        GSide& G = side == 0 ? GA : GB;
        const Pub X = read_pub(gm, body, lane);
        inv_inertia_bwd(X.R, bodies[body].inv_I, G.I, G.R);
        float* o = bm.pairg + ((int64_t)(k * 2 + side) * 18) * 32 + lane;
        o[0 * 32] = G.x.x;
        o[1 * 32] = G.x.y;
        o[2 * 32] = G.x.z;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[(3 + i) * 32] = G.R.m[i];
        o[12 * 32] = G.v.x;
        o[13 * 32] = G.v.y;
        o[14 * 32] = G.v.z;
        o[15 * 32] = G.w.x;
        o[16 * 32] = G.w.y;
        o[17 * 32] = G.w.z;
      }
    }
  }
  group_sync(bar, nthr);
  // ---- reverse K: gather children's adjoints of this body, frame, kinematic
  for (int c = 0; c < bp.n_children; ++c) {
    const float* o = bm.gpub + (bp.children[c] * 18) * 32 + lane;
    gx1 = gx1 + mk3(o[0], o[32], o[64]);
#pragma unroll
    for (int i = 0; i < 9; ++i) gR.m[i] += o[(3 + i) * 32];
    gvm = gvm + mk3(o[12 * 32], o[13 * 32], o[14 * 32]);
    gwm = gwm + mk3(o[15 * 32], o[16 * 32], o[17 * 32]);
  }
  for (int i = 0; kGeneral && i < bp.n_bpairs; ++i) {  // the own pairs' adjoints, in the body's pair order
    const int code = bp.bpair[i];
    if (gm.slot4(code >> 1, 1)[lane].z == 0.f) continue;  // no contact: the pair wrote nothing for this lane
    const float* o = bm.pairg + ((int64_t)code * 18) * 32 + lane;
    gx1 = gx1 + mk3(o[0], o[32], o[64]);
#pragma unroll
    for (int j = 0; j < 9; ++j) gR.m[j] += o[(3 + j) * 32];
    gvm = gvm + mk3(o[12 * 32], o[13 * 32], o[14 * 32]);
    gwm = gwm + mk3(o[15 * 32], o[16 * 32], o[17 * 32]);
  }
  inv_inertia_bwd(f.R, bp.inv_I, gI, gR);
  if (kGeneral && S.gyro) inv_inertia_bwd(f.R, bp.I, gIw, gR);
  float gq1[4] = {g.q[0], g.q[1], g.q[2], g.q[3]};
  qmat_bwd(s.qw, s.qx, s.qy, s.qz, gR, gq1);
  g = kinematic_bwd(bp, h, s_in, gx1, gq1, gvm, gwm);
}

// Register-resident contact point i (0 or 1) of the own body.
__device__ __forceinline__ PointRegs sel_point(int i, const PointRegs* pr) {
  PointRegs p;
  p.o[0] = i ? pr[1].o[0] : pr[0].o[0];
  p.o[1] = i ? pr[1].o[1] : pr[0].o[1];
  p.o[2] = i ? pr[1].o[2] : pr[0].o[2];
  p.r = i ? pr[1].r : pr[0].r;
  p.mu = i ? pr[1].mu : pr[0].mu;
  p.e = i ? pr[1].e : pr[0].e;
  return p;
}

// Whether the own plane-contact point is active (plane_point()'s test: the
// sphere penetrates and the effective mass is positive).
template <class PT>
__device__ __forceinline__ int plane_point_active(const BodyP& bp, const PT& pt, const PlaneP& pl, const Body& s,
                                                  const Frame& f) {
  const V3 ro = mulc(f.R, pt.o);
  const V3 n = ld3(pl.n);
  const float depth = pt.r - dot((s.x + ro) - ld3(pl.p0), n);
  if (!(depth > 0.f)) return 0;
  return eff_mass(bp.flags, bp.inv_mass, f.Ii, fma3(-pt.r, n, ro), n) > 0.f ? 1 : 0;
}

// Reverse of one substep of a hinge-only system whose bodies all have
// isotropic inertia.  Then I_w = R diag(c) R^T = c 1 for every R, so the
// adjoint of I_w reaches no orientation (dI_w/dR = 0) and the summed force
// and torque of the potential integrator, which only that adjoint reads, are
// not needed: no joint is recomputed forward and no child reaction is read.
// What is left needs two group barriers instead of four:
//   K  kinematic + frame, publish; P: adjoints of F and tau -> gwr[b]
//   -- barrier --
//   J  joint (child side; parent adjoints -> gpub[b]), own plane contacts
//   -- barrier --
//   K  gather children's gpub, frame and kinematic integrator.
// Shared memory: a parent's published state and gwr are written before the
// first barrier and read between the two; gpub is written between them and
// read after the second; the next substep writes each only after the
// barrier that follows its last read.
__device__ __forceinline__ void bwd_substep_iso(const SysP& S, const PlaneP* planes, const BodyP& bp,
                                                const HingeRegs& hr, const PointRegs* pr, int b, int lane,
                                                GroupMem& gm, BwdMem& bm, int bar, int nthr, const Body& s_in,
                                                GBody& g, const float* act, float* gact) {
  const float h = S.h;
  Body s = s_in;
  kinematic(bp, h, s);
  const Frame f = make_frame(bp, s);
  if (bp.flags & kPublish) publish<false>(gm, b, lane, s, f, bp);
  // ---- reverse P: v1 = v + h (F/m + g), w1 = w + h Ii tau (+ contact updates)
  V3 gv2 = g.v, gw2 = g.w;
  if (bp.flags & kAnyFrozen) {
    gv2 = mask3(bp.flags, gv2);
    gw2 = mask3(bp.flags >> 3, gw2);
  }
  const V3 gFt = (h * bp.inv_mass) * gv2;
  const V3 gTt = mul(f.Ii, h * gw2);
  {
    float* o = bm.gwr + (b * 6) * 32 + lane;
    o[0] = gFt.x;
    o[32] = gFt.y;
    o[64] = gFt.z;
    o[96] = gTt.x;
    o[128] = gTt.y;
    o[160] = gTt.z;
  }
  group_sync(bar, nthr);
  // ---- reverse J
  V3 gx1 = g.x, gvm = gv2, gwm = gw2;
  M3 gR;
  zero(gR);
  if (bp.flags & kHasParent) {
    const Pub pp = read_pub(gm, bp.parent, lane);
    const float* pg = bm.gwr + (bp.parent * 6) * 32 + lane;
    const V3 gFp = mk3(pg[0], pg[32], pg[64]);
    const V3 gTp = mk3(pg[96], pg[128], pg[160]);
    V3 gxp = zero3(), gvp = zero3(), gwp = zero3();
    M3 gRp;
    zero(gRp);
    joint_hinge_bwd(hr, pp, s, f, act, gFt, gTt, gFp, gTp, gx1, gR, gvm, gwm, gxp, gRp, gvp, gwp, gact);
    float* o = bm.gpub + (b * 18) * 32 + lane;
    o[0] = gxp.x;
    o[32] = gxp.y;
    o[64] = gxp.z;
#pragma unroll
    for (int i = 0; i < 9; ++i) o[(3 + i) * 32] = gRp.m[i];
    o[12 * 32] = gvp.x;
    o[13 * 32] = gvp.y;
    o[14 * 32] = gvp.z;
    o[15 * 32] = gwp.x;
    o[16 * 32] = gwp.y;
    o[17 * 32] = gwp.z;
  }
  // own plane contacts: at most two points a body in this kind of system,
  // both register-resident; one copy of each loop body
  const int np = bp.n_points;
  int n = 0;
#pragma unroll 1
  for (int i = 0; i < np; ++i) n += plane_point_active(bp, sel_point(i, pr), planes[bp.pt[i].plane], s, f);
  if (n > 0) {
    const float inv = (S.average && n > 1) ? __fdividef(1.f, (float)n) : 1.f;
    const V3 gdv = inv * g.v, gdw = inv * g.w;
    S6 gI;  // the adjoint of I_w, which reaches nothing here
    zero(gI);
#pragma unroll 1
    for (int i = 0; i < np; ++i)
      plane_point_bwd(S, bp, sel_point(i, pr), planes[bp.pt[i].plane], s, f, gdv, gdw, gx1, gR, gI, gvm, gwm);
  }
  group_sync(bar, nthr);
  // ---- reverse K
  for (int c = 0; c < bp.n_children; ++c) {
    const float* o = bm.gpub + (bp.children[c] * 18) * 32 + lane;
    gx1 = gx1 + mk3(o[0], o[32], o[64]);
#pragma unroll
    for (int i = 0; i < 9; ++i) gR.m[i] += o[(3 + i) * 32];
    gvm = gvm + mk3(o[12 * 32], o[13 * 32], o[14 * 32]);
    gwm = gwm + mk3(o[15 * 32], o[16 * 32], o[17 * 32]);
  }
  float gq1[4] = {g.q[0], g.q[1], g.q[2], g.q[3]};
  qmat_bwd(s.qw, s.qx, s.qy, s.qz, gR, gq1);
  g = kinematic_bwd(bp, h, s_in, gx1, gq1, gvm, gwm);
}

// Reverse pass of a group of 32 environments: checkpoint segments last
// first.  A block runs unit blockIdx.x over all segments or, under a chunked
// schedule (Sched; chunk_steps counts segments, chunk 0 holds the last
// ones), one chunk of the unit of the item it takes; the state adjoint then
// passes from chunk to chunk through the workspace.
template <bool kGeneral, bool kIso>
__device__ __forceinline__ void rollout_bwd_body(const Launch& L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const bool chunked = L.sc.n_chunks > 0;
  int unit = blockIdx.x, c = 0;
  if (chunked) {
    const int n_units = L.sc.n_units, n_items = L.sc.n_chunks * n_units;
    if (threadIdx.x == 0) {
      int ticket;
      const int it = take_item(L.sc, n_items, &ticket);
      if (it == -2) {  // report the timeout to the system of the unit that was waited for
        const int u = ticket % n_units;
        int sj = 0;
        while (sj + 1 < L.n_segs && u >= L.seg[sj].cta_end) ++sj;
        atomicOr(L.seg[sj].status, kStatusTimeout);
      }
      s_item = it;
    }
    group_sync(0, blockDim.x);
    const int it = s_item;
    if (it < 0 || it >= n_items) return;
    unit = it % n_units;
    c = it / n_units;
  }
  int si = 0;
  while (si + 1 < L.n_segs && unit >= L.seg[si].cta_end) ++si;
  const Seg& sg = L.seg[si];
  const unsigned char* blob = c_pool + sg.pool_off;
  const SysP& S = *reinterpret_cast<const SysP*>(blob);
  const BodyP* bodies = reinterpret_cast<const BodyP*>(blob + blob_bodies_off());
  const PairP* pairs = reinterpret_cast<const PairP*>(blob + blob_pairs_off(sg.B));
  const PlaneP* planes = reinterpret_cast<const PlaneP*>(blob + blob_planes_off(sg.B, sg.P));
  const int B = sg.B, P = sg.P;
  const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
  const int lane = threadIdx.x & 31;
  const int g = warp / B, b = warp - g * B;
  if (g >= sg.groups) return;
  const int64_t N = sg.n_envs;
  const int64_t group = (int64_t)(unit - sg.cta_begin) * sg.groups + g;
  const int64_t env = group * 32 + lane;
  const bool valid = env < N;
  float* gbase = reinterpret_cast<float*>(smem) + g * bwd_group_floats(B, P);
  GroupMem gm = group_mem(gbase, B, 0);
  const int K = L.K, T = L.T, nsub = S.substeps;
  float* ws = sg.ws + group * ws_group_floats(B, P, K, nsub);
  if (kGeneral) gm.slot = reinterpret_cast<float4*>(ws + (int64_t)(K + nsub) * 13 * B * 32);  // pair impulses live in the workspace
  BwdMem bm;
  bm.gwr = gbase + bwd_fwd_floats(B, P, false);
  bm.gpub = bm.gwr + B * 6 * 32;
  bm.gacc = bm.gpub + B * 18 * 32;
  bm.pairg = ws + ws_pairg_off(B, P, K, nsub);
  const int bar = 1 + g, nthr = 32 * B;
  const BodyP& bp = bodies[b];
  const int stride = B * 32;
  float* ws_steps = ws + b * 32 + lane;
  float* ws_subs = ws + (int64_t)K * 13 * B * 32 + b * 32 + lane;

  HingeRegs hr;
  PointRegs pr[2];
  if (!kGeneral) {
    if (bp.flags & kHasParent) hr = hinge_regs(bp);
    if (bp.n_points > 0) pr[0] = point_regs(bp.pt[0]);
    if (bp.n_points > 1) pr[1] = point_regs(bp.pt[1]);
  }
  const int nseg = (T + K - 1) / K;
  const int seg_hi = chunked ? nseg - c * L.sc.chunk_steps : nseg;
  const int seg_lo = chunked ? max(0, seg_hi - L.sc.chunk_steps) : 0;
  GBody gs = zero_gbody();
  if (c > 0) {  // L2 loads: the previous chunk may have run on another SM
    // the adjoint carried between chunks (lane-contiguous, like the step states)
    const float* carry = ws_steps + ws_carry_off(B, P, K, nsub);
    float v[13];
#pragma unroll
    for (int i = 0; i < 13; ++i) v[i] = __ldcg(carry + i * stride);
    gs.x = mk3(v[0], v[1], v[2]);
    gs.q[0] = v[3];
    gs.q[1] = v[4];
    gs.q[2] = v[5];
    gs.q[3] = v[6];
    gs.v = mk3(v[7], v[8], v[9]);
    gs.w = mk3(v[10], v[11], v[12]);
  } else if (valid) {
    const float* p = sg.g_state_T + (env * B + b) * 13;
    gs.x = mk3(p[0], p[1], p[2]);
    gs.q[0] = p[3];
    gs.q[1] = p[4];
    gs.q[2] = p[5];
    gs.q[3] = p[6];
    gs.v = mk3(p[7], p[8], p[9]);
    gs.w = mk3(p[10], p[11], p[12]);
  }
  const int A = sg.A;
  float act[3] = {0.f, 0.f, 0.f};
  auto load_act = [&](int t) {
    if (valid && (bp.flags & kHasParent)) {
      const float* ap = sg.actions + ((int64_t)t * N + env) * A;
#pragma unroll
      for (int a = 0; a < 3; ++a) act[a] = bp.act[a] >= 0 ? __ldg(ap + bp.act[a]) : 0.f;
    }
  };
  for (int seg = seg_hi - 1; seg >= seg_lo; --seg) {
    const int t0 = seg * K, t1 = min(T, t0 + K);
    Body s;
    if (valid) {
      load_body(sg.ckpt + (((int64_t)seg * N + env) * B + b) * 13, s);
    } else {
      s.x = ld3(bp.rest_pos);
      s.qw = bp.rest_rot[0];
      s.qx = bp.rest_rot[1];
      s.qy = bp.rest_rot[2];
      s.qz = bp.rest_rot[3];
      s.v = zero3();
      s.w = zero3();
    }
    // recompute the segment's step states
    for (int t = t0; t < t1; ++t) {
      store_body_ws(ws_steps + (int64_t)(t - t0) * 13 * stride, stride, s);
      if (t + 1 < t1) {
        load_act(t);
        for (int k = 0; k < nsub; ++k)
          fwd_substep<kGeneral, kIso>(S, bodies, pairs, planes, bp, hr, pr, b, B, lane, gm, bar, nthr, s, act);
      }
    }
    for (int t = t1 - 1; t >= t0; --t) {
      load_body_ws(ws_steps + (int64_t)(t - t0) * 13 * stride, stride, s);
      load_act(t);
      __syncwarp();
      discard_state_ws(ws_steps - lane + (int64_t)(t - t0) * 13 * stride, stride, lane);
      for (int k = 0; k < nsub; ++k) {
        store_body_ws(ws_subs + (int64_t)k * 13 * stride, stride, s);
        if (k + 1 < nsub)
          fwd_substep<kGeneral, kIso>(S, bodies, pairs, planes, bp, hr, pr, b, B, lane, gm, bar, nthr, s, act);
      }
      if (sg.g_torso && b == 0 && valid) {
        const float* gt = sg.g_torso + ((int64_t)t * N + env) * 3;
        gs.x = gs.x + mk3(gt[0], gt[1], gt[2]);
      }
      float gact[3] = {0.f, 0.f, 0.f};
      for (int k = nsub - 1; k >= 0; --k) {
        Body sin;
        load_body_ws(ws_subs + (int64_t)k * 13 * stride, stride, sin);
        if (kIso)
          bwd_substep_iso(S, planes, bp, hr, pr, b, lane, gm, bm, bar, nthr, sin, gs, act, gact);
        else
          bwd_substep<kGeneral>(S, bodies, pairs, planes, bp, hr, pr, b, B, lane, gm, bm, bar, nthr, sin, gs, act,
                                gact);
        __syncwarp();
        discard_state_ws(ws_subs - lane + (int64_t)k * 13 * stride, stride, lane);
      }
      if (valid && sg.g_actions && (bp.flags & kHasParent)) {
        float* ga = sg.g_actions + ((int64_t)t * N + env) * A;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (bp.act[a] >= 0) ga[bp.act[a]] = gact[a];
      }
    }
  }
  if (seg_lo > 0) {  // not the first segments yet: hand the adjoint to the next chunk
    float* carry = ws_steps + ws_carry_off(B, P, K, nsub);
    const float v[13] = {gs.x.x, gs.x.y, gs.x.z, gs.q[0], gs.q[1], gs.q[2], gs.q[3],
                         gs.v.x, gs.v.y, gs.v.z, gs.w.x, gs.w.y, gs.w.z};
#pragma unroll
    for (int i = 0; i < 13; ++i) __stcg(carry + i * stride, v[i]);
  } else if (valid && sg.g_state0) {
    float* p = sg.g_state0 + (env * B + b) * 13;
    p[0] = gs.x.x;
    p[1] = gs.x.y;
    p[2] = gs.x.z;
    p[3] = gs.q[0];
    p[4] = gs.q[1];
    p[5] = gs.q[2];
    p[6] = gs.q[3];
    p[7] = gs.v.x;
    p[8] = gs.v.y;
    p[9] = gs.v.z;
    p[10] = gs.w.x;
    p[11] = gs.w.y;
    p[12] = gs.w.z;
  }
  if (chunked) {  // the item is done: its stores are made visible, then the unit's flag says so
    __threadfence();
    group_sync(0, 32 * B * sg.groups);
    if (threadIdx.x == 0) store_release(L.sc.sched + 32 + unit, c + 1);
  }
}

// Launch-bounds variants 0..3 (as the forward kernels), and variant 4: at
// most 112 registers a thread (blocks of up to 576 threads; two 9-warp
// groups per SM), which holds more of the adjoint's live values than the
// 96 registers (576, 1) gives.  Each is compiled for three kinds of system:
// hinge-only, hinge-only with isotropic inertia (bwd_substep_iso), general.
template <int MAXT, int MINB, bool kGeneral, bool kIso>
__global__ void __launch_bounds__(MAXT, MINB) rollout_bwd_kernel(const __grid_constant__ Launch L) {
  rollout_bwd_body<kGeneral, kIso>(L);
}
template <bool kGeneral, bool kIso>
__global__ void __maxnreg__(112) rollout_bwd_kernel_r112(const __grid_constant__ Launch L) {
  rollout_bwd_body<kGeneral, kIso>(L);
}

using BwdKernel = void (*)(const Launch);
template <bool G, bool I>
static BwdKernel bwd_kernel_t(int variant) {
  switch (variant) {
    case 0: return rollout_bwd_kernel<384, 2, G, I>;
    case 1: return rollout_bwd_kernel<576, 1, G, I>;
    case 3: return rollout_bwd_kernel<288, 3, G, I>;
    case 4: return rollout_bwd_kernel_r112<G, I>;
    default: return rollout_bwd_kernel<1024, 1, G, I>;
  }
}
static BwdKernel bwd_kernel(int variant, bool general, bool iso) {
  if (general) return bwd_kernel_t<true, false>(variant);
  return iso ? bwd_kernel_t<false, true>(variant) : bwd_kernel_t<false, false>(variant);
}

int backward_blocks_per_sm(int variant, bool general, bool iso, int threads, size_t smem) {
  const BwdKernel k = bwd_kernel(variant, general, iso);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

int backward_variant_max_threads(int variant) {
  static const int t[5] = {384, 576, 1024, 288, 576};
  return (variant >= 0 && variant < 5) ? t[variant] : 0;
}

cudaError_t launch_rollout_backward(const Launch& L, int grid, int threads, size_t smem, int variant, bool general,
                                    bool iso, cudaStream_t st) {
  const BwdKernel k = bwd_kernel(variant, general, iso);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t upload_pool_backward(int off, const void* data, size_t bytes) {
  return cudaMemcpyToSymbol(c_pool, data, bytes, (size_t)off, cudaMemcpyHostToDevice);
}

size_t backward_smem_bytes(int B, int P, int groups) { return (size_t)groups * bwd_group_floats(B, P) * sizeof(float); }
int64_t backward_ws_floats_per_group(int B, int P, int K, int S) { return ws_group_floats(B, P, K, S); }

}  // namespace brax

// ------------------------------------------------------------------ reverse mode without allocation
// Some callers cannot allocate device memory at the time they need a
// gradient: for example a host framework whose allocator owns all device
// memory and offers no hook to foreign code, or a deployment that fixes its
// memory footprint when it starts.  brax_rollout_backward_noalloc serves them
// with a scratch array that lives in this library's own device image: a
// file-scope __device__ array of BRAX_NOALLOC_SCRATCH_BYTES bytes, which every
// GPU that loads the library holds until the process exits.
//
// In host code `g_noalloc_scratch` names a host-side stand-in, not a device
// address, so it is never passed to a kernel directly.  The first call on a
// device looks up the array's device address with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any stream
// capture.  All calls share the one array and it keeps the last call's
// contents; nothing in it needs to start at zero (the reverse kernel writes
// every scratch word before reading it).  Calls whose kernels overlap on the
// GPU (different streams, or different threads) race on the array.
namespace brax {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BRAX_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int noalloc_fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

// Device address of the scratch array on the current device (set up once per device).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace brax

extern "C" int brax_rollout_backward_noalloc(const brax_system* s, int64_t n_envs, int32_t T, int32_t K,
                                             const float* state0, const float* actions, const float* checkpoints,
                                             const float* g_state_T, const float* g_torso_traj, float* g_actions,
                                             float* g_state0, void* stream) {
  using namespace brax;
  if (!s || n_envs < 0 || T < 0 || K < 1)
    return noalloc_fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward_noalloc: bad arguments");
  const size_t need = backward_workspace_bytes(s, n_envs, std::min(K, std::max(T, 1)));
  if (need > (size_t)BRAX_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(BRAX_ERR_WORKSPACE,
                        "brax_rollout_backward_noalloc: this rollout needs " + std::to_string(need) +
                            " bytes of scratch, more than the " + std::to_string((size_t)BRAX_NOALLOC_SCRATCH_BYTES) +
                            " bytes this entry point holds; use brax_rollout_backward with a caller workspace");
  void* ws = nullptr;
  cudaError_t e = noalloc_scratch(&ws);
  if (e != cudaSuccess)
    return noalloc_fail(BRAX_ERR_CUDA, std::string("brax_rollout_backward_noalloc: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e));
  // The array holds the reverse pass's workspace first and, behind it (at a
  // 256-byte boundary), the region a chunked schedule takes its ticket
  // counter and flags from; when that region does not fit the launch takes
  // the static schedule.  Either way nothing is allocated.
  const size_t ws_bytes = (need + 255) & ~(size_t)255;
  unsigned char* base = static_cast<unsigned char*>(ws);
  return rollout_backward_fixed_sched(s, n_envs, T, K, state0, actions, checkpoints, g_state_T, g_torso_traj, g_actions,
                                      g_state0, ws, ws_bytes, reinterpret_cast<int32_t*>(base + ws_bytes),
                                      (size_t)BRAX_NOALLOC_SCRATCH_BYTES - ws_bytes, stream);
}
