// Device-side parameter layout of one system (host and device).
//
// brax_system_create flattens a validated descriptor into one blob:
//   SysP | BodyP[B] | PairP[P] | PlaneP[n_planes]
// which every thread block copies into shared memory before stepping.  All
// geometry is pre-resolved to what a body's warp needs: its inverse mass and
// inertia, its parent joint (a body is the child of at most one joint), its
// plane-contact points (capsule end spheres, box corners) and the body-body
// pairs it takes part in.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#include "../../include/brax.h"

namespace brax {

enum BodyFlags : uint32_t {
  kFrozenPos0 = 1u << 0,  // bits 0..2: frozen world position axes
  kFrozenRot0 = 1u << 3,  // bits 3..5: frozen world rotation axes
  kAnyFrozen = 1u << 6,
  kHasParent = 1u << 7,   // the body is the child of a joint
  kPublish = 1u << 8,     // other warps read this body's substep state
  kInPair = 1u << 9,      // the body takes part in a body-body pair
};

// A plane-contact point of a body: a sphere of radius r centred at o (body
// frame) tested against plane `plane`.  Capsules give their two end spheres
// (one when the segment has zero length), boxes their eight corners (r = 0).
struct PointP {
  float o[3];
  float r;
  float mu, e;
  int32_t plane;
  int32_t pad;
};

struct BodyP {
  float inv_mass;
  float inv_I[3];
  uint32_t flags;
  int32_t parent;  // parent body of the joint whose child this body is, -1 if none
  int32_t dof;     // 1 or 3
  int32_t joint;   // that joint's index
  float off_p[3], off_c[3];
  float ap[9];     // joint frame axes x, y, z in the parent's body frame
  float ac[9];     // joint frame axes x, y, z in this body's frame
  float k, c, ka, ca, kl;
  float lo[3], hi[3];  // radians
  int32_t act[3];      // actuator index per joint axis, -1 none
  float gear[3];
  // target-angle actuators (bit a: axis a's actuator drives the angle toward
  // act_mid[a] + clamp(action) act_half[a], the middle and half width of the
  // axis' limit range, with stiffness gear[a]); 0: all torque actuators
  int32_t act_angle;
  float act_mid[3], act_half[3];
  float I[3];          // principal inertia (the gyroscopic term)
  int32_t n_children;
  int32_t children[BRAX_MAX_CHILDREN];
  int32_t n_points;
  PointP pt[BRAX_MAX_POINTS];
  int32_t n_bpairs;
  int32_t bpair[BRAX_MAX_BODY_PAIRS];  // (pair index << 1) | side; side 0: +J (body a), 1: -J (body b)
  // default_qp: rest pose for roots
  float rest_pos[3];
  float rest_rot[4];
  float frame_p[4], frame_c[4];  // joint frame quaternions (normalised)
  int32_t dof_offset;            // first joint-angle index of the parent joint
  int32_t tree_slot;             // index among bodies with children (-1: none); names its two tree barriers
  // The body's collider in body-body pairs when it has exactly one (-1: none
  // or several): its world geometry is computed once per substep and
  // published (capsule: g0, g1 = segment end points; box: g0 = centre,
  // g1 = axes, row-major), instead of once per pair.
  int32_t gtype;  // -1, 0 capsule, 1 box
  float g0[3];
  float g1[9];
};

enum PairType : int32_t { kCapsuleCapsule = 0, kCapsuleBox = 1 };

// A body-body pair: capsule a (segment a0..a1 in body a's frame, radius ra)
// against capsule b (segment b0..b1, radius rb) or against box b (centre b0,
// half extents b1, axes bR columns, all in body b's frame).
struct PairP {
  int32_t type;
  int32_t ba, bb;
  int32_t geo;  // bit 0 / bit 1: body a's / body b's collider geometry is published by the body
  float mu, e;
  float ra, rb;
  float a0[3], a1[3];
  float b0[3], b1[3];
  float bR[9];
  // Broadphase: the two colliders' bounding spheres (centred at the capsule
  // segment's midpoint, at the box centre) are disjoint, so the pair cannot
  // touch, when the centres are more than sqrt(bound2) apart.  bound2 is the
  // square of the summed radii (half segment + r; |half extents|) with a
  // relative margin of 1e-4 and 1e-5 m, far above FP32 rounding.
  float bound2;
  // capsule a's segment midpoint offset from its start along its direction
  // (0.5) is implicit; for a box the centre is b0.
};

struct PlaneP {
  float p0[3];
  float n[3];
};

struct SysP {
  int32_t B, J, A, D, P, n_planes, substeps, average;
  float h, beta_h, eps;  // beta_h = baumgarte / h
  float lin_damp;        // global linear damping (1/s) of the potential integrator, 0: none
  float g[3];
  float ang_damp;        // global angular damping (1/s), 0: none
  int32_t general;   // 1: the system has a 3-DOF joint or a body-body pair
  int32_t paired;    // 1: the blob carries SysP2/BodyP2 (two environments per thread)
  int32_t pair_off;  // byte offset of SysP2 in the blob
  int32_t flat;      // 1: every plane's normal is the world z axis (plane contacts drop n's zero components)
  int32_t joint_order[BRAX_MAX_BODIES];  // child bodies in topological order (for default_qp)
  int32_t n_order;
  int32_t n_parents;  // bodies with at least one child
  int32_t gyro;       // 1: the potential integrator adds the gyroscopic torque -w x (I_w w)
  int32_t variants;   // 1: damping, gyroscopic term or target-angle actuators (general kernel only)
  int32_t iso;        // 1: every body's inertia is isotropic (I_w = I for every orientation)
};

// Two environments per thread (systems with hinge joints only and at most
// two plane-contact points per body).  The floating-point parameters a warp
// uses every substep, each duplicated into a (value, value) pair so that it
// is a ready operand of the packed FP32 instructions; appended to the blob.
// Negated copies (m*) let the kernel write a - b*c as one fused multiply-add:
// the packed instructions take no negated operand.
struct SysP2 {
  float2 h, mhh, beta_h, eps2;  // h, -h/2, baumgarte/h, contact_eps^2
  float2 g[3];
  float2 one, mone;             // (1, 1), (-1, -1)
  float2 hh;                    // h/2
};
struct PointP2 {
  float2 o[3];          // sphere centre, body frame
  float2 r, mr, mu, me; // radius, -radius, friction, -elasticity
  float2 n[3], p0[3];   // its plane's normal and a point on it
};
struct BodyP2 {
  float2 off_p[3], off_c[3];
  float2 ap[6], ac[6];  // joint frame x and y axes in the parent's / this body's frame
  float2 k, mc, ka, mca, kl, lo, hi, gear;  // mc = -c, mca = -ca
  float2 inv_mass, inv_I[3];
  PointP2 pt[2];
};

// Byte offsets inside the blob.
__host__ __device__ inline int blob_bodies_off() { return (int)sizeof(SysP); }
__host__ __device__ inline int blob_pairs_off(int B) { return blob_bodies_off() + B * (int)sizeof(BodyP); }
__host__ __device__ inline int blob_planes_off(int B, int P) { return blob_pairs_off(B) + P * (int)sizeof(PairP); }
__host__ __device__ inline int blob_bytes(int B, int P, int n_planes) {
  int b = blob_planes_off(B, P) + n_planes * (int)sizeof(PlaneP);
  return (b + 15) & ~15;
}
// The paired section (SysP2, BodyP2[B]) starts at blob_bytes(B, P, n_planes).
__host__ __device__ inline int blob_pair_bytes(int B) { return (int)sizeof(SysP2) + B * (int)sizeof(BodyP2); }

// Shared memory of one group of 32 environments (floats), after the blob.
constexpr int kPubFields = 36;    // x[3], R[9], v[3], w[3], Ii[6], pair geometry[12]: nine float4 per lane
constexpr int kReactFields = 8;   // F[3], tau[3], 2 pad: two float4 per lane
constexpr int kSlotFields = 8;    // J[3], p[3], active flag, pad: two float4 per lane
// Tree barriers (one group per block): parent slot k owns named barrier
// 2 + 2k (its published state, parent -> children) and 3 + 2k (its
// children's reactions, children -> parent); each counts the parent's warp and
// its children's warps.  Barrier 1 is the group barrier; 0 is __syncthreads.
__host__ __device__ inline bool tree_barriers_fit(int n_parents) { return 3 + 2 * n_parents <= 16; }

__host__ __device__ inline int group_floats(int B, int P) {
  return B * kPubFields * 32 + B * kReactFields * 32 + P * kSlotFields * 32 + 32;
}

}  // namespace brax
