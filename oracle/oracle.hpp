// FP64 oracle of the batched rigid-body step (Brax, arXiv 2106.13281).
//
// TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct CPU
// statement of what the CUDA path computes.  It shares no code with the CUDA
// path; only the tests, the smoke check and the CPU baseline of the benchmark
// may build or call it.
//
// What it follows:
//   * State: per body position, orientation quaternion (w,x,y,z), velocity and
//     angular velocity - the QP primitive of Sec. 3.
//   * One substep is Algorithm 1 of Sec. 3, in its order: the kinematic
//     integrator; then joints, actuators and colliders, all evaluated on the
//     same post-kinematic state and summed ("collected in parallel"); then the
//     potential integrator with the joint + actuator updates; then the
//     collision integrator with the contact updates.
//   * A step is `substeps` substeps of length dt/substeps (Sec. 3, App. A).
//   * Joints are springs (Sec. 7.1 "Spring Joints"); contacts are
//     velocity-level with Baumgarte stabilisation and every listed pair is
//     tested every substep (Sec. 7.2 "Collisions").
// The paper prints no force law; every formula below that it does not fix is
// one of the readings listed in the design notes and is marked READING.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "scalars.hpp"

namespace orc {

// ============================================================ small algebra
template <class T> struct V3 {
  T x, y, z;
};
template <class T> struct Q4 {
  T w, x, y, z;
};
template <class T> struct M3 {
  T m[3][3];
};

template <class T> inline V3<T> mk(T x, T y, T z) { return V3<T>{x, y, z}; }
template <class T> inline V3<T> cst(const double* p) { return V3<T>{T(p[0]), T(p[1]), T(p[2])}; }
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a) { return {-a.x, -a.y, -a.z}; }
template <class T> inline V3<T> operator*(const T& s, const V3<T>& a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> inline T norm(const V3<T>& a) { return sqrt(dot(a, a)); }
// R * o for a constant body-frame vector o.
template <class T> inline V3<T> mulc(const M3<T>& R, const double* o) {
  return {R.m[0][0] * T(o[0]) + R.m[0][1] * T(o[1]) + R.m[0][2] * T(o[2]),
          R.m[1][0] * T(o[0]) + R.m[1][1] * T(o[1]) + R.m[1][2] * T(o[2]),
          R.m[2][0] * T(o[0]) + R.m[2][1] * T(o[1]) + R.m[2][2] * T(o[2])};
}
template <class T> inline V3<T> mul(const M3<T>& R, const V3<T>& o) {
  return {R.m[0][0] * o.x + R.m[0][1] * o.y + R.m[0][2] * o.z,
          R.m[1][0] * o.x + R.m[1][1] * o.y + R.m[1][2] * o.z,
          R.m[2][0] * o.x + R.m[2][1] * o.y + R.m[2][2] * o.z};
}
template <class T> inline V3<T> mulT(const M3<T>& R, const V3<T>& o) {
  return {R.m[0][0] * o.x + R.m[1][0] * o.y + R.m[2][0] * o.z,
          R.m[0][1] * o.x + R.m[1][1] * o.y + R.m[2][1] * o.z,
          R.m[0][2] * o.x + R.m[1][2] * o.y + R.m[2][2] * o.z};
}
// Hamilton product.
template <class T> inline Q4<T> qmul(const Q4<T>& a, const Q4<T>& b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
// Rotation matrix of a unit quaternion (body-to-world).
template <class T> inline M3<T> qmat(const Q4<T>& q) {
  T xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
  T xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
  T wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
  M3<T> R;
  R.m[0][0] = T(1.0) - T(2.0) * (yy + zz);
  R.m[0][1] = T(2.0) * (xy - wz);
  R.m[0][2] = T(2.0) * (xz + wy);
  R.m[1][0] = T(2.0) * (xy + wz);
  R.m[1][1] = T(1.0) - T(2.0) * (xx + zz);
  R.m[1][2] = T(2.0) * (yz - wx);
  R.m[2][0] = T(2.0) * (xz - wy);
  R.m[2][1] = T(2.0) * (yz + wx);
  R.m[2][2] = T(1.0) - T(2.0) * (xx + yy);
  return R;
}

// Double-precision constant helpers (scene geometry, not differentiated).
inline void cq_rotate(const double q[4], const double v[3], double out[3]) {
  // out = q v q^-1 for a unit quaternion q
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  for (int i = 0; i < 3; ++i) out[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
}
inline void cq_normalize(double q[4]) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] /= n;
}

// ============================================================ system
enum ColType { COL_PLANE = 0, COL_CAPSULE = 1, COL_BOX = 2 };

struct System {
  int B = 0, J = 0, A = 0, C = 0, P = 0, substeps = 1;
  double dt = 0.01, g[3] = {0, 0, 0}, baumgarte = 0.1, eps = 1e-6;
  bool average = true;
  // bodies
  std::vector<double> mass, inertia;     // [B], [B*3]
  std::vector<uint8_t> fpos, frot;       // [B*3], 1 = frozen
  std::vector<double> rest_pos, rest_rot;  // [B*3], [B*4]
  // joints
  std::vector<int> parent, child, dof;
  std::vector<double> off_p, off_c;      // [J*3]
  std::vector<double> axp, axc;          // [J*9]: joint frame axes (x,y,z) in parent / child body frame
  std::vector<double> frame_p, frame_c;  // [J*4]
  std::vector<double> k, c, ka, ca, kl;  // [J]
  std::vector<double> lo, hi;            // [J*3] radians
  // actuators
  std::vector<int> act_joint, act_axis;
  std::vector<double> gear;
  std::vector<int> act_type;  // [A] 0: torque, 1: target angle
  // variants of the potential integrator (0 / false: off)
  double lin_damp = 0.0, ang_damp = 0.0;
  bool gyro = false;
  // colliders
  std::vector<int> col_body, col_type;
  std::vector<double> col_pos, col_rot, radius, length, half, friction, elasticity;
  // pairs
  std::vector<int> pair_a, pair_b;
  // derived
  std::vector<int> joint_order;  // topological order (parents placed first)
  std::vector<int> is_child;     // [B]: 1 if body is the child of a joint
  int D = 0;                     // total joint DOF
  std::vector<int> dof_offset;   // [J]: first angle index of joint j

  double h() const { return dt / substeps; }
  bool any_frozen(int b) const {
    for (int i = 0; i < 3; ++i)
      if (fpos[3 * b + i] || frot[3 * b + i]) return true;
    return false;
  }
  // joint frame axis `a` (0=x,1=y,2=z) in the parent / child body frame
  const double* ap(int j, int a) const { return &axp[9 * j + 3 * a]; }
  const double* ac(int j, int a) const { return &axc[9 * j + 3 * a]; }

  void derive() {
    axp.assign(9 * J, 0.0);
    axc.assign(9 * J, 0.0);
    const double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int j = 0; j < J; ++j) {
      double fp[4], fc[4];
      for (int i = 0; i < 4; ++i) { fp[i] = frame_p[4 * j + i]; fc[i] = frame_c[4 * j + i]; }
      cq_normalize(fp);
      cq_normalize(fc);
      for (int a = 0; a < 3; ++a) {
        cq_rotate(fp, e[a], &axp[9 * j + 3 * a]);
        cq_rotate(fc, e[a], &axc[9 * j + 3 * a]);
      }
    }
    is_child.assign(B, 0);
    for (int j = 0; j < J; ++j) is_child[child[j]] = 1;
    std::vector<int> placed(B, 0);
    for (int b = 0; b < B; ++b) placed[b] = !is_child[b];
    joint_order.clear();
    std::vector<int> done(J, 0);
    for (int pass = 0; pass < J + 1; ++pass)
      for (int j = 0; j < J; ++j)
        if (!done[j] && placed[parent[j]]) {
          joint_order.push_back(j);
          done[j] = 1;
          placed[child[j]] = 1;
        }
    dof_offset.assign(J, 0);
    D = 0;
    for (int j = 0; j < J; ++j) { dof_offset[j] = D; D += dof[j]; }
  }
};

// Per-body state, the QP primitive of Sec. 3: 13 numbers per body.
template <class T> struct Body {
  V3<T> x;  // position of the centre of mass (world)
  Q4<T> q;  // orientation, body-to-world, (w,x,y,z)
  V3<T> v;  // linear velocity (world)
  V3<T> w;  // angular velocity (world)
};

template <class T> struct Frame {
  M3<T> R;   // rotation matrix of q
  M3<T> Ii;  // inverse inertia in world coordinates, R diag(1/I) R^T
};

struct Diag {
  int64_t active_contacts = 0;
  uint64_t branch_hash = 1469598103934665603ull;  // FNV-1a over every branch decision taken
  void branch(int code) {
    branch_hash ^= (uint64_t)(code + 1);
    branch_hash *= 1099511628211ull;
  }
};
inline thread_local Diag* tl_diag = nullptr;
inline void note_branch(int code) {
  if (tl_diag) tl_diag->branch(code);
}

inline void set_cat(int c) {
  if (tl_flops) tl_flops->cat = c;
}

// Frozen axes (App. A "frozen"): READING - a 1 freezes that world axis; the
// velocity component is held at zero at every write.
template <class T> inline V3<T> mask(const System& s, const uint8_t* f, const V3<T>& a) {
  (void)s;
  return {f[0] ? T(0.0) : a.x, f[1] ? T(0.0) : a.y, f[2] ? T(0.0) : a.z};
}

// ============================================================ kinematic integrator
// Sec. 3 / Algorithm 1 first line: positions and orientations advance with the
// current velocities.  x <- x + h v;  q <- normalize(q + h/2 (0, w) (x) q), with w
// the world-frame angular velocity (READING: Hamilton product, world frame on
// the left).
template <class T> inline void kinematic(const System& s, int b, Body<T>& qp) {
  const double h = s.h();
  qp.v = mask(s, &s.fpos[3 * b], qp.v);
  qp.w = mask(s, &s.frot[3 * b], qp.w);
  qp.x = qp.x + T(h) * qp.v;
  Q4<T> wq{T(0.0), qp.w.x, qp.w.y, qp.w.z};
  Q4<T> d = qmul(wq, qp.q);
  T hh(0.5 * h);
  Q4<T> q{qp.q.w + hh * d.w, qp.q.x + hh * d.x, qp.q.y + hh * d.y, qp.q.z + hh * d.z};
  T n = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  qp.q = Q4<T>{q.w / n, q.x / n, q.y / n, q.z / n};
}

template <class T> inline Frame<T> frame(const System& s, int b, const Body<T>& qp) {
  Frame<T> f;
  f.R = qmat(qp.q);
  T d[3] = {T(1.0 / s.inertia[3 * b + 0]), T(1.0 / s.inertia[3 * b + 1]), T(1.0 / s.inertia[3 * b + 2])};
  T A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) A[i][k] = f.R.m[i][k] * d[k];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      T v = A[i][0] * f.R.m[j][0] + A[i][1] * f.R.m[j][1] + A[i][2] * f.R.m[j][2];
      f.Ii.m[i][j] = v;
      f.Ii.m[j][i] = v;
    }
  return f;
}

// ============================================================ joints
// Sec. 3 (joint.revolute bundles a 1-DOF constraint between parent and child)
// and Sec. 7.1 (joints are springs).  READING: a linear spring-damper joins
// the two anchor points; a hinge additionally has an alignment spring between
// the hinge axes; an angular damper acts on the relative angular velocity;
// limits (App. A angle_limit, degrees) are one-sided linear springs on the
// joint angle.  Every term is equal and opposite on parent and child.
template <class T> struct Wrench {
  V3<T> F, tau;
};

// Joint angles measured in the parent's joint frame.  For a hinge: the angle
// of the child's joint-frame y axis about the parent's hinge axis.  For a
// 3-DOF joint: intrinsic X-Y-Z Euler angles of the relative rotation.
template <class T> inline void joint_angles(const System& s, int j, const Frame<T>& fp, const Frame<T>& fc, T* ang,
                                            V3<T>* P) {
  for (int a = 0; a < 3; ++a) P[a] = mulc(fp.R, s.ap(j, a));
  if (s.dof[j] == 1) {
    V3<T> yc = mulc(fc.R, s.ac(j, 1));
    ang[0] = atan2(dot(cross(P[1], yc), P[0]), dot(P[1], yc));
  } else {
    V3<T> C0 = mulc(fc.R, s.ac(j, 0)), C1 = mulc(fc.R, s.ac(j, 1)), C2 = mulc(fc.R, s.ac(j, 2));
    T m00 = dot(P[0], C0), m01 = dot(P[0], C1), m02 = dot(P[0], C2);
    T m12 = dot(P[1], C2), m22 = dot(P[2], C2);
    ang[0] = atan2(-m12, m22);
    ang[1] = atan2(m02, sqrt(m00 * m00 + m01 * m01));
    ang[2] = atan2(-m01, m00);
  }
}

template <class T> inline void joint_apply(const System& s, int j, const Body<T>* qp, const Frame<T>* fr,
                                           Wrench<T>* dp) {
  const int p = s.parent[j], c = s.child[j];
  const Body<T>& bp = qp[p];
  const Body<T>& bc = qp[c];
  // anchors and their velocities
  V3<T> rp = mulc(fr[p].R, &s.off_p[3 * j]);
  V3<T> rc = mulc(fr[c].R, &s.off_c[3 * j]);
  V3<T> pp = bp.x + rp, pc = bc.x + rc;
  V3<T> up = bp.v + cross(bp.w, rp), uc = bc.v + cross(bc.w, rc);
  // linear spring-damper: F on the child at its anchor, -F on the parent at its anchor
  V3<T> F = T(s.k[j]) * (pp - pc) - T(s.c[j]) * (uc - up);
  V3<T> tc = cross(rc, F);
  V3<T> tp = -cross(rp, F);
  T ang[3];
  V3<T> P[3];
  joint_angles(s, j, fr[p], fr[c], ang, P);
  // angular damper on the relative angular velocity: about the hinge axis for
  // a hinge, in full 3-D for a 3-DOF joint (READING)
  V3<T> wr = bc.w - bp.w;
  V3<T> td = (s.dof[j] == 1) ? (T(-s.ca[j]) * dot(wr, P[0])) * P[0] : T(-s.ca[j]) * wr;
  tc = tc + td;
  tp = tp - td;
  if (s.dof[j] == 1) {
    // hinge alignment spring, potential ka (1 - Ac.Ap)
    V3<T> Ac = mulc(fr[c].R, s.ac(j, 0));
    V3<T> ta = T(s.ka[j]) * cross(Ac, P[0]);
    tc = tc + ta;
    tp = tp - ta;
  }
  for (int a = 0; a < s.dof[j]; ++a) {
    const double lo = s.lo[3 * j + a], hi = s.hi[3 * j + a];
    T th = ang[a];
    T L(0.0);
    if (val(th) < lo) L = T(s.kl[j]) * (T(lo) - th);
    else if (val(th) > hi) L = T(s.kl[j]) * (T(hi) - th);
    note_branch(val(th) < lo ? 1 : (val(th) > hi ? 2 : 3));
    V3<T> tl = L * P[a];
    tc = tc + tl;
    tp = tp - tl;
  }
  if (s.dof[j] == 2) {
    // 2-DOF (universal) joint, READING: the twist about the third joint axis
    // is held at 0 by a spring of the alignment stiffness ka, as the hinge's
    // off-axis rotations are
    V3<T> tw = (T(-s.ka[j]) * ang[2]) * P[2];
    tc = tc + tw;
    tp = tp - tw;
  }
  dp[c].F = dp[c].F + F;
  dp[c].tau = dp[c].tau + tc;
  dp[p].F = dp[p].F - F;
  dp[p].tau = dp[p].tau + tp;
}

// ============================================================ actuators
// Sec. 3: actuators turn `actions` into torques.  READING: a torque actuator
// applies gear * clamp(a, -1, 1) about the joint's world axis, on the child
// and the opposite on the parent.
// Torque actuator: tau = gear clamp(a, -1, 1) about the joint axis.
// Target-angle actuator (Sec. 3: actions are "torques or target angles";
// READING): the action picks a target angle in the axis' limit range,
// theta* = (lo + hi)/2 + clamp(a, -1, 1) (hi - lo)/2, and the actuator is a
// spring of stiffness gear toward it, tau = gear (theta* - theta), about the
// same axis (the joint's angular damper damps it).
template <class T> inline void actuator_apply(const System& s, int k, const T* act, const Frame<T>* fr,
                                              Wrench<T>* dp) {
  const int j = s.act_joint[k];
  const int p = s.parent[j], c = s.child[j];
  const int axis = s.act_axis[k];
  V3<T> ax = mulc(fr[p].R, s.ap(j, axis));
  T a = vclamp(act[k], -1.0, 1.0);
  note_branch(40 + (val(act[k]) >= 1.0 ? 1 : (val(act[k]) <= -1.0 ? 2 : 0)));
  T mag = T(s.gear[k]) * a;
  if (!s.act_type.empty() && s.act_type[k] == 1) {
    T ang[3];
    V3<T> P[3];
    joint_angles(s, j, fr[p], fr[c], ang, P);
    const double lo = s.lo[3 * j + axis], hi = s.hi[3 * j + axis];
    T target = T(0.5 * (lo + hi)) + T(0.5 * (hi - lo)) * a;
    mag = T(s.gear[k]) * (target - ang[axis]);
  }
  V3<T> tau = mag * ax;
  dp[c].tau = dp[c].tau + tau;
  dp[p].tau = dp[p].tau - tau;
}

// ============================================================ colliders: detection
template <class T> struct Contact {
  V3<T> n;  // unit normal, pointing from body b toward body a
  V3<T> p;  // contact point (world)
  T depth;  // penetration depth (> 0 when active)
  int a, b;  // body receiving +J, body receiving -J (-1: static world)
  double mu, e;
};

// Closest points of two segments P1 + s d1 and P2 + t d2, s,t in [0,1]
// (the clamped minimisation in Ericson, Real-Time Collision Detection 5.1.9).
// READING: zero-length segments reduce to points; near-parallel segments
// (a e - b^2 <= 1e-5 a e) take s = 0.
template <class T> inline void segment_closest(const V3<T>& P1, const V3<T>& d1, const V3<T>& P2, const V3<T>& d2,
                                               T& s, T& t) {
  V3<T> r = P1 - P2;
  T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  const double tiny = 1e-12;
  if (val(a) <= tiny && val(e) <= tiny) {
    s = T(0.0);
    t = T(0.0);
    return;
  }
  if (val(a) <= tiny) {
    s = T(0.0);
    t = vclamp(f / e, 0.0, 1.0);
    return;
  }
  T cc = dot(d1, r);
  if (val(e) <= tiny) {
    t = T(0.0);
    s = vclamp(-cc / a, 0.0, 1.0);
    return;
  }
  T b = dot(d1, d2);
  T ae = a * e;
  T denom = ae - b * b;
  count_flop();  // the relative parallel test multiplies ae by a constant
  if (val(denom) > 1e-5 * val(ae)) s = vclamp((b * f - cc * e) / denom, 0.0, 1.0);
  else s = T(0.0);
  t = (b * s + f) / e;
  note_branch(60 + (val(t) < 0.0 ? 1 : (val(t) > 1.0 ? 2 : 0)) + (val(denom) > 1e-5 * val(ae) ? 4 : 0));
  if (val(t) < 0.0) {
    t = T(0.0);
    s = vclamp(-cc / a, 0.0, 1.0);
  } else if (val(t) > 1.0) {
    t = T(1.0);
    s = vclamp((b - cc) / a, 0.0, 1.0);
  }
  // which parameters ended on an end point of their segment (clamped)
  note_branch(100 + (val(s) == 0.0 ? 1 : 0) + (val(s) == 1.0 ? 2 : 0) + (val(t) == 0.0 ? 4 : 0) +
              (val(t) == 1.0 ? 8 : 0));
}

// Capsule geometry: `length` is the total tip-to-tip length (READING); the
// segment half length is max(length/2 - radius, 0), along the collider's z.
inline double capsule_half(const System& s, int c) { return std::max(0.5 * s.length[c] - s.radius[c], 0.0); }
inline void capsule_local(const System& s, int c, double e0[3], double e1[3]) {
  double ez[3] = {0, 0, 1}, ax[3];
  cq_rotate(&s.col_rot[4 * c], ez, ax);
  double hs = capsule_half(s, c);
  for (int i = 0; i < 3; ++i) {
    e0[i] = s.col_pos[3 * c + i] - hs * ax[i];
    e1[i] = s.col_pos[3 * c + i] + hs * ax[i];
  }
}
inline void plane_of(const System& s, int c, double p0[3], double n[3]) {
  double ez[3] = {0, 0, 1};
  cq_rotate(&s.col_rot[4 * c], ez, n);
  for (int i = 0; i < 3; ++i) p0[i] = s.col_pos[3 * c + i];
}

// Sphere (centre e, radius r) against a static plane.
template <class T> inline void sphere_plane(const V3<T>& e, double r, const double* p0, const double* n, int body,
                                            double mu, double el, std::vector<Contact<T>>& out) {
  V3<T> N = cst<T>(n);
  T dist = dot(e - cst<T>(p0), N);
  T depth = T(r) - dist;
  if (val(depth) > 0.0) out.push_back(Contact<T>{N, e - T(r) * N, depth, body, -1, mu, el});
}

// Exact minimiser of the squared distance from the segment Pl + t dl,
// t in [0, 1], to the axis-aligned box |x_i| <= he_i (box frame).
// READING: the squared distance is a convex piecewise quadratic in t whose
// pieces end where a coordinate crosses a face plane (t = (+-he_i - Pl_i) /
// dl_i).  Each piece is minimised in closed form (its stationary point,
// clamped to the piece) and the smallest value wins; where a piece is flat
// (no active coordinate, or the segment parallel to the active faces) its
// midpoint is taken.  The parameter is a value decision (zero derivative).
template <class T> inline double seg_box_param(const V3<T>& Pl, const V3<T>& dl, const double* he) {
  const double P[3] = {val(Pl.x), val(Pl.y), val(Pl.z)};
  const double D[3] = {val(dl.x), val(dl.y), val(dl.z)};
  // The search runs in plain doubles (its result carries no derivative); its
  // arithmetic is still counted: 7 flops per coordinate of one distance.
  auto d2 = [&](double t) {
    count_flop(21);
    double acc = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double e = P[i] + t * D[i];
      const double r = e - std::min(std::max(e, -he[i]), he[i]);
      acc += r * r;
    }
    return acc;
  };
  std::vector<double> knots = {0.0, 1.0};
  for (int i = 0; i < 3; ++i) {
    if (D[i] == 0.0) continue;
    for (double face : {-he[i], he[i]}) {
      const double t = (face - P[i]) / D[i];
      count_flop(2);
      if (t > 0.0 && t < 1.0) knots.push_back(t);
    }
  }
  std::sort(knots.begin(), knots.end());
  double best_t = 0.0, best = d2(0.0);
  for (size_t j = 0; j + 1 < knots.size(); ++j) {
    const double lo = knots[j], hi = knots[j + 1];
    if (!(hi > lo)) continue;
    const double mid = 0.5 * (lo + hi);
    count_flop(8);
    // On this piece d2(t) = A t^2 + 2 Bc t + const, from the coordinates outside the box.
    double A = 0.0, Bc = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double e = P[i] + mid * D[i];
      if (e > he[i]) {
        A += D[i] * D[i];
        Bc += D[i] * (P[i] - he[i]);
        count_flop(5);
      } else if (e < -he[i]) {
        A += D[i] * D[i];
        Bc += D[i] * (P[i] + he[i]);
        count_flop(5);
      }
    }
    count_flop(4);
    const double t = A > 0.0 ? std::min(std::max(-Bc / A, lo), hi) : mid;
    const double v = d2(t);
    if (v < best) {
      best = v;
      best_t = t;
    }
  }
  return best_t;
}

// Parameter of the segment point closest to the box centre (box frame),
// clamped to [0, 1]; a value decision (zero derivative).
template <class T> inline double seg_center_param(const V3<T>& Pl, const V3<T>& dl) {
  count_flop(14);
  const double dd = val(dl.x) * val(dl.x) + val(dl.y) * val(dl.y) + val(dl.z) * val(dl.z);
  if (!(dd > 0.0)) return 0.0;
  const double t = -(val(Pl.x) * val(dl.x) + val(Pl.y) * val(dl.y) + val(Pl.z) * val(dl.z)) / dd;
  return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

// Capsule (segment P + t d, radius r, body ba) against a box (centre cb,
// rotation Rb, half extents he, body bb).  READING: contact at the closest
// segment point; outside the box the normal is the separation direction, the
// contact point is midway between the capsule surface and the box point;
// when the segment meets the box, at the segment point closest to the box
// centre, with the normal of that point's face of least penetration.
template <class T> inline void capsule_box(const V3<T>& P, const V3<T>& d, double r, int ba, const V3<T>& cb,
                                           const M3<T>& Rb, const double* he, int bb, double mu, double el,
                                           std::vector<Contact<T>>& out) {
  V3<T> Pl = mulT(Rb, P - cb);
  V3<T> dl = mulT(Rb, d);
  double t = seg_box_param(Pl, dl, he);
  V3<T> el3 = Pl + T(t) * dl;
  T e[3] = {el3.x, el3.y, el3.z};
  T q[3], dv[3];
  for (int i = 0; i < 3; ++i) {
    q[i] = vclamp(e[i], -he[i], he[i]);
    dv[i] = e[i] - q[i];
  }
  T d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
  V3<T> nl, pl;
  T depth;
  const double eps = 1e-6;
  note_branch(val(d2) > eps * eps ? 80 : 81);
  if (val(d2) > eps * eps) {
    int pattern = 0;  // which box-frame coordinates were clamped to a face, and to which
    for (int i = 0; i < 3; ++i) pattern = 3 * pattern + (val(e[i]) >= he[i] ? 1 : (val(e[i]) <= -he[i] ? 2 : 0));
    note_branch(120 + pattern);
    T dist = sqrt(d2);
    nl = mk(dv[0] / dist, dv[1] / dist, dv[2] / dist);
    depth = T(r) - dist;
    V3<T> qv = mk(q[0], q[1], q[2]);
    pl = T(0.5) * ((el3 - T(r) * nl) + qv);
  } else {
    t = seg_center_param(Pl, dl);
    el3 = Pl + T(t) * dl;
    e[0] = el3.x;
    e[1] = el3.y;
    e[2] = el3.z;
    int k = 0;
    double best = 1e300;
    for (int i = 0; i < 3; ++i) {
      double pen = he[i] - std::fabs(val(e[i]));
      if (pen < best) { best = pen; k = i; }
    }
    double sg = val(e[k]) >= 0.0 ? 1.0 : -1.0;
    note_branch(50 + 2 * k + (sg > 0.0 ? 1 : 0));
    T pen = T(he[k]) - T(sg) * e[k];
    T z(0.0);
    nl = mk(k == 0 ? T(sg) : z, k == 1 ? T(sg) : z, k == 2 ? T(sg) : z);
    depth = T(r) + pen;
    pl = el3 + (T(0.5) * (pen - T(r))) * nl;
  }
  if (val(depth) > 0.0) out.push_back(Contact<T>{mul(Rb, nl), cb + mul(Rb, pl), depth, ba, bb, mu, el});
}

// Every listed pair, every substep (Sec. 7.2: naive pair enumeration).
template <class T> inline void detect(const System& s, const Body<T>* qp, const Frame<T>* fr,
                                      std::vector<Contact<T>>& out) {
  // World geometry of a collider, computed once per substep however many
  // pairs it is in (a property of the collider's body, not of the pair):
  // capsule end points P, Q (Q = P for a sphere); box axes Rb (body rotation
  // times collider rotation, as columns) and centre.
  const int C = s.C;
  std::vector<V3<T>> wP(C), wQ(C), wc(C);
  std::vector<M3<T>> wR(C);
  std::vector<char> have(C, 0);
  auto world = [&](int c) {
    if (have[c]) return;
    have[c] = 1;
    const int b = s.col_body[c];
    if (s.col_type[c] == COL_CAPSULE) {
      double e0[3], e1[3];
      capsule_local(s, c, e0, e1);
      wP[c] = qp[b].x + mulc(fr[b].R, e0);
      wQ[c] = capsule_half(s, c) > 0.0 ? qp[b].x + mulc(fr[b].R, e1) : wP[c];
    } else if (s.col_type[c] == COL_BOX) {
      double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0}, ez[3] = {0, 0, 1}, cx[3], cy[3], cz[3];
      cq_rotate(&s.col_rot[4 * c], ex, cx);
      cq_rotate(&s.col_rot[4 * c], ey, cy);
      cq_rotate(&s.col_rot[4 * c], ez, cz);
      V3<T> X = mulc(fr[b].R, cx), Y = mulc(fr[b].R, cy), Z = mulc(fr[b].R, cz);
      M3<T>& Rb = wR[c];
      Rb.m[0][0] = X.x; Rb.m[0][1] = Y.x; Rb.m[0][2] = Z.x;
      Rb.m[1][0] = X.y; Rb.m[1][1] = Y.y; Rb.m[1][2] = Z.y;
      Rb.m[2][0] = X.z; Rb.m[2][1] = Y.z; Rb.m[2][2] = Z.z;
      wc[c] = qp[b].x + mulc(fr[b].R, &s.col_pos[3 * c]);
    }
  };
  for (int k = 0; k < s.P; ++k) {
    int ca = s.pair_a[k], cbk = s.pair_b[k];
    // order: the static plane, if any, second; a box second against a capsule
    if (s.col_type[ca] == COL_PLANE || (s.col_type[ca] == COL_BOX && s.col_type[cbk] == COL_CAPSULE)) std::swap(ca, cbk);
    const int ta = s.col_type[ca], tb = s.col_type[cbk];
    const double mu = s.friction[ca] * s.friction[cbk];
    const double el = s.elasticity[ca] * s.elasticity[cbk];
    const int ba = s.col_body[ca], bb = s.col_body[cbk];
    if (tb == COL_PLANE) {
      double p0[3], n[3];
      plane_of(s, cbk, p0, n);
      if (ta == COL_CAPSULE) {
        world(ca);
        sphere_plane(wP[ca], s.radius[ca], p0, n, ba, mu, el, out);
        if (capsule_half(s, ca) > 0.0) sphere_plane(wQ[ca], s.radius[ca], p0, n, ba, mu, el, out);
      } else if (ta == COL_BOX) {
        const double* he = &s.half[3 * ca];
        for (int m = 0; m < 8; ++m) {
          double cl[3] = {(m & 1) ? he[0] : -he[0], (m & 2) ? he[1] : -he[1], (m & 4) ? he[2] : -he[2]};
          double cr[3], co[3];
          cq_rotate(&s.col_rot[4 * ca], cl, cr);
          for (int i = 0; i < 3; ++i) co[i] = s.col_pos[3 * ca + i] + cr[i];
          sphere_plane(qp[ba].x + mulc(fr[ba].R, co), 0.0, p0, n, ba, mu, el, out);
        }
      }
    } else if (ta == COL_CAPSULE && tb == COL_CAPSULE) {
      world(ca);
      world(cbk);
      const V3<T>& P1 = wP[ca];
      const V3<T>& P2 = wP[cbk];
      V3<T> d1 = wQ[ca] - P1, d2 = wQ[cbk] - P2;
      T sp, tp;
      segment_closest(P1, d1, P2, d2, sp, tp);
      V3<T> c1 = P1 + sp * d1, c2 = P2 + tp * d2;
      V3<T> df = c1 - c2;
      T dl = norm(df);
      if (val(dl) < s.eps) continue;
      T depth = T(s.radius[ca] + s.radius[cbk]) - dl;
      if (val(depth) <= 0.0) continue;
      V3<T> n = mk(df.x / dl, df.y / dl, df.z / dl);
      V3<T> p = T(0.5) * ((c1 - T(s.radius[ca]) * n) + (c2 + T(s.radius[cbk]) * n));
      out.push_back(Contact<T>{n, p, depth, ba, bb, mu, el});
    } else if (ta == COL_CAPSULE && tb == COL_BOX) {
      world(ca);
      world(cbk);
      capsule_box(wP[ca], wQ[ca] - wP[ca], s.radius[ca], ba, wc[cbk], wR[cbk], &s.half[3 * cbk], bb, mu, el, out);
    }
  }
}

// ============================================================ colliders: response
// Sec. 7.2: velocity-level update with Baumgarte stabilisation.  READING:
//   u_n target = max(beta depth / h, -e u_n);  j_n = max(0, (target - u_n)/k_n);
//   Coulomb friction j_t = min(|u_t|/k_t, mu j_n) against the sliding direction;
//   each body's velocity update is the mean over its active contacts.
template <class T> inline T eff_mass_term(const System& s, int b, const Frame<T>& f, const V3<T>& l, const V3<T>& dir) {
  // change of the contact-point velocity along dir per unit impulse along dir
  V3<T> dm = mask(s, &s.fpos[3 * b], dir);
  T lin = dot(dm, dir) / T(s.mass[b]);
  V3<T> ld = cross(l, dir);
  V3<T> om = mask(s, &s.frot[3 * b], mul(f.Ii, ld));
  return lin + dot(om, ld);
}

template <class T> struct Accum {
  V3<T> dv, dw;
  int n = 0;
};

template <class T> inline void respond(const System& s, const Contact<T>& ct, const Body<T>* qp, const Frame<T>* fr,
                                       Accum<T>* acc, Diag* dg) {
  const double h = s.h();
  const int a = ct.a, b = ct.b;
  V3<T> la = ct.p - qp[a].x;
  V3<T> u = qp[a].v + cross(qp[a].w, la);
  V3<T> lb{T(0.0), T(0.0), T(0.0)};
  if (b >= 0) {
    lb = ct.p - qp[b].x;
    u = u - (qp[b].v + cross(qp[b].w, lb));
  }
  T kn = eff_mass_term(s, a, fr[a], la, ct.n);
  if (b >= 0) kn = kn + eff_mass_term(s, b, fr[b], lb, ct.n);
  if (!(val(kn) > 0.0)) return;
  T un = dot(u, ct.n);
  T t_pen = T(s.baumgarte / h) * ct.depth;
  T t_rest = T(-ct.e) * un;
  const bool rest_wins = !(val(t_pen) > val(t_rest));
  T target = vmax(t_pen, t_rest);
  T jn = vmax((target - un) / kn, T(0.0));
  note_branch(10 + (val(jn) > 0.0 ? 1 : 0) + (rest_wins ? 2 : 0));
  V3<T> J = jn * ct.n;
  V3<T> ut = u - un * ct.n;
  T ut2 = dot(ut, ut);
  if (val(ut2) > s.eps * s.eps) {
    T utn = sqrt(ut2);
    V3<T> tt = mk(ut.x / utn, ut.y / utn, ut.z / utn);
    T kt = eff_mass_term(s, a, fr[a], la, tt);
    if (b >= 0) kt = kt + eff_mass_term(s, b, fr[b], lb, tt);
    T jt = vmin(utn / kt, T(ct.mu) * jn);
    note_branch(val(utn / kt) < val(T(ct.mu) * jn) ? 20 : 21);
    J = J - jt * tt;
  } else {
    note_branch(22);
  }
  acc[a].dv = acc[a].dv + mask(s, &s.fpos[3 * a], T(1.0 / s.mass[a]) * J);
  acc[a].dw = acc[a].dw + mask(s, &s.frot[3 * a], mul(fr[a].Ii, cross(la, J)));
  acc[a].n += 1;
  if (b >= 0) {
    acc[b].dv = acc[b].dv - mask(s, &s.fpos[3 * b], T(1.0 / s.mass[b]) * J);
    acc[b].dw = acc[b].dw - mask(s, &s.frot[3 * b], mul(fr[b].Ii, cross(lb, J)));
    acc[b].n += 1;
  }
  if (dg) dg->active_contacts += 1;
  note_branch(30 + ct.a * 64 + (ct.b + 1));
}

// ============================================================ one substep (Algorithm 1)
template <class T> void substep(const System& s, Body<T>* qp, const T* act, Diag* dg) {
  const int B = s.B;
  const double h = s.h();
  // kinematic integrator, then per-body frames
  set_cat(FC_BODY);
  for (int b = 0; b < B; ++b) kinematic(s, b, qp[b]);
  std::vector<Frame<T>> fr(B);
  for (int b = 0; b < B; ++b) fr[b] = frame(s, b, qp[b]);
  // joints and actuators: dp_j + dp_a, all from the same post-kinematic qp
  std::vector<Wrench<T>> dp(B);
  for (int b = 0; b < B; ++b) dp[b] = Wrench<T>{mk(T(0.0), T(0.0), T(0.0)), mk(T(0.0), T(0.0), T(0.0))};
  set_cat(FC_JOINT);
  for (int j = 0; j < s.J; ++j) joint_apply(s, j, qp, fr.data(), dp.data());
  set_cat(FC_ACT);
  for (int k = 0; k < s.A; ++k) actuator_apply(s, k, act, fr.data(), dp.data());
  // colliders: dp_c, from the same post-kinematic qp (velocities before the
  // potential update - Algorithm 1 applies colliders before that line)
  set_cat(FC_DETECT);
  std::vector<Contact<T>> contacts;
  detect(s, qp, fr.data(), contacts);
  set_cat(FC_RESPONSE);
  std::vector<Accum<T>> acc(B);
  for (int b = 0; b < B; ++b) acc[b] = Accum<T>{mk(T(0.0), T(0.0), T(0.0)), mk(T(0.0), T(0.0), T(0.0)), 0};
  for (const auto& ct : contacts) respond(s, ct, qp, fr.data(), acc.data(), dg);
  // potential integrator: v += h (F/m + g);  w += h I_w^-1 tau.  READING: by
  // default no gyroscopic term and no global damping.  Variants (Sec. 6's
  // conservation study and the usual engine options): global damping
  // v += h (... - lin_damp v), w += h (... - ang_damp w); the gyroscopic
  // torque -w x (I_w w), I_w = R diag(I) R^T, added to tau (Euler's equations
  // of a free rigid body in the world frame).
  set_cat(FC_INTEGRATE);
  for (int b = 0; b < B; ++b) {
    V3<T> a = T(1.0 / s.mass[b]) * dp[b].F + cst<T>(s.g);
    if (s.lin_damp != 0.0) a = a - T(s.lin_damp) * qp[b].v;
    V3<T> tau = dp[b].tau;
    if (s.gyro) {
      const M3<T>& R = fr[b].R;
      V3<T> wl = mulT(R, qp[b].w);
      V3<T> Lw = mul(R, mk(T(s.inertia[3 * b]) * wl.x, T(s.inertia[3 * b + 1]) * wl.y, T(s.inertia[3 * b + 2]) * wl.z));
      tau = tau - cross(qp[b].w, Lw);
    }
    V3<T> alpha = mul(fr[b].Ii, tau);
    if (s.ang_damp != 0.0) alpha = alpha - T(s.ang_damp) * qp[b].w;
    qp[b].v = mask(s, &s.fpos[3 * b], qp[b].v + T(h) * a);
    qp[b].w = mask(s, &s.frot[3 * b], qp[b].w + T(h) * alpha);
  }
  // collision integrator: mean contact update per body
  for (int b = 0; b < B; ++b) {
    if (acc[b].n == 0) continue;
    if (s.average && acc[b].n > 1) {
      T inv(1.0 / acc[b].n);
      qp[b].v = qp[b].v + inv * acc[b].dv;
      qp[b].w = qp[b].w + inv * acc[b].dw;
    } else {
      qp[b].v = qp[b].v + acc[b].dv;
      qp[b].w = qp[b].w + acc[b].dw;
    }
  }
  set_cat(FC_OTHER);
}

// One environment step: `substeps` substeps with the step's actions held.
template <class T> void step(const System& s, Body<T>* qp, const T* act, Diag* dg) {
  for (int i = 0; i < s.substeps; ++i) substep(s, qp, act, dg);
}

// ============================================================ default_qp (Sec. 4.1)
// Places every body of a joint tree in a valid joint configuration: walking
// the tree from its roots, R_c = R_p F_p Rot(angles) F_c^-1 and the child's
// anchor coincides with the parent's anchor.  Roots keep their rest pose;
// body 0 may be given its own pose.  Velocities are zero.
inline void dq_mul(const double* a, const double* b, double* o) {
  double r[4] = {a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3], a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                 a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1], a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]};
  for (int i = 0; i < 4; ++i) o[i] = r[i];
}
inline void default_qp(const System& s, const double* root_pos, const double* root_rot, const double* angles,
                       double* out /*[B*13]*/) {
  for (int b = 0; b < s.B; ++b) {
    double* o = out + 13 * b;
    for (int i = 0; i < 3; ++i) o[i] = s.rest_pos[3 * b + i];
    for (int i = 0; i < 4; ++i) o[3 + i] = s.rest_rot[4 * b + i];
    for (int i = 7; i < 13; ++i) o[i] = 0.0;
  }
  if (root_pos)
    for (int i = 0; i < 3; ++i) out[i] = root_pos[i];
  if (root_rot)
    for (int i = 0; i < 4; ++i) out[3 + i] = root_rot[i];
  for (int j : s.joint_order) {
    const int p = s.parent[j], c = s.child[j];
    double qp_[4], fp[4], fc[4], rel[4] = {1, 0, 0, 0};
    for (int i = 0; i < 4; ++i) { qp_[i] = out[13 * p + 3 + i]; fp[i] = s.frame_p[4 * j + i]; fc[i] = s.frame_c[4 * j + i]; }
    cq_normalize(qp_);
    cq_normalize(fp);
    cq_normalize(fc);
    for (int a = 0; a < s.dof[j]; ++a) {
      double th = angles ? angles[s.dof_offset[j] + a] : 0.0;
      double r[4] = {std::cos(0.5 * th), 0, 0, 0};
      r[1 + a] = std::sin(0.5 * th);
      dq_mul(rel, r, rel);
    }
    double fci[4] = {fc[0], -fc[1], -fc[2], -fc[3]};
    double qc[4];
    dq_mul(qp_, fp, qc);
    dq_mul(qc, rel, qc);
    dq_mul(qc, fci, qc);
    cq_normalize(qc);
    double rp[3], rc[3];
    cq_rotate(qp_, &s.off_p[3 * j], rp);
    cq_rotate(qc, &s.off_c[3 * j], rc);
    for (int i = 0; i < 3; ++i) out[13 * c + i] = out[13 * p + i] + rp[i] - rc[i];
    for (int i = 0; i < 4; ++i) out[13 * c + 3 + i] = qc[i];
  }
}

// ============================================================ diagnostics
// Energy: kinetic + joint spring potentials + limit potentials - m g.x
// (the quantities of the Sec. 6 conservation experiment).
inline double energy(const System& s, const Body<double>* qp) {
  std::vector<Frame<double>> fr(s.B);
  double E = 0.0;
  for (int b = 0; b < s.B; ++b) {
    fr[b] = frame(s, b, qp[b]);
    const M3<double>& R = fr[b].R;
    V3<double> wl = mulT(R, qp[b].w);
    E += 0.5 * s.mass[b] * dot(qp[b].v, qp[b].v);
    E += 0.5 * (s.inertia[3 * b] * wl.x * wl.x + s.inertia[3 * b + 1] * wl.y * wl.y + s.inertia[3 * b + 2] * wl.z * wl.z);
    E -= s.mass[b] * (s.g[0] * qp[b].x.x + s.g[1] * qp[b].x.y + s.g[2] * qp[b].x.z);
  }
  for (int j = 0; j < s.J; ++j) {
    const int p = s.parent[j], c = s.child[j];
    V3<double> pp = qp[p].x + mulc(fr[p].R, &s.off_p[3 * j]);
    V3<double> pc = qp[c].x + mulc(fr[c].R, &s.off_c[3 * j]);
    V3<double> d = pp - pc;
    E += 0.5 * s.k[j] * dot(d, d);
    double ang[3];
    V3<double> P[3];
    joint_angles(s, j, fr[p], fr[c], ang, P);
    if (s.dof[j] == 1) {
      V3<double> Ac = mulc(fr[c].R, s.ac(j, 0));
      E += s.ka[j] * (1.0 - dot(Ac, P[0]));
    }
    if (s.dof[j] == 2) E += 0.5 * s.ka[j] * ang[2] * ang[2];
    for (int a = 0; a < s.dof[j]; ++a) {
      double lo = s.lo[3 * j + a], hi = s.hi[3 * j + a], ex = 0.0;
      if (ang[a] < lo) ex = lo - ang[a];
      else if (ang[a] > hi) ex = ang[a] - hi;
      E += 0.5 * s.kl[j] * ex * ex;
    }
  }
  return E;
}

// Linear and angular momentum about the world origin.
inline void momentum(const System& s, const Body<double>* qp, double* out6) {
  for (int i = 0; i < 6; ++i) out6[i] = 0.0;
  for (int b = 0; b < s.B; ++b) {
    Frame<double> f = frame(s, b, qp[b]);
    const double m = s.mass[b];
    V3<double> p = m * qp[b].v;
    V3<double> wl = mulT(f.R, qp[b].w);
    V3<double> Lb = mul(f.R, mk(s.inertia[3 * b] * wl.x, s.inertia[3 * b + 1] * wl.y, s.inertia[3 * b + 2] * wl.z));
    V3<double> L = cross(qp[b].x, p) + Lb;
    out6[0] += p.x; out6[1] += p.y; out6[2] += p.z;
    out6[3] += L.x; out6[4] += L.y; out6[5] += L.z;
  }
}

}  // namespace orc
