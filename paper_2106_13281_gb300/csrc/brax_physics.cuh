// Forward physics of one substep for one (body, environment) thread.
//
// A group of 32 environments runs as B warps, warp b = body b, lane = env.
// One substep is Algorithm 1 (Sec. 3) split at two group barriers:
//   phase K  kinematic integrator of the own body, its frame, publish;
//   -- barrier --
//   phase J  the parent joint and its actuators (the own body is the joint's
//            child; the reaction on the parent goes to shared memory), the
//            own plane contacts, the body-body pairs this warp owns;
//   -- barrier --
//   phase P  sum the reactions of the children and the pair impulses,
//            potential integrator, collision integrator.
// Joints, actuators and contacts all read the same post-kinematic state and
// the velocities before the potential update (Algorithm 1 applies colliders
// before the potential integrator).
#pragma once
#include "brax_device.cuh"

namespace brax {

struct Body {
  V3 x;
  float qw, qx, qy, qz;
  V3 v, w;
};

struct Frame {
  M3 R;
  S6 Ii;
};

struct Wrench {
  V3 F, tau;
};

struct Acc {
  V3 dv, dw;
  int n;
};

// ------------------------------------------------------------------ state I/O (QP layout, 13 floats)
__device__ __forceinline__ void load_body(const float* p, Body& s) {
  s.x = mk3(p[0], p[1], p[2]);
  s.qw = p[3];
  s.qx = p[4];
  s.qy = p[5];
  s.qz = p[6];
  s.v = mk3(p[7], p[8], p[9]);
  s.w = mk3(p[10], p[11], p[12]);
}
// The same through L2 only: a chunk of a chunked rollout schedule starts from
// a state that a block on another SM stored, which this SM's L1 may hold an
// older copy of.
__device__ __forceinline__ void load_body_l2(const float* p, Body& s) {
  s.x = mk3(__ldcg(p + 0), __ldcg(p + 1), __ldcg(p + 2));
  s.qw = __ldcg(p + 3);
  s.qx = __ldcg(p + 4);
  s.qy = __ldcg(p + 5);
  s.qz = __ldcg(p + 6);
  s.v = mk3(__ldcg(p + 7), __ldcg(p + 8), __ldcg(p + 9));
  s.w = mk3(__ldcg(p + 10), __ldcg(p + 11), __ldcg(p + 12));
}
__device__ __forceinline__ void store_body(float* p, const Body& s) {
  p[0] = s.x.x;
  p[1] = s.x.y;
  p[2] = s.x.z;
  p[3] = s.qw;
  p[4] = s.qx;
  p[5] = s.qy;
  p[6] = s.qz;
  p[7] = s.v.x;
  p[8] = s.v.y;
  p[9] = s.v.z;
  p[10] = s.w.x;
  p[11] = s.w.y;
  p[12] = s.w.z;
}
__device__ __forceinline__ bool body_finite(const Body& s) {
  const float t = s.x.x + s.x.y + s.x.z + s.qw + s.qx + s.qy + s.qz + s.v.x + s.v.y + s.v.z + s.w.x + s.w.y + s.w.z;
  return fabsf(t) < INFINITY;
}

// ------------------------------------------------------------------ phase K
// Kinematic integrator (Algorithm 1, first line): x += h v;
// q <- normalize(q + h/2 (0, w) (x) q), w in world frame.  Frozen axes hold
// zero velocity.
__device__ __forceinline__ void kinematic(const BodyP& bp, float h, Body& s) {
  if (bp.flags & kAnyFrozen) {
    s.v = mask3(bp.flags, s.v);
    s.w = mask3(bp.flags >> 3, s.w);
  }
  s.x = fma3(h, s.v, s.x);
  const float hh = 0.5f * h;
  const float nw = fmaf(-hh, fmaf(s.w.x, s.qx, fmaf(s.w.y, s.qy, s.w.z * s.qz)), s.qw);
  const float nx = fmaf(hh, fmaf(s.qw, s.w.x, fmaf(s.w.y, s.qz, -s.w.z * s.qy)), s.qx);
  const float ny = fmaf(hh, fmaf(s.qw, s.w.y, fmaf(s.w.z, s.qx, -s.w.x * s.qz)), s.qy);
  const float nz = fmaf(hh, fmaf(s.qw, s.w.z, fmaf(s.w.x, s.qy, -s.w.y * s.qx)), s.qz);
  const float inv = rsqrtf(fmaf(nw, nw, fmaf(nx, nx, fmaf(ny, ny, nz * nz))));
  s.qw = nw * inv;
  s.qx = nx * inv;
  s.qy = ny * inv;
  s.qz = nz * inv;
}

__device__ __forceinline__ Frame make_frame(const BodyP& bp, const Body& s) {
  Frame f;
  f.R = qmat(s.qw, s.qx, s.qy, s.qz);
  f.Ii = inv_inertia_world(f.R, bp.inv_I);
  return f;
}

// World geometry of a body's pair collider (the expressions pair_forward
// and pair_bwd use): capsule segment start P and direction d; box axes Rb
// (row-major, R_body * R_collider) and centre cb.
__device__ __forceinline__ void capsule_world(const M3& R, V3 x, const float* e0, const float* e1, V3& P, V3& d) {
  P = x + mulc(R, e0);
  d = mulc(R, e1) - mulc(R, e0);
}
__device__ __forceinline__ void box_world(const M3& R, V3 x, const float* c0, const float* bR, M3& Rb, V3& cb) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rb.m[3 * i + j] = fmaf(R.m[3 * i + 0], bR[0 * 3 + j], fmaf(R.m[3 * i + 1], bR[1 * 3 + j], R.m[3 * i + 2] * bR[2 * 3 + j]));
  cb = x + mulc(R, c0);
}

template <bool kIi>
__device__ __forceinline__ void publish(GroupMem& gm, int b, int lane, const Body& s, const Frame& f,
                                        const BodyP& bp) {
  float4* p = gm.pub4(b, 0) + lane;
  p[0] = make_float4(s.x.x, s.x.y, s.x.z, f.R.m[0]);
  p[32] = make_float4(f.R.m[1], f.R.m[2], f.R.m[3], f.R.m[4]);
  p[64] = make_float4(f.R.m[5], f.R.m[6], f.R.m[7], f.R.m[8]);
  p[96] = make_float4(s.v.x, s.v.y, s.v.z, s.w.x);
  if (kIi) {
    p[128] = make_float4(s.w.y, s.w.z, f.Ii.a[0], f.Ii.a[1]);
    p[160] = make_float4(f.Ii.a[2], f.Ii.a[3], f.Ii.a[4], f.Ii.a[5]);
    if (bp.gtype == 0) {
      V3 P, d;
      capsule_world(f.R, s.x, bp.g0, bp.g1, P, d);
      p[192] = make_float4(P.x, P.y, P.z, d.x);
      st2(p + 224, d.y, d.z);
    } else if (bp.gtype == 1) {
      M3 Rb;
      V3 cb;
      box_world(f.R, s.x, bp.g0, bp.g1, Rb, cb);
      p[192] = make_float4(cb.x, cb.y, cb.z, Rb.m[0]);
      p[224] = make_float4(Rb.m[1], Rb.m[2], Rb.m[3], Rb.m[4]);
      p[256] = make_float4(Rb.m[5], Rb.m[6], Rb.m[7], Rb.m[8]);
    }
  } else {
    st2(p + 128, s.w.y, s.w.z);
  }
}
__device__ __forceinline__ void read_capsule_world(GroupMem& gm, int b, int lane, V3& P, V3& d) {
  const float4* p = gm.pub4(b, 6) + lane;
  const float4 c0 = p[0];
  const float2 c1 = ld2(p + 32);
  P = mk3(c0.x, c0.y, c0.z);
  d = mk3(c0.w, c1.x, c1.y);
}
__device__ __forceinline__ void read_box_world(GroupMem& gm, int b, int lane, M3& Rb, V3& cb) {
  const float4* p = gm.pub4(b, 6) + lane;
  const float4 c0 = p[0], c1 = p[32], c2 = p[64];
  cb = mk3(c0.x, c0.y, c0.z);
  Rb.m[0] = c0.w;
  Rb.m[1] = c1.x;
  Rb.m[2] = c1.y;
  Rb.m[3] = c1.z;
  Rb.m[4] = c1.w;
  Rb.m[5] = c2.x;
  Rb.m[6] = c2.y;
  Rb.m[7] = c2.z;
  Rb.m[8] = c2.w;
}

struct Pub {
  V3 x;
  M3 R;
  V3 v, w;
};
__device__ __forceinline__ Pub read_pub(GroupMem& gm, int b, int lane) {
  const float4* p = gm.pub4(b, 0) + lane;
  const float4 c0 = p[0], c1 = p[32], c2 = p[64], c3 = p[96];
  const float2 c4 = ld2(p + 128);
  Pub o;
  o.x = mk3(c0.x, c0.y, c0.z);
  o.R.m[0] = c0.w;
  o.R.m[1] = c1.x;
  o.R.m[2] = c1.y;
  o.R.m[3] = c1.z;
  o.R.m[4] = c1.w;
  o.R.m[5] = c2.x;
  o.R.m[6] = c2.y;
  o.R.m[7] = c2.z;
  o.R.m[8] = c2.w;
  o.v = mk3(c3.x, c3.y, c3.z);
  o.w = mk3(c3.w, c4.x, c4.y);
  return o;
}
__device__ __forceinline__ S6 read_pub_Ii(GroupMem& gm, int b, int lane) {
  const float4* p = gm.pub4(b, 4) + lane;
  const float2 a = ld2hi(p);
  const float4 c = p[32];
  S6 s;
  s.a[0] = a.x;
  s.a[1] = a.y;
  s.a[2] = c.x;
  s.a[3] = c.y;
  s.a[4] = c.z;
  s.a[5] = c.w;
  return s;
}

// ------------------------------------------------------------------ register-resident parameters
// The hinge parameters and the first two plane-contact points of a warp's
// body, copied into registers once per launch.  The copy goes through an
// opaque move so the compiler keeps the values in registers instead of
// reloading them from the constant pool every substep.
__device__ __forceinline__ float keep(float x) {
  float y;
  asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
struct HingeRegs {
  float off_p[3], off_c[3], ap[6], ac[6];
  float k, c, ka, ca, kl;
  float lo[1], hi[1], gear[1];
  int act[1];
  int dof;
  // systems with target-angle actuators run the general kernel (BodyP)
  static constexpr int act_angle = 0;
  float act_mid[1], act_half[1];
};
__device__ __forceinline__ HingeRegs hinge_regs(const BodyP& bp) {
  HingeRegs r;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.off_p[i] = keep(bp.off_p[i]);
    r.off_c[i] = keep(bp.off_c[i]);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    r.ap[i] = keep(bp.ap[i]);
    r.ac[i] = keep(bp.ac[i]);
  }
  r.k = keep(bp.k);
  r.c = keep(bp.c);
  r.ka = keep(bp.ka);
  r.ca = keep(bp.ca);
  r.kl = keep(bp.kl);
  r.lo[0] = keep(bp.lo[0]);
  r.hi[0] = keep(bp.hi[0]);
  r.gear[0] = keep(bp.gear[0]);
  r.act[0] = bp.act[0];
  r.dof = 1;
  return r;
}
struct PointRegs {
  float o[3];
  float r, mu, e;
};
__device__ __forceinline__ PointRegs point_regs(const PointP& p) {
  PointRegs r;
  r.o[0] = keep(p.o[0]);
  r.o[1] = keep(p.o[1]);
  r.o[2] = keep(p.o[2]);
  r.r = keep(p.r);
  r.mu = p.mu;
  r.e = p.e;
  return r;
}

// ------------------------------------------------------------------ phase J: joint
// Spring joint (Sec. 3 joint.revolute, Sec. 7.1): anchor spring-damper F on
// the child at its anchor and -F on the parent at its anchor; hinge-axis
// alignment spring; angular damper (hinge: about the axis, 3-DOF: 3-D);
// one-sided limit springs on the joint angles (App. A angle_limit); torque
// actuators gear * clamp(a, -1, 1) about the joint axes (Sec. 3).  Returns
// the child's wrench; writes the parent's to the react buffer.
template <bool kGeneral, class JP>
__device__ __forceinline__ Wrench joint_forward(const JP& bp, const Pub& pp, const Body& s, const Frame& f,
                                                const float* act, float4* react_out /* react4(b,0)+lane */) {
  const V3 rp = mulc(pp.R, bp.off_p);
  const V3 rc = mulc(f.R, bp.off_c);
  const V3 dpc = (pp.x + rp) - (s.x + rc);
  const V3 up = cross_add(pp.w, rp, pp.v);
  const V3 uc = cross_add(s.w, rc, s.v);
  const V3 F = bp.k * dpc - bp.c * (uc - up);
  V3 tc = cross(rc, F);
  V3 tp = cross(F, rp);
  const V3 P0 = mulc(pp.R, bp.ap + 0);
  const V3 P1 = mulc(pp.R, bp.ap + 3);
  const V3 wr = s.w - pp.w;
  V3 tj;
  if (!kGeneral || bp.dof == 1) {
    const V3 Ac = mulc(f.R, bp.ac + 0);
    const V3 yc = mulc(f.R, bp.ac + 3);
    const float th = fast_atan2(dot(cross(P1, yc), P0), dot(P1, yc));
    float L = 0.f;
    if (th < bp.lo[0]) L = bp.kl * (bp.lo[0] - th);
    else if (th > bp.hi[0]) L = bp.kl * (bp.hi[0] - th);
    float sc = L - bp.ca * dot(wr, P0);
    if (bp.act[0] >= 0) {
      if (bp.act_angle & 1)  // target-angle actuator: a spring toward the picked angle
        sc = fmaf(bp.gear[0], fmaf(bp.act_half[0], clamp1(act[0]), bp.act_mid[0]) - th, sc);
      else
        sc = fmaf(bp.gear[0], clamp1(act[0]), sc);
    }
    tj = fma3(sc, P0, bp.ka * cross(Ac, P0));
  } else {
    const V3 P2 = mulc(pp.R, bp.ap + 6);
    const V3 C0 = mulc(f.R, bp.ac + 0);
    const V3 C1 = mulc(f.R, bp.ac + 3);
    const V3 C2 = mulc(f.R, bp.ac + 6);
    const float m00 = dot(P0, C0), m01 = dot(P0, C1), m02 = dot(P0, C2);
    const float m12 = dot(P1, C2), m22 = dot(P2, C2);
    float th[3];
    th[0] = fast_atan2(-m12, m22);
    th[1] = fast_atan2(m02, sqrtf(fmaf(m00, m00, m01 * m01)));
    th[2] = fast_atan2(-m01, m00);
    tj = -bp.ca * wr;
    const V3 Pk[3] = {P0, P1, P2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float L = 0.f;
      if (th[a] < bp.lo[a]) L = bp.kl * (bp.lo[a] - th[a]);
      else if (th[a] > bp.hi[a]) L = bp.kl * (bp.hi[a] - th[a]);
      // 2-DOF (universal) joint: the twist about the third axis is held at 0
      // by a spring of the alignment stiffness (its limits never fire)
      if (a == 2 && bp.dof == 2) L = -bp.ka * th[2];
      if (bp.act[a] >= 0) {
        if (bp.act_angle & (1 << a))
          L = fmaf(bp.gear[a], fmaf(bp.act_half[a], clamp1(act[a]), bp.act_mid[a]) - th[a], L);
        else
          L = fmaf(bp.gear[a], clamp1(act[a]), L);
      }
      tj = fma3(L, Pk[a], tj);
    }
  }
  tc = tc + tj;
  tp = tp - tj;
  react_out[0] = make_float4(-F.x, -F.y, -F.z, tp.x);
  st2(react_out + 32, tp.y, tp.z);
  return Wrench{F, tc};
}

// ------------------------------------------------------------------ phase J: contacts
// Velocity change at a body's contact point along `dir` per unit impulse
// along `dir` (frozen axes excluded).
__device__ __forceinline__ float eff_mass(uint32_t flags, float inv_m, const S6& Ii, V3 l, V3 dir) {
  V3 dm = dir;
  V3 ld = cross(l, dir);
  V3 om = mul(Ii, ld);
  if (flags & kAnyFrozen) {
    dm = mask3(flags, dm);
    om = mask3(flags >> 3, om);
  }
  return fmaf(dot(dm, dir), inv_m, dot(om, ld));
}

// Velocity-level contact with Baumgarte stabilisation (Sec. 7.2): normal
// impulse toward the target max(beta depth / h, -e u_n), Coulomb friction
// against the sliding direction.  u is the relative contact velocity (a - b),
// k_n/k_t the summed effective inverse masses.  Returns the impulse on a.
struct Eff {
  uint32_t flags;
  float inv_m;
};

// Velocity-level response of one contact of the own body against a static
// plane: l is the contact point relative to the centre of mass, n the plane
// normal, depth > 0 the penetration.
__device__ __forceinline__ void point_response(const SysP& S, const BodyP& bp, V3 l, V3 n, float depth, float mu,
                                               float e, const Body& s, const Frame& f, Acc& acc) {
  const V3 u = cross_add(s.w, l, s.v);
  const float kn = eff_mass(bp.flags, bp.inv_mass, f.Ii, l, n);
  if (!(kn > 0.f)) return;
  const float un = dot(u, n);
  const float target = fmaxf(S.beta_h * depth, -e * un);
  const float jn = fmaxf(__fdividef(target - un, kn), 0.f);
  V3 J = jn * n;
  const V3 ut = fma3(-un, n, u);
  const float ut2 = dot(ut, ut);
  if (ut2 > S.eps * S.eps) {
    const float rinv = rsqrtf(ut2);
    const float utn = ut2 * rinv;
    const V3 t = rinv * ut;
    const float kt = eff_mass(bp.flags, bp.inv_mass, f.Ii, l, t);
    const float jt = fminf(__fdividef(utn, kt), mu * jn);
    J = fma3(-jt, t, J);
  }
  V3 dv = bp.inv_mass * J;
  V3 dw = mul(f.Ii, cross(l, J));
  if (bp.flags & kAnyFrozen) {
    dv = mask3(bp.flags, dv);
    dw = mask3(bp.flags >> 3, dw);
  }
  acc.dv = acc.dv + dv;
  acc.dw = acc.dw + dw;
  acc.n += 1;
}

// Plane contact of the own body: sphere (centre R o + x, radius r).
template <class PT>
__device__ __forceinline__ void plane_point(const SysP& S, const BodyP& bp, const PT& pt, const PlaneP& pl,
                                            const Body& s, const Frame& f, Acc& acc) {
  const V3 ro = mulc(f.R, pt.o);
  const V3 n = ld3(pl.n);
  const float dist = dot((s.x + ro) - ld3(pl.p0), n);
  const float depth = pt.r - dist;
  if (!(depth > 0.f)) return;
  point_response(S, bp, fma3(-pt.r, n, ro), n, depth, pt.mu, pt.e, s, f, acc);
}

// Up to two register-resident contact points of the own body.  Both are
// detected; then each lane handles its active points in order, so the warp
// runs the response as many times as the largest per-lane active count
// (a warp whose lanes touch the plane at different points runs it once).
__device__ __forceinline__ void plane_points_regs(const SysP& S, const BodyP& bp, const PointRegs* pr,
                                                  const PlaneP* planes, int np, const Body& s, const Frame& f,
                                                  Acc& acc) {
  if (np <= 0) return;
  const PlaneP& pl0 = planes[bp.pt[0].plane];
  const V3 n0 = ld3(pl0.n);
  const V3 ro0 = mulc(f.R, pr[0].o);
  const float dep0 = pr[0].r - dot((s.x + ro0) - ld3(pl0.p0), n0);
  V3 n1 = n0, ro1 = ro0;
  float dep1 = -1.f;
  if (np > 1) {
    const PlaneP& pl1 = planes[bp.pt[1].plane];
    n1 = ld3(pl1.n);
    ro1 = mulc(f.R, pr[1].o);
    dep1 = pr[1].r - dot((s.x + ro1) - ld3(pl1.p0), n1);
  }
  const bool a0 = dep0 > 0.f, a1 = dep1 > 0.f;
  const int cnt = (int)a0 + (int)a1;
  const int maxc = __reduce_max_sync(0xffffffffu, cnt);
  for (int it = 0; it < maxc; ++it) {
    if (it < cnt) {
      const bool p1 = it > 0 || !a0;
      const V3 n = p1 ? n1 : n0;
      const V3 ro = p1 ? ro1 : ro0;
      const float r = p1 ? pr[1].r : pr[0].r;
      const float depth = p1 ? dep1 : dep0;
      const float mu = p1 ? pr[1].mu : pr[0].mu;
      const float e = p1 ? pr[1].e : pr[0].e;
      point_response(S, bp, fma3(-r, n, ro), n, depth, mu, e, s, f, acc);
    }
  }
}

// Closest points of segments P1 + s d1 and P2 + t d2 (s, t in [0, 1]);
// zero-length segments reduce to points, near-parallel ones take s = 0.
__device__ __forceinline__ void segment_closest(V3 P1, V3 d1, V3 P2, V3 d2, float& s, float& t) {
  const V3 r = P1 - P2;
  const float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  const float tiny = 1e-12f;
  if (a <= tiny && e <= tiny) {
    s = 0.f;
    t = 0.f;
    return;
  }
  if (a <= tiny) {
    s = 0.f;
    t = fminf(fmaxf(__fdividef(f, e), 0.f), 1.f);
    return;
  }
  const float c = dot(d1, r);
  if (e <= tiny) {
    t = 0.f;
    s = fminf(fmaxf(__fdividef(-c, a), 0.f), 1.f);
    return;
  }
  const float b = dot(d1, d2);
  const float ae = a * e;
  const float denom = ae - b * b;
  s = (denom > 1e-5f * ae) ? fminf(fmaxf(__fdividef(fmaf(b, f, -c * e), denom), 0.f), 1.f) : 0.f;
  t = __fdividef(fmaf(b, s, f), e);
  if (t < 0.f) {
    t = 0.f;
    s = fminf(fmaxf(__fdividef(-c, a), 0.f), 1.f);
  } else if (t > 1.f) {
    t = 1.f;
    s = fminf(fmaxf(__fdividef(b - c, a), 0.f), 1.f);
  }
}

// Parameter of the segment point closest to the box centre, clamped to
// [0, 1]; used when the segment meets the box.  A value decision (no
// derivative flows through it).
__device__ __forceinline__ float seg_center_param(V3 Pl, V3 dl) {
  const float dd = dot(dl, dl);
  if (!(dd > 0.f)) return 0.f;
  return fminf(fmaxf(-__fdividef(dot(Pl, dl), dd), 0.f), 1.f);
}

// Half the derivative in t of the squared distance from the point e(t) of
// the segment (direction dl) to the box: sum_i dl_i (e_i - clamp(e_i)).
__device__ __forceinline__ float box_dist_slope(V3 e, V3 dl, const float* he) {
  const float rx = e.x - fminf(fmaxf(e.x, -he[0]), he[0]);
  const float ry = e.y - fminf(fmaxf(e.y, -he[1]), he[1]);
  const float rz = e.z - fminf(fmaxf(e.z, -he[2]), he[2]);
  return fmaf(dl.x, rx, fmaf(dl.y, ry, dl.z * rz));
}

// Exact minimiser over t in [0, 1] of the squared distance from Pl + t dl to
// the box (box frame).  The squared distance is convex and C1 with a
// piecewise-linear, non-decreasing slope whose kinks are the face-plane
// crossings t = (+-he_i - Pl_i) / dl_i.  The root of the slope is bracketed
// by the kinks (each kink inside the current bracket replaces the end whose
// slope sign it shares) and, with no kink left inside, found by linear
// interpolation.  A value decision (no derivative flows through it).
__device__ __forceinline__ float seg_box_param(V3 Pl, V3 dl, const float* he) {
  float gl = box_dist_slope(Pl, dl, he);
  if (gl >= 0.f) return 0.f;
  float gr = box_dist_slope(Pl + dl, dl, he);
  if (gr <= 0.f) return 1.f;
  float tl = 0.f, tr = 1.f;
  const float P[3] = {Pl.x, Pl.y, Pl.z}, D[3] = {dl.x, dl.y, dl.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (D[i] == 0.f) continue;
    const float inv = 1.f / D[i];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const float t = ((side ? he[i] : -he[i]) - P[i]) * inv;
      if (t > tl && t < tr) {
        const float g = box_dist_slope(fma3(t, dl, Pl), dl, he);
        if (g == 0.f) return t;
        if (g < 0.f) {
          tl = t;
          gl = g;
        } else {
          tr = t;
          gr = g;
        }
      }
    }
  }
  return fmaf(tr - tl, __fdividef(gl, gl - gr), tl);
}

// Detect one body-body pair; on contact compute the impulse on body a and
// write (J, p, 1) to the pair's slot, else (0, 0, 0).
__device__ __forceinline__ int pair_forward(const SysP& S, const BodyP* bodies, const PairP& pr, GroupMem& gm,
                                            int k, int lane) {
  // detection needs only the colliders' world geometry: published by the
  // bodies (computed once per substep), else computed here
  V3 P1, d1;
  if (pr.geo & 1) {
    read_capsule_world(gm, pr.ba, lane, P1, d1);
  } else {
    const Pub A = read_pub(gm, pr.ba, lane);
    capsule_world(A.R, A.x, pr.a0, pr.a1, P1, d1);
  }
  V3 n, p;
  float depth;
  bool hit = false;
  if (pr.type == kCapsuleCapsule) {
    V3 P2, d2;
    if (pr.geo & 2) {
      read_capsule_world(gm, pr.bb, lane, P2, d2);
    } else {
      const Pub Bq = read_pub(gm, pr.bb, lane);
      capsule_world(Bq.R, Bq.x, pr.b0, pr.b1, P2, d2);
    }
    // broadphase (Sec. 7.2's future work): disjoint bounding spheres cannot
    // touch; when no environment of the warp needs the narrow phase, skip it
    // (an environment that does not need it would find no contact there)
    const V3 dm = fma3(0.5f, d1, P1) - fma3(0.5f, d2, P2);
    if (__all_sync(0xffffffffu, dot(dm, dm) > pr.bound2)) {
      float4* sl = gm.slot4(k, 0) + lane;
      sl[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      sl[32] = make_float4(0.f, 0.f, 0.f, 0.f);
      return 0;
    }
    float sp, tp;
    segment_closest(P1, d1, P2, d2, sp, tp);
    const V3 c1 = fma3(sp, d1, P1), c2 = fma3(tp, d2, P2);
    const V3 df = c1 - c2;
    const float dl2 = dot(df, df);
    const float dl = sqrtf(dl2);
    depth = pr.ra + pr.rb - dl;
    if (dl >= S.eps && depth > 0.f) {
      const float inv = __fdividef(1.f, dl);
      n = inv * df;
      p = 0.5f * (fma3(-pr.ra, n, c1) + fma3(pr.rb, n, c2));
      hit = true;
    }
  } else {
    // box frame: rotation Rb = R_b * bR, centre cb
    M3 Rb;
    V3 cb;
    if (pr.geo & 2) {
      read_box_world(gm, pr.bb, lane, Rb, cb);
    } else {
      const Pub Bq = read_pub(gm, pr.bb, lane);
      box_world(Bq.R, Bq.x, pr.b0, pr.bR, Rb, cb);
    }
    const V3 dm = fma3(0.5f, d1, P1) - cb;  // broadphase, as for two capsules
    if (__all_sync(0xffffffffu, dot(dm, dm) > pr.bound2)) {
      float4* sl = gm.slot4(k, 0) + lane;
      sl[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      sl[32] = make_float4(0.f, 0.f, 0.f, 0.f);
      return 0;
    }
    const V3 Pl = mulT(Rb, P1 - cb);
    const V3 dl = mulT(Rb, d1);
    const float* he = pr.b1;
    float t = seg_box_param(Pl, dl, he);
    V3 e = fma3(t, dl, Pl);
    const V3 q = mk3(fminf(fmaxf(e.x, -he[0]), he[0]), fminf(fmaxf(e.y, -he[1]), he[1]),
                     fminf(fmaxf(e.z, -he[2]), he[2]));
    const V3 dv = e - q;
    const float d2 = dot(dv, dv);
    V3 nl, pl;
    if (d2 > 1e-12f) {
      const float dist = sqrtf(d2);
      const float inv = __fdividef(1.f, dist);
      nl = inv * dv;
      depth = pr.ra - dist;
      pl = 0.5f * (fma3(-pr.ra, nl, e) + q);
    } else {
      t = seg_center_param(Pl, dl);
      e = fma3(t, dl, Pl);
      const float px = he[0] - fabsf(e.x), py = he[1] - fabsf(e.y), pz = he[2] - fabsf(e.z);
      int kk = 0;
      float pen = px;
      if (py < pen) { pen = py; kk = 1; }
      if (pz < pen) { pen = pz; kk = 2; }
      const float ek = kk == 0 ? e.x : (kk == 1 ? e.y : e.z);
      const float sg = ek >= 0.f ? 1.f : -1.f;
      nl = mk3(kk == 0 ? sg : 0.f, kk == 1 ? sg : 0.f, kk == 2 ? sg : 0.f);
      depth = pr.ra + pen;
      pl = fma3(0.5f * (pen - pr.ra), nl, e);
    }
    if (depth > 0.f) {
      n = mul(Rb, nl);
      p = cb + mul(Rb, pl);
      hit = true;
    }
  }
  float4* sl = gm.slot4(k, 0) + lane;
  if (!hit) {
    sl[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    sl[32] = make_float4(0.f, 0.f, 0.f, 0.f);
    return 0;
  }
  const Pub A = read_pub(gm, pr.ba, lane);
  const Pub Bq = read_pub(gm, pr.bb, lane);
  const BodyP& ba = bodies[pr.ba];
  const BodyP& bb = bodies[pr.bb];
  const S6 Ia = read_pub_Ii(gm, pr.ba, lane);
  const S6 Ib = read_pub_Ii(gm, pr.bb, lane);
  const V3 la = p - A.x, lb = p - Bq.x;
  const V3 u = (A.v + cross(A.w, la)) - (Bq.v + cross(Bq.w, lb));
  const float kn = eff_mass(ba.flags, ba.inv_mass, Ia, la, n) + eff_mass(bb.flags, bb.inv_mass, Ib, lb, n);
  if (!(kn > 0.f)) {
    sl[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    sl[32] = make_float4(0.f, 0.f, 0.f, 0.f);
    return 0;
  }
  const float un = dot(u, n);
  const float target = fmaxf(S.beta_h * depth, -pr.e * un);
  const float jn = fmaxf(__fdividef(target - un, kn), 0.f);
  V3 J = jn * n;
  const V3 ut = fma3(-un, n, u);
  const float ut2 = dot(ut, ut);
  if (ut2 > S.eps * S.eps) {
    const float rinv = rsqrtf(ut2);
    const float utn = ut2 * rinv;
    const V3 t = rinv * ut;
    const float kt = eff_mass(ba.flags, ba.inv_mass, Ia, la, t) + eff_mass(bb.flags, bb.inv_mass, Ib, lb, t);
    const float jt = fminf(__fdividef(utn, kt), pr.mu * jn);
    J = fma3(-jt, t, J);
  }
  sl[0] = make_float4(J.x, J.y, J.z, p.x);
  sl[32] = make_float4(p.y, p.z, 1.f, 0.f);
  return 1;
}

// ------------------------------------------------------------------ environment layer
// Observation of a body's parent joint (the gym-like environment layer): its
// angles, measured as the limits measure them, and the relative angular
// velocity w - w_p along its world axes R_p (parent joint-frame axis k).
// Rp, wp: the parent's rotation and angular velocity; R, w: this body's.
template <bool kGeneral>
__device__ __forceinline__ void joint_obs(const BodyP& bp, const M3& Rp, V3 wp, const M3& R, V3 w, float* ang,
                                          float* rate) {
  const V3 P0 = mulc(Rp, bp.ap + 0);
  const V3 P1 = mulc(Rp, bp.ap + 3);
  const V3 wr = w - wp;
  if (!kGeneral || bp.dof == 1) {
    const V3 yc = mulc(R, bp.ac + 3);
    ang[0] = fast_atan2(dot(cross(P1, yc), P0), dot(P1, yc));
    rate[0] = dot(wr, P0);
  } else {
    const V3 P2 = mulc(Rp, bp.ap + 6);
    const V3 C0 = mulc(R, bp.ac + 0);
    const V3 C1 = mulc(R, bp.ac + 3);
    const V3 C2 = mulc(R, bp.ac + 6);
    const float m00 = dot(P0, C0), m01 = dot(P0, C1), m02 = dot(P0, C2);
    const float m12 = dot(P1, C2), m22 = dot(P2, C2);
    ang[0] = fast_atan2(-m12, m22);
    ang[1] = fast_atan2(m02, sqrtf(fmaf(m00, m00, m01 * m01)));
    ang[2] = fast_atan2(-m01, m00);
    rate[0] = dot(wr, P0);
    rate[1] = dot(wr, P1);
    rate[2] = dot(wr, P2);
  }
}

// The root body's part of the environment layer after a step: its
// observation fields (height, quaternion, velocity, angular velocity), the
// step's reward and whether the episode ended.  x0: its x position before
// the step; ctrl: the sum of the squared clamped actions.
__device__ __forceinline__ bool root_env(const Seg& sg, const Body& s, float x0, float ctrl, float* ob, float* rew,
                                         uint8_t* dn) {
  ob[0] = s.x.z;
  ob[1] = s.qw;
  ob[2] = s.qx;
  ob[3] = s.qy;
  ob[4] = s.qz;
  ob[5] = s.v.x;
  ob[6] = s.v.y;
  ob[7] = s.v.z;
  ob[8] = s.w.x;
  ob[9] = s.w.y;
  ob[10] = s.w.z;
  const bool done = s.x.z < sg.min_z || s.x.z > sg.max_z;
  *rew = fmaf(sg.fwd_w_dt, s.x.x - x0, done ? 0.f : sg.healthy) - sg.ctrl_cost * ctrl;
  *dn = done ? 1 : 0;
  return done;
}

// ------------------------------------------------------------------ phase P
// Add a child's joint reaction (force, torque on this body) to wr.
__device__ __forceinline__ void add_reaction(GroupMem& gm, int child, int lane, Wrench& wr) {
  const float4* r = gm.react4(child, 0) + lane;
  const float4 a = r[0];
  const float2 b = ld2(r + 32);
  wr.F = wr.F + mk3(a.x, a.y, a.z);
  wr.tau = wr.tau + mk3(a.w, b.x, b.y);
}

// Potential integrator: v += h (F/m + g), w += h Ii tau; collision
// integrator: the mean (or sum) of the contact velocity changes.
template <bool kGeneral>
__device__ __forceinline__ void integrate(const SysP& S, const BodyP& bp, GroupMem& gm, int lane, Body& s,
                                          const Frame& f, Wrench wr, Acc acc) {
  for (int c = 0; c < bp.n_children; ++c) add_reaction(gm, bp.children[c], lane, wr);
  for (int i = 0; kGeneral && i < bp.n_bpairs; ++i) {
    const int code = bp.bpair[i];
    const float4* sl = gm.slot4(code >> 1, 0) + lane;
    const float4 c1 = sl[32];
    if (c1.z != 0.f) {
      const float4 c0 = sl[0];
      const float sg = (code & 1) ? -1.f : 1.f;
      const V3 J = sg * mk3(c0.x, c0.y, c0.z);
      const V3 l = mk3(c0.w, c1.x, c1.y) - s.x;
      V3 dv = bp.inv_mass * J;
      V3 dw = mul(f.Ii, cross(l, J));
      if (bp.flags & kAnyFrozen) {
        dv = mask3(bp.flags, dv);
        dw = mask3(bp.flags >> 3, dw);
      }
      acc.dv = acc.dv + dv;
      acc.dw = acc.dw + dw;
      acc.n += 1;
    }
  }
  const float h = S.h;
  V3 v, w;
  if (kGeneral && S.variants) {
    // variants: global damping and the gyroscopic torque -w x (I_w w)
    V3 a = fma3(bp.inv_mass, wr.F, ld3(S.g));
    a = fma3(-S.lin_damp, s.v, a);
    V3 tau = wr.tau;
    if (S.gyro) tau = tau - cross(s.w, mul(inv_inertia_world(f.R, bp.I), s.w));
    const V3 alpha = fma3(-S.ang_damp, s.w, mul(f.Ii, tau));
    v = fma3(h, a, s.v);
    w = fma3(h, alpha, s.w);
  } else {
    v = fma3(h, fma3(bp.inv_mass, wr.F, ld3(S.g)), s.v);
    w = fma3(h, mul(f.Ii, wr.tau), s.w);
  }
  if (bp.flags & kAnyFrozen) {
    v = mask3(bp.flags, v);
    w = mask3(bp.flags >> 3, w);
  }
  if (acc.n > 0) {
    const float inv = (S.average && acc.n > 1) ? __fdividef(1.f, (float)acc.n) : 1.f;
    v = fma3(inv, acc.dv, v);
    w = fma3(inv, acc.dw, w);
  }
  s.v = v;
  s.w = w;
}

}  // namespace brax
