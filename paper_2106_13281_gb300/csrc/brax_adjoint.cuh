// Reverse-mode (vector-Jacobian) building blocks of one substep.
//
// Each *_bwd function takes the forward inputs, recomputes the intermediates
// it needs and accumulates the adjoints of its inputs from the adjoints of
// its outputs.  Branches (max, min, clamp, limits, contact activation) take
// the derivative of the branch the forward took; at an exact tie max(a, b)
// is taken as b, matching the oracle.
#pragma once
#include "brax_physics.cuh"

namespace brax {

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ V3 zero3() { return mk3(0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero(M3& m) {
#pragma unroll
  for (int i = 0; i < 9; ++i) m.m[i] = 0.f;
}
__device__ __forceinline__ void zero(S6& s) {
#pragma unroll
  for (int i = 0; i < 6; ++i) s.a[i] = 0.f;
}
// c = a x b:  ga += b x gc,  gb += gc x a
__device__ __forceinline__ void cross_bwd(V3 a, V3 b, V3 gc, V3& ga, V3& gb) {
  ga = ga + cross(b, gc);
  gb = gb + cross(gc, a);
}
// y = R o (o constant): gR += gy o^T
__device__ __forceinline__ void mulc_bwd(M3& gR, V3 gy, const float* o) {
  const float o0 = o[0], o1 = o[1], o2 = o[2];
  gR.m[0] = fmaf(gy.x, o0, gR.m[0]);
  gR.m[1] = fmaf(gy.x, o1, gR.m[1]);
  gR.m[2] = fmaf(gy.x, o2, gR.m[2]);
  gR.m[3] = fmaf(gy.y, o0, gR.m[3]);
  gR.m[4] = fmaf(gy.y, o1, gR.m[4]);
  gR.m[5] = fmaf(gy.y, o2, gR.m[5]);
  gR.m[6] = fmaf(gy.z, o0, gR.m[6]);
  gR.m[7] = fmaf(gy.z, o1, gR.m[7]);
  gR.m[8] = fmaf(gy.z, o2, gR.m[8]);
}
// y = Ii v (Ii symmetric, 6 stored entries): gIi += sym(gy v^T), gv += Ii gy
__device__ __forceinline__ void s6_mul_bwd(const S6& I, V3 v, V3 gy, S6& gI, V3& gv) {
  gI.a[0] = fmaf(gy.x, v.x, gI.a[0]);
  gI.a[1] += fmaf(gy.x, v.y, gy.y * v.x);
  gI.a[2] += fmaf(gy.x, v.z, gy.z * v.x);
  gI.a[3] = fmaf(gy.y, v.y, gI.a[3]);
  gI.a[4] += fmaf(gy.y, v.z, gy.z * v.y);
  gI.a[5] = fmaf(gy.z, v.z, gI.a[5]);
  gv = gv + mul(I, gy);
}
// Ii = R diag(d) R^T:  gR_ik += d_k (M R)_ik with M = [[2g0,g1,g2],[g1,2g3,g4],[g2,g4,2g5]]
__device__ __forceinline__ void inv_inertia_bwd(const M3& R, const float* d, const S6& g, M3& gR) {
  const float M[9] = {2.f * g.a[0], g.a[1], g.a[2], g.a[1], 2.f * g.a[3], g.a[4], g.a[2], g.a[4], 2.f * g.a[5]};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float mr = fmaf(M[3 * i], R.m[k], fmaf(M[3 * i + 1], R.m[3 + k], M[3 * i + 2] * R.m[6 + k]));
      gR.m[3 * i + k] = fmaf(d[k], mr, gR.m[3 * i + k]);
    }
}
// R = qmat(q): accumulate dL/dq from dL/dR
__device__ __forceinline__ void qmat_bwd(float w, float x, float y, float z, const M3& g, float* gq) {
  const float* G = g.m;
  gq[0] += 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  gq[1] += 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.f * x * G[8]);
  gq[2] += 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.f * y * G[8]);
  gq[3] += 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

// Adjoint of a body's substep state: position, quaternion, velocity, angular velocity.
struct GBody {
  V3 x;
  float q[4];
  V3 v, w;
};
__device__ __forceinline__ GBody zero_gbody() {
  GBody g;
  g.x = zero3();
  g.q[0] = g.q[1] = g.q[2] = g.q[3] = 0.f;
  g.v = zero3();
  g.w = zero3();
  return g;
}

// ------------------------------------------------------------------ kinematic
// Forward (see kinematic()): vm = mask(v), wm = mask(w); x1 = x + h vm;
// qq = q + h/2 (0, wm) (x) q;  q1 = qq / |qq|.
// Inputs: s_in (substep input state), adjoints gx1, gq1 (of x1, q1) and
// gvm, gwm (of the masked velocities).  Returns the input-state adjoint.
__device__ __forceinline__ GBody kinematic_bwd(const BodyP& bp, float h, const Body& s_in, V3 gx1, const float* gq1,
                                               V3 gvm, V3 gwm) {
  V3 wm = s_in.w;
  if (bp.flags & kAnyFrozen) wm = mask3(bp.flags >> 3, wm);
  const float hh = 0.5f * h;
  const float qw = s_in.qw, qx = s_in.qx, qy = s_in.qy, qz = s_in.qz;
  const float nw = fmaf(-hh, fmaf(wm.x, qx, fmaf(wm.y, qy, wm.z * qz)), qw);
  const float nx = fmaf(hh, fmaf(qw, wm.x, fmaf(wm.y, qz, -wm.z * qy)), qx);
  const float ny = fmaf(hh, fmaf(qw, wm.y, fmaf(wm.z, qx, -wm.x * qz)), qy);
  const float nz = fmaf(hh, fmaf(qw, wm.z, fmaf(wm.x, qy, -wm.y * qx)), qz);
  const float r = rsqrtf(fmaf(nw, nw, fmaf(nx, nx, fmaf(ny, ny, nz * nz))));
  const float q1w = nw * r, q1x = nx * r, q1y = ny * r, q1z = nz * r;
  // q1 = qq r:  gqq = r (gq1 - q1 (q1 . gq1))
  const float dq = q1w * gq1[0] + q1x * gq1[1] + q1y * gq1[2] + q1z * gq1[3];
  const float gPw = r * (gq1[0] - q1w * dq), gPx = r * (gq1[1] - q1x * dq);
  const float gPy = r * (gq1[2] - q1y * dq), gPz = r * (gq1[3] - q1z * dq);
  GBody g;
  g.q[0] = gPw + hh * (wm.x * gPx + wm.y * gPy + wm.z * gPz);
  g.q[1] = gPx + hh * (-wm.x * gPw + wm.z * gPy - wm.y * gPz);
  g.q[2] = gPy + hh * (-wm.y * gPw - wm.z * gPx + wm.x * gPz);
  g.q[3] = gPz + hh * (-wm.z * gPw + wm.y * gPx - wm.x * gPy);
  gwm.x += hh * (-qx * gPw + qw * gPx - qz * gPy + qy * gPz);
  gwm.y += hh * (-qy * gPw + qz * gPx + qw * gPy - qx * gPz);
  gwm.z += hh * (-qz * gPw - qy * gPx + qx * gPy + qw * gPz);
  g.x = gx1;
  gvm = fma3(h, gx1, gvm);
  if (bp.flags & kAnyFrozen) {
    gvm = mask3(bp.flags, gvm);
    gwm = mask3(bp.flags >> 3, gwm);
  }
  g.v = gvm;
  g.w = gwm;
  return g;
}

// ------------------------------------------------------------------ effective mass
// e = invm |mp . dir|^2-form + (mr . Ii (l x dir)) . (l x dir); accumulate gl, gdir, gIi.
__device__ __forceinline__ void eff_mass_bwd(uint32_t flags, float inv_m, const S6& Ii, V3 l, V3 dir, float ge,
                                             V3& gl, V3& gdir, S6& gI, bool want_gdir) {
  const V3 ld = cross(l, dir);
  const V3 Ild = mul(Ii, ld);
  V3 gld;
  if (flags & kAnyFrozen) {
    const V3 mp = mask3(flags, mk3(1.f, 1.f, 1.f));
    const V3 mr = mask3(flags >> 3, mk3(1.f, 1.f, 1.f));
    if (want_gdir) gdir = gdir + (2.f * ge * inv_m) * mk3(mp.x * dir.x, mp.y * dir.y, mp.z * dir.z);
    const V3 mld = mk3(mr.x * ld.x, mr.y * ld.y, mr.z * ld.z);
    gld = ge * (mk3(mr.x * Ild.x, mr.y * Ild.y, mr.z * Ild.z) + mul(Ii, mld));
    gI.a[0] += ge * mr.x * ld.x * ld.x;
    gI.a[1] += ge * (mr.x + mr.y) * ld.x * ld.y;
    gI.a[2] += ge * (mr.x + mr.z) * ld.x * ld.z;
    gI.a[3] += ge * mr.y * ld.y * ld.y;
    gI.a[4] += ge * (mr.y + mr.z) * ld.y * ld.z;
    gI.a[5] += ge * mr.z * ld.z * ld.z;
  } else {
    if (want_gdir) gdir = fma3(2.f * ge * inv_m, dir, gdir);
    gld = (2.f * ge) * Ild;
    gI.a[0] = fmaf(ge * ld.x, ld.x, gI.a[0]);
    gI.a[1] = fmaf(2.f * ge * ld.x, ld.y, gI.a[1]);
    gI.a[2] = fmaf(2.f * ge * ld.x, ld.z, gI.a[2]);
    gI.a[3] = fmaf(ge * ld.y, ld.y, gI.a[3]);
    gI.a[4] = fmaf(2.f * ge * ld.y, ld.z, gI.a[4]);
    gI.a[5] = fmaf(ge * ld.z, ld.z, gI.a[5]);
  }
  V3 gdir2 = zero3();
  cross_bwd(l, dir, gld, gl, gdir2);
  if (want_gdir) gdir = gdir + gdir2;
}

// ------------------------------------------------------------------ plane contact point
// Adjoint of one plane-contact point (plane_point()) given the adjoints gdv,
// gdw of the body's summed contact update.  Accumulates into the own body's
// x1, R, Ii, vm, wm adjoints.
template <class PT>
__device__ __forceinline__ void plane_point_bwd(const SysP& S, const BodyP& bp, const PT& pt, const PlaneP& pl,
                                                const Body& s, const Frame& f, V3 gdv, V3 gdw, V3& gx, M3& gR,
                                                S6& gI, V3& gv, V3& gw) {
  const V3 ro = mulc(f.R, pt.o);
  const V3 n = ld3(pl.n);
  const float dist = dot((s.x + ro) - ld3(pl.p0), n);
  const float depth = pt.r - dist;
  if (!(depth > 0.f)) return;
  const V3 l = fma3(-pt.r, n, ro);
  const V3 u = s.v + cross(s.w, l);
  const float kn = eff_mass(bp.flags, bp.inv_mass, f.Ii, l, n);
  if (!(kn > 0.f)) return;
  const float un = dot(u, n);
  const float t1 = S.beta_h * depth, t2 = -pt.e * un;
  const bool first = t1 > t2;
  const float target = first ? t1 : t2;
  const float qn = __fdividef(target - un, kn);
  const bool pos = qn > 0.f;
  const float jn = pos ? qn : 0.f;
  V3 J = jn * n;
  const V3 ut = fma3(-un, n, u);
  const float ut2 = dot(ut, ut);
  const bool fric = ut2 > S.eps * S.eps;
  float rinv = 0.f, utn = 0.f, kt = 1.f, r1 = 0.f, jt = 0.f;
  bool stick = false;
  V3 t = zero3();
  if (fric) {
    rinv = rsqrtf(ut2);
    utn = ut2 * rinv;
    t = rinv * ut;
    kt = eff_mass(bp.flags, bp.inv_mass, f.Ii, l, t);
    r1 = __fdividef(utn, kt);
    stick = r1 < pt.mu * jn;
    jt = stick ? r1 : pt.mu * jn;
    J = fma3(-jt, t, J);
  }
  // ---- reverse
  if (bp.flags & kAnyFrozen) {
    gdv = mask3(bp.flags, gdv);
    gdw = mask3(bp.flags >> 3, gdw);
  }
  V3 gJ = bp.inv_mass * gdv;
  const V3 lJ = cross(l, J);
  V3 glJ = zero3();
  s6_mul_bwd(f.Ii, lJ, gdw, gI, glJ);
  V3 gl = zero3();
  cross_bwd(l, J, glJ, gl, gJ);
  float gjn = dot(gJ, n);
  V3 gu = zero3();
  float gun = 0.f;
  if (fric) {
    const float gjt = -dot(gJ, t);
    V3 gt = (-jt) * gJ;
    float gutn = 0.f, gkt = 0.f;
    if (stick) {
      gutn = __fdividef(gjt, kt);
      gkt = -gjt * __fdividef(r1, kt);
    } else {
      gjn = fmaf(pt.mu, gjt, gjn);
    }
    eff_mass_bwd(bp.flags, bp.inv_mass, f.Ii, l, t, gkt, gl, gt, gI, true);
    const V3 gut = fma3(gutn, t, rinv * fma3(-dot(t, gt), t, gt));
    gu = gu + gut;
    gun -= dot(gut, n);
  }
  float gdepth = 0.f;
  if (pos) {
    const float gq = gjn;
    const float gtarget = __fdividef(gq, kn);
    gun -= gtarget;
    const float gkn = -gq * __fdividef(qn, kn);
    if (first) gdepth = S.beta_h * gtarget;
    else gun = fmaf(-pt.e, gtarget, gun);
    V3 dummy = zero3();
    eff_mass_bwd(bp.flags, bp.inv_mass, f.Ii, l, n, gkn, gl, dummy, gI, false);
  }
  gu = fma3(gun, n, gu);
  gv = gv + gu;
  gw = gw + cross(l, gu);
  gl = gl + cross(gu, s.w);
  V3 gro = gl;
  const float gdist = -gdepth;
  gx = fma3(gdist, n, gx);
  gro = fma3(gdist, n, gro);
  mulc_bwd(gR, gro, pt.o);
}

// ------------------------------------------------------------------ hinge joint
// Adjoint of joint_forward() on the hinge path.  gFc, gTc: adjoints of the
// child's summed force and torque; gFp, gTp: the parent's.  Accumulates the
// own (child) adjoints and returns the parent's through gp_* outputs.
template <class JP>
__device__ __forceinline__ void joint_hinge_bwd(const JP& bp, const Pub& pp, const Body& s, const Frame& f,
                                                const float* act, V3 gFc, V3 gTc, V3 gFp, V3 gTp, V3& gx, M3& gR,
                                                V3& gv, V3& gw, V3& gxp, M3& gRp, V3& gvp, V3& gwp, float* gact) {
  // forward recompute
  const V3 rp = mulc(pp.R, bp.off_p);
  const V3 rc = mulc(f.R, bp.off_c);
  const V3 dpc = (pp.x + rp) - (s.x + rc);
  const V3 up = pp.v + cross(pp.w, rp);
  const V3 uc = s.v + cross(s.w, rc);
  const V3 F = bp.k * dpc - bp.c * (uc - up);
  const V3 P0 = mulc(pp.R, bp.ap + 0);
  const V3 P1 = mulc(pp.R, bp.ap + 3);
  const V3 wr = s.w - pp.w;
  const V3 Ac = mulc(f.R, bp.ac + 0);
  const V3 yc = mulc(f.R, bp.ac + 3);
  const V3 cr = cross(P1, yc);
  const float sy = dot(cr, P0), cx = dot(P1, yc);
  const float th = fast_atan2(sy, cx);
  float L = 0.f;
  int lim = 0;
  if (th < bp.lo[0]) {
    L = bp.kl * (bp.lo[0] - th);
    lim = 1;
  } else if (th > bp.hi[0]) {
    L = bp.kl * (bp.hi[0] - th);
    lim = 1;
  }
  float sc = L - bp.ca * dot(wr, P0);
  const bool has_act = bp.act[0] >= 0;
  const bool angle_act = has_act && (bp.act_angle & 1);
  if (has_act) {
    if (angle_act) sc = fmaf(bp.gear[0], fmaf(bp.act_half[0], clamp1(act[0]), bp.act_mid[0]) - th, sc);
    else sc = fmaf(bp.gear[0], clamp1(act[0]), sc);
  }
  // ---- reverse
  // child gets F, tc = rc x F + tj; parent gets -F, tp = -(rp x F) - tj
  V3 gF = gFc - gFp;
  const V3 gtj = gTc - gTp;
  V3 grc = zero3(), grp = zero3();
  cross_bwd(rc, F, gTc, grc, gF);
  cross_bwd(rp, F, -gTp, grp, gF);
  // tj = sc P0 + ka (Ac x P0)
  const float gsc = dot(gtj, P0);
  V3 gP0 = sc * gtj;
  V3 gAc = zero3();
  cross_bwd(Ac, P0, bp.ka * gtj, gAc, gP0);
  // sc = L - ca (wr . P0) + gear clamp(a)
  const float gL = gsc;
  const V3 gwr = (-bp.ca * gsc) * P0;
  gP0 = fma3(-bp.ca * gsc, wr, gP0);
  if (has_act) {
    const float a = act[0];
    if (a > -1.f && a < 1.f) gact[0] = fmaf(angle_act ? bp.gear[0] * bp.act_half[0] : bp.gear[0], gsc, gact[0]);
  }
  // limit spring: d L / d th = -kl when active; a target-angle actuator adds -gear
  float gth = lim ? -bp.kl * gL : 0.f;
  if (angle_act) gth = fmaf(-bp.gear[0], gsc, gth);
  const float r2 = fmaf(sy, sy, cx * cx);
  const float inv_r2 = r2 > 0.f ? __fdividef(1.f, r2) : 0.f;
  const float gsy = cx * inv_r2 * gth, gcx = -sy * inv_r2 * gth;
  V3 gcr = gsy * P0;
  gP0 = fma3(gsy, cr, gP0);
  V3 gP1 = zero3(), gyc = zero3();
  cross_bwd(P1, yc, gcr, gP1, gyc);
  gP1 = fma3(gcx, yc, gP1);
  gyc = fma3(gcx, P1, gyc);
  // F = k dpc - c (uc - up)
  const V3 gdpc = bp.k * gF;
  const V3 guc = (-bp.c) * gF;
  const V3 gup = bp.c * gF;
  gv = gv + guc;
  cross_bwd(s.w, rc, guc, gw, grc);
  gvp = gvp + gup;
  cross_bwd(pp.w, rp, gup, gwp, grp);
  gxp = gxp + gdpc;
  grp = grp + gdpc;
  gx = gx - gdpc;
  grc = grc - gdpc;
  gw = gw + gwr;
  gwp = gwp - gwr;
  mulc_bwd(gRp, grp, bp.off_p);
  mulc_bwd(gR, grc, bp.off_c);
  mulc_bwd(gRp, gP0, bp.ap + 0);
  mulc_bwd(gRp, gP1, bp.ap + 3);
  mulc_bwd(gR, gAc, bp.ac + 0);
  mulc_bwd(gR, gyc, bp.ac + 3);
}

// ------------------------------------------------------------------ 3-DOF joint
// Adjoint of joint_forward() on the 3-DOF path (intrinsic X-Y-Z angles,
// per-axis limits and actuators about the parent's joint axes, 3-D angular
// damper, no alignment spring).
__device__ __forceinline__ void atan2_bwd(float y, float x, float g, float& gy, float& gx) {
  const float r2 = fmaf(y, y, x * x);
  const float inv = r2 > 0.f ? __fdividef(1.f, r2) : 0.f;
  gy += x * inv * g;
  gx -= y * inv * g;
}

__device__ __forceinline__ void joint3_bwd(const BodyP& bp, const Pub& pp, const Body& s, const Frame& f,
                                           const float* act, V3 gFc, V3 gTc, V3 gFp, V3 gTp, V3& gx, M3& gR, V3& gv,
                                           V3& gw, V3& gxp, M3& gRp, V3& gvp, V3& gwp, float* gact) {
  const V3 rp = mulc(pp.R, bp.off_p);
  const V3 rc = mulc(f.R, bp.off_c);
  const V3 dpc = (pp.x + rp) - (s.x + rc);
  const V3 up = pp.v + cross(pp.w, rp);
  const V3 uc = s.v + cross(s.w, rc);
  const V3 F = bp.k * dpc - bp.c * (uc - up);
  const V3 P[3] = {mulc(pp.R, bp.ap + 0), mulc(pp.R, bp.ap + 3), mulc(pp.R, bp.ap + 6)};
  const V3 Cc[3] = {mulc(f.R, bp.ac + 0), mulc(f.R, bp.ac + 3), mulc(f.R, bp.ac + 6)};
  const float m00 = dot(P[0], Cc[0]), m01 = dot(P[0], Cc[1]), m02 = dot(P[0], Cc[2]);
  const float m12 = dot(P[1], Cc[2]), m22 = dot(P[2], Cc[2]);
  const float sq = sqrtf(fmaf(m00, m00, m01 * m01));
  float th[3];
  th[0] = fast_atan2(-m12, m22);
  th[1] = fast_atan2(m02, sq);
  th[2] = fast_atan2(-m01, m00);
  float L[3];
  int lim[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    L[a] = 0.f;
    lim[a] = 0;
    if (th[a] < bp.lo[a]) {
      L[a] = bp.kl * (bp.lo[a] - th[a]);
      lim[a] = 1;
    } else if (th[a] > bp.hi[a]) {
      L[a] = bp.kl * (bp.hi[a] - th[a]);
      lim[a] = 1;
    }
    if (a == 2 && bp.dof == 2) L[a] = -bp.ka * th[2];  // the 2-DOF joint's twist spring
    if (bp.act[a] >= 0) {
      if (bp.act_angle & (1 << a))
        L[a] = fmaf(bp.gear[a], fmaf(bp.act_half[a], clamp1(act[a]), bp.act_mid[a]) - th[a], L[a]);
      else
        L[a] = fmaf(bp.gear[a], clamp1(act[a]), L[a]);
    }
  }
  // ---- reverse
  V3 gF = gFc - gFp;
  const V3 gtj = gTc - gTp;
  V3 grc = zero3(), grp = zero3();
  cross_bwd(rc, F, gTc, grc, gF);
  cross_bwd(rp, F, -gTp, grp, gF);
  const V3 gwr = (-bp.ca) * gtj;
  V3 gP[3], gC[3];
  float gth[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gP[a] = L[a] * gtj;
    gC[a] = zero3();
    const float gL = dot(gtj, P[a]);
    gth[a] = lim[a] ? -bp.kl * gL : 0.f;
    if (a == 2 && bp.dof == 2) gth[a] = -bp.ka * gL;
    if (bp.act[a] >= 0) {
      const bool angle_act = (bp.act_angle & (1 << a)) != 0;
      const float av = act[a];
      if (av > -1.f && av < 1.f) gact[a] = fmaf(angle_act ? bp.gear[a] * bp.act_half[a] : bp.gear[a], gL, gact[a]);
      if (angle_act) gth[a] = fmaf(-bp.gear[a], gL, gth[a]);
    }
  }
  float gm00 = 0.f, gm01 = 0.f, gm02 = 0.f, gm12 = 0.f, gm22 = 0.f;
  {  // th0 = atan2(-m12, m22)
    float gy = 0.f, gxx = 0.f;
    atan2_bwd(-m12, m22, gth[0], gy, gxx);
    gm12 -= gy;
    gm22 += gxx;
  }
  {  // th1 = atan2(m02, sqrt(m00^2 + m01^2))
    float gy = 0.f, gs = 0.f;
    atan2_bwd(m02, sq, gth[1], gy, gs);
    gm02 += gy;
    if (sq > 0.f) {
      const float is = __fdividef(1.f, sq);
      gm00 += gs * m00 * is;
      gm01 += gs * m01 * is;
    }
  }
  {  // th2 = atan2(-m01, m00)
    float gy = 0.f, gxx = 0.f;
    atan2_bwd(-m01, m00, gth[2], gy, gxx);
    gm01 -= gy;
    gm00 += gxx;
  }
  gP[0] = fma3(gm00, Cc[0], fma3(gm01, Cc[1], fma3(gm02, Cc[2], gP[0])));
  gP[1] = fma3(gm12, Cc[2], gP[1]);
  gP[2] = fma3(gm22, Cc[2], gP[2]);
  gC[0] = gm00 * P[0];
  gC[1] = gm01 * P[0];
  gC[2] = fma3(gm02, P[0], fma3(gm12, P[1], gm22 * P[2]));
  // anchor spring-damper, as in the hinge
  const V3 gdpc = bp.k * gF;
  const V3 guc = (-bp.c) * gF;
  const V3 gup = bp.c * gF;
  gv = gv + guc;
  cross_bwd(s.w, rc, guc, gw, grc);
  gvp = gvp + gup;
  cross_bwd(pp.w, rp, gup, gwp, grp);
  gxp = gxp + gdpc;
  grp = grp + gdpc;
  gx = gx - gdpc;
  grc = grc - gdpc;
  gw = gw + gwr;
  gwp = gwp - gwr;
  mulc_bwd(gRp, grp, bp.off_p);
  mulc_bwd(gR, grc, bp.off_c);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mulc_bwd(gRp, gP[a], bp.ap + 3 * a);
    mulc_bwd(gR, gC[a], bp.ac + 3 * a);
  }
}

// ------------------------------------------------------------------ body-body pairs
// Adjoint state of one side of a pair (written to the workspace; the body
// adds its pairs' contributions in its own pair order).
struct GSide {
  V3 x, v, w;
  M3 R;
  S6 I;
};
__device__ __forceinline__ void zero(GSide& g) {
  g.x = zero3();
  g.v = zero3();
  g.w = zero3();
  zero(g.R);
  zero(g.I);
}

// Closest-point parameters of two segments: adjoint through the branch taken.
__device__ __forceinline__ void segment_closest_bwd(V3 P1, V3 d1, V3 P2, V3 d2, float gs, float gt, V3& gP1, V3& gd1,
                                                    V3& gP2, V3& gd2) {
  const V3 r = P1 - P2;
  const float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  const float tiny = 1e-12f;
  float ga = 0.f, ge = 0.f, gf = 0.f, gc = 0.f, gb = 0.f;
  const float c = dot(d1, r);
  if (a <= tiny && e <= tiny) return;
  if (a <= tiny) {
    const float t = __fdividef(f, e);
    if (t > 0.f && t < 1.f) {
      gf += __fdividef(gt, e);
      ge -= gt * __fdividef(t, e);
    }
  } else if (e <= tiny) {
    const float s = __fdividef(-c, a);
    if (s > 0.f && s < 1.f) {
      gc -= __fdividef(gs, a);
      ga -= gs * __fdividef(s, a);
    }
  } else {
    const float b = dot(d1, d2);
    const float ae = a * e;
    const float denom = ae - b * b;
    const bool gen = denom > 1e-5f * ae;
    const float s0raw = gen ? __fdividef(fmaf(b, f, -c * e), denom) : 0.f;
    const float s0 = gen ? fminf(fmaxf(s0raw, 0.f), 1.f) : 0.f;
    const float t0 = __fdividef(fmaf(b, s0, f), e);
    if (t0 < 0.f) {
      const float s = __fdividef(-c, a);
      if (s > 0.f && s < 1.f) {
        gc -= __fdividef(gs, a);
        ga -= gs * __fdividef(s, a);
      }
    } else if (t0 > 1.f) {
      const float s = __fdividef(b - c, a);
      if (s > 0.f && s < 1.f) {
        const float ia = __fdividef(1.f, a);
        gb += gs * ia;
        gc -= gs * ia;
        ga -= gs * s * ia;
      }
    } else {
      const float ie = __fdividef(1.f, e);
      gb += gt * s0 * ie;
      float gs0 = gs + gt * b * ie;
      gf += gt * ie;
      ge -= gt * t0 * ie;
      if (gen && s0raw > 0.f && s0raw < 1.f) {
        const float id = __fdividef(1.f, denom);
        const float gnum = gs0 * id;
        const float gden = -gs0 * s0raw * id;
        gb += gnum * f;
        gf += gnum * b;
        gc -= gnum * e;
        ge -= gnum * c;
        ga += gden * e;
        ge += gden * a;
        gb -= 2.f * b * gden;
      }
    }
  }
  gd1 = fma3(2.f * ga, d1, gd1);
  gd2 = fma3(2.f * ge, d2, gd2);
  gd2 = fma3(gf, r, gd2);
  V3 gr = gf * d2;
  gd1 = fma3(gc, r, gd1);
  gr = fma3(gc, d1, gr);
  gd1 = fma3(gb, d2, gd1);
  gd2 = fma3(gb, d1, gd2);
  gP1 = gP1 + gr;
  gP2 = gP2 - gr;
}

// Reverse of one body-body pair.  Recomputes the detection and the impulse,
// forms the impulse/contact-point adjoints from both bodies' contact-update
// adjoints (gacc), and returns the adjoints of both bodies' x1, R, v, w, Ii.
__device__ __forceinline__ void pair_bwd(const SysP& S, const BodyP* bodies, const PairP& pr, GroupMem& gm,
                                         const float* gacc, int lane, GSide& GA, GSide& GB) {
  const Pub A = read_pub(gm, pr.ba, lane);
  const Pub Bq = read_pub(gm, pr.bb, lane);
  const V3 P1 = A.x + mulc(A.R, pr.a0);
  const V3 d1 = mulc(A.R, pr.a1) - mulc(A.R, pr.a0);
  V3 n, p;
  float depth = 0.f;
  bool hit = false;
  // capsule-capsule intermediates
  V3 P2 = zero3(), d2 = zero3(), c1 = zero3(), c2 = zero3(), df = zero3();
  float sp = 0.f, tpar = 0.f, dl = 0.f;
  // capsule-box intermediates
  M3 Rb;
  V3 cb = zero3(), Pl = zero3(), dlv = zero3(), e = zero3(), q = zero3(), nl = zero3(), pl = zero3();
  float tbox = 0.f, dist = 0.f;
  int inside = 0, kk = 0;
  float sgk = 1.f, pen = 0.f;
  if (pr.type == kCapsuleCapsule) {
    P2 = Bq.x + mulc(Bq.R, pr.b0);
    d2 = mulc(Bq.R, pr.b1) - mulc(Bq.R, pr.b0);
    segment_closest(P1, d1, P2, d2, sp, tpar);
    c1 = fma3(sp, d1, P1);
    c2 = fma3(tpar, d2, P2);
    df = c1 - c2;
    dl = sqrtf(dot(df, df));
    depth = pr.ra + pr.rb - dl;
    if (dl >= S.eps && depth > 0.f) {
      n = __fdividef(1.f, dl) * df;
      p = 0.5f * (fma3(-pr.ra, n, c1) + fma3(pr.rb, n, c2));
      hit = true;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Rb.m[3 * i + j] = fmaf(Bq.R.m[3 * i + 0], pr.bR[0 * 3 + j],
                               fmaf(Bq.R.m[3 * i + 1], pr.bR[1 * 3 + j], Bq.R.m[3 * i + 2] * pr.bR[2 * 3 + j]));
    cb = Bq.x + mulc(Bq.R, pr.b0);
    Pl = mulT(Rb, P1 - cb);
    dlv = mulT(Rb, d1);
    const float* he = pr.b1;
    tbox = seg_box_param(Pl, dlv, he);
    e = fma3(tbox, dlv, Pl);
    q = mk3(fminf(fmaxf(e.x, -he[0]), he[0]), fminf(fmaxf(e.y, -he[1]), he[1]), fminf(fmaxf(e.z, -he[2]), he[2]));
    const V3 dv = e - q;
    const float d2s = dot(dv, dv);
    if (d2s > 1e-12f) {
      dist = sqrtf(d2s);
      nl = __fdividef(1.f, dist) * dv;
      depth = pr.ra - dist;
      pl = 0.5f * (fma3(-pr.ra, nl, e) + q);
    } else {
      inside = 1;
      tbox = seg_center_param(Pl, dlv);
      e = fma3(tbox, dlv, Pl);
      const float px = he[0] - fabsf(e.x), py = he[1] - fabsf(e.y), pz = he[2] - fabsf(e.z);
      kk = 0;
      pen = px;
      if (py < pen) { pen = py; kk = 1; }
      if (pz < pen) { pen = pz; kk = 2; }
      const float ek = kk == 0 ? e.x : (kk == 1 ? e.y : e.z);
      sgk = ek >= 0.f ? 1.f : -1.f;
      nl = mk3(kk == 0 ? sgk : 0.f, kk == 1 ? sgk : 0.f, kk == 2 ? sgk : 0.f);
      depth = pr.ra + pen;
      pl = fma3(0.5f * (pen - pr.ra), nl, e);
    }
    if (depth > 0.f) {
      n = mul(Rb, nl);
      p = cb + mul(Rb, pl);
      hit = true;
    }
  }
  if (!hit) return;
  const BodyP& ba = bodies[pr.ba];
  const BodyP& bb = bodies[pr.bb];
  const S6 Ia = read_pub_Ii(gm, pr.ba, lane);
  const S6 Ib = read_pub_Ii(gm, pr.bb, lane);
  const V3 la = p - A.x, lb = p - Bq.x;
  const V3 u = (A.v + cross(A.w, la)) - (Bq.v + cross(Bq.w, lb));
  const float kn = eff_mass(ba.flags, ba.inv_mass, Ia, la, n) + eff_mass(bb.flags, bb.inv_mass, Ib, lb, n);
  if (!(kn > 0.f)) return;
  const float un = dot(u, n);
  const float t1 = S.beta_h * depth, t2 = -pr.e * un;
  const bool first = t1 > t2;
  const float target = first ? t1 : t2;
  const float qn = __fdividef(target - un, kn);
  const bool pos = qn > 0.f;
  const float jn = pos ? qn : 0.f;
  V3 J = jn * n;
  const V3 ut = fma3(-un, n, u);
  const float ut2 = dot(ut, ut);
  const bool fric = ut2 > S.eps * S.eps;
  float rinv = 0.f, utn = 0.f, kt = 1.f, r1 = 0.f, jt = 0.f;
  bool stick = false;
  V3 t = zero3();
  if (fric) {
    rinv = rsqrtf(ut2);
    utn = ut2 * rinv;
    t = rinv * ut;
    kt = eff_mass(ba.flags, ba.inv_mass, Ia, la, t) + eff_mass(bb.flags, bb.inv_mass, Ib, lb, t);
    r1 = __fdividef(utn, kt);
    stick = r1 < pr.mu * jn;
    jt = stick ? r1 : pr.mu * jn;
    J = fma3(-jt, t, J);
  }
  // ---- adjoints of J and p from the two bodies' velocity-update adjoints
  V3 gJ = zero3(), gp = zero3();
  for (int side = 0; side < 2; ++side) {
    const BodyP& bs = side == 0 ? ba : bb;
    const int body = side == 0 ? pr.ba : pr.bb;
    const float sgn = side == 0 ? 1.f : -1.f;
    const float* ga = gacc + (body * 6) * 32 + lane;
    V3 gdv = mk3(ga[0], ga[32], ga[64]);
    V3 gdw = mk3(ga[96], ga[128], ga[160]);
    if (bs.flags & kAnyFrozen) {
      gdv = mask3(bs.flags, gdv);
      gdw = mask3(bs.flags >> 3, gdw);
    }
    const S6& I = side == 0 ? Ia : Ib;
    const V3 x = side == 0 ? A.x : Bq.x;
    GSide& G = side == 0 ? GA : GB;
    gJ = fma3(sgn * bs.inv_mass, gdv, gJ);
    const V3 l = p - x;
    const V3 lJ = cross(l, J);
    V3 glJ = zero3();
    s6_mul_bwd(I, sgn * lJ, gdw, G.I, glJ);
    glJ = sgn * glJ;
    V3 gl = zero3();
    cross_bwd(l, J, glJ, gl, gJ);
    gp = gp + gl;
    G.x = G.x - gl;
  }
  // ---- response reverse (two bodies)
  float gjn = dot(gJ, n);
  V3 gn = jn * gJ;
  V3 gu = zero3(), gla = zero3(), glb = zero3();
  float gun = 0.f;
  if (fric) {
    const float gjt = -dot(gJ, t);
    V3 gt = (-jt) * gJ;
    float gutn = 0.f, gkt = 0.f;
    if (stick) {
      gutn = __fdividef(gjt, kt);
      gkt = -gjt * __fdividef(r1, kt);
    } else {
      gjn = fmaf(pr.mu, gjt, gjn);
    }
    eff_mass_bwd(ba.flags, ba.inv_mass, Ia, la, t, gkt, gla, gt, GA.I, true);
    eff_mass_bwd(bb.flags, bb.inv_mass, Ib, lb, t, gkt, glb, gt, GB.I, true);
    const V3 gut = fma3(gutn, t, rinv * fma3(-dot(t, gt), t, gt));
    gu = gu + gut;
    gun -= dot(gut, n);
    gn = fma3(-un, gut, gn);
  }
  float gdepth = 0.f;
  if (pos) {
    const float gq = gjn;
    const float gtarget = __fdividef(gq, kn);
    gun -= gtarget;
    const float gkn = -gq * __fdividef(qn, kn);
    if (first) gdepth = S.beta_h * gtarget;
    else gun = fmaf(-pr.e, gtarget, gun);
    eff_mass_bwd(ba.flags, ba.inv_mass, Ia, la, n, gkn, gla, gn, GA.I, true);
    eff_mass_bwd(bb.flags, bb.inv_mass, Ib, lb, n, gkn, glb, gn, GB.I, true);
  }
  gu = fma3(gun, n, gu);
  gn = fma3(gun, u, gn);
  GA.v = GA.v + gu;
  GA.w = GA.w + cross(la, gu);
  gla = gla + cross(gu, A.w);
  GB.v = GB.v - gu;
  GB.w = GB.w - cross(lb, gu);
  glb = glb - cross(gu, Bq.w);
  gp = gp + gla + glb;
  GA.x = GA.x - gla;
  GB.x = GB.x - glb;
  // ---- detection reverse
  V3 gP1 = zero3(), gd1 = zero3();
  if (pr.type == kCapsuleCapsule) {
    V3 gc1 = 0.5f * gp, gc2 = 0.5f * gp;
    gn = fma3(0.5f * (pr.rb - pr.ra), gp, gn);
    const float idl = __fdividef(1.f, dl);
    V3 gdf = idl * fma3(-dot(n, gn), n, gn);
    gdf = fma3(-gdepth, n, gdf);  // depth = ra + rb - |df|
    gc1 = gc1 + gdf;
    gc2 = gc2 - gdf;
    V3 gP2 = gc2, gd2 = tpar * gc2;
    gP1 = gc1;
    gd1 = sp * gc1;
    const float gsp = dot(gc1, d1), gtp = dot(gc2, d2);
    segment_closest_bwd(P1, d1, P2, d2, gsp, gtp, gP1, gd1, gP2, gd2);
    GB.x = GB.x + gP2;
    mulc_bwd(GB.R, gP2, pr.b0);
    const float db[3] = {pr.b1[0] - pr.b0[0], pr.b1[1] - pr.b0[1], pr.b1[2] - pr.b0[2]};
    mulc_bwd(GB.R, gd2, db);
  } else {
    M3 gRb;
    zero(gRb);
    // n = Rb nl, p = cb + Rb pl
    V3 gnl = mulT(Rb, gn);
    V3 gpl = mulT(Rb, gp);
    V3 gcb = gp;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float gni = i == 0 ? gn.x : (i == 1 ? gn.y : gn.z);
      const float gpi = i == 0 ? gp.x : (i == 1 ? gp.y : gp.z);
      gRb.m[3 * i + 0] += gni * nl.x + gpi * pl.x;
      gRb.m[3 * i + 1] += gni * nl.y + gpi * pl.y;
      gRb.m[3 * i + 2] += gni * nl.z + gpi * pl.z;
    }
    V3 ge = zero3();
    const float* he = pr.b1;
    if (!inside) {
      ge = 0.5f * gpl;
      gnl = fma3(-0.5f * pr.ra, gpl, gnl);
      V3 gq = 0.5f * gpl;
      const float idist = __fdividef(1.f, dist);
      V3 gdv = idist * fma3(-dot(nl, gnl), nl, gnl);
      gdv = fma3(-gdepth, nl, gdv);  // depth = ra - |dv|
      ge = ge + gdv;
      gq = gq - gdv;
      ge.x += (e.x > -he[0] && e.x < he[0]) ? gq.x : 0.f;
      ge.y += (e.y > -he[1] && e.y < he[1]) ? gq.y : 0.f;
      ge.z += (e.z > -he[2] && e.z < he[2]) ? gq.z : 0.f;
    } else {
      ge = gpl;
      const float gpen = 0.5f * dot(gpl, nl) + gdepth;
      if (kk == 0) ge.x -= sgk * gpen;
      else if (kk == 1) ge.y -= sgk * gpen;
      else ge.z -= sgk * gpen;
    }
    // e = Pl + t dl (t fixed)
    const V3 gPl = ge, gdl = tbox * ge;
    // Pl = Rb^T (P1 - cb), dl = Rb^T d1
    const V3 x1 = P1 - cb;
    const V3 gx1 = mul(Rb, gPl);
    gP1 = gx1;
    gcb = gcb - gx1;
    gd1 = mul(Rb, gdl);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float xi = i == 0 ? x1.x : (i == 1 ? x1.y : x1.z);
      const float di = i == 0 ? d1.x : (i == 1 ? d1.y : d1.z);
      gRb.m[3 * i + 0] += xi * gPl.x + di * gdl.x;
      gRb.m[3 * i + 1] += xi * gPl.y + di * gdl.y;
      gRb.m[3 * i + 2] += xi * gPl.z + di * gdl.z;
    }
    // Rb = R_b bR: gR_b += gRb bR^T ; cb = x_b + R_b b0
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        GB.R.m[3 * i + k] += gRb.m[3 * i + 0] * pr.bR[3 * k + 0] + gRb.m[3 * i + 1] * pr.bR[3 * k + 1] +
                             gRb.m[3 * i + 2] * pr.bR[3 * k + 2];
    GB.x = GB.x + gcb;
    mulc_bwd(GB.R, gcb, pr.b0);
  }
  GA.x = GA.x + gP1;
  mulc_bwd(GA.R, gP1, pr.a0);
  const float da[3] = {pr.a1[0] - pr.a0[0], pr.a1[1] - pr.a0[1], pr.a1[2] - pr.a0[2]};
  mulc_bwd(GA.R, gd1, da);
}

}  // namespace brax
