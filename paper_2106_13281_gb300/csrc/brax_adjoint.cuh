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
  const float th = atan2f(sy, cx);
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
  if (has_act) sc = fmaf(bp.gear[0], clamp1(act[0]), sc);
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
    if (a > -1.f && a < 1.f) gact[0] = fmaf(bp.gear[0], gsc, gact[0]);
  }
  // limit spring: d L / d th = -kl when active
  const float gth = lim ? -bp.kl * gL : 0.f;
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

}  // namespace brax
