// Two environments per thread: the forward step of hinge-only systems.
//
// Same mapping as the scalar kernel (warp b = body b), but lane i of a group
// carries two environments, A = group*64 + i and B = group*64 + 32 + i.  Every
// floating-point quantity is a float2 (value in A, value in B) and the
// arithmetic is the packed FP32 instructions (two FMAs, adds or multiplies
// per instruction), so the FP32 work of the step takes half the issue slots
// of the one-environment kernel; parameters shared by A and B come from the
// constant pool as (value, value) pairs (SysP2, BodyP2).  Control flow that
// depends on data (limits, contacts, friction) is evaluated per environment
// and merged with selects or 0/1 masks, so both environments always run the
// same instructions.  The steps and their order are those of the scalar
// kernel (Algorithm 1, Sec. 3): kinematic integrator, joints + actuators +
// plane contacts on the post-kinematic state, potential integrator,
// collision integrator (mean of the contact velocity changes).
#pragma once
#include "brax_physics.cuh"

namespace brax {
namespace p2 {

using f2 = float2;

__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b in one packed instruction (there is no packed negation: a negated
// operand is either a negated parameter copy or a subtraction)
__device__ __forceinline__ f2 sub(f2 a, f2 b) {
  unsigned long long ra, rb, rd;
  memcpy(&ra, &a, 8);
  memcpy(&rb, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  f2 d;
  memcpy(&d, &rd, 8);
  return d;
}
__device__ __forceinline__ f2 zero2() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ f2 neg(f2 a) { return sub(zero2(), a); }

struct V {
  f2 x, y, z;
};
__device__ __forceinline__ V vzero() { return V{zero2(), zero2(), zero2()}; }
__device__ __forceinline__ V vadd(V a, V b) { return V{add(a.x, b.x), add(a.y, b.y), add(a.z, b.z)}; }
__device__ __forceinline__ V vsub(V a, V b) { return V{sub(a.x, b.x), sub(a.y, b.y), sub(a.z, b.z)}; }
__device__ __forceinline__ V vscale(f2 s, V a) { return V{mul(s, a.x), mul(s, a.y), mul(s, a.z)}; }
__device__ __forceinline__ V vfma(f2 s, V a, V b) { return V{fma(s, a.x, b.x), fma(s, a.y, b.y), fma(s, a.z, b.z)}; }
__device__ __forceinline__ f2 dot(V a, V b) { return fma(a.x, b.x, fma(a.y, b.y, mul(a.z, b.z))); }
__device__ __forceinline__ V cross(V a, V b) {
  return V{sub(mul(a.y, b.z), mul(a.z, b.y)), sub(mul(a.z, b.x), mul(a.x, b.z)), sub(mul(a.x, b.y), mul(a.y, b.x))};
}
// c + a x b
__device__ __forceinline__ V cross_add(V a, V b, V c) {
  return V{sub(fma(a.y, b.z, c.x), mul(a.z, b.y)), sub(fma(a.z, b.x, c.y), mul(a.x, b.z)),
           sub(fma(a.x, b.y, c.z), mul(a.y, b.x))};
}
__device__ __forceinline__ V vld(const f2* p) { return V{p[0], p[1], p[2]}; }

struct M {
  f2 m[9];
};
__device__ __forceinline__ V mulv(const M& R, V o) {
  return V{fma(R.m[0], o.x, fma(R.m[1], o.y, mul(R.m[2], o.z))), fma(R.m[3], o.x, fma(R.m[4], o.y, mul(R.m[5], o.z))),
           fma(R.m[6], o.x, fma(R.m[7], o.y, mul(R.m[8], o.z)))};
}
__device__ __forceinline__ V mulc(const M& R, const f2* o) { return mulv(R, vld(o)); }

__device__ __forceinline__ M qmat(f2 qw, f2 qx, f2 qy, f2 qz, f2 one) {
  const f2 x2 = add(qx, qx), y2 = add(qy, qy), z2 = add(qz, qz);
  const f2 xx = mul(qx, x2), yy = mul(qy, y2), zz = mul(qz, z2);
  const f2 wx = mul(qw, x2), wy = mul(qw, y2), wz = mul(qw, z2);
  M R;
  R.m[0] = sub(sub(one, yy), zz);
  R.m[1] = sub(mul(qx, y2), wz);
  R.m[2] = fma(qx, z2, wy);
  R.m[3] = fma(qx, y2, wz);
  R.m[4] = sub(sub(one, xx), zz);
  R.m[5] = sub(mul(qy, z2), wx);
  R.m[6] = sub(mul(qx, z2), wy);
  R.m[7] = fma(qy, z2, wx);
  R.m[8] = sub(sub(one, xx), yy);
  return R;
}

// Symmetric world inverse inertia R diag(d) R^T (xx, xy, xz, yy, yz, zz).
struct S6 {
  f2 a[6];
};
__device__ __forceinline__ S6 inv_inertia_world(const M& R, const f2* d) {
  S6 s;
  const f2 r00 = mul(R.m[0], d[0]), r01 = mul(R.m[1], d[1]), r02 = mul(R.m[2], d[2]);
  const f2 r10 = mul(R.m[3], d[0]), r11 = mul(R.m[4], d[1]), r12 = mul(R.m[5], d[2]);
  s.a[0] = fma(r00, R.m[0], fma(r01, R.m[1], mul(r02, R.m[2])));
  s.a[1] = fma(r00, R.m[3], fma(r01, R.m[4], mul(r02, R.m[5])));
  s.a[2] = fma(r00, R.m[6], fma(r01, R.m[7], mul(r02, R.m[8])));
  s.a[3] = fma(r10, R.m[3], fma(r11, R.m[4], mul(r12, R.m[5])));
  s.a[4] = fma(r10, R.m[6], fma(r11, R.m[7], mul(r12, R.m[8])));
  const f2 r20 = mul(R.m[6], d[0]), r21 = mul(R.m[7], d[1]), r22 = mul(R.m[8], d[2]);
  s.a[5] = fma(r20, R.m[6], fma(r21, R.m[7], mul(r22, R.m[8])));
  return s;
}
__device__ __forceinline__ V mul6(const S6& s, V v) {
  return V{fma(s.a[0], v.x, fma(s.a[1], v.y, mul(s.a[2], v.z))), fma(s.a[1], v.x, fma(s.a[3], v.y, mul(s.a[4], v.z))),
           fma(s.a[2], v.x, fma(s.a[4], v.y, mul(s.a[5], v.z)))};
}

__device__ __forceinline__ V mask(uint32_t bits, V a) {
  return V{(bits & 1u) ? zero2() : a.x, (bits & 2u) ? zero2() : a.y, (bits & 4u) ? zero2() : a.z};
}

// Per-environment arctangent (the scalar kernel's fast_atan2: octant
// reduction, the same degree-7 polynomial, octant undone), with the
// polynomial evaluated packed.
__device__ __forceinline__ f2 atan2p(f2 y, f2 x) {
  const float axa = fabsf(x.x), aya = fabsf(y.x), axb = fabsf(x.y), ayb = fabsf(y.y);
  const float mxa = fmaxf(axa, aya), mna = fminf(axa, aya);
  const float mxb = fmaxf(axb, ayb), mnb = fminf(axb, ayb);
  const f2 a = make_float2(mxa > 0.f ? __fdividef(mna, mxa) : 0.f, mxb > 0.f ? __fdividef(mnb, mxb) : 0.f);
  const f2 s = mul(a, a);
  f2 p = make_float2(-0.004037295f, -0.004037295f);
  p = fma(p, s, make_float2(0.021790044f, 0.021790044f));
  p = fma(p, s, make_float2(-0.055787466f, -0.055787466f));
  p = fma(p, s, make_float2(0.096311055f, 0.096311055f));
  p = fma(p, s, make_float2(-0.13903217f, -0.13903217f));
  p = fma(p, s, make_float2(0.19945158f, 0.19945158f));
  p = fma(p, s, make_float2(-0.3332969f, -0.3332969f));
  p = fma(p, s, make_float2(0.9999993f, 0.9999993f));
  const f2 r = mul(a, p);
  float ra = r.x, rb = r.y;
  if (aya > axa) ra = 1.5707963267948966f - ra;
  if (ayb > axb) rb = 1.5707963267948966f - rb;
  if (x.x < 0.f) ra = 3.141592653589793f - ra;
  if (x.y < 0.f) rb = 3.141592653589793f - rb;
  return make_float2(copysignf(ra, y.x), copysignf(rb, y.y));
}

struct Body {
  V x;
  f2 qw, qx, qy, qz;
  V v, w;
};
struct Frame {
  M R;
  S6 Ii;
};
struct Acc {
  V dv, dw;
  int na, nb;  // active contacts of environment A and B
};

// ------------------------------------------------------------------ group shared memory
// Two environments per lane: every field is one float2 (A, B) per lane, so a
// warp moves a field with one 8-byte access per lane.
// pub  [B][18][32] float2: x, R, v, w of a publishing body
// react[B][12][32] float2: a child's joint force F (the parent takes -F) and
//                          torque on its parent, then the joint's force and
//                          torque on the child itself (parked here between
//                          the joint and the integrator to free registers
//                          for the contact response)
constexpr int kPubFields2 = 18;
constexpr int kReactFields2 = 12;
// then the contact counts [64] int, two mbarriers (8 bytes each) and the
// group's action tile, double-buffered: [2][64 environments][A] floats (the
// 64 environments are contiguous in the action array, so one bulk copy brings
// a step's tile; every offset is a multiple of 16 bytes)
__host__ __device__ inline int group_floats2(int B, int A) {
  return 2 * 32 * B * (kPubFields2 + kReactFields2) + 64 + 4 + 2 * 64 * A;
}
struct GroupMem2 {
  f2* pub;
  f2* react;
  int* cnt;        // [64] contact counts (A lanes, then B lanes)
  uint64_t* mbar;  // [2] completion of the action tile's bulk copies
  float* tile;     // [2][64][A] action tiles
  __device__ __forceinline__ f2* pubf(int b, int f) { return pub + (b * kPubFields2 + f) * 32; }
  __device__ __forceinline__ f2* reactf(int b, int f) { return react + (b * kReactFields2 + f) * 32; }
};
__device__ __forceinline__ GroupMem2 group_mem2(float* base, int B) {
  GroupMem2 m;
  m.pub = reinterpret_cast<f2*>(base);
  m.react = m.pub + B * kPubFields2 * 32;
  m.cnt = reinterpret_cast<int*>(m.react + B * kReactFields2 * 32);
  m.mbar = reinterpret_cast<uint64_t*>(m.cnt + 64);
  m.tile = reinterpret_cast<float*>(m.mbar + 2);
  return m;
}

// ------------------------------------------------------------------ action tile (bulk asynchronous copy)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One thread: expect `bytes` on m and copy them from global src to shared dst
// (both 16-byte aligned, bytes a multiple of 16); the copy completes m's phase.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(m))
      : "memory");
}
// One thread: store `bytes` from shared src to global dst (both 16-byte
// aligned, bytes a multiple of 16) as one bulk asynchronous copy, committed
// as a bulk group of its own.
__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until the calling thread's bulk stores have read their shared sources
// (a store from shared to this GPU's memory always finishes).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until the calling thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Wait until m completes the phase of the given parity; gives up (returns
// false) after wait_ns nanoseconds of the global timer.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, int64_t wait_ns) {
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if ((int64_t)(t - t0) > wait_ns) return false;
  }
}

// ------------------------------------------------------------------ phase K
__device__ __forceinline__ void kinematic(const SysP2& S2, uint32_t flags, Body& s) {
  if (flags & kAnyFrozen) {
    s.v = mask(flags, s.v);
    s.w = mask(flags >> 3, s.w);
  }
  s.x = vfma(S2.h, s.v, s.x);
  const f2 hh = S2.hh;
  const f2 nw = fma(S2.mhh, fma(s.w.x, s.qx, fma(s.w.y, s.qy, mul(s.w.z, s.qz))), s.qw);
  const f2 nx = fma(hh, sub(fma(s.qw, s.w.x, mul(s.w.y, s.qz)), mul(s.w.z, s.qy)), s.qx);
  const f2 ny = fma(hh, sub(fma(s.qw, s.w.y, mul(s.w.z, s.qx)), mul(s.w.x, s.qz)), s.qy);
  const f2 nz = fma(hh, sub(fma(s.qw, s.w.z, mul(s.w.x, s.qy)), mul(s.w.y, s.qx)), s.qz);
  const f2 n2 = fma(nw, nw, fma(nx, nx, fma(ny, ny, mul(nz, nz))));
  const f2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
  s.qw = mul(nw, inv);
  s.qx = mul(nx, inv);
  s.qy = mul(ny, inv);
  s.qz = mul(nz, inv);
}

__device__ __forceinline__ void publish(GroupMem2& gm, int b, int lane, const Body& s, const Frame& f) {
  f2* p = gm.pubf(b, 0) + lane;
  p[0 * 32] = s.x.x;
  p[1 * 32] = s.x.y;
  p[2 * 32] = s.x.z;
#pragma unroll
  for (int i = 0; i < 9; ++i) p[(3 + i) * 32] = f.R.m[i];
  p[12 * 32] = s.v.x;
  p[13 * 32] = s.v.y;
  p[14 * 32] = s.v.z;
  p[15 * 32] = s.w.x;
  p[16 * 32] = s.w.y;
  p[17 * 32] = s.w.z;
}
struct Pub {
  V x;
  M R;
  V v, w;
};
__device__ __forceinline__ Pub read_pub(GroupMem2& gm, int b, int lane) {
  const f2* p = gm.pubf(b, 0) + lane;
  Pub o;
  o.x = V{p[0], p[32], p[64]};
#pragma unroll
  for (int i = 0; i < 9; ++i) o.R.m[i] = p[(3 + i) * 32];
  o.v = V{p[12 * 32], p[13 * 32], p[14 * 32]};
  o.w = V{p[15 * 32], p[16 * 32], p[17 * 32]};
  return o;
}

// ------------------------------------------------------------------ phase J: hinge joint
// The scalar kernel's hinge (Sec. 3 joint.revolute, Sec. 7.1, App. A limits,
// torque actuator); returns the child's wrench and writes the parent's.
struct Wrench {
  V F, tau;
};
__device__ __forceinline__ Wrench joint(const BodyP2& q, bool has_act, const Pub& pp, const Body& s, const Frame& f,
                                        f2 act, f2* react_out) {
  const V rp = mulc(pp.R, q.off_p);
  const V rc = mulc(f.R, q.off_c);
  const V dpc = vsub(vadd(pp.x, rp), vadd(s.x, rc));
  const V up = cross_add(pp.w, rp, pp.v);
  const V uc = cross_add(s.w, rc, s.v);
  const V du = vsub(uc, up);
  const V F = V{fma(q.k, dpc.x, mul(q.mc, du.x)), fma(q.k, dpc.y, mul(q.mc, du.y)), fma(q.k, dpc.z, mul(q.mc, du.z))};
  V tc = cross(rc, F);
  V tp = cross(F, rp);
  const V P0 = mulc(pp.R, q.ap + 0);
  const V P1 = mulc(pp.R, q.ap + 3);
  const V wr = vsub(s.w, pp.w);
  const V Ac = mulc(f.R, q.ac + 0);
  const V yc = mulc(f.R, q.ac + 3);
  const f2 th = atan2p(dot(cross(P1, yc), P0), dot(P1, yc));
  // one-sided limit springs, per environment
  const f2 dlo = sub(q.lo, th), dhi = sub(q.hi, th);
  const f2 Ld = make_float2(th.x < q.lo.x ? dlo.x : (th.x > q.hi.x ? dhi.x : 0.f),
                            th.y < q.lo.y ? dlo.y : (th.y > q.hi.y ? dhi.y : 0.f));
  f2 sc = fma(q.kl, Ld, mul(q.mca, dot(wr, P0)));
  if (has_act) {
    const f2 a = make_float2(fminf(fmaxf(act.x, -1.f), 1.f), fminf(fmaxf(act.y, -1.f), 1.f));
    sc = fma(q.gear, a, sc);
  }
  const V tj = vfma(sc, P0, vscale(q.ka, cross(Ac, P0)));
  tc = vadd(tc, tj);
  tp = vsub(tp, tj);
  react_out[0 * 32] = F.x;  // the parent takes -F: it subtracts
  react_out[1 * 32] = F.y;
  react_out[2 * 32] = F.z;
  react_out[3 * 32] = tp.x;
  react_out[4 * 32] = tp.y;
  react_out[5 * 32] = tp.z;
  react_out[6 * 32] = tc.x;  // the child's own torque (its force is F)
  react_out[7 * 32] = tc.y;
  react_out[8 * 32] = tc.z;
  return Wrench{F, tc};
}

// ------------------------------------------------------------------ phase J: plane contacts
__device__ __forceinline__ f2 eff_mass(uint32_t flags, f2 inv_m, const S6& Ii, V l, V dir) {
  V dm = dir;
  const V ld = cross(l, dir);
  V om = mul6(Ii, ld);
  if (flags & kAnyFrozen) {
    dm = mask(flags, dm);
    om = mask(flags >> 3, om);
  }
  return fma(dot(dm, dir), inv_m, dot(om, ld));
}

// Velocity-level response of one contact point for both environments
// (Sec. 7.2: Baumgarte target, Coulomb friction); environment A's result is
// added to acc when ma, B's when mb.  Inactive environments run the same
// instructions on finite values and are masked out.
__device__ __forceinline__ void point_response(const SysP2& S2, uint32_t flags, f2 inv_m, const PointP2& pt, V l, V n,
                                               f2 depth, bool ma, bool mb, const Body& s, const Frame& f, Acc& acc) {
  const V u = cross_add(s.w, l, s.v);
  const f2 kn = eff_mass(flags, inv_m, f.Ii, l, n);
  // a body that cannot move along n takes no impulse (as in the scalar kernel)
  const bool ka = kn.x > 0.f, kb = kn.y > 0.f;
  ma = ma && ka;
  mb = mb && kb;
  const f2 un = dot(u, n);
  const f2 ue = mul(pt.me, un);
  const f2 tb = mul(S2.beta_h, depth);
  const f2 target = make_float2(fmaxf(tb.x, ue.x), fmaxf(tb.y, ue.y));
  const f2 dn = sub(target, un);
  const f2 jn = make_float2(ka ? fmaxf(__fdividef(dn.x, kn.x), 0.f) : 0.f, kb ? fmaxf(__fdividef(dn.y, kn.y), 0.f) : 0.f);
  V J = vscale(jn, n);
  const V ut = vfma(neg(un), n, u);  // u - u_n n
  const f2 ut2 = dot(ut, ut);
  const bool fa = ut2.x > S2.eps2.x, fb = ut2.y > S2.eps2.y;
  if (__any_sync(0xffffffffu, fa || fb)) {
    const f2 rinv = make_float2(fa ? rsqrtf(ut2.x) : 0.f, fb ? rsqrtf(ut2.y) : 0.f);
    const f2 utn = mul(ut2, rinv);
    const V t = vscale(rinv, ut);
    const f2 kt = eff_mass(flags, inv_m, f.Ii, l, t);
    const f2 cap = mul(pt.mu, jn);
    const f2 jt = make_float2(fa && kt.x > 0.f ? fminf(__fdividef(utn.x, kt.x), cap.x) : 0.f,
                              fb && kt.y > 0.f ? fminf(__fdividef(utn.y, kt.y), cap.y) : 0.f);
    J = vfma(neg(jt), t, J);
  }
  V dv = vscale(inv_m, J);
  V dw = mul6(f.Ii, cross(l, J));
  if (flags & kAnyFrozen) {
    dv = mask(flags, dv);
    dw = mask(flags >> 3, dw);
  }
  const f2 m = make_float2(ma ? 1.f : 0.f, mb ? 1.f : 0.f);
  acc.dv = vfma(m, dv, acc.dv);
  acc.dw = vfma(m, dw, acc.dw);
  acc.na += ma ? 1 : 0;
  acc.nb += mb ? 1 : 0;
}

// Sphere-plane points of the own body (at most two): both are detected
// first (the rotation matrix is dead after that), then each point's response
// runs when any environment of the warp touches the plane there.
__device__ __forceinline__ void plane_points(const SysP2& S2, const BodyP2& q, uint32_t flags, int np, const Body& s,
                                             const Frame& f, Acc& acc) {
  V l0, l1;
  f2 d0 = make_float2(-1.f, -1.f), d1 = make_float2(-1.f, -1.f);
  if (np > 0) {
    const V ro = mulc(f.R, q.pt[0].o);
    d0 = sub(q.pt[0].r, dot(vsub(vadd(s.x, ro), vld(q.pt[0].p0)), vld(q.pt[0].n)));
    l0 = vfma(q.pt[0].mr, vld(q.pt[0].n), ro);
  }
  if (np > 1) {
    const V ro = mulc(f.R, q.pt[1].o);
    d1 = sub(q.pt[1].r, dot(vsub(vadd(s.x, ro), vld(q.pt[1].p0)), vld(q.pt[1].n)));
    l1 = vfma(q.pt[1].mr, vld(q.pt[1].n), ro);
  }
  if (np > 0) {
    const bool ma = d0.x > 0.f, mb = d0.y > 0.f;
    if (__any_sync(0xffffffffu, ma || mb))
      point_response(S2, flags, q.inv_mass, q.pt[0], l0, vld(q.pt[0].n), d0, ma, mb, s, f, acc);
  }
  if (np > 1) {
    const bool ma = d1.x > 0.f, mb = d1.y > 0.f;
    if (__any_sync(0xffffffffu, ma || mb))
      point_response(S2, flags, q.inv_mass, q.pt[1], l1, vld(q.pt[1].n), d1, ma, mb, s, f, acc);
  }
}

// ------------------------------------------------------------------ phase J: contacts with a z-up ground
// The same response for planes whose normal is the world z axis, n = (0, 0, 1),
// with the products by n's zero components dropped (they contribute exact
// zeros): l x n = (l.y, -l.x, 0), u_n = u.z, the tangential velocity is
// (u.x, u.y, 0) and the normal impulse acts along z alone.
__device__ __forceinline__ void point_response_z(const SysP2& S2, uint32_t flags, f2 inv_m, const PointP2& pt, V l,
                                                 f2 depth, bool ma, bool mb, const Body& s, const Frame& f,
                                                 Acc& acc) {
  const V u = cross_add(s.w, l, s.v);
  // k_n: linear term (unless z is frozen) + (I_w^-1 (l x n)) . (l x n)
  const f2 nlx = neg(l.x);
  f2 omx = fma(f.Ii.a[0], l.y, mul(f.Ii.a[1], nlx));
  f2 omy = fma(f.Ii.a[1], l.y, mul(f.Ii.a[3], nlx));
  if (flags & kAnyFrozen) {
    if (flags & (kFrozenRot0 << 0)) omx = zero2();
    if (flags & (kFrozenRot0 << 1)) omy = zero2();
  }
  const f2 lin = (flags & (kFrozenPos0 << 2)) ? zero2() : inv_m;
  const f2 kn = add(lin, fma(omx, l.y, mul(omy, nlx)));
  const bool ka = kn.x > 0.f, kb = kn.y > 0.f;
  ma = ma && ka;
  mb = mb && kb;
  const f2 un = u.z;
  const f2 ue = mul(pt.me, un);
  const f2 tb = mul(S2.beta_h, depth);
  const f2 target = make_float2(fmaxf(tb.x, ue.x), fmaxf(tb.y, ue.y));
  const f2 dn = sub(target, un);
  const f2 jn = make_float2(ka ? fmaxf(__fdividef(dn.x, kn.x), 0.f) : 0.f, kb ? fmaxf(__fdividef(dn.y, kn.y), 0.f) : 0.f);
  V J = V{zero2(), zero2(), jn};
  const f2 ut2 = fma(u.x, u.x, mul(u.y, u.y));
  const bool fa = ut2.x > S2.eps2.x, fb = ut2.y > S2.eps2.y;
  if (__any_sync(0xffffffffu, fa || fb)) {
    const f2 rinv = make_float2(fa ? rsqrtf(ut2.x) : 0.f, fb ? rsqrtf(ut2.y) : 0.f);
    const f2 utn = mul(ut2, rinv);
    const V t = V{mul(rinv, u.x), mul(rinv, u.y), zero2()};
    const f2 kt = eff_mass(flags, inv_m, f.Ii, l, t);
    const f2 cap = mul(pt.mu, jn);
    const f2 jt = make_float2(fa && kt.x > 0.f ? fminf(__fdividef(utn.x, kt.x), cap.x) : 0.f,
                              fb && kt.y > 0.f ? fminf(__fdividef(utn.y, kt.y), cap.y) : 0.f);
    const f2 njt = neg(jt);
    J.x = mul(njt, t.x);
    J.y = mul(njt, t.y);
  }
  V dv = vscale(inv_m, J);
  V dw = mul6(f.Ii, cross(l, J));
  if (flags & kAnyFrozen) {
    dv = mask(flags, dv);
    dw = mask(flags >> 3, dw);
  }
  const f2 m = make_float2(ma ? 1.f : 0.f, mb ? 1.f : 0.f);
  acc.dv = vfma(m, dv, acc.dv);
  acc.dw = vfma(m, dw, acc.dw);
  acc.na += ma ? 1 : 0;
  acc.nb += mb ? 1 : 0;
}

// plane_points for z-up planes: depth r - ((x + R o).z - p0.z), lever
// R o - r n = (R o).xy, (R o).z - r.
__device__ __forceinline__ void plane_points_z(const SysP2& S2, const BodyP2& q, uint32_t flags, int np,
                                               const Body& s, const Frame& f, Acc& acc) {
  V l0, l1;
  f2 d0 = make_float2(-1.f, -1.f), d1 = make_float2(-1.f, -1.f);
  if (np > 0) {
    const V ro = mulc(f.R, q.pt[0].o);
    d0 = sub(q.pt[0].r, sub(add(s.x.z, ro.z), q.pt[0].p0[2]));
    l0 = V{ro.x, ro.y, add(ro.z, q.pt[0].mr)};
  }
  if (np > 1) {
    const V ro = mulc(f.R, q.pt[1].o);
    d1 = sub(q.pt[1].r, sub(add(s.x.z, ro.z), q.pt[1].p0[2]));
    l1 = V{ro.x, ro.y, add(ro.z, q.pt[1].mr)};
  }
  if (np > 0) {
    const bool ma = d0.x > 0.f, mb = d0.y > 0.f;
    if (__any_sync(0xffffffffu, ma || mb)) point_response_z(S2, flags, q.inv_mass, q.pt[0], l0, d0, ma, mb, s, f, acc);
  }
  if (np > 1) {
    const bool ma = d1.x > 0.f, mb = d1.y > 0.f;
    if (__any_sync(0xffffffffu, ma || mb)) point_response_z(S2, flags, q.inv_mass, q.pt[1], l1, d1, ma, mb, s, f, acc);
  }
}

// ------------------------------------------------------------------ phase P
__device__ __forceinline__ void integrate(const SysP2& S2, bool average, const BodyP& bp, const BodyP2& q,
                                          GroupMem2& gm, int b, int lane, Body& s, const Frame& f, const Acc& acc) {
  Wrench wr{vzero(), vzero()};
  if (bp.flags & kHasParent) {  // the own joint's wrench, parked by joint()
    const f2* r = gm.reactf(b, 0) + lane;
    wr.F = V{r[0], r[32], r[64]};
    wr.tau = V{r[6 * 32], r[7 * 32], r[8 * 32]};
  }
  for (int c = 0; c < bp.n_children; ++c) {
    const f2* r = gm.reactf(bp.children[c], 0) + lane;
    wr.F = vsub(wr.F, V{r[0], r[32], r[64]});
    wr.tau = vadd(wr.tau, V{r[96], r[128], r[160]});
  }
  const f2 h = S2.h;
  V v = vfma(h, vfma(q.inv_mass, wr.F, vld(S2.g)), s.v);
  V w = vfma(h, mul6(f.Ii, wr.tau), s.w);
  if (bp.flags & kAnyFrozen) {
    v = mask(bp.flags, v);
    w = mask(bp.flags >> 3, w);
  }
  // mean (or sum) of the contact velocity changes; a body without contacts
  // adds its zero accumulator
  const float ia = (average && acc.na > 1) ? __fdividef(1.f, (float)acc.na) : 1.f;
  const float ib = (average && acc.nb > 1) ? __fdividef(1.f, (float)acc.nb) : 1.f;
  const f2 inv = make_float2(ia, ib);
  s.v = vfma(inv, acc.dv, v);
  s.w = vfma(inv, acc.dw, w);
}

}  // namespace p2
}  // namespace brax
