// C ABI of the batched step: descriptor validation, the device parameter
// blob, launch configuration, status words.  Declarations and contracts are
// in include/brax.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/brax.h"
#include "brax_internal.h"
#include "brax_kernels.h"
#include "brax_params.h"

using namespace brax;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(BRAX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ host quaternion helpers (double)
void dq_normalize(double* q) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] /= n;
}
void dq_rotate(const double* q, const double* v, double* o) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  for (int i = 0; i < 3; ++i) o[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
}
void dq_matrix(const double* q, double R[3][3]) {
  double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, c[3];
  for (int j = 0; j < 3; ++j) {
    dq_rotate(q, e[j], c);
    for (int i = 0; i < 3; ++i) R[i][j] = c[i];
  }
}
bool finite_all(const float* p, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

struct Rejected {
  std::string msg;
};
#define REQUIRE(cond, msg)                  \
  do {                                      \
    if (!(cond)) throw Rejected{std::string(msg)}; \
  } while (0)

// Validate a descriptor and flatten it into the parameter blob.
std::vector<unsigned char> build_blob(const brax_desc& d, int* n_planes_out, int* P_out) {
  REQUIRE(d.version == 1 || d.version == BRAX_DESC_VERSION, "version: expected 1 or BRAX_DESC_VERSION");
  // a version-1 descriptor ends before the variant fields: they are off
  const bool v2 = d.version >= 2;
  const float lin_damp = v2 ? d.linear_damping : 0.f, ang_damp = v2 ? d.angular_damping_global : 0.f;
  const int gyro = v2 ? (d.gyroscopic != 0) : 0;
  const int32_t* act_type = v2 ? d.act_type : nullptr;
  REQUIRE(std::isfinite(lin_damp) && lin_damp >= 0.f && std::isfinite(ang_damp) && ang_damp >= 0.f,
          "linear_damping / angular_damping_global: must be finite and >= 0");
  const int B = d.n_bodies, J = d.n_joints, A = d.n_actuators, C = d.n_colliders, P = d.n_pairs;
  REQUIRE(B >= 1 && B <= BRAX_MAX_BODIES, "n_bodies: must be in [1, BRAX_MAX_BODIES]");
  REQUIRE(J >= 0 && J < B, "n_joints: must be in [0, n_bodies - 1]");
  REQUIRE(A >= 0 && C >= 0 && P >= 0, "counts must be non-negative");
  REQUIRE(d.substeps >= 1 && d.substeps <= 1000, "substeps: must be in [1, 1000]");
  REQUIRE(std::isfinite(d.dt) && d.dt > 0.f, "dt: must be positive and finite");
  REQUIRE(finite_all(d.gravity, 3), "gravity: must be finite");
  REQUIRE(std::isfinite(d.baumgarte) && d.baumgarte >= 0.f, "baumgarte: must be finite and >= 0");
  REQUIRE(std::isfinite(d.contact_eps) && d.contact_eps > 0.f, "contact_eps: must be positive");
  REQUIRE(d.mass && d.inertia && d.rest_pos && d.rest_rot && d.frozen_pos && d.frozen_rot, "body arrays: null");
  if (J > 0)
    REQUIRE(d.parent && d.child && d.dof && d.parent_offset && d.child_offset && d.parent_frame && d.child_frame &&
                d.stiffness && d.spring_damping && d.angular_stiffness && d.angular_damping && d.limit_lo &&
                d.limit_hi && d.limit_stiffness,
            "joint arrays: null");
  if (A > 0) REQUIRE(d.act_joint && d.act_axis && d.gear, "actuator arrays: null");
  if (C > 0)
    REQUIRE(d.col_body && d.col_type && d.col_pos && d.col_rot && d.radius && d.length && d.half_extents &&
                d.friction && d.elasticity,
            "collider arrays: null");
  if (P > 0) REQUIRE(d.pair_a && d.pair_b, "pair arrays: null");
  for (int b = 0; b < B; ++b) {
    REQUIRE(std::isfinite(d.mass[b]) && d.mass[b] > 0.f, "mass: must be positive and finite");
    for (int i = 0; i < 3; ++i) REQUIRE(std::isfinite(d.inertia[3 * b + i]) && d.inertia[3 * b + i] > 0.f,
                                        "inertia: must be positive and finite");
  }
  REQUIRE(finite_all(d.rest_pos, 3 * B) && finite_all(d.rest_rot, 4 * B), "rest pose: must be finite");

  const int Pb_max = BRAX_MAX_PAIRS;
  std::vector<SysP> sysv(1);
  SysP& S = sysv[0];
  std::memset(&S, 0, sizeof(S));
  std::vector<BodyP> bodies(B);
  std::memset(bodies.data(), 0, sizeof(BodyP) * B);
  for (int b = 0; b < B; ++b) {
    BodyP& bp = bodies[b];
    bp.inv_mass = (float)(1.0 / d.mass[b]);
    uint32_t fl = 0;
    for (int i = 0; i < 3; ++i) {
      bp.inv_I[i] = (float)(1.0 / d.inertia[3 * b + i]);
      bp.I[i] = d.inertia[3 * b + i];
      if (d.frozen_pos[3 * b + i]) fl |= kFrozenPos0 << i;
      if (d.frozen_rot[3 * b + i]) fl |= kFrozenRot0 << i;
    }
    if (fl) fl |= kAnyFrozen;
    bp.flags = fl;
    bp.parent = -1;
    bp.joint = -1;
    bp.dof = 0;
    for (int i = 0; i < 3; ++i) {
      bp.act[i] = -1;
      bp.rest_pos[i] = d.rest_pos[3 * b + i];
    }
    double rq[4] = {d.rest_rot[4 * b], d.rest_rot[4 * b + 1], d.rest_rot[4 * b + 2], d.rest_rot[4 * b + 3]};
    REQUIRE(rq[0] * rq[0] + rq[1] * rq[1] + rq[2] * rq[2] + rq[3] * rq[3] > 1e-12, "rest_rot: zero quaternion");
    dq_normalize(rq);
    for (int i = 0; i < 4; ++i) bp.rest_rot[i] = (float)rq[i];
  }
  // joints
  const double deg = 3.14159265358979323846 / 180.0;
  int D = 0;
  for (int j = 0; j < J; ++j) {
    const int p = d.parent[j], c = d.child[j];
    REQUIRE(p >= 0 && p < B && c >= 0 && c < B && p != c, "joint parent/child: out of range or equal");
    REQUIRE(d.dof[j] >= 1 && d.dof[j] <= 3, "dof: must be 1, 2 or 3");
    BodyP& bc = bodies[c];
    REQUIRE(bc.joint < 0, "child: a body may be the child of only one joint");
    REQUIRE(bodies[p].n_children < BRAX_MAX_CHILDREN, "parent: more than BRAX_MAX_CHILDREN children");
    bodies[p].children[bodies[p].n_children++] = c;
    bodies[p].flags |= kPublish;
    bc.joint = j;
    bc.parent = p;
    bc.dof = d.dof[j];
    bc.flags |= kHasParent;
    bc.dof_offset = D;
    D += d.dof[j];
    REQUIRE(finite_all(d.parent_offset + 3 * j, 3) && finite_all(d.child_offset + 3 * j, 3), "offsets: not finite");
    for (int i = 0; i < 3; ++i) {
      bc.off_p[i] = d.parent_offset[3 * j + i];
      bc.off_c[i] = d.child_offset[3 * j + i];
    }
    double fp[4], fc[4];
    for (int i = 0; i < 4; ++i) {
      fp[i] = d.parent_frame[4 * j + i];
      fc[i] = d.child_frame[4 * j + i];
    }
    REQUIRE(fp[0] * fp[0] + fp[1] * fp[1] + fp[2] * fp[2] + fp[3] * fp[3] > 1e-12 &&
                fc[0] * fc[0] + fc[1] * fc[1] + fc[2] * fc[2] + fc[3] * fc[3] > 1e-12,
            "joint frames: zero quaternion");
    dq_normalize(fp);
    dq_normalize(fc);
    const double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int a = 0; a < 3; ++a) {
      double o[3];
      dq_rotate(fp, e[a], o);
      for (int i = 0; i < 3; ++i) bc.ap[3 * a + i] = (float)o[i];
      dq_rotate(fc, e[a], o);
      for (int i = 0; i < 3; ++i) bc.ac[3 * a + i] = (float)o[i];
    }
    for (int i = 0; i < 4; ++i) {
      bc.frame_p[i] = (float)fp[i];
      bc.frame_c[i] = (float)fc[i];
    }
    const float kk[5] = {d.stiffness[j], d.spring_damping[j], d.angular_stiffness[j], d.angular_damping[j],
                         d.limit_stiffness[j]};
    for (float v : kk) REQUIRE(std::isfinite(v) && v >= 0.f, "joint constants: must be finite and >= 0");
    bc.k = kk[0];
    bc.c = kk[1];
    bc.ka = kk[2];
    bc.ca = kk[3];
    bc.kl = kk[4];
    for (int a = 0; a < 3; ++a) {
      REQUIRE(std::isfinite(d.limit_lo[3 * j + a]) && std::isfinite(d.limit_hi[3 * j + a]), "limits: not finite");
      bc.lo[a] = (float)(d.limit_lo[3 * j + a] * deg);
      bc.hi[a] = (float)(d.limit_hi[3 * j + a] * deg);
    }
    if (d.dof[j] == 2) {  // the third axis has no limit: its twist spring holds it (joint_forward)
      bc.lo[2] = -3.14159265358979323846f;
      bc.hi[2] = 3.14159265358979323846f;
    }
  }
  // topological order of joints (children of placed bodies)
  {
    std::vector<int> placed(B, 0);
    for (int b = 0; b < B; ++b) placed[b] = bodies[b].joint < 0;
    int n = 0;
    for (int pass = 0; pass <= J && n < J; ++pass)
      for (int b = 0; b < B; ++b)
        if (!placed[b] && bodies[b].joint >= 0 && placed[bodies[b].parent]) {
          S.joint_order[n++] = b;
          placed[b] = 1;
        }
    REQUIRE(n == J, "joints: the joint graph has a cycle");
    S.n_order = n;
    int np = 0;
    for (int b = 0; b < B; ++b) bodies[b].tree_slot = bodies[b].n_children > 0 ? np++ : -1;
    S.n_parents = np;
  }
  // actuators
  for (int k = 0; k < A; ++k) {
    const int j = d.act_joint[k];
    REQUIRE(j >= 0 && j < J, "act_joint: out of range");
    const int c = d.child[j];
    const int ax = d.act_axis[k];
    REQUIRE(ax >= 0 && ax < d.dof[j], "act_axis: out of range for the joint's dof");
    REQUIRE(bodies[c].act[ax] < 0, "actuators: at most one actuator per (joint, axis)");
    REQUIRE(std::isfinite(d.gear[k]), "gear: not finite");
    bodies[c].act[ax] = k;
    bodies[c].gear[ax] = d.gear[k];
    if (act_type) {
      REQUIRE(act_type[k] == 0 || act_type[k] == 1, "act_type: must be 0 (torque) or 1 (target angle)");
      if (act_type[k] == 1) {
        const double lo = d.limit_lo[3 * j + ax] * deg, hi = d.limit_hi[3 * j + ax] * deg;
        bodies[c].act_angle |= 1 << ax;
        bodies[c].act_mid[ax] = (float)(0.5 * (lo + hi));
        bodies[c].act_half[ax] = (float)(0.5 * (hi - lo));
      }
    }
  }
  // colliders, planes
  std::vector<int> plane_slot(C, -1);
  std::vector<PlaneP> planes;
  for (int c = 0; c < C; ++c) {
    const int t = d.col_type[c];
    REQUIRE(t == BRAX_PLANE || t == BRAX_CAPSULE || t == BRAX_BOX, "col_type: unknown");
    REQUIRE(finite_all(d.col_pos + 3 * c, 3) && finite_all(d.col_rot + 4 * c, 4), "collider pose: not finite");
    if (t == BRAX_PLANE) {
      REQUIRE(d.col_body[c] == -1, "planes must be static (col_body -1)");
      REQUIRE((int)planes.size() < BRAX_MAX_PLANES, "more than BRAX_MAX_PLANES planes");
      double q[4] = {d.col_rot[4 * c], d.col_rot[4 * c + 1], d.col_rot[4 * c + 2], d.col_rot[4 * c + 3]};
      dq_normalize(q);
      const double ez[3] = {0, 0, 1};
      double n[3];
      dq_rotate(q, ez, n);
      PlaneP pl;
      for (int i = 0; i < 3; ++i) {
        pl.p0[i] = d.col_pos[3 * c + i];
        pl.n[i] = (float)n[i];
      }
      plane_slot[c] = (int)planes.size();
      planes.push_back(pl);
    } else {
      REQUIRE(d.col_body[c] >= 0 && d.col_body[c] < B, "col_body: capsules and boxes need a body");
      if (t == BRAX_CAPSULE)
        REQUIRE(d.radius[c] > 0.f && d.length[c] >= 0.f && std::isfinite(d.radius[c]) && std::isfinite(d.length[c]),
                "capsule: radius > 0, length >= 0");
      else
        for (int i = 0; i < 3; ++i) REQUIRE(d.half_extents[3 * c + i] > 0.f, "box: half extents must be > 0");
    }
    REQUIRE(std::isfinite(d.friction[c]) && d.friction[c] >= 0.f, "friction: must be finite and >= 0");
    REQUIRE(std::isfinite(d.elasticity[c]) && d.elasticity[c] >= 0.f, "elasticity: must be finite and >= 0");
  }
  auto capsule_local = [&](int c, double* e0, double* e1) {
    double q[4] = {d.col_rot[4 * c], d.col_rot[4 * c + 1], d.col_rot[4 * c + 2], d.col_rot[4 * c + 3]};
    dq_normalize(q);
    const double ez[3] = {0, 0, 1};
    double ax[3];
    dq_rotate(q, ez, ax);
    const double hs = std::max(0.5 * (double)d.length[c] - (double)d.radius[c], 0.0);
    for (int i = 0; i < 3; ++i) {
      e0[i] = d.col_pos[3 * c + i] - hs * ax[i];
      e1[i] = d.col_pos[3 * c + i] + hs * ax[i];
    }
    return hs;
  };
  // pairs
  std::vector<PairP> pairs;
  std::vector<int> body_pcol(B, -1), body_multi(B, 0);  // a body's collider in pairs; several of them
  for (int k = 0; k < P; ++k) {
    int ca = d.pair_a[k], cb = d.pair_b[k];
    REQUIRE(ca >= 0 && ca < C && cb >= 0 && cb < C && ca != cb, "pair: collider index out of range");
    if (d.col_type[ca] == BRAX_PLANE || (d.col_type[ca] == BRAX_BOX && d.col_type[cb] == BRAX_CAPSULE))
      std::swap(ca, cb);
    const int ta = d.col_type[ca], tb = d.col_type[cb];
    const float mu = d.friction[ca] * d.friction[cb];
    const float el = d.elasticity[ca] * d.elasticity[cb];
    REQUIRE(ta != BRAX_PLANE, "pair: plane against plane");
    const int ba = d.col_body[ca];
    if (tb == BRAX_PLANE) {
      BodyP& bp = bodies[ba];
      auto add_point = [&](const double* o, double r) {
        REQUIRE(bp.n_points < BRAX_MAX_POINTS, "body: more than BRAX_MAX_POINTS plane-contact points");
        PointP& pt = bp.pt[bp.n_points++];
        for (int i = 0; i < 3; ++i) pt.o[i] = (float)o[i];
        pt.r = (float)r;
        pt.mu = mu;
        pt.e = el;
        pt.plane = plane_slot[cb];
        pt.pad = 0;
      };
      if (ta == BRAX_CAPSULE) {
        double e0[3], e1[3];
        double hs = capsule_local(ca, e0, e1);
        add_point(e0, d.radius[ca]);
        if (hs > 0.0) add_point(e1, d.radius[ca]);
      } else {
        double q[4] = {d.col_rot[4 * ca], d.col_rot[4 * ca + 1], d.col_rot[4 * ca + 2], d.col_rot[4 * ca + 3]};
        dq_normalize(q);
        const float* he = d.half_extents + 3 * ca;
        for (int m = 0; m < 8; ++m) {
          double cl[3] = {(m & 1) ? he[0] : -he[0], (m & 2) ? he[1] : -he[1], (m & 4) ? he[2] : -he[2]};
          double cr[3], co[3];
          dq_rotate(q, cl, cr);
          for (int i = 0; i < 3; ++i) co[i] = d.col_pos[3 * ca + i] + cr[i];
          add_point(co, 0.0);
        }
      }
    } else {
      REQUIRE(ta == BRAX_CAPSULE, "pair: box-box pairs are not supported");
      const int bb = d.col_body[cb];
      REQUIRE(ba != bb, "pair: both colliders on one body");
      REQUIRE((int)pairs.size() < Pb_max, "more than BRAX_MAX_PAIRS body-body pairs");
      PairP pr;
      std::memset(&pr, 0, sizeof(pr));
      pr.type = tb == BRAX_CAPSULE ? kCapsuleCapsule : kCapsuleBox;
      pr.ba = ba;
      pr.bb = bb;
      pr.mu = mu;
      pr.e = el;
      pr.ra = d.radius[ca];
      double a0[3], a1[3];
      capsule_local(ca, a0, a1);
      for (int i = 0; i < 3; ++i) {
        pr.a0[i] = (float)a0[i];
        pr.a1[i] = (float)a1[i];
      }
      if (tb == BRAX_CAPSULE) {
        double b0[3], b1[3];
        capsule_local(cb, b0, b1);
        pr.rb = d.radius[cb];
        for (int i = 0; i < 3; ++i) {
          pr.b0[i] = (float)b0[i];
          pr.b1[i] = (float)b1[i];
        }
      } else {
        double q[4] = {d.col_rot[4 * cb], d.col_rot[4 * cb + 1], d.col_rot[4 * cb + 2], d.col_rot[4 * cb + 3]};
        dq_normalize(q);
        double R[3][3];
        dq_matrix(q, R);
        for (int i = 0; i < 3; ++i) {
          pr.b0[i] = d.col_pos[3 * cb + i];
          pr.b1[i] = d.half_extents[3 * cb + i];
          for (int j = 0; j < 3; ++j) pr.bR[3 * i + j] = (float)R[i][j];
        }
      }
      {  // broadphase bound (PairP::bound2)
        auto seg_half = [&](int ci) {
          double e0[3], e1[3];
          capsule_local(ci, e0, e1);
          const double dx = e1[0] - e0[0], dy = e1[1] - e0[1], dz = e1[2] - e0[2];
          return 0.5 * std::sqrt(dx * dx + dy * dy + dz * dz);
        };
        double ra = seg_half(ca) + d.radius[ca], rb;
        if (tb == BRAX_CAPSULE) {
          rb = seg_half(cb) + d.radius[cb];
        } else {
          const float* he = d.half_extents + 3 * cb;
          rb = std::sqrt((double)he[0] * he[0] + (double)he[1] * he[1] + (double)he[2] * he[2]);
        }
        const double bnd = (ra + rb) * (1.0 + 1e-4) + 1e-5;
        pr.bound2 = (float)(bnd * bnd);
      }
      const int idx = (int)pairs.size();
      pairs.push_back(pr);
      for (int side = 0; side < 2; ++side) {
        const int bi = side == 0 ? ba : bb, ci = side == 0 ? ca : cb;
        if (body_pcol[bi] < 0) body_pcol[bi] = ci;
        else if (body_pcol[bi] != ci) body_multi[bi] = 1;
        BodyP& bp = bodies[side == 0 ? ba : bb];
        REQUIRE(bp.n_bpairs < BRAX_MAX_BODY_PAIRS, "body: more than BRAX_MAX_BODY_PAIRS body-body pairs");
        bp.bpair[bp.n_bpairs++] = (idx << 1) | side;
        bp.flags |= kPublish | kInPair;
      }
    }
  }
  const int Pb = (int)pairs.size();
  // bodies with exactly one collider in pairs publish its world geometry
  for (int b = 0; b < B; ++b) {
    BodyP& bp = bodies[b];
    bp.gtype = -1;
    const int c = body_pcol[b];
    if (c < 0 || body_multi[b]) continue;
    if (d.col_type[c] == BRAX_CAPSULE) {
      double e0[3], e1[3];
      capsule_local(c, e0, e1);
      bp.gtype = 0;
      for (int i = 0; i < 3; ++i) {
        bp.g0[i] = (float)e0[i];
        bp.g1[i] = (float)e1[i];
      }
    } else {
      double q[4] = {d.col_rot[4 * c], d.col_rot[4 * c + 1], d.col_rot[4 * c + 2], d.col_rot[4 * c + 3]};
      dq_normalize(q);
      double Rm[3][3];
      dq_matrix(q, Rm);
      bp.gtype = 1;
      for (int i = 0; i < 3; ++i) {
        bp.g0[i] = d.col_pos[3 * c + i];
        for (int j = 0; j < 3; ++j) bp.g1[3 * i + j] = (float)Rm[i][j];
      }
    }
  }
  for (int k = 0; k < Pb; ++k) {
    pairs[k].geo = 0;
    if (bodies[pairs[k].ba].gtype >= 0) pairs[k].geo |= 1;
    if (bodies[pairs[k].bb].gtype >= 0) pairs[k].geo |= 2;
  }
  S.B = B;
  S.J = J;
  S.A = A;
  S.D = D;
  S.P = Pb;
  S.n_planes = (int)planes.size();
  S.flat = 1;
  for (const PlaneP& pl : planes) S.flat = S.flat && pl.n[0] == 0.f && pl.n[1] == 0.f && pl.n[2] == 1.f;
  S.substeps = d.substeps;
  S.average = d.average_contacts ? 1 : 0;
  S.general = Pb > 0 ? 1 : 0;
  for (int j = 0; j < J; ++j)
    if (d.dof[j] >= 2) S.general = 1;
  // variants run in the general kernel (forward and reverse)
  S.lin_damp = lin_damp;
  S.ang_damp = ang_damp;
  S.gyro = gyro;
  S.variants = (lin_damp != 0.f || ang_damp != 0.f || gyro) ? 1 : 0;
  for (int b = 0; b < B; ++b)
    if (bodies[b].act_angle) S.variants = 1;
  if (S.variants) S.general = 1;
  S.iso = 1;
  for (int b = 0; b < S.B; ++b)
    S.iso = S.iso && bodies[b].inv_I[0] == bodies[b].inv_I[1] && bodies[b].inv_I[1] == bodies[b].inv_I[2];
  const double h = (double)d.dt / d.substeps;
  S.h = (float)h;
  S.beta_h = (float)(d.baumgarte / h);
  S.eps = d.contact_eps;
  for (int i = 0; i < 3; ++i) S.g[i] = d.gravity[i];

  // Two environments per thread need hinge joints only and at most two
  // plane-contact points per body.
  bool paired = !S.general;
  for (int b = 0; b < B; ++b) paired = paired && bodies[b].n_points <= 2;
  const int base_bytes = blob_bytes(B, Pb, S.n_planes);
  S.paired = paired ? 1 : 0;
  S.pair_off = paired ? base_bytes : 0;
  std::vector<unsigned char> blob(base_bytes + (paired ? blob_pair_bytes(B) : 0), 0);
  if (paired) {
    auto f2 = [](float v) { return make_float2(v, v); };
    SysP2 S2;
    std::memset(&S2, 0, sizeof(S2));
    S2.h = f2(S.h);
    S2.mhh = f2(-0.5f * S.h);
    S2.hh = f2(0.5f * S.h);
    S2.beta_h = f2(S.beta_h);
    S2.eps2 = f2(S.eps * S.eps);
    for (int i = 0; i < 3; ++i) S2.g[i] = f2(S.g[i]);
    S2.one = f2(1.f);
    S2.mone = f2(-1.f);
    std::memcpy(blob.data() + base_bytes, &S2, sizeof(S2));
    for (int b = 0; b < B; ++b) {
      const BodyP& bp = bodies[b];
      BodyP2 q;
      std::memset(&q, 0, sizeof(q));
      for (int i = 0; i < 3; ++i) {
        q.off_p[i] = f2(bp.off_p[i]);
        q.off_c[i] = f2(bp.off_c[i]);
        q.inv_I[i] = f2(bp.inv_I[i]);
      }
      for (int i = 0; i < 6; ++i) {
        q.ap[i] = f2(bp.ap[i]);
        q.ac[i] = f2(bp.ac[i]);
      }
      q.k = f2(bp.k);
      q.mc = f2(-bp.c);
      q.ka = f2(bp.ka);
      q.mca = f2(-bp.ca);
      q.kl = f2(bp.kl);
      q.lo = f2(bp.lo[0]);
      q.hi = f2(bp.hi[0]);
      q.gear = f2(bp.gear[0]);
      q.inv_mass = f2(bp.inv_mass);
      for (int k = 0; k < bp.n_points; ++k) {
        const PointP& pt = bp.pt[k];
        const PlaneP& pl = planes[pt.plane];
        for (int i = 0; i < 3; ++i) {
          q.pt[k].o[i] = f2(pt.o[i]);
          q.pt[k].n[i] = f2(pl.n[i]);
          q.pt[k].p0[i] = f2(pl.p0[i]);
        }
        q.pt[k].r = f2(pt.r);
        q.pt[k].mr = f2(-pt.r);
        q.pt[k].mu = f2(pt.mu);
        q.pt[k].me = f2(-pt.e);
      }
      std::memcpy(blob.data() + base_bytes + sizeof(SysP2) + b * sizeof(BodyP2), &q, sizeof(q));
    }
  }
  std::memcpy(blob.data(), &S, sizeof(SysP));
  std::memcpy(blob.data() + blob_bodies_off(), bodies.data(), sizeof(BodyP) * B);
  if (Pb) std::memcpy(blob.data() + blob_pairs_off(B), pairs.data(), sizeof(PairP) * Pb);
  if (!planes.empty()) std::memcpy(blob.data() + blob_planes_off(B, Pb), planes.data(), sizeof(PlaneP) * planes.size());
  *n_planes_out = S.n_planes;
  *P_out = Pb;
  return blob;
}

}  // namespace

namespace {

size_t group_bytes(const brax_system* s) { return (size_t)group_floats(s->B, s->P) * sizeof(float); }

// First-fit allocator of the constant parameter pool, one per device.
// Systems with byte-identical blobs share one range (reference counted), so
// many handles of one scene cost the pool once.
struct PoolRange {
  int device, off, bytes, refs;
  std::vector<unsigned char> content;
};
std::vector<PoolRange> g_pool;
std::mutex g_pool_mu;

// Returns the offset of `blob` in the device's pool (uploading it to the
// constant pools of the kernel translation units when it is new), -1 when
// the pool is full, or -2 - cudaError when the upload failed.
static_assert(alignof(SysP) <= 16 && alignof(BodyP) <= 16 && alignof(PairP) <= 16 && alignof(PlaneP) <= 16 &&
                  alignof(SysP2) <= 16 && alignof(BodyP2) <= 16,
              "blob sections and constant-pool ranges start on 16-byte boundaries");
int pool_acquire(int device, const std::vector<unsigned char>& blob) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto& r : g_pool)
    if (r.device == device && r.content == blob) {
      ++r.refs;
      return r.off;
    }
  const int bytes = (int)blob.size();
  std::vector<const PoolRange*> used;
  for (const auto& r : g_pool)
    if (r.device == device) used.push_back(&r);
  std::sort(used.begin(), used.end(), [](const PoolRange* a, const PoolRange* b) { return a->off < b->off; });
  // first fit; ranges start on 16-byte boundaries (the parameter structs need
  // 8, the blob sections are laid out from 16)
  int off = 0;
  for (const auto* r : used) {
    if (r->off - off >= bytes) break;
    off = std::max(off, (r->off + r->bytes + 15) & ~15);
  }
  if (off + bytes > kPoolBytes) return -1;
  cudaError_t e = upload_pool_forward(off, blob.data(), blob.size());
  if (e == cudaSuccess) e = upload_pool_backward(off, blob.data(), blob.size());
  if (e != cudaSuccess) return -2 - (int)e;
  g_pool.push_back(PoolRange{device, off, bytes, 1, blob});
  return off;
}
void pool_release(int device, int off) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (size_t i = 0; i < g_pool.size(); ++i)
    if (g_pool[i].device == device && g_pool[i].off == off) {
      if (--g_pool[i].refs == 0) g_pool.erase(g_pool.begin() + i);
      return;
    }
}

// Default launch-bounds variant: the smallest that admits the block (the
// autotuner may pick another).
int pick_variant(int threads) {
  static const int order[4] = {3, 0, 1, 2};
  for (int v : order)
    if (threads <= rollout_variant_max_threads(v)) return v;
  return -1;
}
// The reverse kernel's default launch (before any autotuning): the adjoint
// holds more live values than the forward, so the largest register budget
// whose block fits, (576, 1) or (1024, 1); the tighter bounds spill more than
// the extra resident blocks hide (quadruped reverse, 65,536 x 100: 53 ms
// under (288, 3), 41 ms under (576, 1)).
int pick_bwd_variant(int threads) {
  static const int order[2] = {1, 2};
  for (int v : order)
    if (threads <= backward_variant_max_threads(v)) return v;
  return -1;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

Seg make_seg(const brax_system* s, int groups, int64_t n_envs) {
  Seg sg;
  std::memset(&sg, 0, sizeof(sg));
  sg.blob = s->d_blob;
  sg.pool_off = s->pool_off;
  sg.blob_bytes = (int32_t)s->blob.size();
  sg.B = s->B;
  sg.P = s->P;
  sg.A = s->A;
  sg.groups = groups;
  sg.n_envs = n_envs;
  sg.status = s->d_status;
  return sg;
}

// Chunked schedule of a rollout of `units` blocks (Sched), per_sm of which
// are resident per SM, over T steps (reverse pass: T checkpoint segments).
// Taken when the units leave the last resident wave less than 97 % full
// (mode 1), or always (mode 2, chunks of `chunk` steps).  Mode 1 picks the
// chunk length (at least min_chunk steps: 16, or 16 steps' worth of
// segments) that minimises a round model of the launch: items run in rounds
// of `slots` blocks in chunk-major order, a round lasts as long as its
// longest item (a full chunk, or the shorter last chunk), and every item
// costs a quarter step more (a new block, the state through L2, a flag
// check).
struct SchedPlan {
  int n_chunks = 0, chunk_steps = 0;
};
// The plan for `slots` resident blocks (host arithmetic only).
SchedPlan plan_schedule_slots(int mode, int chunk, int64_t units, int T, int64_t slots, int min_chunk) {
  SchedPlan p;
  if (mode == 0 || T < 2 || units < 1 || slots < 1) return p;
  int64_t steps;
  if (mode == 2) {
    steps = std::max(1, chunk);
  } else {
    const int64_t waves = (units + slots - 1) / slots;
    if (units <= slots || (double)units >= 0.97 * (double)(waves * slots)) return p;
    steps = 0;
    double best = 0.0;
    for (int64_t len = std::max(1, min_chunk); len <= (T + 1) / 2; ++len) {
      const int64_t C = (T + len - 1) / len;
      if (C < 2) continue;
      const int64_t last = T - (C - 1) * len;
      const int64_t rounds = (C * units + slots - 1) / slots;
      const int64_t full = std::min(rounds, ((C - 1) * units + slots - 1) / slots);
      const double t = (double)(full * len + (rounds - full) * last) + 0.25 * (double)(C * units) / (double)slots;
      if (steps == 0 || t < best - 1e-9) {
        best = t;
        steps = len;
      }
    }
    if (steps == 0) return p;
  }
  const int64_t C = (T + steps - 1) / steps;
  if (C < 2 || C * units > 0x3fffffff) return p;
  p.n_chunks = (int)C;
  p.chunk_steps = (int)steps;
  return p;
}
SchedPlan plan_schedule(int mode, int chunk, int device, int64_t units, int T, int per_sm, int min_chunk = 16) {
  if (mode == 0 || T < 2 || units < 1 || per_sm < 1) return SchedPlan{};
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return SchedPlan{};
  }
  return plan_schedule_slots(mode, chunk, units, T, (int64_t)per_sm * n_sm, min_chunk);
}

// One region of a scheduler scratch for a launch of `units` units (null when
// it cannot be had: the caller then runs the static schedule).  Growing the
// scratch allocates, which a stream under capture does not allow.
int32_t* sched_region(SchedScratch& sc, int64_t units, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(sc.mu);
  if (units > sc.units) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return nullptr;
    }
    const int64_t cap = std::max<int64_t>(units, 2 * sc.units);
    int32_t* d = nullptr;
    if (cudaMalloc(&d, SchedScratch::kRing * (32 + cap) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    if (sc.d) sc.retired.push_back(sc.d);
    sc.d = d;
    sc.units = cap;
  }
  const int r = sc.next;
  sc.next = (r + 1) % SchedScratch::kRing;
  return sc.d + r * (32 + sc.units);
}
void sched_free(SchedScratch& sc) {
  if (sc.d) cudaFree(sc.d);
  for (int32_t* d : sc.retired) cudaFree(d);
  sc.d = nullptr;
  sc.retired.clear();
}

// A caller-provided scheduler region: `fixed` (device memory of `bytes`
// bytes) is used instead of the system's own scratch; with use = true and a
// region too small (or null) the launch takes the static schedule, so that
// nothing is allocated.
struct FixedRegion {
  bool use = false;
  int32_t* fixed = nullptr;
  size_t bytes = 0;
};

// Fill L.sc for a chunked launch of `units` units when the plan asks for one
// and scratch can be had; returns the grid (one block per item, or `units`).
// Fails only if zeroing the scratch region fails.
cudaError_t apply_schedule(const SchedPlan& pl, SchedScratch& sc, int first_item, int64_t wait_ns, int64_t units,
                           Launch& L, int64_t* grid, cudaStream_t st, const FixedRegion& fr = FixedRegion{}) {
  *grid = units;
  if (pl.n_chunks == 0) return cudaSuccess;
  int32_t* region = nullptr;
  if (fr.use) {
    if (fr.fixed && fr.bytes >= (size_t)(32 + units) * sizeof(int32_t)) region = fr.fixed;
  } else {
    region = sched_region(sc, units, st);
  }
  if (!region) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(region, 0, (32 + units) * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  L.sc.n_chunks = pl.n_chunks;
  L.sc.chunk_steps = pl.chunk_steps;
  L.sc.n_units = (int32_t)units;
  L.sc.first_item = first_item;
  L.sc.sched = region;
  L.sc.wait_ns = wait_ns;
  *grid = (int64_t)pl.n_chunks * units;
  return cudaSuccess;
}

}  // namespace

extern "C" {

const char* brax_last_error(void) { return g_err.c_str(); }

int brax_system_create(const brax_desc* desc, brax_system** out) {
  if (!desc || !out) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_create: null argument");
  *out = nullptr;
  brax_system* s = new brax_system();
  try {
    s->blob = build_blob(*desc, &s->n_planes, &s->P);
  } catch (const Rejected& r) {
    delete s;
    return fail(BRAX_ERR_INVALID_DESCRIPTOR, "brax_system_create: " + r.msg);
  }
  const SysP* S = reinterpret_cast<const SysP*>(s->blob.data());
  s->B = S->B;
  s->A = S->A;
  s->D = S->D;
  s->general = S->general != 0;
  // the isotropic reverse kernel keeps at most two contact points a body in registers
  s->iso = S->iso != 0;
  for (int b = 0; b < S->B; ++b)
    if (reinterpret_cast<const BodyP*>(s->blob.data() + blob_bodies_off())[b].n_points > 2) s->iso = false;
  cudaError_t e = cudaMalloc(&s->d_blob, s->blob.size());
  if (e != cudaSuccess) {
    delete s;
    return e == cudaErrorMemoryAllocation ? fail(BRAX_ERR_OUT_OF_MEMORY, "brax_system_create: cudaMalloc")
                                          : cuda_fail(e, "brax_system_create");
  }
  e = cudaMalloc(&s->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(s->d_blob, s->blob.data(), s->blob.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) {
    const int off = pool_acquire(s->device, s->blob);
    if (off == -1) {
      cudaFree(s->d_blob);
      cudaFree(s->d_status);
      delete s;
      return fail(BRAX_ERR_OUT_OF_MEMORY, "brax_system_create: the constant parameter pool (60 KB per device) is full");
    }
    if (off < -1) e = (cudaError_t)(-2 - off);
    else s->pool_off = off;
  }
  if (e != cudaSuccess) {
    cudaFree(s->d_blob);
    if (s->d_status) cudaFree(s->d_status);
    if (s->pool_off >= 0) pool_release(s->device, s->pool_off);
    delete s;
    return cuda_fail(e, "brax_system_create");
  }
  s->groups = 1;
  s->variant = pick_variant(32 * s->B);
  s->paired = S->paired != 0;
  s->pair_groups = 1;
  s->pair_variant = 0;
  s->pair_mode = (s->paired && 32 * s->B <= pair_variant_max_threads(0)) ? 1 : 0;
  *out = s;
  return BRAX_OK;
}

void brax_system_destroy(brax_system* s) {
  if (!s) return;
  if (s->pool_off >= 0) pool_release(s->device, s->pool_off);
  cudaFree(s->d_blob);
  cudaFree(s->d_status);
  sched_free(s->sched);
  if (s->copy_stream) {
    cudaStreamDestroy(s->copy_stream);
    cudaEventDestroy(s->ev_start);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(s->ev_ready[i]);
      cudaEventDestroy(s->ev_free[i]);
    }
  }
  delete s;
}

int brax_system_info(const brax_system* s, int32_t* n_bodies, int32_t* n_actuators, int32_t* n_dof) {
  if (!s) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_info: null system");
  if (n_bodies) *n_bodies = s->B;
  if (n_actuators) *n_actuators = s->A;
  if (n_dof) *n_dof = s->D;
  return BRAX_OK;
}

// Launch configuration override (groups of 32 environments per block,
// launch-bounds variant); used by the autotuner.  Not part of brax.h's
// stable surface.
int brax_system_set_launch(brax_system* s, int32_t groups, int32_t variant) {
  if (!s || groups < 1 || groups > 15 || variant < 0 || variant > 3)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_launch: bad arguments");
  if (32 * s->B * groups > rollout_variant_max_threads(variant))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_launch: block too large for the variant");
  s->groups = groups;
  s->variant = variant;
  return BRAX_OK;
}

// Two-environments-per-thread launch override (mode 0: off, 1: on; groups of
// 64 environments per block; launch-bounds variant); used by the autotuner.
int brax_system_set_pair_launch(brax_system* s, int32_t mode, int32_t groups, int32_t variant) {
  if (!s || mode < 0 || mode > 1 || groups < 1 || groups > 15 || variant < 0 || variant > 4)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_pair_launch: bad arguments");
  if (mode == 1 && !s->paired)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_pair_launch: the system has no paired kernel");
  if (mode == 1 && 32 * s->B * groups > pair_variant_max_threads(variant))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_pair_launch: block too large for the variant");
  s->pair_mode = mode;
  if (mode == 1) {
    s->pair_groups = groups;
    s->pair_variant = variant;
  }
  return BRAX_OK;
}

// Current launch configuration (for the autotuner's cache): the
// one-environment kernel's groups and variant; the paired mode (-1: the
// system has no paired kernel, else 0/1); the reverse kernel's variant.
int brax_system_get_launch(const brax_system* s, int32_t* groups, int32_t* variant) {
  if (!s || !groups || !variant) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_get_launch: null argument");
  *groups = s->groups;
  *variant = s->variant;
  return BRAX_OK;
}
int brax_internal_plan_schedule(int32_t mode, int32_t chunk_steps, int64_t units, int32_t T, int64_t slots,
                                int32_t min_chunk, int32_t* n_chunks, int32_t* steps) {
  if (!n_chunks || !steps) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_internal_plan_schedule: null argument");
  const SchedPlan p = plan_schedule_slots(mode, chunk_steps, units, T, slots, min_chunk);
  *n_chunks = p.n_chunks;
  *steps = p.chunk_steps;
  return BRAX_OK;
}
int brax_system_set_schedule(brax_system* s, int32_t mode, int32_t chunk_steps, int32_t first_item, int64_t wait_ns) {
  if (!s || mode < 0 || mode > 2 || (mode == 2 && chunk_steps < 1) || first_item < 0 || wait_ns < 1)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_schedule: bad arguments");
  s->sched_mode = mode;
  s->sched_chunk = chunk_steps;
  s->sched_first = first_item;
  s->sched_wait_ns = wait_ns;
  return BRAX_OK;
}
int brax_system_get_pair_launch(const brax_system* s, int32_t* mode) {
  if (!s || !mode) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_get_pair_launch: null argument");
  *mode = s->paired ? s->pair_mode : -1;
  return BRAX_OK;
}
int brax_system_set_backward_launch(brax_system* s, int32_t variant) {
  if (!s || variant < -1 || variant > 4) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_backward_launch: bad arguments");
  if (variant >= 0 && 32 * s->B > backward_variant_max_threads(variant))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_set_backward_launch: block too large for the variant");
  s->bwd_variant = variant;
  return BRAX_OK;
}

int brax_default_qp(const brax_system* s, int64_t n_envs, const float* root_pos, const float* root_rot,
                    const float* joint_angles, float* state_out, void* stream) {
  if (!s || !state_out || n_envs < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_default_qp: bad arguments");
  cudaError_t e = launch_default_qp(s->d_blob, n_envs, root_pos, root_rot, joint_angles, state_out, as_stream(stream));
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_default_qp");
}

}  // extern "C"

namespace {
// Outputs and parameters of the environment layer for one rollout (null: off).
struct EnvOut {
  const brax_env_params* p;
  const float* reset_state;
  float* obs;
  float* reward;
  uint8_t* done;
};
void apply_env(const brax_system* s, Seg& sg, const EnvOut* env) {
  if (!env) return;
  const SysP* S = reinterpret_cast<const SysP*>(s->blob.data());
  sg.obs = env->obs;
  sg.reward = env->reward;
  sg.done = env->done;
  sg.reset_state = env->reset_state;
  sg.obs_dim = 11 + 2 * S->D;
  sg.auto_reset = env->p->auto_reset ? 1 : 0;
  sg.fwd_w_dt = (float)((double)env->p->forward_weight / ((double)S->h * S->substeps));
  sg.healthy = env->p->healthy_reward;
  sg.ctrl_cost = env->p->ctrl_cost;
  sg.min_z = env->p->min_z;
  sg.max_z = env->p->max_z;
}

int rollout_impl(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                 const float* actions, float* state_T, float* checkpoints, float* torso_traj, int32_t* contact_count,
                 void* stream, const EnvOut* env, const FixedRegion& fr = FixedRegion{}) {
  if (!s || n_envs < 0 || T < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: bad arguments");
  if (n_envs > 0 && (!state0 || !state_T || (T > 0 && s->A > 0 && !actions)))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: null state or actions");
  if (checkpoints && K < 1) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: K must be >= 1");
  if (n_envs == 0) return BRAX_OK;
  if (s->variant < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: system too large for one block");
  Launch L;
  std::memset(&L, 0, sizeof(L));
  L.n_segs = 1;
  L.T = T;
  L.K = K < 1 ? 1 : K;
  // Two environments per thread whenever the system has that kernel and it
  // is switched on, checkpointing rollouts included: the reverse pass
  // rebuilds a checkpoint segment's step states with the kernel that wrote
  // the checkpoints (rollout_backward_impl), so gradients do not depend on K.
  if (s->pair_mode == 1) {
    Seg sg = make_seg(s, s->pair_groups, n_envs);
    const int64_t per_cta = 64LL * s->pair_groups;
    const int64_t grid = (n_envs + per_cta - 1) / per_cta;
    if (grid > 0x7fffffff) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: too many environments");
    sg.cta_begin = 0;
    sg.cta_end = (int32_t)grid;
    sg.state0 = state0;
    sg.actions = actions;
    sg.state_T = state_T;
    sg.ckpt = checkpoints;
    sg.torso = torso_traj;
    sg.ccount = contact_count;
    apply_env(s, sg, env);
    L.seg[0] = sg;
    size_t smem = s->pair_groups * pair_group_bytes(s->B, s->A);
    if (checkpoints) {  // checkpoint staging buffers, [64][B][13] floats a group, when they fit
      const size_t with = smem + (size_t)s->pair_groups * 64 * s->B * 13 * sizeof(float);
      int optin = 0;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device) != cudaSuccess) {
        cudaGetLastError();
        optin = 0;
      }
      if (with + 1024 <= (size_t)optin) {
        smem = with;
        L.seg[0].ck_stage = 1;
      }
    }
    const int threads = 32 * s->B * s->pair_groups;
    const SchedPlan pl = plan_schedule(s->sched_mode, s->sched_chunk, s->device, grid, T,
                                       pair_blocks_per_sm(s->pair_variant, threads, smem));
    int64_t launch_grid;
    cudaError_t e = apply_schedule(pl, s->sched, s->sched_first, s->sched_wait_ns, grid, L, &launch_grid,
                                   as_stream(stream), fr);
    s->last_grid = launch_grid;
    s->last_chunks = L.sc.n_chunks;
    s->last_chunk_steps = L.sc.chunk_steps;
    if (e == cudaSuccess)
      e = launch_rollout_pair(L, (int)launch_grid, threads, smem, s->pair_variant,
                              reinterpret_cast<const SysP*>(s->blob.data())->flat != 0, as_stream(stream));
    return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_rollout");
  }
  Seg sg = make_seg(s, s->groups, n_envs);
  const int64_t per_cta = 32LL * s->groups;
  const int64_t grid = (n_envs + per_cta - 1) / per_cta;
  if (grid > 0x7fffffff) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout: too many environments");
  sg.cta_begin = 0;
  sg.cta_end = (int32_t)grid;
  sg.state0 = state0;
  sg.actions = actions;
  sg.state_T = state_T;
  sg.ckpt = checkpoints;
  sg.torso = torso_traj;
  sg.ccount = contact_count;
  apply_env(s, sg, env);
  L.seg[0] = sg;
  const size_t smem = s->groups * group_bytes(s);
  const int threads = 32 * s->B * s->groups;
  const SchedPlan pl = plan_schedule(s->sched_mode, s->sched_chunk, s->device, grid, T,
                                     rollout_blocks_per_sm(s->variant, s->general, threads, smem));
  int64_t launch_grid;
  cudaError_t e = apply_schedule(pl, s->sched, s->sched_first, s->sched_wait_ns, grid, L, &launch_grid,
                                 as_stream(stream), fr);
  s->last_grid = launch_grid;
  s->last_chunks = L.sc.n_chunks;
  s->last_chunk_steps = L.sc.chunk_steps;
  if (e == cudaSuccess) e = launch_rollout(L, (int)launch_grid, threads, smem, s->variant, s->general, as_stream(stream));
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_rollout");
}

}  // namespace

extern "C" {

int brax_rollout(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                 const float* actions, float* state_T, float* checkpoints, float* torso_traj, int32_t* contact_count,
                 void* stream) {
  return rollout_impl(s, n_envs, T, K, state0, actions, state_T, checkpoints, torso_traj, contact_count, stream,
                      nullptr);
}

int brax_streamed_workspace_size(const brax_system* s, int64_t n_envs, int32_t chunk_steps, size_t* bytes) {
  if (!s || !bytes || n_envs < 0 || chunk_steps < 1)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_streamed_workspace_size: bad arguments");
  const size_t act = ((size_t)chunk_steps * n_envs * s->A * sizeof(float) + 255) & ~(size_t)255;
  const size_t st = ((size_t)n_envs * s->B * 13 * sizeof(float) + 255) & ~(size_t)255;
  *bytes = 2 * act + 2 * st;
  return BRAX_OK;
}

int brax_rollout_streamed(const brax_system* s, int64_t n_envs, int32_t T, const float* h_state0,
                          const float* h_actions, float* h_state_T, int32_t chunk_steps, int32_t first_steps,
                          void* workspace, size_t workspace_bytes, void* stream) {
  if (!s || n_envs < 0 || T < 0 || chunk_steps < 1 || first_steps < 1)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_streamed: bad arguments");
  if (n_envs == 0) return BRAX_OK;
  if (!h_state0 || !h_state_T || (T > 0 && s->A > 0 && !h_actions))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_streamed: null host array");
  const int32_t C = std::max(1, std::min(chunk_steps, std::max(T, 1)));
  size_t need = 0;
  brax_streamed_workspace_size(s, n_envs, C, &need);
  if (!workspace || workspace_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(BRAX_ERR_WORKSPACE, "brax_rollout_streamed: workspace missing, too small or not 256-byte aligned");
  brax_system* ms = const_cast<brax_system*>(s);
  std::lock_guard<std::mutex> lk(ms->stream_mu);
  cudaError_t e = cudaSuccess;
  if (!ms->copy_stream) {
    e = cudaStreamCreateWithFlags(&ms->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ms->ev_start, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&ms->ev_ready[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ms->ev_free[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "brax_rollout_streamed: stream/event creation");
  }
  const cudaStream_t st = as_stream(stream), cs = ms->copy_stream;
  const size_t act_bytes = ((size_t)C * n_envs * s->A * sizeof(float) + 255) & ~(size_t)255;
  const size_t state_bytes = (size_t)n_envs * s->B * 13 * sizeof(float);
  const size_t state_pad = (state_bytes + 255) & ~(size_t)255;
  unsigned char* base = static_cast<unsigned char*>(workspace);
  float* act_buf[2] = {reinterpret_cast<float*>(base), reinterpret_cast<float*>(base + act_bytes)};
  float* st_buf[2] = {reinterpret_cast<float*>(base + 2 * act_bytes),
                      reinterpret_cast<float*>(base + 2 * act_bytes + state_pad)};
  // chunks: first_steps, doubling up to C
  std::vector<std::pair<int32_t, int32_t>> chunks;
  for (int32_t t0 = 0, n = std::min(first_steps, C); t0 < T; t0 += n, n = std::min(C, 2 * n))
    chunks.push_back({t0, std::min(T, t0 + n)});
  const size_t row = (size_t)n_envs * s->A * sizeof(float);
  // the copy stream starts after the workspace's previous users on `stream`
  e = cudaEventRecord(ms->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ms->ev_start, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st_buf[0], h_state0, state_bytes, cudaMemcpyHostToDevice, cs);
  auto upload = [&](size_t i) -> cudaError_t {
    const int b = (int)(i % 2);
    cudaError_t r = cudaSuccess;
    if (i >= 2) r = cudaStreamWaitEvent(cs, ms->ev_free[b], 0);  // the buffer's previous chunk is done
    const size_t nb = (size_t)(chunks[i].second - chunks[i].first) * row;
    if (r == cudaSuccess && nb)
      r = cudaMemcpyAsync(act_buf[b], h_actions + (size_t)chunks[i].first * n_envs * s->A, nb,
                          cudaMemcpyHostToDevice, cs);
    if (r == cudaSuccess) r = cudaEventRecord(ms->ev_ready[b], cs);
    return r;
  };
  if (chunks.empty()) {  // T == 0: the state goes back unchanged
    if (e == cudaSuccess) e = cudaEventRecord(ms->ev_ready[0], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ms->ev_ready[0], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_state_T, st_buf[0], state_bytes, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_rollout_streamed");
  }
  if (e == cudaSuccess) e = upload(0);
  int cur = 0;
  for (size_t i = 0; i < chunks.size() && e == cudaSuccess; ++i) {
    if (i + 1 < chunks.size()) e = upload(i + 1);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ms->ev_ready[i % 2], 0);
    if (e != cudaSuccess) break;
    const int rc = brax_rollout(s, n_envs, chunks[i].second - chunks[i].first, 1, st_buf[cur], act_buf[i % 2],
                                st_buf[1 - cur], nullptr, nullptr, nullptr, stream);
    if (rc != BRAX_OK) return rc;
    e = cudaEventRecord(ms->ev_free[i % 2], st);
    cur = 1 - cur;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_state_T, st_buf[cur], state_bytes, cudaMemcpyDeviceToHost, st);
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_rollout_streamed");
}

int brax_env_obs_size(const brax_system* s, int32_t* obs_dim) {
  if (!s || !obs_dim) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_env_obs_size: null argument");
  *obs_dim = 11 + 2 * s->D;
  return BRAX_OK;
}

int brax_env_rollout(const brax_system* s, const brax_env_params* env, int64_t n_envs, int32_t T, const float* state0,
                     const float* reset_state, const float* actions, float* state_T, float* obs, float* reward,
                     uint8_t* done, void* stream) {
  if (!s || !env || n_envs < 0 || T < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_env_rollout: bad arguments");
  if (n_envs > 0 && T > 0 && (!obs || !reward || !done || (env->auto_reset && !reset_state)))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_env_rollout: obs, reward and done are required (and reset_state "
                                           "with auto_reset)");
  if (!(env->min_z <= env->max_z))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_env_rollout: min_z must not exceed max_z");
  EnvOut eo{env, reset_state, obs, reward, done};
  return rollout_impl(s, n_envs, T, 1, state0, actions, state_T, nullptr, nullptr, nullptr, stream, &eo);
}

int brax_step(const brax_system* s, int64_t n_envs, const float* state_in, const float* actions, float* state_out,
              void* stream) {
  return brax_rollout(s, n_envs, 1, 1, state_in, actions, state_out, nullptr, nullptr, nullptr, stream);
}

int brax_sync_status(const brax_system* s, void* stream) {
  if (!s) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_sync_status: null system");
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "brax_sync_status");
  int32_t h = 0;
  e = cudaMemcpy(&h, s->d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h) e = cudaMemset(s->d_status, 0, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_fail(e, "brax_sync_status");
  if (h & kStatusTimeout)
    return fail(BRAX_ERR_TIMEOUT, "brax_sync_status: a rollout block gave up waiting for the previous chunk of its "
                                  "environments (the rollout's outputs are incomplete)");
  if (h) return fail(BRAX_ERR_NONFINITE, "brax_sync_status: a kernel produced a non-finite state");
  return BRAX_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ heterogeneous batch
namespace {
// Groups per block for system s when a block has `warps` warps.
int batch_groups(const brax_system* s, int warps) { return std::max(1, std::min(15, warps / s->B)); }
}  // namespace

extern "C" {

int brax_batch_create(const brax_system* const* systems, const int64_t* n_envs, int32_t n, brax_batch** out) {
  if (!systems || !n_envs || !out || n < 1 || n > BRAX_MAX_SEGS)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_create: need 1..BRAX_MAX_SEGS systems");
  *out = nullptr;
  brax_batch* b = new brax_batch();
  int warps = 0;
  for (int i = 0; i < n; ++i) {
    if (!systems[i] || n_envs[i] < 0) {
      delete b;
      return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_create: null system or negative size");
    }
    b->sys.push_back(systems[i]);
    b->n_envs.push_back(n_envs[i]);
    warps = std::max(warps, systems[i]->B);
  }
  // a block holds one group of the largest system; smaller systems pack
  // several groups of 32 environments into the same block
  b->warps = warps;
  *out = b;
  return BRAX_OK;
}

int brax_batch_set_schedule(brax_batch* b, int32_t mode, int32_t chunk_steps) {
  if (!b || mode < 0 || mode > 2 || (mode == 2 && chunk_steps < 1))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_set_schedule: bad arguments");
  b->sched_mode = mode;
  b->sched_chunk = chunk_steps;
  return BRAX_OK;
}

void brax_batch_destroy(brax_batch* b) {
  if (!b) return;
  sched_free(b->sched);
  delete b;
}

int brax_batch_offsets(const brax_batch* b, int32_t T, int32_t K, int32_t i, int64_t* state_off, int64_t* action_off,
                       int64_t* torso_off, int64_t* ckpt_off) {
  if (!b || i < 0 || i >= (int)b->sys.size() || T < 0 || K < 1)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_offsets: bad arguments");
  int64_t so = 0, ao = 0, to = 0, co = 0;
  const int64_t nck = (T + K - 1) / K;
  for (int k = 0; k < i; ++k) {
    const int64_t N = b->n_envs[k];
    so += N * b->sys[k]->B * 13;
    ao += (int64_t)T * N * b->sys[k]->A;
    to += (int64_t)T * N * 3;
    co += nck * N * b->sys[k]->B * 13;
  }
  if (state_off) *state_off = so;
  if (action_off) *action_off = ao;
  if (torso_off) *torso_off = to;
  if (ckpt_off) *ckpt_off = co;
  return BRAX_OK;
}

}  // extern "C"

namespace brax_batch_impl {
// Fill a launch table for the batch; pointers offset per system.
int make_launch(const brax_batch* b, int32_t T, int32_t K, Launch& L, int* grid, int* threads, size_t* smem,
                bool* general) {
  *general = false;
  std::memset(&L, 0, sizeof(L));
  L.n_segs = (int)b->sys.size();
  L.T = T;
  L.K = K;
  int cta = 0;
  size_t sm = 0;
  for (int i = 0; i < L.n_segs; ++i) {
    const brax_system* s = b->sys[i];
    const int G = batch_groups(s, b->warps);
    Seg sg = make_seg(s, G, b->n_envs[i]);
    const int64_t per = 32LL * G;
    const int64_t nb = (b->n_envs[i] + per - 1) / per;
    sg.cta_begin = cta;
    sg.cta_end = cta + (int)nb;
    cta += (int)nb;
    sm = std::max(sm, (size_t)G * group_bytes(s));
    *general = *general || s->general;
    L.seg[i] = sg;
  }
  *grid = cta;
  *threads = 32 * b->warps;
  *smem = sm;
  return BRAX_OK;
}
}  // namespace brax_batch_impl

extern "C" int brax_batch_rollout(const brax_batch* b, int32_t T, int32_t K, const float* state0, const float* actions,
                                  float* state_T, float* checkpoints, float* torso_traj, void* stream) {
  if (!b || T < 0 || !state0 || !state_T || (checkpoints && K < 1))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_rollout: bad arguments");
  if (K < 1) K = 1;
  Launch L;
  int grid, threads;
  size_t smem;
  bool general;
  brax_batch_impl::make_launch(b, T, K, L, &grid, &threads, &smem, &general);
  for (int i = 0; i < L.n_segs; ++i) {
    int64_t so, ao, to, co;
    brax_batch_offsets(b, T, K, i, &so, &ao, &to, &co);
    L.seg[i].state0 = state0 + so;
    L.seg[i].actions = actions ? actions + ao : nullptr;
    L.seg[i].state_T = state_T + so;
    L.seg[i].ckpt = checkpoints ? checkpoints + co : nullptr;
    L.seg[i].torso = torso_traj ? torso_traj + to : nullptr;
  }
  if (grid == 0) return BRAX_OK;
  const int variant = pick_variant(threads);
  if (variant < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_rollout: block too large");
  int device = 0;
  cudaGetDevice(&device);
  const SchedPlan pl = plan_schedule(b->sched_mode, b->sched_chunk, device, grid, T,
                                     rollout_blocks_per_sm(variant, general, threads, smem));
  int64_t launch_grid;
  cudaError_t e = apply_schedule(pl, b->sched, 0, 2000000000LL, grid, L, &launch_grid, as_stream(stream));
  if (e == cudaSuccess) e = launch_rollout(L, (int)launch_grid, threads, smem, variant, general, as_stream(stream));
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_batch_rollout");
}

// ------------------------------------------------------------------ reverse mode
namespace {

// One group of 32 environments per block for the reverse kernel.
int64_t bwd_groups_total(int64_t n_envs) { return (n_envs + 31) / 32; }

// Scratch of the reverse kernel proper for (n_envs, K).
size_t bwd_kernel_ws_bytes(const brax_system* s, int64_t n_envs, int32_t K) {
  const SysP* S = reinterpret_cast<const SysP*>(s->blob.data());
  return (size_t)bwd_groups_total(n_envs) * (size_t)backward_ws_floats_per_group(s->B, s->P, K, S->substeps) *
         sizeof(float);
}
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// Whether the reverse pass rebuilds each checkpoint segment's step states
// with the forward kernel (the one that wrote the checkpoints) instead of
// recomputing them inside the reverse kernel: whenever a segment has more
// than one step.  The reverse kernel's own step arithmetic agrees with the
// forward kernels' to FP32 rounding but not always bit for bit (the compiled
// code of each kernel decides where a multiply and an add fuse; the biped's
// differs), so only the forward kernel reproduces the forward's step states
// exactly.
bool bwd_by_segments(const brax_system* s, int32_t K) {
  (void)s;
  return K > 1;
}
// Scratch of brax_rollout_backward for (n_envs, K), K already at most T.
// Rebuilding segments: the reverse kernel's scratch for K = 1, the step
// states of one segment [K][N][B][13] and two state adjoints [N][B][13]
// passed from segment to segment.
size_t bwd_ws_bytes(const brax_system* s, int64_t n_envs, int32_t K) {
  if (!bwd_by_segments(s, K)) return bwd_kernel_ws_bytes(s, n_envs, K);
  const size_t st = (size_t)n_envs * s->B * 13 * sizeof(float);
  return align256(bwd_kernel_ws_bytes(s, n_envs, 1)) + align256((size_t)K * st) + 2 * align256(st);
}

}  // namespace

namespace brax {
size_t backward_workspace_bytes(const brax_system* s, int64_t n_envs, int32_t K) { return bwd_ws_bytes(s, n_envs, K); }
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace brax

extern "C" int brax_workspace_size(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, size_t* bytes) {
  if (!s || !bytes || n_envs < 0 || T < 0 || K < 1)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_workspace_size: bad arguments");
  *bytes = bwd_ws_bytes(s, n_envs, std::min(K, std::max(T, 1)));
  return BRAX_OK;
}

namespace {
int rollout_backward_impl(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                          const float* actions, const float* checkpoints, const float* g_state_T,
                          const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                          size_t workspace_bytes, void* stream, const FixedRegion& fr) {
  if (!s || n_envs < 0 || T < 0 || K < 1) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward: bad arguments");
  if (n_envs == 0) return BRAX_OK;
  if (!g_state_T) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward: g_state_T is required");
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (g_state0) {
      cudaError_t e = cudaMemcpyAsync(g_state0, g_state_T, (size_t)n_envs * s->B * 13 * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "brax_rollout_backward");
    }
    return BRAX_OK;
  }
  if (!state0 || !checkpoints || (s->A > 0 && !actions))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward: state0, actions and checkpoints are required");
  const int32_t Ke = std::min(K, T);
  const size_t need = bwd_ws_bytes(s, n_envs, Ke);
  if (!workspace || workspace_bytes < need)
    return fail(BRAX_ERR_WORKSPACE, "brax_rollout_backward: workspace missing or smaller than brax_workspace_size");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(BRAX_ERR_WORKSPACE, "brax_rollout_backward: workspace must be 256-byte aligned");
  if (bwd_by_segments(s, Ke)) {
    // Checkpoint segments, last first: the forward kernel (the one that
    // wrote the checkpoints) rebuilds the segment's step states from its
    // checkpoint, K - 1 steps with a checkpoint every step plus the state
    // after them; then the reverse kernel runs the segment with K = 1 and
    // hands its state adjoint to the next segment.  Bitwise the same step
    // states as the forward, so the gradients do not depend on K.
    const size_t sb = (size_t)n_envs * s->B * 13 * sizeof(float);
    const size_t kern = align256(bwd_kernel_ws_bytes(s, n_envs, 1));
    unsigned char* base = static_cast<unsigned char*>(workspace);
    float* steps = reinterpret_cast<float*>(base + kern);
    float* carry[2] = {reinterpret_cast<float*>(base + kern + align256((size_t)Ke * sb)),
                       reinterpret_cast<float*>(base + kern + align256((size_t)Ke * sb) + align256(sb))};
    const size_t per_state = (size_t)n_envs * s->B * 13, per_act = (size_t)n_envs * s->A;
    const int nseg = (T + K - 1) / K;
    const float* g_in = g_state_T;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
      const int t0 = sgi * K, len = std::min(K, T - t0);
      const float* ck = checkpoints + (size_t)sgi * per_state;
      const float* act = actions ? actions + (size_t)t0 * per_act : nullptr;
      int rc = BRAX_OK;
      if (len > 1) {
        rc = rollout_impl(s, n_envs, len - 1, 1, ck, act, steps + (size_t)(len - 1) * per_state, steps, nullptr,
                          nullptr, stream, nullptr, fr);
      } else {
        cudaError_t e = cudaMemcpyAsync(steps, ck, sb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "brax_rollout_backward");
      }
      if (rc != BRAX_OK) return rc;
      float* g_out = sgi == 0 ? g_state0 : carry[sgi & 1];
      rc = rollout_backward_impl(s, n_envs, len, 1, ck, act, steps, g_in,
                                 g_torso_traj ? g_torso_traj + (size_t)t0 * n_envs * 3 : nullptr,
                                 g_actions ? g_actions + (size_t)t0 * per_act : nullptr, g_out, workspace, kern, stream,
                                 fr);
      if (rc != BRAX_OK) return rc;
      g_in = g_out;
    }
    return BRAX_OK;
  }
  Launch L;
  std::memset(&L, 0, sizeof(L));
  L.n_segs = 1;
  L.T = T;
  L.K = K;  // segment boundaries follow the checkpoints written with K
  Seg sg = make_seg(s, 1, n_envs);
  const int64_t grid = bwd_groups_total(n_envs);
  if (grid > 0x7fffffff) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward: too many environments");
  sg.cta_begin = 0;
  sg.cta_end = (int32_t)grid;
  sg.state0 = state0;
  sg.actions = actions;
  sg.ckpt = const_cast<float*>(checkpoints);
  sg.g_state_T = g_state_T;
  sg.g_torso = g_torso_traj;
  sg.g_actions = g_actions;
  sg.g_state0 = g_state0;
  sg.ws = reinterpret_cast<float*>(workspace);
  L.seg[0] = sg;
  const int threads = 32 * s->B;
  const int variant =
      (s->bwd_variant >= 0 && threads <= backward_variant_max_threads(s->bwd_variant)) ? s->bwd_variant
                                                                                        : pick_bwd_variant(threads);
  if (variant < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_rollout_backward: system too large for one block");
  const size_t smem = backward_smem_bytes(s->B, s->P, 1);
  const int nseg = (T + K - 1) / K;
  const SchedPlan pl = plan_schedule(s->sched_mode, s->sched_chunk, s->device, grid, nseg,
                                     backward_blocks_per_sm(variant, s->general, s->iso, threads, smem),
                                     (16 + K - 1) / K);
  int64_t launch_grid;
  cudaError_t e = apply_schedule(pl, s->sched, s->sched_first, s->sched_wait_ns, grid, L, &launch_grid, st, fr);
  if (e == cudaSuccess)
    e = launch_rollout_backward(L, (int)launch_grid, threads, smem, variant, s->general, s->iso, st);
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_rollout_backward");
}
}  // namespace

extern "C" int brax_rollout_backward(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                                     const float* actions, const float* checkpoints, const float* g_state_T,
                                     const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  return rollout_backward_impl(s, n_envs, T, K, state0, actions, checkpoints, g_state_T, g_torso_traj, g_actions,
                               g_state0, workspace, workspace_bytes, stream, FixedRegion{});
}

namespace brax {
int rollout_backward_fixed_sched(const brax_system* s, int64_t n_envs, int32_t T, int32_t K, const float* state0,
                                 const float* actions, const float* checkpoints, const float* g_state_T,
                                 const float* g_torso_traj, float* g_actions, float* g_state0, void* workspace,
                                 size_t workspace_bytes, int32_t* sched, size_t sched_bytes, void* stream) {
  FixedRegion fr;
  fr.use = true;
  fr.fixed = sched;
  fr.bytes = sched_bytes;
  return rollout_backward_impl(s, n_envs, T, K, state0, actions, checkpoints, g_state_T, g_torso_traj, g_actions,
                               g_state0, workspace, workspace_bytes, stream, fr);
}
}  // namespace brax

namespace {
// Reverse-mode layout of a batch: one launch, system i's blocks hold G_i
// groups of 32 environments, its workspace block starts at ws_off[i].
struct BwdBatchPlan {
  int grid = 0, threads = 0;
  size_t smem = 0, ws_bytes = 0;
  bool general = false, iso = true;
  std::vector<int> groups, cta_begin, cta_end;
  std::vector<size_t> ws_off;
};
BwdBatchPlan plan_batch_backward(const brax_batch* b, int32_t K) {
  BwdBatchPlan pl;
  pl.threads = 32 * b->warps;
  int cta = 0;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    const brax_system* s = b->sys[i];
    const SysP* S = reinterpret_cast<const SysP*>(s->blob.data());
    const int G = batch_groups(s, b->warps);
    const int64_t per = 32LL * G;
    const int nb = (int)((b->n_envs[i] + per - 1) / per);
    pl.groups.push_back(G);
    pl.cta_begin.push_back(cta);
    pl.cta_end.push_back(cta + nb);
    cta += nb;
    pl.ws_off.push_back(pl.ws_bytes);
    const size_t wb = (size_t)nb * G * (size_t)backward_ws_floats_per_group(s->B, s->P, K, S->substeps) * sizeof(float);
    pl.ws_bytes += (wb + 255) & ~size_t(255);
    pl.smem = std::max(pl.smem, backward_smem_bytes(s->B, s->P, G));
    pl.general = pl.general || s->general;
    pl.iso = pl.iso && s->iso;
  }
  pl.grid = cta;
  return pl;
}
}  // namespace

extern "C" int brax_batch_workspace_size(const brax_batch* b, int32_t T, int32_t K, size_t* bytes) {
  if (!b || !bytes || T < 0 || K < 1) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_workspace_size: bad arguments");
  *bytes = plan_batch_backward(b, std::min(K, std::max(T, 1))).ws_bytes;
  return BRAX_OK;
}

extern "C" int brax_batch_rollout_backward(const brax_batch* b, int32_t T, int32_t K, const float* state0,
                                           const float* actions, const float* checkpoints, const float* g_state_T,
                                           const float* g_torso_traj, float* g_actions, float* g_state0,
                                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!b || T < 0 || K < 1 || !g_state_T)
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_rollout_backward: bad arguments");
  cudaStream_t st = as_stream(stream);
  if (T == 0) {
    if (g_state0) {
      int64_t tot = 0;
      for (size_t i = 0; i < b->sys.size(); ++i) tot += b->n_envs[i] * b->sys[i]->B * 13;
      cudaError_t e = cudaMemcpyAsync(g_state0, g_state_T, (size_t)tot * sizeof(float), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "brax_batch_rollout_backward");
    }
    return BRAX_OK;
  }
  if (!state0 || !checkpoints) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_rollout_backward: null inputs");
  const BwdBatchPlan pl = plan_batch_backward(b, std::min(K, T));
  if (!workspace || workspace_bytes < pl.ws_bytes)
    return fail(BRAX_ERR_WORKSPACE, "brax_batch_rollout_backward: workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(BRAX_ERR_WORKSPACE, "brax_batch_rollout_backward: workspace must be 256-byte aligned");
  if (pl.grid == 0) return BRAX_OK;
  Launch L;
  std::memset(&L, 0, sizeof(L));
  L.n_segs = (int)b->sys.size();
  L.T = T;
  L.K = K;
  for (int i = 0; i < L.n_segs; ++i) {
    int64_t so, ao, to, co;
    brax_batch_offsets(b, T, K, i, &so, &ao, &to, &co);
    Seg sg = make_seg(b->sys[i], pl.groups[i], b->n_envs[i]);
    sg.cta_begin = pl.cta_begin[i];
    sg.cta_end = pl.cta_end[i];
    sg.state0 = state0 + so;
    sg.actions = actions ? actions + ao : nullptr;
    sg.ckpt = const_cast<float*>(checkpoints) + co;
    sg.g_state_T = g_state_T + so;
    sg.g_torso = g_torso_traj ? g_torso_traj + to : nullptr;
    sg.g_actions = g_actions ? g_actions + ao : nullptr;
    sg.g_state0 = g_state0 ? g_state0 + so : nullptr;
    sg.ws = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + pl.ws_off[i]);
    L.seg[i] = sg;
  }
  const int variant = pick_bwd_variant(pl.threads);
  if (variant < 0) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_batch_rollout_backward: block too large");
  int device = 0;
  cudaGetDevice(&device);
  const SchedPlan sp = plan_schedule(b->sched_mode, b->sched_chunk, device, pl.grid, (T + K - 1) / K,
                                     backward_blocks_per_sm(variant, pl.general, pl.iso, pl.threads, pl.smem),
                                     (16 + K - 1) / K);
  int64_t launch_grid;
  cudaError_t e = apply_schedule(sp, b->sched, 0, 2000000000LL, pl.grid, L, &launch_grid, st);
  if (e == cudaSuccess)
    e = launch_rollout_backward(L, (int)launch_grid, pl.threads, pl.smem, variant, pl.general, pl.iso, st);
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_batch_rollout_backward");
}

// fast_atan2 of the kernels (and its packed two-environment form) over n
// device elements: the accuracy test's probe (internal, brax_internal.h).
extern "C" int brax_internal_atan2(const float* y, const float* x, float* out, float* out_packed, int64_t n,
                                   void* stream) {
  if (n < 0 || (n > 0 && (!y || !x || !out || !out_packed)))
    return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_internal_atan2: bad arguments");
  cudaError_t e = brax::launch_atan2_probe(y, x, out, out_packed, n, as_stream(stream));
  return e == cudaSuccess ? BRAX_OK : cuda_fail(e, "brax_internal_atan2");
}

extern "C" int brax_system_last_rollout(const brax_system* s, int64_t* grid, int32_t* n_chunks, int32_t* chunk_steps) {
  if (!s) return fail(BRAX_ERR_INVALID_ARGUMENT, "brax_system_last_rollout: null system");
  if (grid) *grid = s->last_grid;
  if (n_chunks) *n_chunks = s->last_chunks;
  if (chunk_steps) *chunk_steps = s->last_chunk_steps;
  return BRAX_OK;
}
