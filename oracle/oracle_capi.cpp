// C entry points of the FP64 oracle, called from Python through ctypes.
//
// TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
// baseline of the benchmark.  The product library never links or calls it.
//
// Arrays follow the QP layout of Sec. 3: state [N, B, 13] with per body
// (pos[3], quat[4] (w,x,y,z), vel[3], angvel[3]); actions [T, N, A].
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "oracle.hpp"

using namespace orc;

extern "C" {

// Flat FP64 descriptor of a system (the oracle's own definition).
typedef struct {
  int32_t n_bodies, n_joints, n_actuators, n_colliders, n_pairs, substeps;
  double dt, gravity[3], baumgarte, contact_eps;
  int32_t average_contacts;
  const double *mass, *inertia, *rest_pos, *rest_rot;
  const uint8_t *frozen_pos, *frozen_rot;
  const int32_t *parent, *child, *dof;
  const double *parent_offset, *child_offset, *parent_frame, *child_frame;
  const double *stiffness, *spring_damping, *angular_stiffness, *angular_damping;
  const double *limit_lo, *limit_hi, *limit_stiffness;
  const int32_t *act_joint, *act_axis;
  const double* gear;
  const int32_t *col_body, *col_type;
  const double *col_pos, *col_rot, *radius, *length, *half_extents, *friction, *elasticity;
  const int32_t *pair_a, *pair_b;
  // variants (zero / NULL: off)
  double linear_damping, angular_damping_global;
  int32_t gyroscopic;
  const int32_t* act_type;
} orc_desc;

}  // extern "C"

namespace {

template <class V, class P> void cp(V& dst, const P* src, int64_t n) { dst.assign(src, src + n); }

System make_system(const orc_desc* d) {
  System s;
  s.B = d->n_bodies;
  s.J = d->n_joints;
  s.A = d->n_actuators;
  s.C = d->n_colliders;
  s.P = d->n_pairs;
  s.substeps = d->substeps;
  s.dt = d->dt;
  for (int i = 0; i < 3; ++i) s.g[i] = d->gravity[i];
  s.baumgarte = d->baumgarte;
  s.eps = d->contact_eps;
  s.average = d->average_contacts != 0;
  s.lin_damp = d->linear_damping;
  s.ang_damp = d->angular_damping_global;
  s.gyro = d->gyroscopic != 0;
  if (d->act_type) cp(s.act_type, d->act_type, d->n_actuators);
  cp(s.mass, d->mass, s.B);
  cp(s.inertia, d->inertia, 3 * s.B);
  cp(s.rest_pos, d->rest_pos, 3 * s.B);
  cp(s.rest_rot, d->rest_rot, 4 * s.B);
  cp(s.fpos, d->frozen_pos, 3 * s.B);
  cp(s.frot, d->frozen_rot, 3 * s.B);
  cp(s.parent, d->parent, s.J);
  cp(s.child, d->child, s.J);
  cp(s.dof, d->dof, s.J);
  cp(s.off_p, d->parent_offset, 3 * s.J);
  cp(s.off_c, d->child_offset, 3 * s.J);
  cp(s.frame_p, d->parent_frame, 4 * s.J);
  cp(s.frame_c, d->child_frame, 4 * s.J);
  cp(s.k, d->stiffness, s.J);
  cp(s.c, d->spring_damping, s.J);
  cp(s.ka, d->angular_stiffness, s.J);
  cp(s.ca, d->angular_damping, s.J);
  cp(s.kl, d->limit_stiffness, s.J);
  // App. A gives limits in degrees
  s.lo.resize(3 * s.J);
  s.hi.resize(3 * s.J);
  const double deg = 3.14159265358979323846 / 180.0;
  for (int i = 0; i < 3 * s.J; ++i) {
    s.lo[i] = d->limit_lo[i] * deg;
    s.hi[i] = d->limit_hi[i] * deg;
  }
  cp(s.act_joint, d->act_joint, s.A);
  cp(s.act_axis, d->act_axis, s.A);
  cp(s.gear, d->gear, s.A);
  cp(s.col_body, d->col_body, s.C);
  cp(s.col_type, d->col_type, s.C);
  cp(s.col_pos, d->col_pos, 3 * s.C);
  cp(s.col_rot, d->col_rot, 4 * s.C);
  cp(s.radius, d->radius, s.C);
  cp(s.length, d->length, s.C);
  cp(s.half, d->half_extents, 3 * s.C);
  cp(s.friction, d->friction, s.C);
  cp(s.elasticity, d->elasticity, s.C);
  cp(s.pair_a, d->pair_a, s.P);
  cp(s.pair_b, d->pair_b, s.P);
  s.derive();
  return s;
}

template <class T> void load_env(const System& s, const double* st, std::vector<Body<T>>& qp) {
  qp.resize(s.B);
  for (int b = 0; b < s.B; ++b) {
    const double* o = st + 13 * b;
    qp[b].x = mk(T(o[0]), T(o[1]), T(o[2]));
    qp[b].q = Q4<T>{T(o[3]), T(o[4]), T(o[5]), T(o[6])};
    qp[b].v = mk(T(o[7]), T(o[8]), T(o[9]));
    qp[b].w = mk(T(o[10]), T(o[11]), T(o[12]));
  }
}
template <class T> void store_env(const System& s, const std::vector<Body<T>>& qp, double* st) {
  for (int b = 0; b < s.B; ++b) {
    double* o = st + 13 * b;
    const Body<T>& q = qp[b];
    double v[13] = {val(q.x.x), val(q.x.y), val(q.x.z), val(q.q.w), val(q.q.x), val(q.q.y), val(q.q.z),
                    val(q.v.x), val(q.v.y), val(q.v.z), val(q.w.x), val(q.w.y), val(q.w.z)};
    std::memcpy(o, v, sizeof(v));
  }
}
template <class T> T* comp(Body<T>& b, int i) {
  switch (i) {
    case 0: return &b.x.x; case 1: return &b.x.y; case 2: return &b.x.z;
    case 3: return &b.q.w; case 4: return &b.q.x; case 5: return &b.q.y; case 6: return &b.q.z;
    case 7: return &b.v.x; case 8: return &b.v.y; case 9: return &b.v.z;
    case 10: return &b.w.x; case 11: return &b.w.y; default: return &b.w.z;
  }
}

template <class F> void parallel_for(int64_t n, int threads, F fn) {
  if (threads <= 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  if (threads > n) threads = (int)n;
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t]() {
      for (int64_t i = t; i < n; i += threads) fn(i);
    });
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// Forward rollout in FP64.  traj (optional): states after every step
// [T, N, B, 13].  contact_count (optional): active contacts summed over all
// substeps, per environment.
int orc_rollout(const orc_desc* d, int64_t N, int32_t T, const double* state0, const double* actions,
                double* state_T, double* traj, int64_t* contact_count, uint64_t* branch_sig, int32_t n_threads) {
  System s = make_system(d);
  const int B = s.B, A = s.A;
  parallel_for(N, n_threads, [&](int64_t n) {
    std::vector<Body<double>> qp;
    load_env(s, state0 + n * B * 13, qp);
    Diag dg;
    tl_diag = &dg;
    std::vector<double> act(A > 0 ? A : 1);
    for (int t = 0; t < T; ++t) {
      for (int a = 0; a < A; ++a) act[a] = actions[((int64_t)t * N + n) * A + a];
      step(s, qp.data(), act.data(), &dg);
      if (traj) store_env(s, qp, traj + ((int64_t)t * N + n) * B * 13);
    }
    tl_diag = nullptr;
    store_env(s, qp, state_T + n * B * 13);
    if (contact_count) contact_count[n] = dg.active_contacts;
    if (branch_sig) branch_sig[n] = dg.branch_hash;
  });
  return 0;
}

// Algorithmic flop count of a rollout, by category (FlopCat), summed over
// environments, plus the number of active contacts.
int orc_flops(const orc_desc* d, int64_t N, int32_t T, const double* state0, const double* actions, int64_t* counts,
              int64_t* n_active) {
  System s = make_system(d);
  const int B = s.B, A = s.A;
  FlopCounter fc;
  int64_t na = 0;
  for (int64_t n = 0; n < N; ++n) {
    std::vector<Body<Flop>> qp;
    load_env(s, state0 + n * B * 13, qp);
    Diag dg;
    std::vector<Flop> act(A > 0 ? A : 1);
    tl_flops = &fc;
    for (int t = 0; t < T; ++t) {
      for (int a = 0; a < A; ++a) act[a] = Flop(actions[((int64_t)t * N + n) * A + a]);
      step(s, qp.data(), act.data(), &dg);
    }
    tl_flops = nullptr;
    na += dg.active_contacts;
  }
  for (int i = 0; i < FC_N; ++i) counts[i] = fc.n[i];
  *n_active = na;
  return 0;
}

// Reverse-mode gradient (vector-Jacobian product) of a rollout through the
// tape type.  Outputs: g_actions [T, N, A], g_state0 [N, B, 13].  g_torso
// (optional) is the cotangent of body 0's position after every step [T, N, 3].
int orc_vjp(const orc_desc* d, int64_t N, int32_t T, const double* state0, const double* actions,
            const double* g_state_T, const double* g_torso, double* g_actions, double* g_state0, int32_t n_threads) {
  System s = make_system(d);
  const int B = s.B, A = s.A;
  parallel_for(N, n_threads, [&](int64_t n) {
    Tape tape;
    tape.nodes.reserve(1 << 20);
    tl_tape = &tape;
    std::vector<Body<Var>> qp(B);
    std::vector<int> in_state(B * 13);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < 13; ++i) {
        Var v = var_leaf(state0[(n * B + b) * 13 + i]);
        *comp(qp[b], i) = v;
        in_state[b * 13 + i] = v.i;
      }
    std::vector<int> in_act((size_t)T * (A > 0 ? A : 1));
    std::vector<int> torso((size_t)T * 3);
    std::vector<Var> act(A > 0 ? A : 1);
    for (int t = 0; t < T; ++t) {
      for (int a = 0; a < A; ++a) {
        act[a] = var_leaf(actions[((int64_t)t * N + n) * A + a]);
        in_act[(size_t)t * A + a] = act[a].i;
      }
      step(s, qp.data(), act.data(), (Diag*)nullptr);
      torso[3 * t + 0] = qp[0].x.x.i;
      torso[3 * t + 1] = qp[0].x.y.i;
      torso[3 * t + 2] = qp[0].x.z.i;
    }
    std::vector<double> adj(tape.nodes.size(), 0.0);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < 13; ++i) {
        Var v = *comp(qp[b], i);
        if (v.i >= 0) adj[v.i] += g_state_T[(n * B + b) * 13 + i];
      }
    if (g_torso)
      for (int t = 0; t < T; ++t)
        for (int i = 0; i < 3; ++i)
          if (torso[3 * t + i] >= 0) adj[torso[3 * t + i]] += g_torso[((int64_t)t * N + n) * 3 + i];
    tape.backward(adj);
    for (int k = 0; k < B * 13; ++k) g_state0[n * B * 13 + k] = adj[in_state[k]];
    for (int t = 0; t < T; ++t)
      for (int a = 0; a < A; ++a) g_actions[((int64_t)t * N + n) * A + a] = adj[in_act[(size_t)t * A + a]];
    tl_tape = nullptr;
  });
  return 0;
}

// Reverse-op count of a rollout's tape (the algorithmic flops of the reverse
// pass): out[0] = 2 flops per tape edge (multiply and accumulate) + the
// flops that formed the local partials; out[1] = tape nodes.  Summed over
// environments.
int orc_reverse_flops(const orc_desc* d, int64_t N, int32_t T, const double* state0, const double* actions,
                      int64_t* out, int32_t n_threads) {
  System s = make_system(d);
  const int B = s.B, A = s.A;
  std::vector<int64_t> flops(N, 0), nodes(N, 0);
  parallel_for(N, n_threads, [&](int64_t n) {
    Tape tape;
    tl_tape = &tape;
    std::vector<Body<Var>> qp(B);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < 13; ++i) *comp(qp[b], i) = var_leaf(state0[(n * B + b) * 13 + i]);
    std::vector<Var> act(A > 0 ? A : 1);
    for (int t = 0; t < T; ++t) {
      for (int a = 0; a < A; ++a) act[a] = var_leaf(actions[((int64_t)t * N + n) * A + a]);
      step(s, qp.data(), act.data(), (Diag*)nullptr);
    }
    flops[n] = 2 * tape.edges() + tape.deriv_flops;
    nodes[n] = (int64_t)tape.nodes.size();
    tl_tape = nullptr;
  });
  out[0] = out[1] = 0;
  for (int64_t n = 0; n < N; ++n) {
    out[0] += flops[n];
    out[1] += nodes[n];
  }
  return 0;
}

// Forward-mode derivative (Jacobian-vector product) of a rollout along the
// direction (d_state0 [N,B,13], d_actions [T,N,A]).  Outputs d_state_T
// [N,B,13] and d_torso [T,N,3] (optional).
int orc_jvp(const orc_desc* d, int64_t N, int32_t T, const double* state0, const double* actions,
            const double* d_state0, const double* d_actions, double* d_state_T, double* d_torso, int32_t n_threads) {
  System s = make_system(d);
  const int B = s.B, A = s.A;
  parallel_for(N, n_threads, [&](int64_t n) {
    std::vector<Body<Dual>> qp(B);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < 13; ++i)
        *comp(qp[b], i) = Dual(state0[(n * B + b) * 13 + i], d_state0[(n * B + b) * 13 + i]);
    std::vector<Dual> act(A > 0 ? A : 1);
    for (int t = 0; t < T; ++t) {
      for (int a = 0; a < A; ++a) {
        int64_t k = ((int64_t)t * N + n) * A + a;
        act[a] = Dual(actions[k], d_actions[k]);
      }
      step(s, qp.data(), act.data(), (Diag*)nullptr);
      if (d_torso) {
        d_torso[((int64_t)t * N + n) * 3 + 0] = qp[0].x.x.d;
        d_torso[((int64_t)t * N + n) * 3 + 1] = qp[0].x.y.d;
        d_torso[((int64_t)t * N + n) * 3 + 2] = qp[0].x.z.d;
      }
    }
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < 13; ++i) d_state_T[(n * B + b) * 13 + i] = comp(qp[b], i)->d;
  });
  return 0;
}

// default_qp (Sec. 4.1).  root_pos [N,3], root_rot [N,4], angles [N,D]
// (radians) may each be NULL.
int orc_default_qp(const orc_desc* d, int64_t N, const double* root_pos, const double* root_rot,
                   const double* angles, double* state_out) {
  System s = make_system(d);
  for (int64_t n = 0; n < N; ++n)
    default_qp(s, root_pos ? root_pos + 3 * n : nullptr, root_rot ? root_rot + 4 * n : nullptr,
               angles ? angles + n * s.D : nullptr, state_out + n * s.B * 13);
  return 0;
}

// Joint angles [N, D] (radians) of states [N, B, 13].
int orc_joint_angles(const orc_desc* d, int64_t N, const double* state, double* out) {
  System s = make_system(d);
  for (int64_t n = 0; n < N; ++n) {
    std::vector<Body<double>> qp;
    load_env(s, state + n * s.B * 13, qp);
    std::vector<Frame<double>> fr(s.B);
    for (int b = 0; b < s.B; ++b) fr[b] = frame(s, b, qp[b]);
    for (int j = 0; j < s.J; ++j) {
      double ang[3];
      V3<double> P[3];
      joint_angles(s, j, fr[s.parent[j]], fr[s.child[j]], ang, P);
      for (int a = 0; a < s.dof[j]; ++a) out[n * s.D + s.dof_offset[j] + a] = ang[a];
    }
  }
  return 0;
}

// Joint angles [N, D] and joint angular rates [N, D]: for each joint DOF the
// relative angular velocity of child and parent, w_c - w_p, along the joint
// axis in the world, R_p (parent joint-frame axis k).  The observation of the
// gym-like environment layer (Sec. 4.2) reads both.
int orc_joint_state(const orc_desc* d, int64_t N, const double* state, double* ang_out, double* rate_out) {
  System s = make_system(d);
  for (int64_t n = 0; n < N; ++n) {
    std::vector<Body<double>> qp;
    load_env(s, state + n * s.B * 13, qp);
    std::vector<Frame<double>> fr(s.B);
    for (int b = 0; b < s.B; ++b) fr[b] = frame(s, b, qp[b]);
    for (int j = 0; j < s.J; ++j) {
      double ang[3];
      V3<double> P[3];
      joint_angles(s, j, fr[s.parent[j]], fr[s.child[j]], ang, P);
      const V3<double> wr = qp[s.child[j]].w - qp[s.parent[j]].w;
      for (int a = 0; a < s.dof[j]; ++a) {
        ang_out[n * s.D + s.dof_offset[j] + a] = ang[a];
        rate_out[n * s.D + s.dof_offset[j] + a] = dot(wr, P[a]);
      }
    }
  }
  return 0;
}

// Energy [N] and momentum [N, 6] (linear, angular about the origin).
int orc_energy(const orc_desc* d, int64_t N, const double* state, double* energy_out, double* momentum_out) {
  System s = make_system(d);
  for (int64_t n = 0; n < N; ++n) {
    std::vector<Body<double>> qp;
    load_env(s, state + n * s.B * 13, qp);
    if (energy_out) energy_out[n] = energy(s, qp.data());
    if (momentum_out) momentum(s, qp.data(), momentum_out + 6 * n);
  }
  return 0;
}

// Active contacts of one state [B, 13]: up to max_out contacts, each
// (a, b) bodies and (depth, n[3], p[3]).  Returns the number detected.
int orc_contacts(const orc_desc* d, const double* state, int32_t max_out, int32_t* bodies, double* geo) {
  System s = make_system(d);
  std::vector<Body<double>> qp;
  load_env(s, state, qp);
  std::vector<Frame<double>> fr(s.B);
  for (int b = 0; b < s.B; ++b) fr[b] = frame(s, b, qp[b]);
  std::vector<Contact<double>> cts;
  detect(s, qp.data(), fr.data(), cts);
  int n = 0;
  for (const auto& c : cts) {
    if (n >= max_out) break;
    bodies[2 * n] = c.a;
    bodies[2 * n + 1] = c.b;
    double g[7] = {c.depth, c.n.x, c.n.y, c.n.z, c.p.x, c.p.y, c.p.z};
    std::memcpy(geo + 7 * n, g, sizeof(g));
    ++n;
  }
  return (int)cts.size();
}

// Closest points of two segments: out = (s, t).
void orc_segment_closest(const double* P1, const double* Q1, const double* P2, const double* Q2, double* out) {
  V3<double> p1{P1[0], P1[1], P1[2]}, q1{Q1[0], Q1[1], Q1[2]}, p2{P2[0], P2[1], P2[2]}, q2{Q2[0], Q2[1], Q2[2]};
  double sp, tp;
  segment_closest(p1, q1 - p1, p2, q2 - p2, sp, tp);
  out[0] = sp;
  out[1] = tp;
}

// Capsule (segment P..Q, radius r) against a box (centre c, rotation quat q,
// half extents he).  out = (depth, n[3], p[3]); returns 1 when active.
int orc_capsule_box(const double* P, const double* Q, double r, const double* c, const double* q, const double* he,
                    double* out) {
  double R[3][3];
  double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0}, ez[3] = {0, 0, 1}, X[3], Y[3], Z[3];
  double qq[4] = {q[0], q[1], q[2], q[3]};
  cq_normalize(qq);
  cq_rotate(qq, ex, X);
  cq_rotate(qq, ey, Y);
  cq_rotate(qq, ez, Z);
  for (int i = 0; i < 3; ++i) { R[i][0] = X[i]; R[i][1] = Y[i]; R[i][2] = Z[i]; }
  M3<double> Rb;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rb.m[i][j] = R[i][j];
  std::vector<Contact<double>> cts;
  V3<double> p{P[0], P[1], P[2]}, qv{Q[0], Q[1], Q[2]}, cc{c[0], c[1], c[2]};
  capsule_box(p, qv - p, r, 0, cc, Rb, he, 1, 1.0, 0.0, cts);
  // report the geometry even when not penetrating: recompute depth sign
  if (cts.empty()) return 0;
  const auto& k = cts[0];
  double g[7] = {k.depth, k.n.x, k.n.y, k.n.z, k.p.x, k.p.y, k.p.z};
  std::memcpy(out, g, sizeof(g));
  return 1;
}

// Golden-section segment parameter of orc_capsule_box, exposed for the
// brute-force test of the minimisation.
double orc_seg_box_param(const double* Pl, const double* dl, const double* he) {
  V3<double> p{Pl[0], Pl[1], Pl[2]}, dd{dl[0], dl[1], dl[2]};
  return seg_box_param(p, dd, he);
}

}  // extern "C"
