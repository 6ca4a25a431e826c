// Scalar types for the FP64 oracle.
//
// TEST INFRASTRUCTURE ONLY: the oracle is the plain, slow reference that the
// CUDA path is checked against.  Only tests, the smoke check and the CPU
// baseline of the benchmark may build or call it; the product path never does.
//
// The physics in oracle.hpp is written once, templated on a scalar type T, and
// instantiated with:
//   double  - the reference values;
//   Flop    - a double that counts the arithmetic it performs (the algorithmic
//             flop count used as the numerator of the roofline fraction);
//   Dual    - forward-mode derivative along one direction (Jacobian-vector
//             products, for the dot-product test of the adjoint);
//   Var     - reverse-mode derivative through a tape (the FP64 oracle adjoint
//             of the differentiable step, Sec. 1 and Sec. 5 "APG").
//
// Branching functions (max, min, clamp, if) take the derivative of the branch
// that is actually executed; comparisons are made on values.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

// ------------------------------------------------------------------ double
inline double val(double a) { return a; }
inline double sqrt(double a) { return std::sqrt(a); }
inline double atan2(double y, double x) { return std::atan2(y, x); }

// ------------------------------------------------------------------ Flop
// Counting rule: add, sub, mul, div, sqrt, atan2, min, max = 1 flop each.
// Negation, comparisons used for branching and copies are free.  A fused
// multiply-add written as a*b+c counts 2 (one mul, one add).
enum FlopCat { FC_BODY = 0, FC_JOINT, FC_ACT, FC_DETECT, FC_RESPONSE, FC_INTEGRATE, FC_OTHER, FC_N };
struct FlopCounter {
  int64_t n[FC_N] = {0, 0, 0, 0, 0, 0, 0};
  int cat = FC_OTHER;
};
inline thread_local FlopCounter* tl_flops = nullptr;
inline void count_flop(int k = 1) {
  if (tl_flops) tl_flops->n[tl_flops->cat] += k;
}
struct Flop {
  double v;
  Flop(double x = 0.0) : v(x) {}
};
inline double val(const Flop& a) { return a.v; }
inline Flop operator+(Flop a, Flop b) { count_flop(); return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { count_flop(); return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { count_flop(); return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { count_flop(); return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop sqrt(Flop a) { count_flop(); return Flop(std::sqrt(a.v)); }
inline Flop atan2(Flop a, Flop b) { count_flop(); return Flop(std::atan2(a.v, b.v)); }

// ------------------------------------------------------------------ Dual
struct Dual {
  double v, d;
  Dual(double x = 0.0) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline double val(const Dual& a) { return a.v; }
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual atan2(Dual y, Dual x) {
  double r2 = x.v * x.v + y.v * y.v;
  double dv = r2 > 0.0 ? (x.v * y.d - y.v * x.d) / r2 : 0.0;
  return Dual(std::atan2(y.v, x.v), dv);
}

// ------------------------------------------------------------------ Var (tape)
struct Tape {
  struct Node { int a, b; double da, db; };
  std::vector<Node> nodes;
  // flops spent forming local partial derivatives (divide, sqrt, atan2) of
  // recorded nodes; with 2 flops per edge of the reverse sweep this is the
  // tape's reverse-op count
  int64_t deriv_flops = 0;
  int64_t edges() const {
    int64_t e = 0;
    for (const Node& n : nodes) e += (n.a >= 0) + (n.b >= 0);
    return e;
  }
  int push(int a, double da, int b, double db) {
    nodes.push_back(Node{a, b, da, db});
    return (int)nodes.size() - 1;
  }
  int leaf() { return push(-1, 0.0, -1, 0.0); }
  // Reverse sweep: adj must have nodes.size() entries, seeded by the caller.
  void backward(std::vector<double>& adj) const {
    for (int i = (int)nodes.size() - 1; i >= 0; --i) {
      double g = adj[i];
      if (g == 0.0) continue;
      const Node& n = nodes[i];
      if (n.a >= 0) adj[n.a] += n.da * g;
      if (n.b >= 0) adj[n.b] += n.db * g;
    }
  }
};
inline thread_local Tape* tl_tape = nullptr;

struct Var {
  double v;
  int i;  // node index on the current tape, -1 for a constant
  Var(double x = 0.0) : v(x), i(-1) {}
  Var(double x, int idx) : v(x), i(idx) {}
};
inline double val(const Var& a) { return a.v; }
inline Var var_leaf(double x) { return Var(x, tl_tape->leaf()); }
inline Var var_un(double v, const Var& a, double da) {
  if (a.i < 0) return Var(v);
  return Var(v, tl_tape->push(a.i, da, -1, 0.0));
}
inline Var var_bin(double v, const Var& a, double da, const Var& b, double db) {
  if (a.i < 0 && b.i < 0) return Var(v);
  return Var(v, tl_tape->push(a.i, da, b.i, db));
}
inline Var operator+(Var a, Var b) { return var_bin(a.v + b.v, a, 1.0, b, 1.0); }
inline Var operator-(Var a, Var b) { return var_bin(a.v - b.v, a, 1.0, b, -1.0); }
inline Var operator*(Var a, Var b) { return var_bin(a.v * b.v, a, b.v, b, a.v); }
inline Var operator/(Var a, Var b) {
  double q = a.v / b.v;
  if (a.i >= 0 || b.i >= 0) tl_tape->deriv_flops += 2;
  return var_bin(q, a, 1.0 / b.v, b, -q / b.v);
}
inline Var operator-(Var a) { return var_un(-a.v, a, -1.0); }
inline Var sqrt(Var a) {
  double s = std::sqrt(a.v);
  if (a.i >= 0) tl_tape->deriv_flops += 1;
  return var_un(s, a, s > 0.0 ? 0.5 / s : 0.0);
}
inline Var atan2(Var y, Var x) {
  if (y.i >= 0 || x.i >= 0) tl_tape->deriv_flops += 5;
  double r2 = x.v * x.v + y.v * y.v;
  double dy = r2 > 0.0 ? x.v / r2 : 0.0;
  double dx = r2 > 0.0 ? -y.v / r2 : 0.0;
  return var_bin(std::atan2(y.v, x.v), y, dy, x, dx);
}

// ------------------------------------------------------------------ generic helpers
// Branch helpers: decide on values, return the operand actually selected so
// that derivatives follow the executed branch.  Each selection between two
// computed values counts as one flop (a min/max instruction).
template <class T> inline T vmax(const T& a, const T& b) {
  count_flop();
  return val(a) > val(b) ? a : b;
}
template <class T> inline T vmin(const T& a, const T& b) {
  count_flop();
  return val(a) < val(b) ? a : b;
}
// clamp(a, lo, hi): the derivative passes only strictly inside (lo, hi).
template <class T> inline T vclamp(const T& a, double lo, double hi) {
  count_flop(2);
  if (val(a) >= hi) return T(hi);
  if (val(a) <= lo) return T(lo);
  return a;
}

}  // namespace orc
