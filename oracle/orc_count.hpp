// FP64 oracle -- TEST INFRASTRUCTURE ONLY.  A counting scalar: the oracle instantiated on
// `cdouble` computes the same doubles and tallies its floating-point operations per phase of the
// substep, for the algorithmic flop count of the step (the roofline's numerator).
//
// What counts.  An operation counts one flop (add, sub, mul, div, sqrt; sin, cos and pow one
// each as transcendentals) when it does work that a model-specialised program must do:
//   * every value derived from the state, the controls or the solver is "variable"; a value
//     built from a double in the code (a literal or a model constant) is "constant";
//   * an operation on constants only is folded (counts nothing), as a compiler folds it;
//   * a product with a constant 0 is the constant 0, a product or quotient with a constant +-1
//     is the other operand (its sign), a sum with a constant 0 is the other operand: none counts
//     (this is what keeps the tally on the tree-sparse pattern: the oracle's dense loops run over
//     zero blocks that are constant zeros here);
//   * every other operation counts one.
// A fused multiply-add is a product and a sum: two flops.  Comparisons count nothing.
#pragma once
#include <cmath>

#include "orc_math.hpp"

namespace orc {

// phases of the substep; PH_DIAG (the solver's contact-force output) is not part of the step
enum CountPhase { PH_KIN = 0, PH_MASS, PH_BIAS, PH_SMOOTH, PH_COLLIDE, PH_ROWS, PH_SOLVE, PH_INTEGRATE, PH_DIAG, PH_N };

struct Counts {
  double add[PH_N], mul[PH_N], div[PH_N], sqrt[PH_N], trans[PH_N];
  int phase = 0;
  void clear() {
    for (int k = 0; k < PH_N; k++) add[k] = mul[k] = div[k] = sqrt[k] = trans[k] = 0.0;
    phase = 0;
  }
};

inline Counts& counts() {
  static thread_local Counts c;
  return c;
}

struct cdouble {
  double v = 0.0;
  bool k = true;   // constant (folded by a specialising compiler)
  cdouble() = default;
  cdouble(double x) : v(x), k(true) {}
  static cdouble var(double x) {
    cdouble r(x);
    r.k = false;
    return r;
  }
};

inline double val(const cdouble& a) { return a.v; }

inline cdouble cvar(double x) { return cdouble::var(x); }
inline bool is_c(const cdouble& a, double x) { return a.k && a.v == x; }

inline cdouble operator+(const cdouble& a, const cdouble& b) {
  if (a.k && b.k) return cdouble(a.v + b.v);
  if (is_c(a, 0.0)) return b;
  if (is_c(b, 0.0)) return a;
  counts().add[counts().phase] += 1;
  return cvar(a.v + b.v);
}
inline cdouble operator-(const cdouble& a) {
  cdouble r = a;
  r.v = -a.v;
  return r;
}
inline cdouble operator-(const cdouble& a, const cdouble& b) {
  if (a.k && b.k) return cdouble(a.v - b.v);
  if (is_c(a, 0.0)) return -b;
  if (is_c(b, 0.0)) return a;
  counts().add[counts().phase] += 1;
  return cvar(a.v - b.v);
}
inline cdouble operator*(const cdouble& a, const cdouble& b) {
  if (a.k && b.k) return cdouble(a.v * b.v);
  if (is_c(a, 0.0) || is_c(b, 0.0)) return cdouble(0.0);
  if (is_c(a, 1.0)) return b;
  if (is_c(b, 1.0)) return a;
  if (is_c(a, -1.0)) return -b;
  if (is_c(b, -1.0)) return -a;
  counts().mul[counts().phase] += 1;
  return cvar(a.v * b.v);
}
inline cdouble operator/(const cdouble& a, const cdouble& b) {
  if (a.k && b.k) return cdouble(a.v / b.v);
  if (is_c(a, 0.0)) return cdouble(0.0);
  if (is_c(b, 1.0)) return a;
  if (is_c(b, -1.0)) return -a;
  counts().div[counts().phase] += 1;
  return cvar(a.v / b.v);
}
inline cdouble operator+(const cdouble& a, double b) { return a + cdouble(b); }
inline cdouble operator+(double a, const cdouble& b) { return cdouble(a) + b; }
inline cdouble operator-(const cdouble& a, double b) { return a - cdouble(b); }
inline cdouble operator-(double a, const cdouble& b) { return cdouble(a) - b; }
inline cdouble operator*(const cdouble& a, double b) { return a * cdouble(b); }
inline cdouble operator*(double a, const cdouble& b) { return cdouble(a) * b; }
inline cdouble operator/(const cdouble& a, double b) { return a / cdouble(b); }
inline cdouble operator/(double a, const cdouble& b) { return cdouble(a) / b; }
inline cdouble& operator+=(cdouble& a, const cdouble& b) { return a = a + b; }
inline cdouble& operator-=(cdouble& a, const cdouble& b) { return a = a - b; }
inline cdouble& operator*=(cdouble& a, const cdouble& b) { return a = a * b; }

inline cdouble sqrt(const cdouble& a) {
  if (a.k) return cdouble(std::sqrt(a.v));
  counts().sqrt[counts().phase] += 1;
  return cvar(std::sqrt(a.v));
}
inline cdouble sin(const cdouble& a) {
  if (a.k) return cdouble(std::sin(a.v));
  counts().trans[counts().phase] += 1;
  return cvar(std::sin(a.v));
}
inline cdouble cos(const cdouble& a) {
  if (a.k) return cdouble(std::cos(a.v));
  counts().trans[counts().phase] += 1;
  return cvar(std::cos(a.v));
}
inline cdouble pow(const cdouble& a, double p) {
  if (a.k) return cdouble(std::pow(a.v, p));
  if (p == 1.0) return a;
  counts().trans[counts().phase] += 1;
  return cvar(std::pow(a.v, p));
}

// the phase hook of orc_step.hpp, and the tree-sparse factorisation, for the counting scalar
template <> struct PhaseHook<cdouble> {
  static void set(int k) { counts().phase = k; }
};
template <> struct TreeMethods<cdouble> {
  static constexpr bool value = true;
};

}  // namespace orc
