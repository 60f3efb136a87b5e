// FP64 oracle -- TEST INFRASTRUCTURE ONLY.  A reverse-mode tape scalar.
//
// Every arithmetic operation on `adouble` values that depend on a registered input appends a
// node (value, up to two parents and the local partial derivatives) to the thread's tape;
// constants never enter the tape.  `backward` sweeps the tape once from the last node to the
// first, accumulating adjoints (the chain rule applied in reverse topological order).
#pragma once
#include <cmath>
#include <vector>

#include "orc_math.hpp"

namespace orc {

struct Tape {
  std::vector<int> p1, p2;
  std::vector<double> d1, d2;
  int push(int a, double da, int b, double db) {
    p1.push_back(a); d1.push_back(da);
    p2.push_back(b); d2.push_back(db);
    return (int)p1.size() - 1;
  }
  void clear() { p1.clear(); p2.clear(); d1.clear(); d2.clear(); }
  size_t size() const { return p1.size(); }
  // adjoints of every node given seeds (node index, adjoint)
  std::vector<double> backward(const std::vector<std::pair<int, double>>& seeds) const {
    std::vector<double> adj(size(), 0.0);
    for (auto& s : seeds)
      if (s.first >= 0) adj[s.first] += s.second;
    for (int n = (int)size() - 1; n >= 0; n--) {
      const double a = adj[n];
      if (a == 0.0) continue;
      if (p1[n] >= 0) adj[p1[n]] += d1[n] * a;
      if (p2[n] >= 0) adj[p2[n]] += d2[n] * a;
    }
    return adj;
  }
};

inline Tape*& tape() {
  static thread_local Tape* t = nullptr;
  return t;
}

struct adouble {
  double v = 0.0;
  int i = -1;   // tape node, -1 for a constant
  adouble() = default;
  adouble(double x) : v(x), i(-1) {}
  static adouble var(double x) {
    adouble r(x);
    r.i = tape()->push(-1, 0.0, -1, 0.0);
    return r;
  }
};

inline double val(const adouble& a) { return a.v; }
template <> struct Taped<adouble> { static constexpr bool value = true; };

inline adouble node(double v, const adouble& a, double da, const adouble& b, double db) {
  adouble r(v);
  if (a.i >= 0 || b.i >= 0) r.i = tape()->push(a.i, a.i >= 0 ? da : 0.0, b.i, b.i >= 0 ? db : 0.0);
  return r;
}
inline adouble node1(double v, const adouble& a, double da) {
  adouble r(v);
  if (a.i >= 0) r.i = tape()->push(a.i, da, -1, 0.0);
  return r;
}

inline adouble operator+(const adouble& a, const adouble& b) { return node(a.v + b.v, a, 1.0, b, 1.0); }
inline adouble operator-(const adouble& a, const adouble& b) { return node(a.v - b.v, a, 1.0, b, -1.0); }
inline adouble operator*(const adouble& a, const adouble& b) { return node(a.v * b.v, a, b.v, b, a.v); }
inline adouble operator/(const adouble& a, const adouble& b) {
  const double q = a.v / b.v;
  return node(q, a, 1.0 / b.v, b, -q / b.v);
}
inline adouble operator-(const adouble& a) { return node1(-a.v, a, -1.0); }
inline adouble operator+(const adouble& a, double b) { return node1(a.v + b, a, 1.0); }
inline adouble operator+(double a, const adouble& b) { return node1(a + b.v, b, 1.0); }
inline adouble operator-(const adouble& a, double b) { return node1(a.v - b, a, 1.0); }
inline adouble operator-(double a, const adouble& b) { return node1(a - b.v, b, -1.0); }
inline adouble operator*(const adouble& a, double b) { return node1(a.v * b, a, b); }
inline adouble operator*(double a, const adouble& b) { return node1(a * b.v, b, a); }
inline adouble operator/(const adouble& a, double b) { return node1(a.v / b, a, 1.0 / b); }
inline adouble operator/(double a, const adouble& b) {
  const double q = a / b.v;
  return node1(q, b, -q / b.v);
}
inline adouble& operator+=(adouble& a, const adouble& b) { return a = a + b; }
inline adouble& operator-=(adouble& a, const adouble& b) { return a = a - b; }
inline adouble& operator*=(adouble& a, const adouble& b) { return a = a * b; }

inline adouble sqrt(const adouble& a) {
  const double s = std::sqrt(a.v);
  return node1(s, a, s > 0 ? 0.5 / s : 0.0);
}
inline adouble sin(const adouble& a) { return node1(std::sin(a.v), a, std::cos(a.v)); }
inline adouble cos(const adouble& a) { return node1(std::cos(a.v), a, -std::sin(a.v)); }
inline adouble pow(const adouble& a, double p) {
  const double r = std::pow(a.v, p);
  return node1(r, a, a.v != 0.0 ? p * r / a.v : (p == 1.0 ? 1.0 : 0.0));
}

}  // namespace orc
