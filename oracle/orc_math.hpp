// FP64 oracle for the batched physics step -- TEST INFRASTRUCTURE ONLY.
//
// Small dense vector / matrix / quaternion helpers, written for readability.  Every
// routine is generic over the scalar type T so that the oracle can be instantiated with
// plain double and with a reverse-mode tape scalar.  `val(x)` returns the double value of
// a scalar and is used for every comparison that decides a branch.
//
// Only tests/, the package's smoke() check and bench.py's CPU-baseline leg may load the
// library built from these files; the product path never does.
#pragma once
#include <array>
#include <cmath>
#include <vector>

namespace orc {

inline double val(double x) { return x; }

template <class T> using V3 = std::array<T, 3>;
template <class T> using M3 = std::array<T, 9>;   // row-major 3x3

template <class T> inline V3<T> v3(T a, T b, T c) { return V3<T>{a, b, c}; }
template <class T> inline V3<T> add(const V3<T>& a, const V3<T>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
template <class T> inline V3<T> sub(const V3<T>& a, const V3<T>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
template <class T, class S> inline V3<T> scl(const V3<T>& a, const S& s) { return {a[0] * s, a[1] * s, a[2] * s}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
template <class T> inline T norm(const V3<T>& a) { using std::sqrt; return sqrt(dot(a, a)); }

template <class T> inline M3<T> eye3() { return M3<T>{T(1), T(0), T(0), T(0), T(1), T(0), T(0), T(0), T(1)}; }
template <class T> inline V3<T> mv(const M3<T>& m, const V3<T>& v) {
  return {m[0] * v[0] + m[1] * v[1] + m[2] * v[2], m[3] * v[0] + m[4] * v[1] + m[5] * v[2],
          m[6] * v[0] + m[7] * v[1] + m[8] * v[2]};
}
template <class T> inline V3<T> mtv(const M3<T>& m, const V3<T>& v) {   // m^T v
  return {m[0] * v[0] + m[3] * v[1] + m[6] * v[2], m[1] * v[0] + m[4] * v[1] + m[7] * v[2],
          m[2] * v[0] + m[5] * v[1] + m[8] * v[2]};
}
template <class T> inline M3<T> mm(const M3<T>& a, const M3<T>& b) {
  M3<T> c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
  return c;
}
template <class T> inline M3<T> mT(const M3<T>& a) { return {a[0], a[3], a[6], a[1], a[4], a[7], a[2], a[5], a[8]}; }
template <class T> inline V3<T> col(const M3<T>& a, int k) { return {a[k], a[3 + k], a[6 + k]}; }

// rotation matrix of a unit quaternion (w, x, y, z), Hamilton convention: v' = q v q*
template <class T> inline M3<T> quat2mat(const T* q) {
  T w = q[0], x = q[1], y = q[2], z = q[3];
  return {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
          2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
          2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
}

// rotation by `angle` about the unit axis `a` (Rodrigues' formula)
template <class T> inline M3<T> axis_angle(const V3<T>& a, const T& angle) {
  using std::cos; using std::sin;
  T c = cos(angle), s = sin(angle), C = 1 - c;
  return {c + a[0] * a[0] * C, a[0] * a[1] * C - a[2] * s, a[0] * a[2] * C + a[1] * s,
          a[1] * a[0] * C + a[2] * s, c + a[1] * a[1] * C, a[1] * a[2] * C - a[0] * s,
          a[2] * a[0] * C - a[1] * s, a[2] * a[1] * C + a[0] * s, c + a[2] * a[2] * C};
}

// Hamilton product p (x) q
template <class T> inline std::array<T, 4> qmul(const std::array<T, 4>& p, const std::array<T, 4>& q) {
  return {p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3],
          p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2],
          p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1],
          p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0]};
}

// rigid transform (R, p): x -> R x + p, i.e. the 4x4 homogeneous matrix [R p; 0 1]
template <class T> struct Xf {
  M3<T> R;
  V3<T> p;
};
template <class T> inline Xf<T> xf_identity() { return Xf<T>{eye3<T>(), V3<T>{T(0), T(0), T(0)}}; }
template <class T> inline Xf<T> compose(const Xf<T>& a, const Xf<T>& b) {   // a * b
  return Xf<T>{mm(a.R, b.R), add(mv(a.R, b.p), a.p)};
}
template <class T> inline V3<T> xform(const Xf<T>& a, const V3<T>& x) { return add(mv(a.R, x), a.p); }

// dense row-major n x n helpers on std::vector
template <class T> using Vec = std::vector<T>;

// Cholesky factor (lower) of a symmetric positive definite matrix; returns false if it fails
template <class T> bool cholesky(Vec<T>& A, int n) {
  using std::sqrt;
  for (int j = 0; j < n; j++) {
    T s = A[j * n + j];
    for (int k = 0; k < j; k++) s = s - A[j * n + k] * A[j * n + k];
    if (!(val(s) > 0.0)) return false;
    T d = sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      T t = A[i * n + j];
      for (int k = 0; k < j; k++) t = t - A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
    for (int i = 0; i < j; i++) A[i * n + j] = T(0);
  }
  return true;
}

// solve (L L^T) x = b in place with the lower factor L
template <class T> void chol_solve(const Vec<T>& L, int n, Vec<T>& b) {
  for (int i = 0; i < n; i++) {
    T s = b[i];
    for (int k = 0; k < i; k++) s = s - L[i * n + k] * b[k];
    b[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; i--) {
    T s = b[i];
    for (int k = i + 1; k < n; k++) s = s - L[k * n + i] * b[k];
    b[i] = s / L[i * n + i];
  }
}

// L^T D L factorisation of a symmetric positive definite matrix, eliminating from the last index
// (A = L^T D L, L unit lower triangular).  For a matrix whose pattern is a tree's ancestor
// pattern with parents before children (a mass matrix in level order) it makes no fill-in.
// The oracle solves with the Cholesky factor; the flop count (orc_count.hpp) takes this one,
// the tree-sparse factorisation of the method.  In place: A_kk = D_k, A_ki = L_ki (i < k);
// returns false if a pivot is not positive.
template <class T> bool ldlt_leaves_first(Vec<T>& A, int n) {
  for (int k = n - 1; k >= 0; k--) {
    if (!(val(A[k * n + k]) > 0.0)) return false;
    for (int i = k - 1; i >= 0; i--) {
      T l = A[k * n + i] / A[k * n + k];
      for (int j = 0; j <= i; j++) A[i * n + j] = A[i * n + j] - l * A[k * n + j];
      A[k * n + i] = l;
    }
  }
  return true;
}

// solve (L^T D L) x = b in place with the factor of ldlt_leaves_first
template <class T> void ldlt_solve(const Vec<T>& A, int n, Vec<T>& b) {
  for (int k = n - 1; k >= 0; k--)
    for (int i = 0; i < k; i++) b[i] = b[i] - A[k * n + i] * b[k];
  for (int k = 0; k < n; k++) b[k] = b[k] / A[k * n + k];
  for (int k = 0; k < n; k++)
    for (int i = 0; i < k; i++) b[k] = b[k] - A[k * n + i] * b[i];
}

// The methods the oracle uses: its plain ones (the mass matrix from the kinetic energy, Cholesky
// solves), except for a counting scalar (orc_count.hpp), which takes the tree methods whose flops
// the step's count is of: CRBA and the leaves-first L^T D L (each pinned against the plain one).
template <class T> struct TreeMethods { static constexpr bool value = false; };
// Whether a scalar records a reverse-mode tape (orc_ad.hpp specialises it for adouble).
template <class T> struct Taped { static constexpr bool value = false; };
template <class T> bool spd_factor(Vec<T>& A, int n) {
  return TreeMethods<T>::value ? ldlt_leaves_first(A, n) : cholesky(A, n);
}
template <class T> void spd_solve(const Vec<T>& A, int n, Vec<T>& b) {
  if (TreeMethods<T>::value) ldlt_solve(A, n, b);
  else chol_solve(A, n, b);
}

// Phases of the substep for a counting scalar's tally (orc_count.hpp); nothing for the others.
template <class T> struct PhaseHook {
  static void set(int) {}
};

}  // namespace orc
