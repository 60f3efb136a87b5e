// FP64 oracle -- TEST INFRASTRUCTURE ONLY.
//
// One physics substep of one environment, written as plainly as possible:
//   kinematics with rigid transforms, the mass matrix from its kinetic-energy definition
//   (sum over bodies of m Jv^T Jv + Jw^T I Jw), bias forces by Newton-Euler on per-body
//   velocities/accelerations projected through the Jacobians, dense Cholesky solves,
//   primitive collision by direct geometry, constraint rows, the capped (or converged)
//   Newton solve with an exact line search on sorted breakpoints, PD/motor actuation and
//   semi-implicit Euler.
//
// The paper (MuJoCo Playground, Sec. 1 and Limitations) runs its environments on MJX and
// does not print the step's mathematics; the formulation below is the textbook rigid-body
// method in generalised coordinates, with these choices fixed (identically on the GPU):
//   * PD law tau = kp (q_des - q) - kd qdot, eq. (pd_mapping), App. B.2.1, held over substeps;
//   * armature I_a = k_g^2 m_r r_r^2 / 2, App. C.2.2;
//   * static candidate pair lists with fixed per-pair slots (Limitations; App. B.2.3);
//   * a Newton solver with a fixed iteration cap (Table dm_control_envs, iterations=1..4);
//   * soft constraints: aref = -b v - k d(r) r, R = (1-d)/d * Ahat with the exact diagonal
//     Ahat = (J M^-1 J^T)_ii, D = 1/R; impedance d(r) from solimp (d0, dwidth, width, mid, p).
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

#include "orc_math.hpp"
#include "orc_model.hpp"

namespace orc {

using std::sqrt;

// Optional differentiable model parameters (a tape scalar can take derivatives through them):
// body masses (a body's inertia scales with its mass, its centre of mass is unchanged), dof
// damping and actuator kp.  A null pointer means the model's own constants.
template <class T> struct Params {
  std::vector<T> mass, damping, kp;
};

template <class T> inline T body_mass(const Model& m, const Params<T>* P, int b) {
  return P ? P->mass[b] : T(m.mass[b]);
}

// ------------------------------------------------------------------------------------
// kinematics
// ------------------------------------------------------------------------------------
template <class T> struct Kin {
  std::vector<Xf<T>> xbody;    // body frames in the world
  std::vector<V3<T>> xcom;     // body centres of mass
  std::vector<M3<T>> Iw;       // body inertia about the COM, world axes
  std::vector<V3<T>> janchor;  // joint anchor (world), taken before the joint moves
  std::vector<V3<T>> jaxis;    // joint axis (world)
  std::vector<Xf<T>> xgeom;    // geom frames
};

template <class T> inline Xf<T> body_offset(const Model& m, int b) {
  T q[4] = {T(m.body_quat[4 * b]), T(m.body_quat[4 * b + 1]), T(m.body_quat[4 * b + 2]), T(m.body_quat[4 * b + 3])};
  return Xf<T>{quat2mat(q), V3<T>{T(m.body_pos[3 * b]), T(m.body_pos[3 * b + 1]), T(m.body_pos[3 * b + 2])}};
}

template <class T> inline V3<T> cv3(const double* p) { return V3<T>{T(p[0]), T(p[1]), T(p[2])}; }

// World frame of every body: X(b) = X(parent) * X_offset(b) * prod_j X_joint(j, q_j).
// Hinge: rotation by q about the axis through the anchor; slide: translation q along the axis;
// free: position qpos[0:3] and the normalised quaternion qpos[3:7] (the parent is the world).
template <class T> void kinematics(const Model& m, const T* qpos, Kin<T>& k, const Params<T>* P = nullptr) {
  k.xbody.assign(m.nbody, xf_identity<T>());
  k.xcom.assign(m.nbody, V3<T>{T(0), T(0), T(0)});
  k.Iw.assign(m.nbody, M3<T>{});
  k.janchor.assign(m.njnt, V3<T>{});
  k.jaxis.assign(m.njnt, V3<T>{});
  for (int b = 1; b < m.nbody; b++) {
    Xf<T> X = compose(k.xbody[m.parent[b]], body_offset<T>(m, b));
    for (int j = m.body_jntadr[b]; j < m.body_jntadr[b] + m.body_jntnum[b]; j++) {
      const T* q = qpos + m.jnt_qposadr[j];
      V3<T> p = cv3<T>(&m.jnt_pos[3 * j]), a = cv3<T>(&m.jnt_axis[3 * j]);
      if (m.jnt_type[j] == FREE) {
        T n = sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5] + q[6] * q[6]);
        T qu[4] = {q[3] / n, q[4] / n, q[5] / n, q[6] / n};
        X = Xf<T>{quat2mat(qu), V3<T>{q[0], q[1], q[2]}};
        k.janchor[j] = X.p;
        k.jaxis[j] = V3<T>{T(0), T(0), T(0)};
      } else {
        k.janchor[j] = xform(X, p);
        k.jaxis[j] = mv(X.R, a);
        if (m.jnt_type[j] == HINGE) {
          Xf<T> to{eye3<T>(), p}, back{eye3<T>(), scl(p, T(-1))}, rot{axis_angle(a, q[0]), V3<T>{T(0), T(0), T(0)}};
          X = compose(X, compose(to, compose(rot, back)));
        } else {
          X = compose(X, Xf<T>{eye3<T>(), scl(a, q[0])});
        }
      }
    }
    k.xbody[b] = X;
    k.xcom[b] = xform(X, cv3<T>(&m.ipos[3 * b]));
    const double* I = &m.inertia[6 * b];
    M3<T> Ib{T(I[0]), T(I[3]), T(I[4]), T(I[3]), T(I[1]), T(I[5]), T(I[4]), T(I[5]), T(I[2])};
    if (P && m.mass[b] > 0)
      for (int q = 0; q < 9; q++) Ib[q] = Ib[q] * (P->mass[b] / m.mass[b]);
    k.Iw[b] = mm(X.R, mm(Ib, mT(X.R)));
  }
  k.xgeom.resize(m.ngeom);
  for (int g = 0; g < m.ngeom; g++) {
    T q[4] = {T(m.geom_quat[4 * g]), T(m.geom_quat[4 * g + 1]), T(m.geom_quat[4 * g + 2]), T(m.geom_quat[4 * g + 3])};
    k.xgeom[g] = compose(k.xbody[m.geom_body[g]], Xf<T>{quat2mat(q), cv3<T>(&m.geom_pos[3 * g])});
  }
}

// Linear (Jv) and angular (Jw) velocity Jacobians, 3 x nv row-major, of the world point P
// moving with body b.  Columns: hinge (a, a x (P - anchor)); slide (0, a); free translation
// (0, e_k) in world axes; free rotation (R e_k, R e_k x (P - x_body)) for the body-local
// angular velocity.
template <class T> void point_jacobian(const Model& m, const Kin<T>& k, int b, const V3<T>& P, std::vector<T>& Jv,
                                       std::vector<T>& Jw) {
  const int nv = m.nv;
  Jv.assign(3 * nv, T(0));
  Jw.assign(3 * nv, T(0));
  for (int bb = b; bb > 0; bb = m.parent[bb]) {
    for (int j = m.body_jntadr[bb]; j < m.body_jntadr[bb] + m.body_jntnum[bb]; j++) {
      int d = m.jnt_dofadr[j];
      if (m.jnt_type[j] == FREE) {
        const M3<T>& R = k.xbody[bb].R;
        for (int c = 0; c < 3; c++) {
          Jv[c * nv + d + c] = T(1);
          V3<T> e = col(R, c);
          V3<T> lin = cross(e, sub(P, k.xbody[bb].p));
          for (int r = 0; r < 3; r++) {
            Jw[r * nv + d + 3 + c] = e[r];
            Jv[r * nv + d + 3 + c] = lin[r];
          }
        }
      } else if (m.jnt_type[j] == HINGE) {
        V3<T> a = k.jaxis[j], lin = cross(a, sub(P, k.janchor[j]));
        for (int r = 0; r < 3; r++) {
          Jw[r * nv + d] = a[r];
          Jv[r * nv + d] = lin[r];
        }
      } else {
        for (int r = 0; r < 3; r++) Jv[r * nv + d] = k.jaxis[j][r];
      }
    }
  }
}

// M = sum_b ( m_b Jv(com_b)^T Jv(com_b) + Jw_b^T Iw_b Jw_b ) + diag(armature):
// the matrix of the kinetic energy 1/2 qdot^T M qdot (rotor inertia on the diagonal).
template <class T> void mass_matrix(const Model& m, const Kin<T>& k, std::vector<T>& M, const Params<T>* P = nullptr) {
  const int nv = m.nv;
  M.assign(nv * nv, T(0));
  std::vector<T> Jv, Jw;
  for (int b = 1; b < m.nbody; b++) {
    point_jacobian(m, k, b, k.xcom[b], Jv, Jw);
    for (int i = 0; i < nv; i++)
      for (int j = 0; j < nv; j++) {
        T s = T(0);
        for (int r = 0; r < 3; r++) s = s + body_mass(m, P, b) * Jv[r * nv + i] * Jv[r * nv + j];
        for (int r = 0; r < 3; r++)
          for (int c = 0; c < 3; c++) s = s + Jw[r * nv + i] * k.Iw[b][3 * r + c] * Jw[c * nv + j];
        M[i * nv + j] = M[i * nv + j] + s;
      }
  }
  for (int i = 0; i < nv; i++) M[i * nv + i] = M[i * nv + i] + T(m.dof_armature[i]);
}

// The same matrix by the composite-rigid-body algorithm (CRBA).  Spatial vectors about the world
// origin: a dof's motion subspace s = (w, v) moves a body point P with velocity v + w x P (hinge
// with axis a through the anchor p: (a, p x a); slide: (0, a); free translation k: (0, e_k); free
// rotation k about the body origin x: (R e_k, x x R e_k)); a body's spatial inertia about the
// origin is (I_O = Iw + m (|c|^2 1 - c c^T), h = m c, m) with c its centre of mass.  Composite
// inertias Ic(b) = own + the children's composites; for dof j on body b the force Ic(b) s_j =
// (I_O w + h x v, m v - h x w), and M_ij = s_i . (Ic(b) s_j) for every dof i on j's chain.
template <class T> void crba_mass_matrix(const Model& m, const Kin<T>& k, std::vector<T>& M, const Params<T>* P = nullptr) {
  const int nv = m.nv;
  M.assign(nv * nv, T(0));
  std::vector<std::array<T, 6>> S(nv);
  std::vector<int> dof_body(nv, 0);
  for (int b = 1; b < m.nbody; b++)
    for (int j = m.body_jntadr[b]; j < m.body_jntadr[b] + m.body_jntnum[b]; j++) {
      const int d = m.jnt_dofadr[j];
      if (m.jnt_type[j] == FREE) {
        const Xf<T>& X = k.xbody[b];
        for (int c = 0; c < 3; c++) {
          S[d + c] = {T(0), T(0), T(0), T(c == 0 ? 1 : 0), T(c == 1 ? 1 : 0), T(c == 2 ? 1 : 0)};
          const V3<T> e = col(X.R, c), v = cross(X.p, e);
          S[d + 3 + c] = {e[0], e[1], e[2], v[0], v[1], v[2]};
          dof_body[d + c] = dof_body[d + 3 + c] = b;
        }
      } else if (m.jnt_type[j] == HINGE) {
        const V3<T> a = k.jaxis[j], v = cross(k.janchor[j], a);
        S[d] = {a[0], a[1], a[2], v[0], v[1], v[2]};
        dof_body[d] = b;
      } else {
        const V3<T> a = k.jaxis[j];
        S[d] = {T(0), T(0), T(0), a[0], a[1], a[2]};
        dof_body[d] = b;
      }
    }
  // spatial inertias about the origin: I_O (Ixx Iyy Izz Ixy Ixz Iyz), h, m
  std::vector<std::array<T, 10>> Ic(m.nbody);
  for (int b = 1; b < m.nbody; b++) {
    const T mb = body_mass(m, P, b);
    const V3<T>& c = k.xcom[b];
    const M3<T>& I = k.Iw[b];
    const T c2 = dot(c, c);
    Ic[b] = {I[0] + mb * (c2 - c[0] * c[0]), I[4] + mb * (c2 - c[1] * c[1]), I[8] + mb * (c2 - c[2] * c[2]),
             I[1] - mb * c[0] * c[1], I[2] - mb * c[0] * c[2], I[5] - mb * c[1] * c[2],
             mb * c[0], mb * c[1], mb * c[2], mb};
  }
  for (int b = m.nbody - 1; b >= 1; b--)
    if (m.parent[b] > 0)
      for (int q = 0; q < 10; q++) Ic[m.parent[b]][q] = Ic[m.parent[b]][q] + Ic[b][q];
  for (int j = 0; j < nv; j++) {
    const std::array<T, 10>& I = Ic[dof_body[j]];
    const V3<T> w{S[j][0], S[j][1], S[j][2]}, v{S[j][3], S[j][4], S[j][5]}, h{I[6], I[7], I[8]};
    const V3<T> fa = add(V3<T>{I[0] * w[0] + I[3] * w[1] + I[4] * w[2], I[3] * w[0] + I[1] * w[1] + I[5] * w[2],
                               I[4] * w[0] + I[5] * w[1] + I[2] * w[2]},
                         cross(h, v));
    const V3<T> fl = sub(scl(v, I[9]), cross(h, w));
    // dof j's chain: the earlier dofs of its body, then every dof of its ancestors
    for (int b = dof_body[j]; b > 0; b = m.parent[b])
      for (int jj = m.body_jntadr[b]; jj < m.body_jntadr[b] + m.body_jntnum[b]; jj++)
        for (int i = m.jnt_dofadr[jj]; i < m.jnt_dofadr[jj] + (m.jnt_type[jj] == FREE ? 6 : 1); i++) {
          if (b == dof_body[j] && i > j) continue;
          const T Mij = S[i][0] * fa[0] + S[i][1] * fa[1] + S[i][2] * fa[2] + S[i][3] * fl[0] + S[i][4] * fl[1] +
                        S[i][5] * fl[2];
          M[j * nv + i] = Mij;
          M[i * nv + j] = Mij;
        }
  }
  for (int i = 0; i < nv; i++) M[i * nv + i] = M[i * nv + i] + T(m.dof_armature[i]);
}

// Per-body angular velocity w and acceleration al, and a reference point r fixed in the body
// with its velocity vr and acceleration ar, propagated from the world along each joint:
//   hinge (axis a through p): move the reference to p (rigid-body formulas), then
//         w += a qd,  al += a qdd + w_before x (a qd);
//   slide (axis a): vr += a qd, ar += a qdd + 2 w x (a qd)   (relative + Coriolis terms);
//   free: w = R qd[3:6], al = R qdd[3:6], r = x_body, vr = qd[0:3], ar = qdd[0:3].
template <class T> struct Motion {
  V3<T> w, al, r, vr, ar;
};

template <class T> void body_motion(const Model& m, const Kin<T>& k, const T* qvel, const T* qacc,
                                    std::vector<Motion<T>>& out) {
  V3<T> z{T(0), T(0), T(0)};
  out.assign(m.nbody, Motion<T>{z, z, z, z, z});
  for (int b = 1; b < m.nbody; b++) {
    Motion<T> s = out[m.parent[b]];
    for (int j = m.body_jntadr[b]; j < m.body_jntadr[b] + m.body_jntnum[b]; j++) {
      int d = m.jnt_dofadr[j];
      if (m.jnt_type[j] == FREE) {
        const M3<T>& R = k.xbody[b].R;
        s.w = mv(R, V3<T>{qvel[d + 3], qvel[d + 4], qvel[d + 5]});
        s.al = mv(R, V3<T>{qacc[d + 3], qacc[d + 4], qacc[d + 5]});
        s.r = k.xbody[b].p;
        s.vr = V3<T>{qvel[d], qvel[d + 1], qvel[d + 2]};
        s.ar = V3<T>{qacc[d], qacc[d + 1], qacc[d + 2]};
      } else if (m.jnt_type[j] == HINGE) {
        V3<T> p = k.janchor[j], a = k.jaxis[j], rp = sub(p, s.r);
        s.vr = add(s.vr, cross(s.w, rp));
        s.ar = add(add(s.ar, cross(s.al, rp)), cross(s.w, cross(s.w, rp)));
        s.r = p;
        s.al = add(add(s.al, scl(a, qacc[d])), cross(s.w, scl(a, qvel[d])));
        s.w = add(s.w, scl(a, qvel[d]));
      } else {
        V3<T> a = k.jaxis[j];
        s.vr = add(s.vr, scl(a, qvel[d]));
        s.ar = add(add(s.ar, scl(a, qacc[d])), scl(cross(s.w, scl(a, qvel[d])), T(2)));
      }
    }
    out[b] = s;
  }
}

template <class T> inline V3<T> point_vel(const Motion<T>& s, const V3<T>& P) { return add(s.vr, cross(s.w, sub(P, s.r))); }
template <class T> inline V3<T> point_acc(const Motion<T>& s, const V3<T>& P) {
  V3<T> d = sub(P, s.r);
  return add(add(s.ar, cross(s.al, d)), cross(s.w, cross(s.w, d)));
}

// Inverse dynamics tau = M(q) qdd + c(q, qd) by Newton-Euler: per body the force
// m (a_com - g) and the torque about the COM Iw al + w x Iw w, mapped to generalised forces
// with the body's Jacobians (virtual work); plus armature * qdd.
template <class T> void inverse_dynamics(const Model& m, const Kin<T>& k, const T* qvel, const T* qacc, std::vector<T>& tau,
                                         const Params<T>* P = nullptr) {
  const int nv = m.nv;
  std::vector<Motion<T>> mo;
  body_motion(m, k, qvel, qacc, mo);
  tau.assign(nv, T(0));
  V3<T> g{T(m.gravity[0]), T(m.gravity[1]), T(m.gravity[2])};
  std::vector<T> Jv, Jw;
  for (int b = 1; b < m.nbody; b++) {
    V3<T> ac = point_acc(mo[b], k.xcom[b]);
    V3<T> F = scl(sub(ac, g), body_mass(m, P, b));
    V3<T> Iwv = mv(k.Iw[b], mo[b].w);
    V3<T> N = add(mv(k.Iw[b], mo[b].al), cross(mo[b].w, Iwv));
    point_jacobian(m, k, b, k.xcom[b], Jv, Jw);
    for (int i = 0; i < nv; i++) {
      T s = T(0);
      for (int r = 0; r < 3; r++) s = s + Jv[r * nv + i] * F[r] + Jw[r * nv + i] * N[r];
      tau[i] = tau[i] + s;
    }
  }
  for (int i = 0; i < nv; i++) tau[i] = tau[i] + T(m.dof_armature[i]) * qacc[i];
}

// ------------------------------------------------------------------------------------
// collision
// ------------------------------------------------------------------------------------
template <class T> struct Contact {
  bool active = false;
  T dist = T(0);
  V3<T> pos{}, n{}, t1{}, t2{};
};

// Tangent frame: t1 = normalise(n x e_k), e_k the world axis with the smallest |n_k|
// (ties to the lowest k); t2 = n x t1.
template <class T> void contact_frame(Contact<T>& c) {
  double a0 = std::fabs(val(c.n[0])), a1 = std::fabs(val(c.n[1])), a2 = std::fabs(val(c.n[2]));
  int kmin = 0;
  if (a1 < a0) kmin = 1;
  if (a2 < (kmin == 0 ? a0 : a1)) kmin = 2;
  V3<T> e{T(0), T(0), T(0)};
  e[kmin] = T(1);
  V3<T> t = cross(c.n, e);
  c.t1 = scl(t, T(1) / norm(t));
  c.t2 = cross(c.n, c.t1);
}

// Two spheres (c1, r1) -> (c2, r2); normal from the first to the second; the contact point is
// the midpoint of the two surface points.  Coincident centres use the normal +z.
template <class T> Contact<T> sphere_sphere(const V3<T>& c1, T r1, const V3<T>& c2, T r2) {
  Contact<T> c;
  V3<T> d = sub(c2, c1);
  T L = norm(d);
  if (val(L) > 1e-12) c.n = scl(d, T(1) / L);
  else c.n = V3<T>{T(0), T(0), T(1)};
  c.dist = L - r1 - r2;
  V3<T> s1 = add(c1, scl(c.n, r1)), s2 = sub(c2, scl(c.n, r2));
  c.pos = scl(add(s1, s2), T(0.5));
  return c;
}

// Sphere (c, r) against a plane through p0 with unit normal nz (the plane is geom1).
template <class T> Contact<T> plane_sphere(const V3<T>& p0, const V3<T>& nz, const V3<T>& c, T r) {
  Contact<T> out;
  T h = dot(nz, sub(c, p0));
  out.n = nz;
  out.dist = h - r;
  V3<T> s_sphere = sub(c, scl(nz, r)), s_plane = sub(c, scl(nz, h));
  out.pos = scl(add(s_sphere, s_plane), T(0.5));
  return out;
}

// Sphere (c, r) (geom1) against a box (frame X, half-sizes h) (geom2).  Outside: the closest
// box point by clamping; inside: the face of least penetration (ties to the lowest axis).
template <class T> Contact<T> sphere_box(const V3<T>& c, T r, const Xf<T>& X, const double* h) {
  Contact<T> out;
  V3<T> p = mtv(X.R, sub(c, X.p));
  V3<T> q;
  bool inside = true;
  for (int k = 0; k < 3; k++) {
    T hk = T(h[k]);
    if (val(p[k]) > h[k]) { q[k] = hk; inside = false; }
    else if (val(p[k]) < -h[k]) { q[k] = -hk; inside = false; }
    else q[k] = p[k];
  }
  V3<T> out_dir;   // unit direction from the box towards the sphere (world)
  V3<T> surf;      // box surface point (box frame)
  if (!inside) {
    V3<T> d = sub(p, q);
    T L = norm(d);
    out_dir = mv(X.R, scl(d, T(1) / L));
    surf = q;
    out.dist = L - r;
  } else {
    int kb = 0;
    double best = h[0] - std::fabs(val(p[0]));
    for (int k = 1; k < 3; k++) {
      double s = h[k] - std::fabs(val(p[k]));
      if (s < best) { best = s; kb = k; }
    }
    T sg = val(p[kb]) >= 0 ? T(1) : T(-1);
    V3<T> e{T(0), T(0), T(0)};
    e[kb] = sg;
    out_dir = mv(X.R, e);
    surf = p;
    surf[kb] = sg * T(h[kb]);
    T pen = T(h[kb]) - sg * p[kb];
    out.dist = -pen - r;
  }
  out.n = scl(out_dir, T(-1));
  V3<T> s_box = xform(X, surf), s_sph = add(c, scl(out.n, r));
  out.pos = scl(add(s_box, s_sph), T(0.5));
  return out;
}

// Closest points of the segments c1 + u a1 (|u| <= h1) and c2 + v a2 (|v| <= h2), unit axes:
// u from the unconstrained solution (u = 0 when the axes are parallel, 1 - (a1.a2)^2 <= 1e-10),
// clamped; then v optimal for u, clamped; then u optimal for v, clamped.
template <class T> void segment_segment(const V3<T>& c1, const V3<T>& a1, T h1, const V3<T>& c2, const V3<T>& a2, T h2,
                                        T& u, T& v) {
  V3<T> r = sub(c1, c2);
  T b = dot(a1, a2), c = dot(a1, r), f = dot(a2, r);
  T den = T(1) - b * b;
  auto clamp = [](T x, T lo, T hi) { return val(x) < val(lo) ? lo : (val(x) > val(hi) ? hi : x); };
  if (val(den) > 1e-10) u = clamp((b * f - c) / den, -h1, h1);
  else u = T(0);
  v = clamp(b * u + f, -h2, h2);
  u = clamp(b * v - c, -h1, h1);
}

template <class T> inline V3<T> seg_axis(const Xf<T>& X) { return col(X.R, 2); }

// Closest points of the segments c1 + u a1 (|u| <= h1) and c2 + v a2 (|v| <= h2) by exhaustion of
// the parameter rectangle: the unconstrained stationary point when it lies inside, and the best
// point of each of the rectangle's four sides (one parameter fixed at a bound, the other clamped
// to its own optimum); the candidate of least distance wins (ties to the first listed).
template <class T> void segment_pair_exhaustive(const V3<T>& c1, const V3<T>& a1, double h1, const V3<T>& c2,
                                                const V3<T>& a2, double h2, T& u_out, T& v_out) {
  const V3<T> r = sub(c1, c2);
  const T b = dot(a1, a2), c = dot(a1, r), f = dot(a2, r);
  auto clampd = [](T x, double lo, double hi) { return val(x) < lo ? T(lo) : (val(x) > hi ? T(hi) : x); };
  auto dist2 = [&](const T& u, const T& v) {
    const V3<T> d = sub(add(c1, scl(a1, u)), add(c2, scl(a2, v)));
    return dot(d, d);
  };
  std::vector<std::pair<T, T>> cand;
  const T den = T(1) - b * b;
  if (val(den) > 1e-12) {
    const T u = (b * f - c) / den, v = (f - b * c) / den;
    if (std::fabs(val(u)) <= h1 && std::fabs(val(v)) <= h2) cand.push_back({u, v});
  }
  for (double us : {-h1, h1}) cand.push_back({T(us), clampd(b * T(us) + f, -h2, h2)});
  for (double vs : {-h2, h2}) cand.push_back({clampd(b * T(vs) - c, -h1, h1), T(vs)});
  size_t best = 0;
  for (size_t k = 1; k < cand.size(); k++)
    if (val(dist2(cand[k].first, cand[k].second)) < val(dist2(cand[best].first, cand[best].second))) best = k;
  u_out = cand[best].first;
  v_out = cand[best].second;
}

// Box-box by the separating-axis test over the 15 candidate axes (3 face normals of each box and
// the 9 edge-edge cross products; a cross product shorter than 1e-6 is no axis).  Overlap along a
// unit axis L: sum_k hA_k |L.A_k| + sum_k hB_k |L.B_k| - |L.(cB - cA)|.  If any axis separates,
// every slot stays inactive.  Axis choice (R15): the best face axis of box 1, replaced by box 2's
// best face axis only if that is smaller by more than tol = 1e-5 (1 + overlap), then by the best
// edge axis only if smaller again by more than tol (ties to the lower index throughout).
//   Face case: the box owning the axis is the reference; its face with outward normal nref along
//   the axis (towards the other box) is the reference face; the incident face is the other box's
//   face whose outward normal is most opposed to nref.  The contact polygon is the part of the
//   incident face inside the reference face's prism (the reference face swept along nref).  Its
//   vertices are constructed directly: (a) incident-face corners inside the prism, (b) crossings
//   of the incident face's edges with the prism's side planes that lie inside the prism, (c)
//   the prism's side edges (through the reference face's corners, along nref) piercing the
//   incident face inside it; duplicates merged, then ordered by angle about their centroid in
//   the reference face's plane.  Vertices below the reference face (depth >= 0) are contacts,
//   at the midpoint between the vertex and its projection on the reference face.  More than 4:
//   the deepest, the farthest from it, the one of largest triangle area with those two, then the
//   one farthest outside that triangle (largest sum of the three sub-triangle areas), each with
//   ties to the first in that order; kept in that order.
//   Edge case: the closest points of the two edges (one per box, parallel to the axis's two
//   factors) that are furthest along +n on box 1 and along -n on box 2; one contact.
// The normal points from box 1 to box 2.
template <class T> void box_box(const Xf<T>& XA, const double* hA, const Xf<T>& XB, const double* hB, Contact<T>* out) {
  for (int i = 0; i < 4; i++) { out[i].dist = T(1); out[i].n = V3<T>{T(0), T(0), T(1)}; out[i].pos = XA.p; }
  const V3<T> axA[3] = {col(XA.R, 0), col(XA.R, 1), col(XA.R, 2)};
  const V3<T> axB[3] = {col(XB.R, 0), col(XB.R, 1), col(XB.R, 2)};
  const V3<T> d = sub(XB.p, XA.p);
  auto absv = [](const T& x) { return val(x) < 0 ? -x : x; };
  auto overlap_along = [&](const V3<T>& L) {
    T reach = T(0);
    for (int k = 0; k < 3; k++) reach = reach + T(hA[k]) * absv(dot(L, axA[k])) + T(hB[k]) * absv(dot(L, axB[k]));
    return reach - absv(dot(L, d));
  };
  // candidate axes in the order: box 1 faces, box 2 faces, edge pairs (i of box 1, j of box 2)
  struct Axis { V3<T> L; T ov; bool ok; };
  std::vector<Axis> ax;
  for (int k = 0; k < 3; k++) ax.push_back({axA[k], T(0), true});
  for (int k = 0; k < 3; k++) ax.push_back({axB[k], T(0), true});
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      const V3<T> c = cross(axA[i], axB[j]);
      const T len = norm(c);
      ax.push_back({val(len) > 1e-6 ? scl(c, T(1) / len) : c, T(0), val(len) > 1e-6});
    }
  for (Axis& a : ax) {
    if (!a.ok) continue;
    a.ov = overlap_along(a.L);
    if (val(a.ov) < 0) return;   // a separating axis
  }
  auto least = [&](int lo, int hi) {
    int w = -1;
    for (int k = lo; k < hi; k++)
      if (ax[k].ok && (w < 0 || val(ax[k].ov) < val(ax[w].ov))) w = k;
    return w;
  };
  int pick = least(0, 3);
  const int f2 = least(3, 6), e = least(6, 15);
  if (val(ax[f2].ov) < val(ax[pick].ov) - 1e-5 * (1 + val(ax[pick].ov))) pick = f2;
  if (e >= 0 && val(ax[e].ov) < val(ax[pick].ov) - 1e-5 * (1 + val(ax[pick].ov))) pick = e;
  const T depth = ax[pick].ov;
  const V3<T> n = val(dot(ax[pick].L, d)) < 0 ? scl(ax[pick].L, T(-1)) : ax[pick].L;   // box 1 -> box 2
  if (pick >= 6) {
    const int i = (pick - 6) / 3, j = (pick - 6) % 3;
    // of the 4 edges of a box parallel to an axis, the one whose midpoint is furthest along s
    auto support_edge_mid = [](const Xf<T>& X, const V3<T>* axes, const double* h, int along, const V3<T>& s) {
      V3<T> best_mid = X.p;
      double best_val = -1e300;
      for (int corner = 0; corner < 4; corner++) {
        V3<T> mid = X.p;
        int bit = 0;
        for (int k = 0; k < 3; k++) {
          if (k == along) continue;
          const double sg = ((corner >> bit) & 1) ? 1.0 : -1.0;
          mid = add(mid, scl(axes[k], T(sg * h[k])));
          bit++;
        }
        const double v = val(dot(mid, s));
        if (v > best_val) { best_val = v; best_mid = mid; }
      }
      return best_mid;
    };
    const V3<T> ma = support_edge_mid(XA, axA, hA, i, n), mb = support_edge_mid(XB, axB, hB, j, scl(n, T(-1)));
    T u, v;
    segment_pair_exhaustive(ma, axA[i], hA[i], mb, axB[j], hB[j], u, v);
    out[0].n = n;
    out[0].dist = -depth;
    out[0].pos = scl(add(add(ma, scl(axA[i], u)), add(mb, scl(axB[j], v))), T(0.5));
    return;
  }
  // ---- face case ----
  const bool refA = pick < 3;
  const Xf<T>& XR = refA ? XA : XB;
  const Xf<T>& XI = refA ? XB : XA;
  const double* hR = refA ? hA : hB;
  const double* hI = refA ? hB : hA;
  const int kr = refA ? pick : pick - 3;
  const V3<T> nref = refA ? n : scl(n, T(-1));   // out of the reference face, towards the incident box
  const int r1 = (kr + 1) % 3, r2 = (kr + 2) % 3;
  const V3<T> tu = col(XR.R, r1), tv = col(XR.R, r2);
  // reference-face coordinates of a point: (along tu, along tv) relative to the face centre, and
  // its depth below the face
  auto face_uv = [&](const V3<T>& p) {
    const V3<T> q = sub(p, XR.p);
    return std::array<T, 2>{dot(q, tu), dot(q, tv)};
  };
  auto depth_of = [&](const V3<T>& p) { return T(hR[kr]) - dot(sub(p, XR.p), nref); };
  const double tol = 1e-12 * (1 + std::max(std::max(hR[r1], hR[r2]), std::max(hI[0], std::max(hI[1], hI[2]))));
  auto in_prism = [&](const V3<T>& p) {
    const std::array<T, 2> uv = face_uv(p);
    return std::fabs(val(uv[0])) <= hR[r1] + tol && std::fabs(val(uv[1])) <= hR[r2] + tol;
  };
  // the incident face: outward normal (axis fk, sign fs) most opposed to nref (ties to the lower
  // axis, + before -)
  int fk = 0;
  double fs = 1, most = 2;
  for (int k = 0; k < 3; k++)
    for (double sg : {1.0, -1.0}) {
      const double c = sg * val(dot(col(XI.R, k), nref));
      if (c < most) { most = c; fk = k; fs = sg; }
    }
  const int i1 = (fk + 1) % 3, i2 = (fk + 2) % 3;
  const V3<T> fc = add(XI.p, scl(col(XI.R, fk), T(fs * hI[fk])));      // incident face centre
  const V3<T> iu = col(XI.R, i1), iv = col(XI.R, i2), inrm = scl(col(XI.R, fk), T(fs));
  std::vector<V3<T>> corners;
  for (double a : {-1.0, 1.0})
    for (double b : {-1.0, 1.0}) corners.push_back(add(fc, add(scl(iu, T(a * hI[i1])), scl(iv, T(b * hI[i2])))));
  const int edges[4][2] = {{0, 1}, {1, 3}, {3, 2}, {2, 0}};   // the face's boundary, corner pairs
  std::vector<V3<T>> pts;
  auto add_point = [&](const V3<T>& p) {
    for (const V3<T>& q : pts)
      if (val(norm(sub(p, q))) <= 1e3 * tol) return;
    pts.push_back(p);
  };
  for (const V3<T>& c : corners)                                          // (a)
    if (in_prism(c)) add_point(c);
  for (const auto& ed : edges) {                                          // (b)
    const V3<T> &P = corners[ed[0]], &Q = corners[ed[1]];
    const std::array<T, 2> up = face_uv(P), uq = face_uv(Q);
    for (int coord = 0; coord < 2; coord++)
      for (double side : {-1.0, 1.0}) {
        const double lim = side * (coord == 0 ? hR[r1] : hR[r2]);
        const T a = up[coord] - T(lim), b = uq[coord] - T(lim);
        if ((val(a) < 0) == (val(b) < 0) || val(a) == val(b)) continue;   // no crossing
        const T t = a / (a - b);
        const V3<T> X = add(P, scl(sub(Q, P), t));
        if (in_prism(X)) add_point(X);
      }
  }
  const T den = dot(nref, inrm);
  if (std::fabs(val(den)) > 1e-12)                                        // (c)
    for (double a : {-1.0, 1.0})
      for (double b : {-1.0, 1.0}) {
        const V3<T> base = add(XR.p, add(scl(tu, T(a * hR[r1])), scl(tv, T(b * hR[r2]))));
        const T s = dot(sub(fc, base), inrm) / den;                    // base + s nref on the face plane
        const V3<T> X = add(base, scl(nref, s));
        const V3<T> q = sub(X, fc);
        if (std::fabs(val(dot(q, iu))) <= hI[i1] + tol && std::fabs(val(dot(q, iv))) <= hI[i2] + tol) add_point(X);
      }
  if (pts.empty()) return;
  // angular order about the centroid, in the reference face's (tu, tv) plane
  V3<T> cen{T(0), T(0), T(0)};
  for (const V3<T>& p : pts) cen = add(cen, p);
  cen = scl(cen, T(1.0 / pts.size()));
  std::vector<std::pair<double, int>> ang;
  for (size_t k = 0; k < pts.size(); k++) {
    const V3<T> q = sub(pts[k], cen);
    ang.push_back({std::atan2(val(dot(q, tv)), val(dot(q, tu))), (int)k});
  }
  std::sort(ang.begin(), ang.end());
  std::vector<V3<T>> poly;
  std::vector<T> dep;
  for (const auto& a : ang) {
    const T dd = depth_of(pts[a.second]);
    if (val(dd) >= 0) { poly.push_back(pts[a.second]); dep.push_back(dd); }
  }
  std::vector<int> keep;
  for (size_t k = 0; k < poly.size(); k++) keep.push_back((int)k);
  if (poly.size() > 4) {
    auto area2 = [&](int a, int b, int c) { return val(norm(cross(sub(poly[b], poly[a]), sub(poly[c], poly[a])))); };
    auto argmax = [&](auto score, const std::vector<int>& taken) {
      int w = -1;
      double bv = -1;
      for (int k = 0; k < (int)poly.size(); k++) {
        if (std::find(taken.begin(), taken.end(), k) != taken.end()) continue;
        const double v = score(k);
        if (w < 0 || v > bv) { bv = v; w = k; }
      }
      return w;
    };
    std::vector<int> sel;
    sel.push_back(argmax([&](int k) { return val(dep[k]); }, sel));
    sel.push_back(argmax([&](int k) { return val(norm(sub(poly[k], poly[sel[0]]))); }, sel));
    sel.push_back(argmax([&](int k) { return area2(sel[0], sel[1], k); }, sel));
    sel.push_back(argmax([&](int k) { return area2(sel[0], sel[1], k) + area2(sel[1], sel[2], k) + area2(sel[2], sel[0], k); },
                         sel));
    keep = sel;
  }
  for (size_t c = 0; c < keep.size(); c++) {
    const int k = keep[c];
    out[c].n = n;
    out[c].dist = -dep[k];
    out[c].pos = add(poly[k], scl(nref, dep[k] * T(0.5)));
  }
}

// ---- heightfield ------------------------------------------------------------------
// The surface is the grid's triangulation: cell (i, j) (i < nrow - 1, j < ncol - 1) with corners
// v00 = (i, j), v01 = (i, j + 1), v10 = (i + 1, j), v11 = (i + 1, j + 1) is split along its
// v00-v11 diagonal into (v00, v01, v11) and (v00, v11, v10).

template <class T> V3<T> hf_vertex(const HField& hf, const double* size, int i, int j) {
  const double dx = 2 * size[0] / (hf.ncol - 1), dy = 2 * size[1] / (hf.nrow - 1);
  return V3<T>{T(-size[0] + j * dx), T(-size[1] + i * dy), T(size[2] * hf.e[(size_t)i * hf.ncol + j])};
}

template <class T> void hf_triangle(const HField& hf, const double* size, int i, int j, int t, V3<T> v[3]) {
  v[0] = hf_vertex<T>(hf, size, i, j);
  v[1] = t == 0 ? hf_vertex<T>(hf, size, i, j + 1) : hf_vertex<T>(hf, size, i + 1, j + 1);
  v[2] = t == 0 ? hf_vertex<T>(hf, size, i + 1, j + 1) : hf_vertex<T>(hf, size, i + 1, j);
}

// closest point to p on the triangle v: the projection onto its plane when that falls inside
// (all barycentric weights >= 0), else the nearest of the three edges' clamped projections
template <class T> V3<T> closest_on_triangle(const V3<T>& p, const V3<T> v[3]) {
  V3<T> n = cross(sub(v[1], v[0]), sub(v[2], v[0]));
  T nn = dot(n, n);
  V3<T> q = sub(p, scl(n, dot(n, sub(p, v[0])) / nn));
  T w0 = dot(cross(sub(v[2], v[1]), sub(q, v[1])), n) / nn;
  T w1 = dot(cross(sub(v[0], v[2]), sub(q, v[2])), n) / nn;
  if (val(w0) >= 0 && val(w1) >= 0 && val(w0) + val(w1) <= 1) return q;
  V3<T> best{};
  double bd = 1e300;
  for (int k = 0; k < 3; k++) {
    const V3<T>& a = v[k];
    const V3<T>& b = v[(k + 1) % 3];
    V3<T> ab = sub(b, a);
    T t = dot(sub(p, a), ab) / dot(ab, ab);
    if (val(t) < 0) t = T(0);
    if (val(t) > 1) t = T(1);
    V3<T> c = add(a, scl(ab, t));
    double d = val(dot(sub(p, c), sub(p, c)));
    if (d < bd) { bd = d; best = c; }
  }
  return best;
}

// Heightfield (geom1: frame X, size (hx, hy, hz), grid hf) against a sphere (c, r).
//   * Centre outside the grid's xy footprint: no contact (dist = 1e30).
//   * Centre on or below the triangle under it (signed distance s <= 0 to that triangle's plane,
//     normal pointing up): dist = s - r along that normal.
//   * Otherwise: the closest point q over the triangles of the cells that meet the square of
//     half-width r around the centre (ties to the first in cell row, column, triangle order);
//     normal (c - q) / |c - q|, dist = |c - q| - r.
// The contact point is midway between the sphere's deepest point and the surface point.
template <class T> Contact<T> hfield_sphere(const Xf<T>& X, const double* size, const HField& hf, const V3<T>& cw, T r) {
  Contact<T> out;
  V3<T> c = mtv(X.R, sub(cw, X.p));
  const double hx = size[0], hy = size[1];
  const double dx = 2 * hx / (hf.ncol - 1), dy = 2 * hy / (hf.nrow - 1);
  if (val(c[0]) < -hx || val(c[0]) > hx || val(c[1]) < -hy || val(c[1]) > hy) {
    out.dist = T(1e30);
    out.n = col(X.R, 2);
    out.pos = cw;
    return out;
  }
  auto cell = [](double u, double d, int n) { int k = (int)std::floor(u / d); return k < 0 ? 0 : (k > n - 2 ? n - 2 : k); };
  const int i = cell(val(c[1]) + hy, dy, hf.nrow), j = cell(val(c[0]) + hx, dx, hf.ncol);
  const double fu = (val(c[0]) + hx) / dx - j, fv = (val(c[1]) + hy) / dy - i;
  V3<T> tri[3];
  hf_triangle(hf, size, i, j, fu >= fv ? 0 : 1, tri);
  V3<T> nt = cross(sub(tri[1], tri[0]), sub(tri[2], tri[0]));
  nt = scl(nt, T(1) / norm(nt));
  T sd = dot(nt, sub(c, tri[0]));
  V3<T> nl;
  T d;
  if (val(sd) <= 0) {
    nl = nt;
    d = sd;
  } else {
    const double rr = val(r);
    const int i0 = cell(val(c[1]) - rr + hy, dy, hf.nrow), i1 = cell(val(c[1]) + rr + hy, dy, hf.nrow);
    const int j0 = cell(val(c[0]) - rr + hx, dx, hf.ncol), j1 = cell(val(c[0]) + rr + hx, dx, hf.ncol);
    double best = 1e300;
    V3<T> q{};
    for (int a = i0; a <= i1; a++)
      for (int b = j0; b <= j1; b++)
        for (int t = 0; t < 2; t++) {
          hf_triangle(hf, size, a, b, t, tri);
          V3<T> p = closest_on_triangle(c, tri);
          double dd = val(dot(sub(c, p), sub(c, p)));
          if (dd < best) { best = dd; q = p; }
        }
    V3<T> e = sub(c, q);
    d = norm(e);
    nl = scl(e, T(1) / d);
  }
  out.n = mv(X.R, nl);
  out.dist = d - r;
  out.pos = sub(cw, scl(out.n, r + out.dist * T(0.5)));
  return out;
}

// Cylinder (frame X, radius r, half-length hl along its z axis a) against a plane (point p0,
// unit normal n).  The deepest point of a cylinder over a plane lies on a rim circle, on the
// radius along which the rim falls fastest: e = -(n - (n.a) a) / |n - (n.a) a|.  When the axis
// lies within 1e-4 of the normal every rim point is equally deep and e is the cylinder's own x
// axis.  The lower cap is the one at -hl when n.a >= 0, else the one at +hl; with b = a x e the
// four candidate points are
//   0: lower cap + r e   (the deepest point)        1: upper cap + r e
//   2: lower cap + r (-e/2 + (sqrt 3)/2 b)        3: lower cap + r (-e/2 - (sqrt 3)/2 b)
// so that a cylinder standing on a cap rests on a tripod of rim points 120 degrees apart and one
// lying on its side on the two rims' lowest points.  Each has normal n, distance n.(p - p0) and
// its contact point midway between p and the plane.
template <class T> void plane_cylinder(const V3<T>& p0, const V3<T>& n, const Xf<T>& X, T r, T hl, Contact<T>* out) {
  const V3<T> a = col(X.R, 2);
  const T s = dot(n, a);
  V3<T> perp = sub(n, scl(a, s));
  const T pl = norm(perp);
  V3<T> e = val(pl) < 1e-4 ? col(X.R, 0) : scl(perp, T(-1) / pl);
  const V3<T> b = cross(a, e);
  const T sg = val(s) >= 0 ? T(-1) : T(1);
  const V3<T> clo = add(X.p, scl(a, sg * hl)), chi = sub(X.p, scl(a, sg * hl));
  const T c3 = T(std::sqrt(3.0) / 2);
  V3<T> p[4] = {add(clo, scl(e, r)), add(chi, scl(e, r)), add(clo, scl(add(scl(e, T(-0.5)), scl(b, c3)), r)),
                add(clo, scl(sub(scl(e, T(-0.5)), scl(b, c3)), r))};
  for (int k = 0; k < 4; k++) {
    out[k].n = n;
    out[k].dist = dot(n, sub(p[k], p0));
    out[k].pos = sub(p[k], scl(n, out[k].dist * T(0.5)));
  }
}

// ---- convex solids (boxes and meshes) --------------------------------------------
// A box of half sizes h as a Solid: corner i at (+-h0, +-h1, +-h2), + on axis k when bit k of i is
// set; faces -x, +x, -y, +y, -z, +z.
inline Solid box_solid(const double* h) {
  Solid sd;
  for (int i = 0; i < 8; i++)
    for (int k = 0; k < 3; k++) sd.vert.push_back(((i >> k) & 1) ? h[k] : -h[k]);
  for (int f = 0; f < 6; f++) {
    double pl[4] = {0, 0, 0, h[f / 2]};
    pl[f / 2] = (f % 2) ? 1.0 : -1.0;
    sd.plane.insert(sd.plane.end(), pl, pl + 4);
  }
  return sd;
}

template <class T> struct Candidate {
  Contact<T> c;
  int order;
};

// the 4 deepest candidates (ties: the earlier in the list), written to out in list order
template <class T> void keep_deepest4(std::vector<Candidate<T>> cand, Contact<T>* out) {
  std::stable_sort(cand.begin(), cand.end(), [](const Candidate<T>& a, const Candidate<T>& b) {
    return val(a.c.dist) < val(b.c.dist);
  });
  if (cand.size() > 4) cand.resize(4);
  std::sort(cand.begin(), cand.end(), [](const Candidate<T>& a, const Candidate<T>& b) { return a.order < b.order; });
  for (size_t i = 0; i < cand.size(); i++) out[i] = cand[i].c;
}

// Plane (point p0, unit normal n) against a convex solid in frame X: each vertex at its distance
// n.(v - p0); the 4 deepest (ties: lower vertex index) in vertex order, each midway between the
// vertex and the plane.
template <class T> void plane_solid(const V3<T>& p0, const V3<T>& n, const Xf<T>& X, const Solid& sd, Contact<T>* out) {
  std::vector<Candidate<T>> cand;
  for (int i = 0; i < sd.nv(); i++) {
    V3<T> w = xform(X, V3<T>{T(sd.vert[3 * i]), T(sd.vert[3 * i + 1]), T(sd.vert[3 * i + 2])});
    Candidate<T> k;
    k.c.n = n;
    k.c.dist = dot(n, sub(w, p0));
    k.c.pos = sub(w, scl(n, k.c.dist * T(0.5)));
    k.order = i;
    cand.push_back(k);
  }
  keep_deepest4(cand, out);
}

// The triangle of the grid under the grid-frame point (x, y) inside the footprint: its cell by
// floor (clamped to the last cell), then triangle 0 when the point's offset in the cell has
// fu >= fv, else triangle 1; returned as its upward unit normal and its first vertex.
template <class T> void hf_under(const HField& hf, const double* size, double x, double y, V3<T>& nt, V3<T>& v0) {
  const double hx = size[0], hy = size[1];
  const double dx = 2 * hx / (hf.ncol - 1), dy = 2 * hy / (hf.nrow - 1);
  auto cell = [](double u, double d, int n) { int k = (int)std::floor(u / d); return k < 0 ? 0 : (k > n - 2 ? n - 2 : k); };
  const int i = cell(y + hy, dy, hf.nrow), j = cell(x + hx, dx, hf.ncol);
  const double fu = (x + hx) / dx - j, fv = (y + hy) / dy - i;
  V3<T> tri[3];
  hf_triangle(hf, size, i, j, fu >= fv ? 0 : 1, tri);
  nt = cross(sub(tri[1], tri[0]), sub(tri[2], tri[0]));
  nt = scl(nt, T(1) / norm(nt));
  v0 = tri[0];
}

// Heightfield (geom1: frame X1, size, grid hf) against a convex solid (frame X2).  Candidates:
//   first every vertex over the grid's footprint, at its signed distance to the plane of the
//   triangle under it, along that triangle's upward normal;
//   then every grid vertex (row-major) strictly inside the solid, at the depth of its nearest
//   face (the largest of its negative distances to the face planes; ties: lower face index),
//   normal minus that face's outward normal.
// The 4 deepest (ties: candidate order) in candidate order, each midway between the surfaces.
template <class T> void hfield_solid(const Xf<T>& X1, const double* size, const HField& hf, const Xf<T>& X2,
                                     const Solid& sd, Contact<T>* out) {
  std::vector<Candidate<T>> cand;
  for (int i = 0; i < sd.nv(); i++) {
    V3<T> w = xform(X2, V3<T>{T(sd.vert[3 * i]), T(sd.vert[3 * i + 1]), T(sd.vert[3 * i + 2])});
    V3<T> p = mtv(X1.R, sub(w, X1.p));
    if (val(p[0]) < -size[0] || val(p[0]) > size[0] || val(p[1]) < -size[1] || val(p[1]) > size[1]) continue;
    V3<T> nt, v0;
    hf_under(hf, size, val(p[0]), val(p[1]), nt, v0);
    Candidate<T> k;
    k.c.dist = dot(nt, sub(p, v0));
    k.c.n = mv(X1.R, nt);
    k.c.pos = add(X1.p, mv(X1.R, sub(p, scl(nt, k.c.dist * T(0.5)))));
    k.order = i;
    cand.push_back(k);
  }
  for (int a = 0; a < hf.nrow; a++)
    for (int b = 0; b < hf.ncol; b++) {
      V3<T> q = add(X1.p, mv(X1.R, hf_vertex<T>(hf, size, a, b)));
      V3<T> ql = mtv(X2.R, sub(q, X2.p));
      int best = -1;
      T bd = T(0);
      for (int f = 0; f < sd.nf(); f++) {
        T s = T(sd.plane[4 * f]) * ql[0] + T(sd.plane[4 * f + 1]) * ql[1] + T(sd.plane[4 * f + 2]) * ql[2] -
              T(sd.plane[4 * f + 3]);
        if (best < 0 || val(s) > val(bd)) { best = f; bd = s; }
      }
      if (!(val(bd) < 0)) continue;
      V3<T> nf = mv(X2.R, V3<T>{T(sd.plane[4 * best]), T(sd.plane[4 * best + 1]), T(sd.plane[4 * best + 2])});
      Candidate<T> k;
      k.c.dist = bd;
      k.c.n = scl(nf, T(-1));
      k.c.pos = sub(q, scl(nf, bd * T(0.5)));
      k.order = sd.nv() + a * hf.ncol + b;
      cand.push_back(k);
    }
  keep_deepest4(cand, out);
}

// All candidate contacts of one pair, written to out[0 .. pair_max_points); slots without a
// candidate keep dist = 1 (inactive).  mesh2: geom2's solid when it is a mesh.
template <class T> void collide_pair(int t1, const Xf<T>& X1, const double* s1, int t2, const Xf<T>& X2, const double* s2,
                                     Contact<T>* out, const HField& hf = HField(), const Solid* mesh2 = nullptr) {
  if ((t1 == HFIELD && (t2 == BOX || t2 == MESH)) || (t1 == PLANE && t2 == MESH))   // 4 slots, maybe not all filled
    for (int i = 0; i < 4; i++) { out[i].dist = T(1); out[i].n = V3<T>{T(0), T(0), T(1)}; out[i].pos = X1.p; }
  if (t1 == HFIELD && (t2 == BOX || t2 == MESH)) {
    hfield_solid(X1, s1, hf, X2, t2 == BOX ? box_solid(s2) : *mesh2, out);
  } else if (t1 == PLANE && t2 == MESH) {
    plane_solid(X1.p, col(X1.R, 2), X2, *mesh2, out);
  } else if (t1 == HFIELD) {
    // a sphere; a capsule meets the terrain at its two end spheres
    if (t2 == SPHERE) {
      out[0] = hfield_sphere(X1, s1, hf, X2.p, T(s2[0]));
    } else if (t2 == CAPSULE) {
      V3<T> a = seg_axis(X2);
      for (int e = 0; e < 2; e++) {
        T sgn = e == 0 ? T(-1) : T(1);
        out[e] = hfield_sphere(X1, s1, hf, add(X2.p, scl(a, sgn * T(s2[1]))), T(s2[0]));
      }
    }
  } else if (t1 == PLANE) {
    V3<T> nz = col(X1.R, 2), p0 = X1.p;
    if (t2 == SPHERE) {
      out[0] = plane_sphere(p0, nz, X2.p, T(s2[0]));
    } else if (t2 == CAPSULE) {
      V3<T> a = seg_axis(X2);
      for (int e = 0; e < 2; e++) {
        T sgn = e == 0 ? T(-1) : T(1);
        out[e] = plane_sphere(p0, nz, add(X2.p, scl(a, sgn * T(s2[1]))), T(s2[0]));
      }
    } else if (t2 == BOX) {
      // the 4 deepest of the 8 corners (ties to the lower corner index), kept in corner order
      T d[8];
      V3<T> cp[8];
      for (int v = 0; v < 8; v++) {
        V3<T> l{T((v & 1) ? s2[0] : -s2[0]), T((v & 2) ? s2[1] : -s2[1]), T((v & 4) ? s2[2] : -s2[2])};
        cp[v] = xform(X2, l);
        d[v] = dot(nz, sub(cp[v], p0));
      }
      int order[8] = {0, 1, 2, 3, 4, 5, 6, 7};
      std::stable_sort(order, order + 8, [&](int a, int b) { return val(d[a]) < val(d[b]); });
      int keep[4] = {order[0], order[1], order[2], order[3]};
      std::sort(keep, keep + 4);
      for (int i = 0; i < 4; i++) {
        int v = keep[i];
        out[i].n = nz;
        out[i].dist = d[v];
        out[i].pos = sub(cp[v], scl(nz, d[v] * T(0.5)));
      }
    } else if (t2 == CYLINDER) {
      plane_cylinder(p0, nz, X2, T(s2[0]), T(s2[1]), out);
    }
  } else if (t1 == SPHERE) {
    if (t2 == SPHERE) {
      out[0] = sphere_sphere(X1.p, T(s1[0]), X2.p, T(s2[0]));
    } else if (t2 == CAPSULE) {
      V3<T> a = seg_axis(X2);
      T t = dot(sub(X1.p, X2.p), a);
      T h = T(s2[1]);
      if (val(t) > val(h)) t = h;
      if (val(t) < -val(h)) t = -h;
      out[0] = sphere_sphere(X1.p, T(s1[0]), add(X2.p, scl(a, t)), T(s2[0]));
    } else if (t2 == BOX) {
      out[0] = sphere_box(X1.p, T(s1[0]), X2, s2);
    }
  } else if (t1 == CAPSULE) {
    if (t2 == CAPSULE) {
      V3<T> a1 = seg_axis(X1), a2 = seg_axis(X2);
      T u, v;
      segment_segment(X1.p, a1, T(s1[1]), X2.p, a2, T(s2[1]), u, v);
      out[0] = sphere_sphere(add(X1.p, scl(a1, u)), T(s1[0]), add(X2.p, scl(a2, v)), T(s2[0]));
    } else if (t2 == BOX) {
      V3<T> a = seg_axis(X1);
      for (int e = 0; e < 2; e++) {
        T sgn = e == 0 ? T(-1) : T(1);
        out[e] = sphere_box(add(X1.p, scl(a, sgn * T(s1[1]))), T(s1[0]), X2, s2);
      }
    }
  } else if (t1 == BOX && t2 == BOX) {
    box_box(X1, s1, X2, s2, out);
  }
  for (int i = 0; i < pair_max_points(t1, t2); i++) contact_frame(out[i]);
}

// ------------------------------------------------------------------------------------
// constraint rows
// ------------------------------------------------------------------------------------
template <class T> struct Rows {
  int n = 0;
  std::vector<T> J;                          // n x nv
  std::vector<T> r, v, aref, D, Ahat, imp;   // per row
  std::vector<int> slot;                     // contact slot (or -1 - joint for a limit)
  // row kind: 0 one-sided scalar row (pyramid edge, frictionless normal, joint limit);
  // 1 normal row of an elliptic contact, followed by its 2 tangent rows (kind 2);
  // 3 joint friction-loss row (two-sided, its force bounded by mu)
  std::vector<int> kind;
  std::vector<double> mu;                    // friction of an elliptic contact's rows; a friction-loss row's bound
};

// Friction-loss row with residual x = J a - aref, regulariser R = 1 / D and force bound F: the
// soft cost is the Huber function of x that keeps the row's force -s'(x) inside [-F, F]:
//   |x| <= R F   s = D x^2 / 2           (zone 1)
//   x > R F      s = F x - R F^2 / 2     (zone 2)
//   x < -R F     s = -F x - R F^2 / 2    (zone 0)
template <class T> int fric_zone(const T& x, const T& D, double F) {
  const double rf = F / val(D);
  return val(x) > rf ? 2 : (val(x) < -rf ? 0 : 1);
}
template <class T> T fric_cost(const T& x, const T& D, double F) {
  const int z = fric_zone(x, D, F);
  if (z == 1) return T(0.5) * D * x * x;
  return (z == 2 ? T(F) * x : -T(F) * x) - T(0.5 * F * F) / D;
}

// Soft cost of an elliptic contact with residual x = (x_n, x_1, x_2) = J a - aref: half D times
// the squared distance from x to the dual cone K* = {x_n >= mu |x_t|}.  With t = |x_t|:
//   x_n >= mu t                (inside K*)          s = 0
//   mu x_n + t <= 0            (inside -K, polar)   s = D |x|^2 / 2
//   otherwise                  (projection on the boundary)  s = D (x_n - mu t)^2 / (2 (1 + mu^2))
// zone: 0 / 2 / 1 respectively.  Gradient and Hessian of s in the same zones.
template <class T> int cone_zone(const T* x, double mu) {
  double t = std::sqrt(val(x[1]) * val(x[1]) + val(x[2]) * val(x[2]));
  if (val(x[0]) >= mu * t) return 0;
  if (mu * val(x[0]) + t <= 0) return 2;
  return 1;
}
template <class T> T cone_cost(const T* x, const T& D, double mu) {
  int z = cone_zone(x, mu);
  if (z == 0) return T(0);
  if (z == 2) return T(0.5) * D * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  T t = sqrt(x[1] * x[1] + x[2] * x[2]);
  T ph = x[0] - T(mu) * t;
  return T(0.5) * D * ph * ph / T(1 + mu * mu);
}
template <class T> void cone_grad_hess(const T* x, const T& D, double mu, T* g, T* H) {
  for (int i = 0; i < 3; i++) { g[i] = T(0); for (int j = 0; j < 3; j++) H[3 * i + j] = T(0); }
  int z = cone_zone(x, mu);
  if (z == 0) return;
  if (z == 2) {
    for (int i = 0; i < 3; i++) { g[i] = D * x[i]; H[4 * i] = D; }
    return;
  }
  T t = sqrt(x[1] * x[1] + x[2] * x[2]);
  T u[2] = {x[1] / t, x[2] / t};
  T ph = x[0] - T(mu) * t, k = D / T(1 + mu * mu);
  T dphi[3] = {T(1), -T(mu) * u[0], -T(mu) * u[1]};
  for (int i = 0; i < 3; i++) {
    g[i] = k * ph * dphi[i];
    for (int j = 0; j < 3; j++) H[3 * i + j] = k * dphi[i] * dphi[j];
  }
  // phi times the Hessian of phi: -mu (I - u u^T) / t on the tangent block
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) H[3 * (i + 1) + (j + 1)] = H[3 * (i + 1) + (j + 1)] - k * ph * T(mu) * (T(i == j ? 1 : 0) - u[i] * u[j]) / t;
}

// Impedance d(r) from solimp = (d0, dwidth, width, mid, power): x = min(|r| / width, 1),
// y = x^p / mid^(p-1) for x <= mid, else 1 - (1-x)^p / (1-mid)^(p-1); d = d0 + y (dwidth - d0).
template <class T> T impedance(const T& r, const double* solimp) {
  using std::pow;
  double d0 = solimp[0], d1 = solimp[1], width = solimp[2], mid = solimp[3], p = solimp[4];
  T x = (val(r) < 0 ? -r : r) / T(width);
  if (val(x) >= 1.0) return T(d1);
  T y;
  if (val(x) <= mid) y = pow(x, p) / std::pow(mid, p - 1);
  else y = T(1) - pow(T(1) - x, p) / std::pow(1 - mid, p - 1);
  return T(d0) + y * T(d1 - d0);
}

// ------------------------------------------------------------------------------------
// the convex soft-constraint problem and its Newton solver
// ------------------------------------------------------------------------------------
// f(a) = 1/2 (a - a0)^T M (a - a0) + sum_i 1/2 D_i min(0, J_i a - aref_i)^2
template <class T> T cost(int nv, const std::vector<T>& M, const std::vector<T>& a0, const Rows<T>& R,
                          const std::vector<T>& a) {
  T f = T(0);
  std::vector<T> t(nv);
  for (int j = 0; j < nv; j++) t[j] = a[j] - a0[j];
  for (int i = 0; i < nv; i++) {
    T s = T(0);
    for (int j = 0; j < nv; j++) s = s + M[i * nv + j] * t[j];
    f = f + T(0.5) * t[i] * s;
  }
  for (int i = 0; i < R.n; i++) {
    if (R.kind[i] == 2) continue;
    if (R.kind[i] == 1) {
      T x[3];
      for (int e = 0; e < 3; e++) {
        x[e] = -R.aref[i + e];
        for (int j = 0; j < nv; j++) x[e] = x[e] + R.J[(i + e) * nv + j] * a[j];
      }
      f = f + cone_cost(x, R.D[i], R.mu[i]);
      continue;
    }
    T jar = -R.aref[i];
    for (int j = 0; j < nv; j++) jar = jar + R.J[i * nv + j] * a[j];
    if (R.kind[i] == 3) f = f + fric_cost(jar, R.D[i], R.mu[i]);
    else if (val(jar) < 0) f = f + T(0.5) * R.D[i] * jar * jar;
  }
  return f;
}

// Minimiser over alpha >= 0 of the convex phi(alpha) = f(a + alpha p) when elliptic contacts make
// it non-quadratic: bracket the root of phi' (phi'(0) < 0; double alpha from 1 until phi' >= 0),
// then safeguarded Newton steps on phi' (a bisection whenever the Newton point leaves the
// bracket), until the bracket or |phi'| is at rounding level.
template <class T> T smooth_line_search(int nv, const std::vector<T>& M, const std::vector<T>& a0, const Rows<T>& R,
                                        const std::vector<T>& a, const std::vector<T>& p) {
  std::vector<T> jar(R.n), Jp(R.n);
  for (int i = 0; i < R.n; i++) {
    T s = -R.aref[i], t = T(0);
    for (int j = 0; j < nv; j++) {
      s = s + R.J[i * nv + j] * a[j];
      t = t + R.J[i * nv + j] * p[j];
    }
    jar[i] = s;
    Jp[i] = t;
  }
  T quad = T(0), lin = T(0);
  for (int i = 0; i < nv; i++) {
    T Mp = T(0), Md = T(0);
    for (int j = 0; j < nv; j++) {
      Mp = Mp + M[i * nv + j] * p[j];
      Md = Md + M[i * nv + j] * (a[j] - a0[j]);
    }
    quad = quad + p[i] * Mp;
    lin = lin + p[i] * Md;
  }
  // phi'(alpha) and phi''(alpha)
  auto deriv = [&](const T& al, T& d2) {
    T d1 = lin + al * quad;
    d2 = quad;
    for (int i = 0; i < R.n; i++) {
      if (R.kind[i] == 2) continue;
      if (R.kind[i] == 1) {
        T x[3], y[3], g[3], H[9];
        for (int e = 0; e < 3; e++) { x[e] = jar[i + e] + al * Jp[i + e]; y[e] = Jp[i + e]; }
        cone_grad_hess(x, R.D[i], R.mu[i], g, H);
        for (int e = 0; e < 3; e++) {
          d1 = d1 + g[e] * y[e];
          for (int f = 0; f < 3; f++) d2 = d2 + y[e] * H[3 * e + f] * y[f];
        }
        continue;
      }
      T x = jar[i] + al * Jp[i];
      if (R.kind[i] == 3) {   // friction loss: D x inside the band |x| <= F / D, the bound +-F beyond
        const int z = fric_zone(x, R.D[i], R.mu[i]);
        if (z == 1) { d1 = d1 + R.D[i] * x * Jp[i]; d2 = d2 + R.D[i] * Jp[i] * Jp[i]; }
        else d1 = d1 + (z == 2 ? T(R.mu[i]) : -T(R.mu[i])) * Jp[i];
        continue;
      }
      if (val(x) < 0) { d1 = d1 + R.D[i] * x * Jp[i]; d2 = d2 + R.D[i] * Jp[i] * Jp[i]; }
    }
    return d1;
  };
  T d2;
  T g0 = deriv(T(0), d2);
  if (!(val(g0) < 0)) return T(0);
  T lo = T(0), hi = T(1);
  for (int k = 0; k < 200 && val(deriv(hi, d2)) < 0; k++) { lo = hi; hi = hi * T(2); }
  T al = lo;
  T glo = deriv(lo, d2);
  for (int it = 0; it < 200; it++) {
    T cand = al - glo / d2;
    if (!(val(cand) > val(lo) && val(cand) < val(hi))) cand = T(0.5) * (lo + hi);
    T d2c;
    T gc = deriv(cand, d2c);
    if (val(gc) < 0) { lo = cand; al = cand; glo = gc; d2 = d2c; }
    else { hi = cand; al = cand; glo = gc; d2 = d2c; }
    if (val(hi) - val(lo) <= 1e-15 * val(hi) || std::fabs(val(gc)) <= 1e-14 * std::fabs(val(g0))) break;
  }
  return al;
}

template <class T> struct SolveResult {
  std::vector<T> qacc, force;
  int iterations = 0;
  bool converged = false;
  bool warm_used = false;
};

// Exact minimiser over alpha of f(a + alpha p) (piecewise quadratic, convex): sort the
// breakpoints alpha_i = -jar_i / Jp_i > 0 (ties by row index) and walk the segments until the
// derivative phi'(alpha) = alpha (p^T M p + sum_act D Jp^2) + (p^T M (a-a0) + sum_act D Jp jar)
// changes sign.
template <class T> T exact_line_search(int nv, const std::vector<T>& M, const std::vector<T>& a0, const Rows<T>& R,
                                       const std::vector<T>& a, const std::vector<T>& p) {
  std::vector<T> jar(R.n), Jp(R.n);
  for (int i = 0; i < R.n; i++) {
    T s = -R.aref[i], t = T(0);
    for (int j = 0; j < nv; j++) {
      s = s + R.J[i * nv + j] * a[j];
      t = t + R.J[i * nv + j] * p[j];
    }
    jar[i] = s;
    Jp[i] = t;
  }
  T quad = T(0), lin = T(0);
  for (int i = 0; i < nv; i++) {
    T Mp = T(0), Md = T(0);
    for (int j = 0; j < nv; j++) {
      Mp = Mp + M[i * nv + j] * p[j];
      Md = Md + M[i * nv + j] * (a[j] - a0[j]);
    }
    quad = quad + p[i] * Mp;
    lin = lin + p[i] * Md;
  }
  // phi'(alpha) = lin + quad alpha between breakpoints.  A one-sided row is quadratic while
  // jar + alpha Jp < 0 (one breakpoint); a friction-loss row is quadratic inside its band
  // |x| <= R F and linear outside it (two breakpoints), contributing +-F Jp there.
  std::vector<char> act(R.n, 0);
  struct Event { double alpha; int row; double x; };   // x: the residual value at the crossing
  std::vector<Event> ev;
  for (int i = 0; i < R.n; i++) {
    const double x0 = val(jar[i]), jp = val(Jp[i]);
    if (R.kind[i] == 3) {
      const double rf = R.mu[i] / val(R.D[i]);
      // zone just after alpha = 0
      int z = x0 > rf ? 2 : (x0 < -rf ? 0 : 1);
      if (x0 == rf && jp > 0) z = 2;
      if (x0 == -rf && jp < 0) z = 0;
      act[i] = (char)z;
      if (z == 1) { quad = quad + R.D[i] * Jp[i] * Jp[i]; lin = lin + R.D[i] * Jp[i] * jar[i]; }
      else lin = lin + (z == 2 ? T(R.mu[i]) : -T(R.mu[i])) * Jp[i];
      for (double edge : {-rf, rf})
        if (jp != 0 && (edge - x0) / jp > 0) ev.push_back({(edge - x0) / jp, i, edge});
      continue;
    }
    bool on = x0 < 0 || (x0 == 0 && jp < 0);
    act[i] = on;
    if (on) { quad = quad + R.D[i] * Jp[i] * Jp[i]; lin = lin + R.D[i] * Jp[i] * jar[i]; }
    if (jp != 0 && -x0 / jp > 0) ev.push_back({-x0 / jp, i, 0.0});
  }
  std::stable_sort(ev.begin(), ev.end(), [](const Event& x, const Event& y) { return x.alpha < y.alpha; });
  for (size_t k = 0; k <= ev.size(); k++) {
    T root = -lin / quad;
    if (k == ev.size() || val(root) <= ev[k].alpha) return root;
    const int i = ev[k].row;
    if (R.kind[i] == 3) {   // leave the current zone, enter the one the motion leads to
      const double jp = val(Jp[i]);
      const int z = act[i];
      const int zn = z == 1 ? (jp > 0 ? 2 : 0) : 1;
      if (z == 1) { quad = quad - R.D[i] * Jp[i] * Jp[i]; lin = lin - R.D[i] * Jp[i] * jar[i]; }
      else lin = lin - (z == 2 ? T(R.mu[i]) : -T(R.mu[i])) * Jp[i];
      if (zn == 1) { quad = quad + R.D[i] * Jp[i] * Jp[i]; lin = lin + R.D[i] * Jp[i] * jar[i]; }
      else lin = lin + (zn == 2 ? T(R.mu[i]) : -T(R.mu[i])) * Jp[i];
      act[i] = (char)zn;
      continue;
    }
    // crossing this breakpoint toggles row i
    if (act[i]) { quad = quad - R.D[i] * Jp[i] * Jp[i]; lin = lin - R.D[i] * Jp[i] * jar[i]; act[i] = 0; }
    else { quad = quad + R.D[i] * Jp[i] * Jp[i]; lin = lin + R.D[i] * Jp[i] * jar[i]; act[i] = 1; }
  }
  return -lin / quad;
}

// Newton's method on f: g = M(a - a0) + J_A^T D_A (J_A a - aref_A), H = M + J_A^T D_A J_A,
// p = -H^-1 g (dense Cholesky), exact line search, a += alpha p.  It stops at the iteration cap
// or as soon as the active set after the step equals the one used to build H (then the step
// was exact and a is the minimiser).  Warm start: qacc_warm if f(qacc_warm) < f(a0), else a0.
template <class T> SolveResult<T> newton_solve(int nv, const std::vector<T>& M, const std::vector<T>& a0,
                                               const Rows<T>& R, const T* warm, int cap) {
  SolveResult<T> out;
  std::vector<T> a = a0;
  if (R.n == 0) {
    out.qacc = a0;
    out.converged = true;
    return out;
  }
  if (warm) {
    std::vector<T> w(warm, warm + nv);
    if (val(cost(nv, M, a0, R, w)) < val(cost(nv, M, a0, R, a0))) { a = w; out.warm_used = true; }
  }
  bool elliptic = false;
  for (int i = 0; i < R.n; i++) elliptic = elliptic || R.kind[i] == 1;
  // active set: per scalar row jar < 0; per elliptic contact its zone (on its normal row)
  auto active_set = [&](const std::vector<T>& x) {
    std::vector<char> s(R.n, 0);
    for (int i = 0; i < R.n; i++) {
      if (R.kind[i] == 2) continue;
      if (R.kind[i] == 1) {
        T y[3];
        for (int e = 0; e < 3; e++) {
          y[e] = -R.aref[i + e];
          for (int j = 0; j < nv; j++) y[e] = y[e] + R.J[(i + e) * nv + j] * x[j];
        }
        s[i] = (char)cone_zone(y, R.mu[i]);
        continue;
      }
      T jar = -R.aref[i];
      for (int j = 0; j < nv; j++) jar = jar + R.J[i * nv + j] * x[j];
      s[i] = R.kind[i] == 3 ? (char)fric_zone(jar, R.D[i], R.mu[i]) : (char)(val(jar) < 0);
    }
    return s;
  };
  T f_cur = elliptic ? cost(nv, M, a0, R, a) : T(0);   // (the stopping rule of elliptic contacts)
  // g and the lower triangle of H at `at` with the active set A (the factorisations read only that
  // triangle; it is mirrored before them)
  auto grad_hess = [&](const std::vector<T>& at, const std::vector<char>& A, std::vector<T>& g, std::vector<T>& H) {
    g.assign(nv, T(0));
    H = M;
    std::vector<T> t(nv);
    for (int j = 0; j < nv; j++) t[j] = at[j] - a0[j];
    for (int i = 0; i < nv; i++) {
      T s = T(0);
      for (int j = 0; j < nv; j++) s = s + M[i * nv + j] * t[j];
      g[i] = s;
    }
    for (int r = 0; r < R.n; r++) {
      if (R.kind[r] == 3 && A[r] != 1) {   // friction loss outside its band: the constant force bound
        const T Fs = A[r] == 2 ? T(R.mu[r]) : -T(R.mu[r]);
        for (int i = 0; i < nv; i++) g[i] = g[i] + Fs * R.J[r * nv + i];
        continue;
      }
      if (!A[r] || R.kind[r] == 2) continue;
      if (R.kind[r] == 1) {   // J_c^T grad s and J_c^T hess s J_c over the contact's 3 rows
        T x[3], gc[3], Hc[9];
        for (int e = 0; e < 3; e++) {
          x[e] = -R.aref[r + e];
          for (int j = 0; j < nv; j++) x[e] = x[e] + R.J[(r + e) * nv + j] * at[j];
        }
        cone_grad_hess(x, R.D[r], R.mu[r], gc, Hc);
        for (int i = 0; i < nv; i++)
          for (int e = 0; e < 3; e++) {
            g[i] = g[i] + R.J[(r + e) * nv + i] * gc[e];
            for (int j = 0; j <= i; j++)
              for (int f = 0; f < 3; f++) H[i * nv + j] = H[i * nv + j] + R.J[(r + e) * nv + i] * Hc[3 * e + f] * R.J[(r + f) * nv + j];
          }
        continue;
      }
      T jar = -R.aref[r];
      for (int j = 0; j < nv; j++) jar = jar + R.J[r * nv + j] * at[j];
      const T Djar = R.D[r] * jar;
      for (int i = 0; i < nv; i++) {
        g[i] = g[i] + Djar * R.J[r * nv + i];
        const T DJ = R.D[r] * R.J[r * nv + i];
        for (int j = 0; j <= i; j++) H[i * nv + j] = H[i * nv + j] + DJ * R.J[r * nv + j];
      }
    }
    for (int i = 0; i < nv; i++)
      for (int j = i + 1; j < nv; j++) H[i * nv + j] = H[j * nv + i];
  };
  for (int it = 0; it < cap; it++) {
    std::vector<char> A = active_set(a);
    std::vector<T> g, H;
    grad_hess(a, A, g, H);
    out.iterations = it + 1;
    bool zero = true;
    for (int i = 0; i < nv; i++) zero = zero && val(g[i]) == 0;
    if (zero) { out.converged = true; break; }
    if (!spd_factor(H, nv)) break;
    std::vector<T> p(g);
    spd_solve(H, nv, p);
    for (int i = 0; i < nv; i++) p[i] = -p[i];
    T alpha = elliptic ? smooth_line_search(nv, M, a0, R, a, p) : exact_line_search(nv, M, a0, R, a, p);
    for (int i = 0; i < nv; i++) a[i] = a[i] + alpha * p[i];
    std::vector<char> A2 = active_set(a);
    if (!elliptic) {
      if (A2 == A) { out.converged = true; break; }
      continue;
    }
    // elliptic contacts: the Newton step is exact only when no contact sits in the middle zone
    // (there s is not quadratic); otherwise stop when f no longer decreases
    bool middle = false;
    for (int i = 0; i < R.n; i++) middle = middle || (R.kind[i] == 1 && A2[i] == 1);
    T f_new = cost(nv, M, a0, R, a);
    if ((A2 == A && !middle) || !(val(f_new) < val(f_cur))) { out.converged = true; break; }
    f_cur = f_new;
  }
  // Reverse mode differentiates the solve through its iterations.  At the minimiser, one Newton
  // step with the final active set held, a - H^-1 g(a), leaves the value where it is (g(a) = 0 to
  // rounding) and carries exactly the implicit derivative of the minimiser, -H^-1 dg/dtheta,
  // whatever the iterates before it (g is affine in a for a fixed active set, so
  // a - H^-1 g(a) = a* identically).  Without it, a solve that starts at the minimiser (warm-started
  // from the previous substep) ends on a step of rounding size, whose line-search factor, and with
  // it the derivative that factor scales, is rounding noise.  Taped instantiations only: the
  // values of the plain and counting ones are untouched.
  if (Taped<T>::value && out.converged && !elliptic) {
    std::vector<char> A = active_set(a);
    std::vector<T> g, H;
    grad_hess(a, A, g, H);
    if (spd_factor(H, nv)) {
      spd_solve(H, nv, g);
      for (int i = 0; i < nv; i++) a[i] = a[i] - g[i];
    }
  }
  out.qacc = a;
  PhaseHook<T>::set(8);   // the contact forces: an output, not part of the step's work
  out.force.assign(R.n, T(0));
  for (int i = 0; i < R.n; i++) {
    if (R.kind[i] == 2) continue;
    if (R.kind[i] == 1) {   // force = -grad s
      T x[3], gc[3], Hc[9];
      for (int e = 0; e < 3; e++) {
        x[e] = -R.aref[i + e];
        for (int j = 0; j < nv; j++) x[e] = x[e] + R.J[(i + e) * nv + j] * a[j];
      }
      cone_grad_hess(x, R.D[i], R.mu[i], gc, Hc);
      for (int e = 0; e < 3; e++) out.force[i + e] = -gc[e];
      continue;
    }
    T jar = -R.aref[i];
    for (int j = 0; j < nv; j++) jar = jar + R.J[i * nv + j] * a[j];
    if (R.kind[i] == 3) {
      const int z = fric_zone(jar, R.D[i], R.mu[i]);
      out.force[i] = z == 1 ? -R.D[i] * jar : (z == 2 ? -T(R.mu[i]) : T(R.mu[i]));
    } else if (val(jar) < 0) {
      out.force[i] = -R.D[i] * jar;
    }
  }
  return out;
}

// ------------------------------------------------------------------------------------
// one substep
// ------------------------------------------------------------------------------------
template <class T> struct Forward {
  Kin<T> kin;
  std::vector<T> M, bias, passive, actuator, a0;
  std::vector<Contact<T>> con;
  Rows<T> rows;
  SolveResult<T> sol;
  uint32_t status = 0;
};

// Actuation: motor tau += gear * u (u clamped to ctrlrange when ctrllimited);
// position (PD, eq. pd_mapping) tau += kp (u - q) - kd qdot on the actuated joint.
template <class T> void actuation(const Model& m, const T* qpos, const T* qvel, const T* ctrl, std::vector<T>& tau,
                                  const Params<T>* P = nullptr) {
  tau.assign(m.nv, T(0));
  for (int a = 0; a < m.nu; a++) {
    int j = m.act_jnt[a], d = m.jnt_dofadr[j], qa = m.jnt_qposadr[j];
    T u = ctrl[a];
    if (m.act_ctrllimited[a]) {
      if (val(u) < m.act_ctrlrange[2 * a]) u = T(m.act_ctrlrange[2 * a]);
      if (val(u) > m.act_ctrlrange[2 * a + 1]) u = T(m.act_ctrlrange[2 * a + 1]);
    }
    T f = m.act_type[a] == MOTOR ? T(m.act_gear[a]) * u
                                  : (P ? P->kp[a] : T(m.act_kp[a])) * (u - qpos[qa]) - T(m.act_kd[a]) * qvel[d];
    if (m.act_forcelimited[a]) {   // torque limits: the force is clipped to its range
      if (val(f) < m.act_forcerange[2 * a]) f = T(m.act_forcerange[2 * a]);
      if (val(f) > m.act_forcerange[2 * a + 1]) f = T(m.act_forcerange[2 * a + 1]);
    }
    tau[d] = tau[d] + f;
  }
}

template <class T> void build_rows(const Model& m, const Forward<T>& F, const T* qpos, const T* qvel, Rows<T>& R,
                                   const std::vector<T>& Mchol) {
  const int nv = m.nv;
  R = Rows<T>();
  std::vector<T> Jv1, Jw1, Jv2, Jw2;
  auto push = [&](const std::vector<T>& Jrow, T r, int slot, int kind = 0, double mu = 0.0) {
    R.J.insert(R.J.end(), Jrow.begin(), Jrow.end());
    R.r.push_back(r);
    R.slot.push_back(slot);
    R.kind.push_back(kind);
    R.mu.push_back(mu);
    R.n++;
  };
  for (int p = 0; p < m.npair; p++) {
    int g1 = m.pair_g1[p], g2 = m.pair_g2[p];
    int b1 = m.geom_body[g1], b2 = m.geom_body[g2];
    for (int s = m.pair_slotadr[p]; s < m.pair_slotadr[p] + m.pair_nslot[p]; s++) {
      const Contact<T>& c = F.con[s];
      if (!c.active) continue;
      point_jacobian(m, F.kin, b1, c.pos, Jv1, Jw1);
      point_jacobian(m, F.kin, b2, c.pos, Jv2, Jw2);
      std::vector<T> Jn(nv), Jt1(nv), Jt2(nv);
      for (int i = 0; i < nv; i++) {
        V3<T> dj{Jv2[i] - Jv1[i], Jv2[nv + i] - Jv1[nv + i], Jv2[2 * nv + i] - Jv1[2 * nv + i]};
        Jn[i] = dot(c.n, dj);
        Jt1[i] = dot(c.t1, dj);
        Jt2[i] = dot(c.t2, dj);
      }
      if (m.pair_condim[p] == 1) {
        push(Jn, c.dist, s);
      } else if (m.cone == ELLIPTIC) {
        push(Jn, c.dist, s, 1, m.pair_friction[p]);
        push(Jt1, T(0), s, 2, m.pair_friction[p]);
        push(Jt2, T(0), s, 2, m.pair_friction[p]);
      } else {
        T mu = T(m.pair_friction[p]);
        std::vector<T> e(nv);
        for (int k = 0; k < 4; k++) {
          const std::vector<T>& Jt = k < 2 ? Jt1 : Jt2;
          T sg = (k % 2 == 0) ? mu : -mu;
          for (int i = 0; i < nv; i++) e[i] = Jn[i] + sg * Jt[i];
          push(e, c.dist, s);
        }
      }
    }
  }
  for (int j = 0; j < m.njnt; j++) {
    if (!m.jnt_limited[j] || m.jnt_type[j] == FREE) continue;
    T q = qpos[m.jnt_qposadr[j]];
    int d = m.jnt_dofadr[j];
    std::vector<T> e(nv, T(0));
    if (val(q) - m.jnt_range[2 * j] < m.margin) {
      e[d] = T(1);
      push(e, q - T(m.jnt_range[2 * j]), -1 - j);
    } else if (m.jnt_range[2 * j + 1] - val(q) < m.margin) {
      e[d] = T(-1);
      push(e, T(m.jnt_range[2 * j + 1]) - q, -1 - j);
    }
  }
  // joint friction loss: one two-sided row per dof with a positive loss, at zero position (its
  // reference acceleration is the damping term alone)
  for (int d = 0; d < nv; d++) {
    if (!(m.dof_frictionloss[d] > 0)) continue;
    std::vector<T> e(nv, T(0));
    e[d] = T(1);
    push(e, T(0), -100000 - d, 3, m.dof_frictionloss[d]);
  }
  // reference acceleration and regularisation per row
  double h = m.timestep;
  double tc = std::max(m.solref[0], 2 * h), zeta = m.solref[1], dmax = m.solimp[1];
  double kk = 1.0 / (dmax * dmax * tc * tc * zeta * zeta), bb = 2.0 / (dmax * tc);
  R.v.resize(R.n); R.aref.resize(R.n); R.D.resize(R.n); R.Ahat.resize(R.n); R.imp.resize(R.n);
  for (int i = 0; i < R.n; i++) {
    T v = T(0);
    for (int j = 0; j < nv; j++) v = v + R.J[i * nv + j] * qvel[j];
    R.v[i] = v;
    if (R.kind[i] == 2) {   // elliptic tangent row: the normal row's impedance, Ahat and D
      const int n0 = R.kind[i - 1] == 1 ? i - 1 : i - 2;
      R.Ahat[i] = R.Ahat[n0];
      R.imp[i] = R.imp[n0];
      R.aref[i] = -T(bb) * v - T(kk) * R.imp[n0] * R.r[i];
      R.D[i] = R.D[n0] * T(m.impratio);
      continue;
    }
    std::vector<T> x(R.J.begin() + i * nv, R.J.begin() + (i + 1) * nv);
    spd_solve(Mchol, nv, x);
    T A = T(0);
    for (int j = 0; j < nv; j++) A = A + R.J[i * nv + j] * x[j];
    T d = impedance(R.r[i], m.solimp);
    R.Ahat[i] = A;
    R.imp[i] = d;
    R.aref[i] = -T(bb) * v - T(kk) * d * R.r[i];
    R.D[i] = d / ((T(1) - d) * A);
  }
}

// solver_cap < 0 selects the converged mode (cap 200, exact termination only)
template <class T> void forward(const Model& m, const T* qpos, const T* qvel, const T* qacc_warm, const T* ctrl,
                                int solver_cap, Forward<T>& F, const Params<T>* P = nullptr) {
  const int nv = m.nv;
  PhaseHook<T>::set(0);   // kinematics
  kinematics(m, qpos, F.kin, P);
  PhaseHook<T>::set(1);   // mass matrix
  if (TreeMethods<T>::value) crba_mass_matrix(m, F.kin, F.M, P);
  else mass_matrix(m, F.kin, F.M, P);
  PhaseHook<T>::set(2);   // bias forces
  std::vector<T> zero(nv, T(0));
  inverse_dynamics(m, F.kin, qvel, zero.data(), F.bias, P);
  PhaseHook<T>::set(3);   // passive and actuator forces, the smooth acceleration
  F.passive.assign(nv, T(0));
  for (int i = 0; i < nv; i++) F.passive[i] = -(P ? P->damping[i] : T(m.dof_damping[i])) * qvel[i];
  actuation(m, qpos, qvel, ctrl, F.actuator, P);
  std::vector<T> Mchol(F.M);
  if (!spd_factor(Mchol, nv)) F.status |= ST_NAN;
  F.a0.assign(nv, T(0));
  for (int i = 0; i < nv; i++) F.a0[i] = F.actuator[i] + F.passive[i] - F.bias[i];
  spd_solve(Mchol, nv, F.a0);
  PhaseHook<T>::set(4);   // collision
  // collision over the static pair list; then the active-contact cap in slot order
  F.con.assign(m.nslot, Contact<T>());
  for (int p = 0; p < m.npair; p++) {
    int g1 = m.pair_g1[p], g2 = m.pair_g2[p];
    collide_pair(m.geom_type[g1], F.kin.xgeom[g1], &m.geom_size[3 * g1], m.geom_type[g2], F.kin.xgeom[g2],
                 &m.geom_size[3 * g2], &F.con[m.pair_slotadr[p]], m.hf(),
                 m.geom_meshid[g2] >= 0 ? &m.meshes[m.geom_meshid[g2]] : nullptr);
  }
  int nact = 0;
  for (int s = 0; s < m.nslot; s++) {
    F.con[s].active = val(F.con[s].dist) < m.margin;
    if (F.con[s].active) {
      if (nact >= m.max_contacts) { F.con[s].active = false; F.status |= ST_CAPACITY; }
      else nact++;
    }
  }
  PhaseHook<T>::set(5);   // constraint rows
  build_rows(m, F, qpos, qvel, F.rows, Mchol);
  PhaseHook<T>::set(6);   // the Newton solve
  bool warm_ok = true;
  for (int i = 0; i < nv; i++) warm_ok = warm_ok && std::isfinite(val(qacc_warm[i]));
  if (!warm_ok) F.status |= ST_WARM_RESET;
  int cap = solver_cap < 0 ? 200 : solver_cap;
  F.sol = newton_solve(nv, F.M, F.a0, F.rows, warm_ok ? qacc_warm : nullptr, cap);
  if (!F.sol.converged) F.status |= ST_NOT_CONVERGED;
}

// Semi-implicit Euler: qvel += h qacc, then positions with the new velocity; the free joint's
// quaternion is multiplied by the rotation of angle h |w| about w (body-local w) and normalised.
template <class T> void integrate_pos(const Model& m, T* qpos, const T* qvel, double h) {
  for (int j = 0; j < m.njnt; j++) {
    T* q = qpos + m.jnt_qposadr[j];
    const T* v = qvel + m.jnt_dofadr[j];
    if (m.jnt_type[j] == FREE) {
      for (int k = 0; k < 3; k++) q[k] = q[k] + T(h) * v[k];
      T wn = sqrt(v[3] * v[3] + v[4] * v[4] + v[5] * v[5]);
      std::array<T, 4> qq{q[3], q[4], q[5], q[6]};
      if (val(wn) > 1e-8) {
        using std::cos; using std::sin;
        T ang = T(h) * wn, s = sin(ang * T(0.5)) / wn;
        std::array<T, 4> dq{cos(ang * T(0.5)), v[3] * s, v[4] * s, v[5] * s};
        qq = qmul(qq, dq);
      } else {
        // the same rotation by its series (cos(h|w|/2), (h/2) w (1 - O(h^2 |w|^2))): at w = 0 it is
        // the identity, and its derivative (h/2 along w) survives in reverse mode, which the
        // closed form through |w| cannot give there
        const T hh = T(0.5 * h);
        std::array<T, 4> dq{T(1) - T(0.5) * hh * hh * (v[3] * v[3] + v[4] * v[4] + v[5] * v[5]), v[3] * hh, v[4] * hh,
                            v[5] * hh};
        qq = qmul(qq, dq);
      }
      T n = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
      for (int k = 0; k < 4; k++) q[3 + k] = qq[k] / n;
    } else {
      q[0] = q[0] + T(h) * v[0];
    }
  }
}

template <class T> uint32_t substep(const Model& m, T* qpos, T* qvel, T* qacc_warm, const T* ctrl, int solver_cap,
                                    Forward<T>* keep = nullptr, const Params<T>* P = nullptr) {
  Forward<T> local;
  Forward<T>& F = keep ? *keep : local;
  F = Forward<T>();
  forward(m, qpos, qvel, qacc_warm, ctrl, solver_cap, F, P);
  PhaseHook<T>::set(7);   // integration
  const int nv = m.nv;
  for (int i = 0; i < nv; i++) qvel[i] = qvel[i] + T(m.timestep) * F.sol.qacc[i];
  integrate_pos(m, qpos, qvel, m.timestep);
  for (int i = 0; i < nv; i++) qacc_warm[i] = F.sol.qacc[i];
  uint32_t st = F.status;
  for (int i = 0; i < nv; i++)
    if (!std::isfinite(val(qvel[i])) || !std::isfinite(val(F.sol.qacc[i]))) st |= ST_NAN;
  for (int i = 0; i < m.nq; i++)
    if (!std::isfinite(val(qpos[i]))) st |= ST_NAN;
  return st;
}

}  // namespace orc
