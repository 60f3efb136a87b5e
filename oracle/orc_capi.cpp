// FP64 oracle -- TEST INFRASTRUCTURE ONLY.  C API of the oracle (loaded with ctypes by the
// tests, by the package's smoke() check and by bench.py's CPU-baseline leg).
//
// Arrays are environment-major ([env][coord]) doubles.  Every function returns 0 on success
// and a negative value on a bad argument.
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "orc_ad.hpp"
#include "orc_model.hpp"
#include "orc_step.hpp"
#include "orc_count.hpp"

using orc::Model;

extern "C" {

void* orc_model_new(const orc::Desc* d, char* err, int errlen) {
  Model* m = new Model();
  std::string e = orc::compile_model(*d, *m);
  if (!e.empty()) {
    if (err && errlen > 0) { std::strncpy(err, e.c_str(), errlen - 1); err[errlen - 1] = 0; }
    delete m;
    return nullptr;
  }
  return m;
}

void orc_model_free(void* h) { delete static_cast<Model*>(h); }

// nq nv nu nbody ngeom nslot nrow_max njnt npair nlimited max_contacts
int orc_model_sizes(void* h, int* out) {
  const Model& m = *static_cast<Model*>(h);
  int v[11] = {m.nq, m.nv, m.nu, m.nbody, m.ngeom, m.nslot, m.nrow_max, m.njnt, m.npair, m.nlimited, m.max_contacts};
  std::memcpy(out, v, sizeof(v));
  return 0;
}

int orc_model_massprops(void* h, double* mass, double* ipos, double* inertia, double* armature) {
  const Model& m = *static_cast<Model*>(h);
  std::memcpy(mass, m.mass.data(), sizeof(double) * m.nbody);
  std::memcpy(ipos, m.ipos.data(), sizeof(double) * 3 * m.nbody);
  std::memcpy(inertia, m.inertia.data(), sizeof(double) * 6 * m.nbody);
  std::memcpy(armature, m.dof_armature.data(), sizeof(double) * m.nv);
  return 0;
}

// Advance n_envs independent environments by n_steps control steps of n_substeps substeps
// each (controls held over a control step).  solver_cap >= 1: capped Newton; < 0: converged.
int orc_rollout(void* h, int n_envs, int n_steps, int n_substeps, double* qpos, double* qvel, double* qacc_warm,
                const double* ctrl, uint32_t* status, int solver_cap, int nthreads, double* traj_qpos,
                double* traj_qvel) {
  const Model& m = *static_cast<Model*>(h);
  if (n_envs < 0 || n_steps < 0 || n_substeps < 1) return -1;
  if (nthreads < 1) nthreads = 1;
  auto work = [&](int lo, int hi) {
    for (int e = lo; e < hi; e++) {
      double* q = qpos + (size_t)e * m.nq;
      double* v = qvel + (size_t)e * m.nv;
      double* w = qacc_warm + (size_t)e * m.nv;
      for (int t = 0; t < n_steps; t++) {
        const double* u = ctrl + ((size_t)t * n_envs + e) * m.nu;
        for (int s = 0; s < n_substeps; s++) status[e] |= orc::substep(m, q, v, w, u, solver_cap);
        if (traj_qpos) std::memcpy(traj_qpos + ((size_t)t * n_envs + e) * m.nq, q, sizeof(double) * m.nq);
        if (traj_qvel) std::memcpy(traj_qvel + ((size_t)t * n_envs + e) * m.nv, v, sizeof(double) * m.nv);
      }
    }
  };
  if (nthreads == 1 || n_envs <= 1) {
    work(0, n_envs);
  } else {
    std::vector<std::thread> pool;
    int per = (n_envs + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; t++) {
      int lo = t * per, hi = std::min(n_envs, lo + per);
      if (lo < hi) pool.emplace_back(work, lo, hi);
    }
    for (auto& th : pool) th.join();
  }
  return 0;
}

// Offsets (in doubles) of the per-substep diagnostic record written by orc_forward:
// 0 xpos[nbody][3]  1 xmat[nbody][9]  2 xcom[nbody][3]  3 M[nv][nv]  4 bias[nv]  5 passive[nv]
// 6 actuator[nv]  7 a0[nv]  8 contacts[nslot][14] (active, dist, pos3, n3, t1 3, t2 3)
// 9 nrow  10 rows[nrow_max][nv + 7] (J[nv], r, v, aref, D, Ahat, imp, force)  11 qacc[nv]
// 12 iterations  13 status  14 qpos_next[nq]  15 qvel_next[nv]  16 total
int orc_forward_layout(void* h, int* off) {
  const Model& m = *static_cast<Model*>(h);
  int sz[16] = {3 * m.nbody, 9 * m.nbody, 3 * m.nbody, m.nv * m.nv, m.nv, m.nv, m.nv, m.nv, 14 * m.nslot, 1,
                m.nrow_max * (m.nv + 7), m.nv, 1, 1, m.nq, m.nv};
  off[0] = 0;
  for (int i = 0; i < 16; i++) off[i + 1] = off[i] + sz[i];
  return 0;
}

int orc_forward(void* h, const double* qpos, const double* qvel, const double* qacc_warm, const double* ctrl,
                int solver_cap, double* out) {
  const Model& m = *static_cast<Model*>(h);
  int off[17];
  orc_forward_layout(h, off);
  std::memset(out, 0, sizeof(double) * off[16]);
  std::vector<double> q(qpos, qpos + m.nq), v(qvel, qvel + m.nv), w(qacc_warm, qacc_warm + m.nv);
  orc::Forward<double> F;
  uint32_t st = orc::substep(m, q.data(), v.data(), w.data(), ctrl, solver_cap, &F);
  for (int b = 0; b < m.nbody; b++) {
    for (int k = 0; k < 3; k++) out[off[0] + 3 * b + k] = F.kin.xbody[b].p[k];
    for (int k = 0; k < 9; k++) out[off[1] + 9 * b + k] = F.kin.xbody[b].R[k];
    for (int k = 0; k < 3; k++) out[off[2] + 3 * b + k] = F.kin.xcom[b][k];
  }
  std::memcpy(out + off[3], F.M.data(), sizeof(double) * m.nv * m.nv);
  std::memcpy(out + off[4], F.bias.data(), sizeof(double) * m.nv);
  std::memcpy(out + off[5], F.passive.data(), sizeof(double) * m.nv);
  std::memcpy(out + off[6], F.actuator.data(), sizeof(double) * m.nv);
  std::memcpy(out + off[7], F.a0.data(), sizeof(double) * m.nv);
  for (int s = 0; s < m.nslot; s++) {
    double* c = out + off[8] + 14 * s;
    const orc::Contact<double>& k = F.con[s];
    c[0] = k.active ? 1 : 0;
    c[1] = k.dist;
    for (int i = 0; i < 3; i++) { c[2 + i] = k.pos[i]; c[5 + i] = k.n[i]; c[8 + i] = k.t1[i]; c[11 + i] = k.t2[i]; }
  }
  out[off[9]] = F.rows.n;
  for (int r = 0; r < F.rows.n && r < m.nrow_max; r++) {
    double* o = out + off[10] + r * (m.nv + 7);
    for (int j = 0; j < m.nv; j++) o[j] = F.rows.J[r * m.nv + j];
    o[m.nv] = F.rows.r[r];
    o[m.nv + 1] = F.rows.v[r];
    o[m.nv + 2] = F.rows.aref[r];
    o[m.nv + 3] = F.rows.D[r];
    o[m.nv + 4] = F.rows.Ahat[r];
    o[m.nv + 5] = F.rows.imp[r];
    o[m.nv + 6] = F.sol.force.empty() ? 0.0 : F.sol.force[r];
  }
  std::memcpy(out + off[11], F.sol.qacc.data(), sizeof(double) * m.nv);
  out[off[12]] = F.sol.iterations;
  out[off[13]] = st;
  std::memcpy(out + off[14], q.data(), sizeof(double) * m.nq);
  std::memcpy(out + off[15], v.data(), sizeof(double) * m.nv);
  return 0;
}

int orc_inverse_dynamics(void* h, const double* qpos, const double* qvel, const double* qacc, double* tau) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> t;
  orc::inverse_dynamics(m, k, qvel, qacc, t);
  std::memcpy(tau, t.data(), sizeof(double) * m.nv);
  return 0;
}

int orc_mass_matrix(void* h, const double* qpos, double* M) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> Mm;
  orc::mass_matrix(m, k, Mm);
  std::memcpy(M, Mm.data(), sizeof(double) * m.nv * m.nv);
  return 0;
}

// per body: R (9, row-major), x (3), com (3)
// the mass matrix by CRBA (the counted method), row-major nv x nv
int orc_mass_matrix_crba(void* h, const double* qpos, double* M) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> Mv;
  orc::crba_mass_matrix(m, k, Mv);
  std::memcpy(M, Mv.data(), sizeof(double) * m.nv * m.nv);
  return 0;
}

int orc_body_frames(void* h, const double* qpos, double* out) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  for (int b = 0; b < m.nbody; b++) {
    for (int i = 0; i < 9; i++) out[15 * b + i] = k.xbody[b].R[i];
    for (int i = 0; i < 3; i++) out[15 * b + 9 + i] = k.xbody[b].p[i];
    for (int i = 0; i < 3; i++) out[15 * b + 12 + i] = k.xcom[b][i];
  }
  return 0;
}

// per geom: R (9), x (3)
int orc_geom_frames(void* h, const double* qpos, double* out) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  for (int g = 0; g < m.ngeom; g++) {
    for (int i = 0; i < 9; i++) out[12 * g + i] = k.xgeom[g].R[i];
    for (int i = 0; i < 3; i++) out[12 * g + 9 + i] = k.xgeom[g].p[i];
  }
  return 0;
}

// kinetic energy from per-body velocities (sum 1/2 m |v_com|^2 + 1/2 w^T Iw w, plus
// 1/2 armature qdot^2) and potential energy -sum m g . com
int orc_energy(void* h, const double* qpos, const double* qvel, double* out) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> zero(m.nv, 0.0);
  std::vector<orc::Motion<double>> mo;
  orc::body_motion(m, k, qvel, zero.data(), mo);
  double T = 0, U = 0;
  for (int b = 1; b < m.nbody; b++) {
    orc::V3<double> vc = orc::point_vel(mo[b], k.xcom[b]);
    orc::V3<double> Iw = orc::mv(k.Iw[b], mo[b].w);
    T += 0.5 * m.mass[b] * orc::dot(vc, vc) + 0.5 * orc::dot(mo[b].w, Iw);
    U -= m.mass[b] * (m.gravity[0] * k.xcom[b][0] + m.gravity[1] * k.xcom[b][1] + m.gravity[2] * k.xcom[b][2]);
  }
  for (int i = 0; i < m.nv; i++) T += 0.5 * m.dof_armature[i] * qvel[i] * qvel[i];
  out[0] = T;
  out[1] = U;
  return 0;
}

// linear momentum P, angular momentum about the system COM, and the COM
int orc_momentum(void* h, const double* qpos, const double* qvel, double* out) {
  const Model& m = *static_cast<Model*>(h);
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> zero(m.nv, 0.0);
  std::vector<orc::Motion<double>> mo;
  orc::body_motion(m, k, qvel, zero.data(), mo);
  orc::V3<double> P{0, 0, 0}, C{0, 0, 0}, L{0, 0, 0};
  double Mt = 0;
  for (int b = 1; b < m.nbody; b++) {
    Mt += m.mass[b];
    C = orc::add(C, orc::scl(k.xcom[b], m.mass[b]));
  }
  C = orc::scl(C, 1.0 / Mt);
  for (int b = 1; b < m.nbody; b++) {
    orc::V3<double> vc = orc::point_vel(mo[b], k.xcom[b]);
    P = orc::add(P, orc::scl(vc, m.mass[b]));
    L = orc::add(L, orc::add(orc::mv(k.Iw[b], mo[b].w), orc::scl(orc::cross(orc::sub(k.xcom[b], C), vc), m.mass[b])));
  }
  for (int i = 0; i < 3; i++) { out[i] = P[i]; out[3 + i] = L[i]; out[6 + i] = C[i]; }
  return 0;
}

int orc_point_jacobian(void* h, const double* qpos, int body, const double* point, double* Jv, double* Jw) {
  const Model& m = *static_cast<Model*>(h);
  if (body < 0 || body >= m.nbody) return -1;
  orc::Kin<double> k;
  orc::kinematics(m, qpos, k);
  std::vector<double> a, b;
  orc::point_jacobian(m, k, body, orc::V3<double>{point[0], point[1], point[2]}, a, b);
  std::memcpy(Jv, a.data(), sizeof(double) * 3 * m.nv);
  std::memcpy(Jw, b.data(), sizeof(double) * 3 * m.nv);
  return 0;
}

int orc_integrate_pos(void* h, double* qpos, const double* qvel, double dt) {
  orc::integrate_pos(*static_cast<Model*>(h), qpos, qvel, dt);
  return 0;
}

// Model-free collision of one primitive pair; frames given as R (row-major 3x3) and p.
// Writes pair_max_points records of 13 doubles: dist, pos3, n3, t1 3, t2 3.  Returns the count.
int orc_collide(int t1, const double* R1, const double* p1, const double* s1, int t2, const double* R2,
                const double* p2, const double* s2, double* out) {
  int n = orc::pair_max_points(t1, t2);
  if (n < 0 || t2 == orc::MESH) return -1;
  orc::Xf<double> X1, X2;
  for (int i = 0; i < 9; i++) { X1.R[i] = R1[i]; X2.R[i] = R2[i]; }
  for (int i = 0; i < 3; i++) { X1.p[i] = p1[i]; X2.p[i] = p2[i]; }
  orc::Contact<double> c[4];
  orc::collide_pair(t1, X1, s1, t2, X2, s2, c);
  for (int i = 0; i < n; i++) {
    double* o = out + 13 * i;
    o[0] = c[i].dist;
    for (int k = 0; k < 3; k++) { o[1 + k] = c[i].pos[k]; o[4 + k] = c[i].n[k]; o[7 + k] = c[i].t1[k]; o[10 + k] = c[i].t2[k]; }
  }
  return n;
}

// Model-free collision of a heightfield (geom1: frame R1/p1, size s1, grid nrow x ncol of
// elevations) with a sphere or capsule (geom2); the same records as orc_collide.
int orc_collide_hfield(const double* R1, const double* p1, const double* s1, int nrow, int ncol, const double* elev,
                       int t2, const double* R2, const double* p2, const double* s2, double* out) {
  int n = orc::pair_max_points(orc::HFIELD, t2);
  if (n < 0 || nrow < 2 || ncol < 2 || !elev || t2 == orc::MESH) return -1;
  orc::Xf<double> X1, X2;
  for (int i = 0; i < 9; i++) { X1.R[i] = R1[i]; X2.R[i] = R2[i]; }
  for (int i = 0; i < 3; i++) { X1.p[i] = p1[i]; X2.p[i] = p2[i]; }
  orc::Contact<double> c[4];
  orc::collide_pair(orc::HFIELD, X1, s1, t2, X2, s2, c, orc::HField{nrow, ncol, elev});
  for (int i = 0; i < n; i++) {
    double* o = out + 13 * i;
    o[0] = c[i].dist;
    for (int k = 0; k < 3; k++) { o[1 + k] = c[i].pos[k]; o[4 + k] = c[i].n[k]; o[7 + k] = c[i].t1[k]; o[10 + k] = c[i].t2[k]; }
  }
  return n;
}

// Model-free collision of a plane (t1 = PLANE; frame R1/p1) or a heightfield (t1 = HFIELD; size s1,
// grid nrow x ncol) with a convex mesh (vertices nvert x 3, outward triangles nface x 3, in the
// frame R2/p2); the same records as orc_collide, 4 of them.  -1 on a bad pair or mesh.
int orc_collide_mesh(int t1, const double* R1, const double* p1, const double* s1, int nrow, int ncol, const double* elev,
                     int nvert, const double* vert, int nface, const int* face, const double* R2, const double* p2,
                     double* out) {
  if (t1 != orc::PLANE && !(t1 == orc::HFIELD && nrow >= 2 && ncol >= 2 && elev)) return -1;
  orc::Solid sd;
  if (!orc::mesh_solid(vert, nvert, face, nface, sd).empty()) return -1;
  orc::Xf<double> X1, X2;
  for (int i = 0; i < 9; i++) { X1.R[i] = R1[i]; X2.R[i] = R2[i]; }
  for (int i = 0; i < 3; i++) { X1.p[i] = p1[i]; X2.p[i] = p2[i]; }
  orc::Contact<double> c[4];
  const double zero[3] = {0, 0, 0};
  orc::collide_pair(t1, X1, s1 ? s1 : zero, orc::MESH, X2, zero, c, orc::HField{nrow, ncol, elev}, &sd);
  for (int i = 0; i < 4; i++) {
    double* o = out + 13 * i;
    o[0] = c[i].dist;
    for (int k = 0; k < 3; k++) { o[1 + k] = c[i].pos[k]; o[4 + k] = c[i].n[k]; o[7 + k] = c[i].t1[k]; o[10 + k] = c[i].t2[k]; }
  }
  return 4;
}

// The Newton solver on raw data (M, a0, rows J/aref/D); cap < 0 selects the converged mode.
// Rows from raw arrays; kind / mu NULL: every row a one-sided scalar row
static orc::Rows<double> raw_rows(int nv, int nr, const double* J, const double* aref, const double* D, const int* kind,
                                  const double* mu) {
  orc::Rows<double> R;
  R.n = nr;
  R.J.assign(J, J + nr * nv);
  R.aref.assign(aref, aref + nr);
  R.D.assign(D, D + nr);
  R.kind.assign(nr, 0);
  R.mu.assign(nr, 0.0);
  for (int i = 0; i < nr; i++) {
    if (kind) R.kind[i] = kind[i];
    if (mu) R.mu[i] = mu[i];
  }
  return R;
}

int orc_solve(int nv, const double* M, const double* a0, int nr, const double* J, const double* aref, const double* D,
              const double* warm, int cap, double* qacc, double* force, int* iters, const int* kind, const double* mu) {
  std::vector<double> Mm(M, M + nv * nv), a(a0, a0 + nv);
  orc::Rows<double> R = raw_rows(nv, nr, J, aref, D, kind, mu);
  orc::SolveResult<double> s = orc::newton_solve(nv, Mm, a, R, warm, cap < 0 ? 200 : cap);
  std::memcpy(qacc, s.qacc.data(), sizeof(double) * nv);
  if (nr > 0) std::memcpy(force, s.force.data(), sizeof(double) * nr);
  *iters = s.iterations;
  return s.converged ? 1 : 0;
}

double orc_cost(int nv, const double* M, const double* a0, int nr, const double* J, const double* aref, const double* D,
                const double* a, const int* kind, const double* mu) {
  std::vector<double> Mm(M, M + nv * nv), aa(a0, a0 + nv), x(a, a + nv);
  orc::Rows<double> R = raw_rows(nv, nr, J, aref, D, kind, mu);
  return orc::cost(nv, Mm, aa, R, x);
}

// the elliptic contact cost, its zone, gradient and Hessian at x (3), for pins
double orc_cone_cost(const double* x, double D, double mu, double* g, double* H, int* zone) {
  orc::cone_grad_hess(x, D, mu, g, H);
  *zone = orc::cone_zone(x, mu);
  return orc::cone_cost(x, D, mu);
}

// ---- rollout loss and its reverse-mode gradient ----------------------------------------
// Loss over a rollout of T control steps (n_substeps each) from (q0, v0) with controls
// ctrl[T][nu]:  L = sum_{t=1..T} sum_i wq_i (q_t,i - qs_i)^2 + sum_i wv_i (v_t,i - vs_i)^2.
// Optional parameters (NULL = the model's): body masses [nbody], dof damping [nv], kp [nu].
static orc::Params<double> make_params(const Model& m, const double* mass, const double* damp, const double* kp) {
  orc::Params<double> P;
  P.mass = mass ? std::vector<double>(mass, mass + m.nbody) : m.mass;
  P.damping = damp ? std::vector<double>(damp, damp + m.nv) : m.dof_damping;
  P.kp.resize(m.nu);
  for (int a = 0; a < m.nu; a++) P.kp[a] = kp ? kp[a] : m.act_kp[a];
  return P;
}

static double step_loss(const Model& m, const double* q, const double* v, const double* wq, const double* qs,
                        const double* wv, const double* vs) {
  double L = 0;
  for (int i = 0; i < m.nq; i++) L += wq[i] * (q[i] - qs[i]) * (q[i] - qs[i]);
  for (int i = 0; i < m.nv; i++) L += wv[i] * (v[i] - vs[i]) * (v[i] - vs[i]);
  return L;
}

double orc_rollout_loss(void* h, const double* q0, const double* v0, const double* ctrl, int T, int n_substeps,
                        int solver_cap, const double* mass, const double* damp, const double* kp, const double* wq,
                        const double* qs, const double* wv, const double* vs) {
  const Model& m = *static_cast<Model*>(h);
  orc::Params<double> P = make_params(m, mass, damp, kp);
  std::vector<double> q(q0, q0 + m.nq), v(v0, v0 + m.nv), w(m.nv, 0.0);
  double L = 0;
  for (int t = 0; t < T; t++) {
    for (int s = 0; s < n_substeps; s++) orc::substep<double>(m, q.data(), v.data(), w.data(), ctrl + (size_t)t * m.nu, solver_cap, nullptr, &P);
    L += step_loss(m, q.data(), v.data(), wq, qs, wv, vs);
  }
  return L;
}

// Reverse mode through one control step (n_substeps substeps) from (q, v) with controls u: the
// adjoint (bq, bv) of the post-step state is replaced by the adjoint of the pre-step state;
// control adjoints are written to gu and parameter adjoints added to gmass / gdamp / gkp.  The
// warm start enters as a constant.
static void control_step_vjp(const Model& m, const orc::Params<double>& P, const double* q0, const double* v0,
                             const double* w0, const double* u0, int n_substeps, int solver_cap, double* bq, double* bv,
                             double* gu, double* gmass, double* gdamp, double* gkp) {
  using orc::adouble;
  const int nq = m.nq, nv = m.nv, nu = m.nu, nb = m.nbody;
  orc::Tape tp;
  orc::Tape* prev = orc::tape();
  orc::tape() = &tp;
  std::vector<adouble> q(nq), v(nv), u(nu), w(nv);
  for (int i = 0; i < nq; i++) q[i] = adouble::var(q0[i]);
  for (int i = 0; i < nv; i++) v[i] = adouble::var(v0[i]);
  for (int i = 0; i < nu; i++) u[i] = adouble::var(u0[i]);
  for (int i = 0; i < nv; i++) w[i] = adouble(w0 ? w0[i] : 0.0);
  orc::Params<adouble> PA;
  for (int b = 0; b < nb; b++) PA.mass.push_back(adouble::var(P.mass[b]));
  for (int i = 0; i < nv; i++) PA.damping.push_back(adouble::var(P.damping[i]));
  for (int a = 0; a < nu; a++) PA.kp.push_back(adouble::var(P.kp[a]));
  std::vector<int> iq(nq), iv(nv), iu(nu);
  for (int i = 0; i < nq; i++) iq[i] = q[i].i;
  for (int i = 0; i < nv; i++) iv[i] = v[i].i;
  for (int i = 0; i < nu; i++) iu[i] = u[i].i;
  for (int s = 0; s < n_substeps; s++) orc::substep<adouble>(m, q.data(), v.data(), w.data(), u.data(), solver_cap, nullptr, &PA);
  std::vector<std::pair<int, double>> seeds;
  for (int i = 0; i < nq; i++) seeds.push_back({q[i].i, bq[i]});
  for (int i = 0; i < nv; i++) seeds.push_back({v[i].i, bv[i]});
  std::vector<double> adj = tp.backward(seeds);
  for (int i = 0; i < nq; i++) bq[i] = adj[iq[i]];
  for (int i = 0; i < nv; i++) bv[i] = adj[iv[i]];
  for (int i = 0; i < nu; i++) gu[i] = adj[iu[i]];
  for (int b = 0; b < nb; b++) gmass[b] += adj[PA.mass[b].i];
  for (int i = 0; i < nv; i++) gdamp[i] += adj[PA.damping[i].i];
  for (int a = 0; a < nu; a++) gkp[a] += adj[PA.kp[a].i];
  orc::tape() = prev;
}

// One control step's vector-Jacobian product at a given state (see control_step_vjp); the
// parameter adjoints are accumulated (+=) into gmass / gdamp / gkp.
int orc_step_vjp(void* h, const double* q, const double* v, const double* u, int n_substeps, int solver_cap,
                 const double* mass, const double* damp, const double* kp, double* bq, double* bv, double* gu,
                 double* gmass, double* gdamp, double* gkp) {
  const Model& m = *static_cast<Model*>(h);
  orc::Params<double> P = make_params(m, mass, damp, kp);
  control_step_vjp(m, P, q, v, nullptr, u, n_substeps, solver_cap, bq, bv, gu, gmass, gdamp, gkp);
  return 0;
}

// Gradient of orc_rollout_loss by reverse mode: states are kept after every control step and
// each step is taped from its start state (inputs q, v, u and the parameters; the solver's
// warm start enters as a constant), then swept backward with the state adjoint of the next step.
int orc_rollout_grad(void* h, const double* q0, const double* v0, const double* ctrl, int T, int n_substeps,
                     int solver_cap, const double* mass, const double* damp, const double* kp, const double* wq,
                     const double* qs, const double* wv, const double* vs, double* gq0, double* gv0, double* gu,
                     double* gmass, double* gdamp, double* gkp, double* loss) {
  const Model& m = *static_cast<Model*>(h);
  const int nq = m.nq, nv = m.nv, nu = m.nu, nb = m.nbody;
  orc::Params<double> P = make_params(m, mass, damp, kp);
  std::vector<std::vector<double>> Q(T + 1), V(T + 1), Wm(T + 1);
  Q[0].assign(q0, q0 + nq); V[0].assign(v0, v0 + nv); Wm[0].assign(nv, 0.0);
  double L = 0;
  for (int t = 0; t < T; t++) {
    Q[t + 1] = Q[t]; V[t + 1] = V[t]; Wm[t + 1] = Wm[t];
    for (int s = 0; s < n_substeps; s++)
      orc::substep<double>(m, Q[t + 1].data(), V[t + 1].data(), Wm[t + 1].data(), ctrl + (size_t)t * nu, solver_cap, nullptr, &P);
    L += step_loss(m, Q[t + 1].data(), V[t + 1].data(), wq, qs, wv, vs);
  }
  if (loss) *loss = L;
  std::vector<double> bq(nq), bv(nv);
  for (int i = 0; i < nq; i++) bq[i] = 2 * wq[i] * (Q[T][i] - qs[i]);
  for (int i = 0; i < nv; i++) bv[i] = 2 * wv[i] * (V[T][i] - vs[i]);
  std::fill(gmass, gmass + nb, 0.0);
  std::fill(gdamp, gdamp + nv, 0.0);
  std::fill(gkp, gkp + nu, 0.0);
  for (int t = T - 1; t >= 0; t--) {
    control_step_vjp(m, P, Q[t].data(), V[t].data(), Wm[t].data(), ctrl + (size_t)t * nu, n_substeps, solver_cap,
                     bq.data(), bv.data(), gu + (size_t)t * nu, gmass, gdamp, gkp);
    if (t >= 1) {
      for (int i = 0; i < nq; i++) bq[i] += 2 * wq[i] * (Q[t][i] - qs[i]);
      for (int i = 0; i < nv; i++) bv[i] += 2 * wv[i] * (V[t][i] - vs[i]);
    }
  }
  std::memcpy(gq0, bq.data(), sizeof(double) * nq);
  std::memcpy(gv0, bv.data(), sizeof(double) * nv);
  return 0;
}

double orc_impedance(double r, const double* solimp) { return orc::impedance(r, solimp); }

void orc_solid_inertia(int type, const double* size, double m, double* out) { orc::solid_inertia(type, size, m, out); }

double orc_rotor_armature(double kg, double mr, double rr) { return orc::rotor_armature(kg, mr, rr); }

// Counting-scalar checks on textbook kernels of size n (all entries variable unless stated):
//   0 dense matrix-vector product y = A x                      (expect 2 n^2 - n)
//   1 the same with A a constant zero matrix                    (expect 0)
//   2 dense Cholesky factor and solve of an SPD matrix          (see the test for the formula)
//   3 leaves-first L^T D L factor and solve of an arrowhead (tree) matrix: dense diagonal,
//     first row/column, constant zeros elsewhere                 (no fill: 3 (n - 1) + ... )
// Returns the counted flops (all kinds summed) in *out.
int orc_count_selftest(int which, int n, double* out) {
  using orc::cdouble;
  if (n < 1) return -1;
  orc::Counts& C = orc::counts();
  C.clear();
  std::vector<cdouble> A((size_t)n * n), x(n), y(n);
  for (int i = 0; i < n; i++) {
    x[i] = cdouble::var(1.0 + 0.1 * i);
    for (int j = 0; j < n; j++) {
      const double v = (i == j ? n + 1.0 : 1.0 / (1.0 + i + j));
      if (which == 1) A[i * n + j] = cdouble(0.0);
      else if (which == 3 && i != j && i != 0 && j != 0) A[i * n + j] = cdouble(0.0);
      else A[i * n + j] = cdouble::var(v);
    }
  }
  if (which == 0 || which == 1) {
    for (int i = 0; i < n; i++) {
      cdouble s(0.0);
      for (int j = 0; j < n; j++) s = s + A[i * n + j] * x[j];
      y[i] = s;
    }
  } else if (which == 2) {
    if (!orc::cholesky(A, n)) return -2;
    orc::chol_solve(A, n, x);
  } else if (which == 3) {
    if (!orc::ldlt_leaves_first(A, n)) return -2;
    orc::ldlt_solve(A, n, x);
  } else {
    return -1;
  }
  double t = 0;
  for (int k = 0; k < orc::PH_N; k++) t += C.add[k] + C.mul[k] + C.div[k] + C.sqrt[k] + C.trans[k];
  *out = t;
  return 0;
}

// Counted flops of n_substeps substeps of one environment from (qpos, qvel, qacc_warm) with the
// controls ctrl held: the oracle on the counting scalar (orc_count.hpp).  Per substep s:
// counts[(s * 9 + phase) * 5 + {add, mul, div, sqrt, transcendental}] (phase 8: the contact-force
// output, not part of the step), rows[s] (constraint rows
// assembled) and iters[s] (Newton iterations).  The state is advanced in place.
int orc_count_substeps(void* h, double* qpos, double* qvel, double* qacc_warm, const double* ctrl, int n_substeps,
                       int solver_cap, double* counts, int* rows, int* iters) {
  const Model& m = *static_cast<Model*>(h);
  if (n_substeps < 1) return -1;
  using orc::cdouble;
  std::vector<cdouble> q(m.nq), v(m.nv), w(m.nv), u(std::max(m.nu, 1));
  for (int i = 0; i < m.nq; i++) q[i] = cdouble::var(qpos[i]);
  for (int i = 0; i < m.nv; i++) { v[i] = cdouble::var(qvel[i]); w[i] = cdouble::var(qacc_warm[i]); }
  for (int i = 0; i < m.nu; i++) u[i] = cdouble::var(ctrl[i]);
  orc::Counts& C = orc::counts();
  for (int s = 0; s < n_substeps; s++) {
    C.clear();
    orc::Forward<cdouble> F;
    orc::substep(m, q.data(), v.data(), w.data(), u.data(), solver_cap, &F);
    for (int k = 0; k < orc::PH_N; k++) {
      double* o = counts + ((size_t)s * orc::PH_N + k) * 5;
      o[0] = C.add[k]; o[1] = C.mul[k]; o[2] = C.div[k]; o[3] = C.sqrt[k]; o[4] = C.trans[k];
    }
    rows[s] = F.rows.n;
    iters[s] = F.sol.iterations;
  }
  for (int i = 0; i < m.nq; i++) qpos[i] = q[i].v;
  for (int i = 0; i < m.nv; i++) { qvel[i] = v[i].v; qacc_warm[i] = w[i].v; }
  return 0;
}

}  // extern "C"
