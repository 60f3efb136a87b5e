// FP64 oracle -- TEST INFRASTRUCTURE ONLY.  Derived model tables.
#include "orc_model.hpp"

#include <algorithm>
#include <cmath>

namespace orc {

static M3<double> quat_rot(const double* q) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double u[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
  return quat2mat(u);
}

std::string mesh_solid(const double* vert, int nv, const int* face, int nf, Solid& sd) {
  if (nv < 4 || nf < 4) return "a mesh needs at least 4 vertices and 4 faces";
  sd.vert.assign(vert, vert + 3 * (size_t)nv);
  sd.plane.clear();
  for (int t = 0; t < nf; t++) {
    V3<double> v[3];
    for (int j = 0; j < 3; j++) {
      const int i = face[3 * t + j];
      if (i < 0 || i >= nv) return "mesh face index out of range";
      v[j] = V3<double>{sd.vert[3 * i], sd.vert[3 * i + 1], sd.vert[3 * i + 2]};
    }
    V3<double> n = cross(sub(v[1], v[0]), sub(v[2], v[0]));
    n = scl(n, 1.0 / norm(n));
    const double off = dot(n, v[0]);
    for (int i = 0; i < nv; i++)
      if (n[0] * sd.vert[3 * i] + n[1] * sd.vert[3 * i + 1] + n[2] * sd.vert[3 * i + 2] > off + 1e-6)
        return "mesh is not convex or a face is not outward";
    sd.plane.insert(sd.plane.end(), {n[0], n[1], n[2], off});
  }
  return "";
}

// Volume, centroid and inertia about the centroid (unit density, the mesh's own axes) of the solid
// bounded by outward triangles: the sum over triangles of the tetrahedra they span with the
// vertices' mean o (an interior point of a convex hull), each by the exact integrals of a
// tetrahedron with one vertex at o -- volume det(a, b, c) / 6 and second moment
// V / 20 (a a^T + b b^T + c c^T + s s^T), s = a + b + c (positions relative to o).
static void mesh_mass(const Solid& sd, const int* face, int nface, double& vol, double com[3], double I[9]) {
  double o[3] = {0, 0, 0};
  const int nv = sd.nv();
  for (int i = 0; i < nv; i++)
    for (int k = 0; k < 3; k++) o[k] += sd.vert[3 * i + k] / nv;
  double first[3] = {0, 0, 0}, S[9] = {0};
  vol = 0;
  for (int t = 0; t < nface; t++) {
    double p[3][3];
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++) p[j][k] = sd.vert[3 * face[3 * t + j] + k] - o[k];
    const double V = (p[0][0] * (p[1][1] * p[2][2] - p[1][2] * p[2][1]) - p[0][1] * (p[1][0] * p[2][2] - p[1][2] * p[2][0]) +
                      p[0][2] * (p[1][0] * p[2][1] - p[1][1] * p[2][0])) / 6.0;
    double sum[3];
    for (int k = 0; k < 3; k++) sum[k] = p[0][k] + p[1][k] + p[2][k];
    vol += V;
    for (int k = 0; k < 3; k++) first[k] += V * sum[k] / 4.0;   // centroid of the tetrahedron: (0 + a + b + c) / 4
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++)
        S[3 * r + c] += V / 20.0 * (p[0][r] * p[0][c] + p[1][r] * p[1][c] + p[2][r] * p[2][c] + sum[r] * sum[c]);
  }
  double g[3];   // the centroid relative to o
  for (int k = 0; k < 3; k++) { g[k] = first[k] / vol; com[k] = o[k] + g[k]; }
  // second moment about the centroid, then inertia = tr(S) 1 - S
  double Sc[9];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) Sc[3 * r + c] = S[3 * r + c] - vol * g[r] * g[c];
  const double tr = Sc[0] + Sc[4] + Sc[8];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) I[3 * r + c] = (r == c ? tr : 0.0) - Sc[3 * r + c];
}

std::string compile_model(const Desc& d, Model& m) {
  if (d.nbody < 1) return "nbody must be >= 1 (body 0 is the world)";
  m.nbody = d.nbody; m.njnt = d.njnt; m.ngeom = d.ngeom; m.npair = d.npair; m.nu = d.nu;
  m.parent.assign(d.body_parent, d.body_parent + d.nbody);
  m.parent[0] = -1;
  for (int b = 1; b < m.nbody; b++)
    if (m.parent[b] < 0 || m.parent[b] >= b) return "body_parent must satisfy 0 <= parent[i] < i (level order)";
  m.body_pos.assign(d.body_pos, d.body_pos + 3 * d.nbody);
  m.body_quat.assign(d.body_quat, d.body_quat + 4 * d.nbody);
  for (int b = 0; b < m.nbody; b++) {   // normalise the offset quaternions
    double* q = &m.body_quat[4 * b];
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(n > 0)) return "body_quat must be non-zero";
    for (int k = 0; k < 4; k++) q[k] /= n;
  }
  // joints
  m.jnt_type.assign(d.jnt_type, d.jnt_type + d.njnt);
  m.jnt_body.assign(d.jnt_body, d.jnt_body + d.njnt);
  m.jnt_pos.assign(d.jnt_pos, d.jnt_pos + 3 * d.njnt);
  m.jnt_axis.assign(d.jnt_axis, d.jnt_axis + 3 * d.njnt);
  m.jnt_limited.assign(d.jnt_limited, d.jnt_limited + d.njnt);
  m.jnt_range.assign(d.jnt_range, d.jnt_range + 2 * d.njnt);
  m.body_jntadr.assign(m.nbody, 0);
  m.body_jntnum.assign(m.nbody, 0);
  m.nq = m.nv = 0;
  for (int j = 0; j < m.njnt; j++) {
    int b = m.jnt_body[j], t = m.jnt_type[j];
    if (b < 1 || b >= m.nbody) return "jnt_body out of range";
    if (j > 0 && m.jnt_body[j - 1] > b) return "joints must be grouped by body in body order";
    if (t != FREE && t != HINGE && t != SLIDE) return "unknown joint type";
    if (m.body_jntnum[b] == 0) m.body_jntadr[b] = j;
    m.body_jntnum[b]++;
    m.jnt_qposadr.push_back(m.nq);
    m.jnt_dofadr.push_back(m.nv);
    m.nq += t == FREE ? 7 : 1;
    m.nv += t == FREE ? 6 : 1;
    if (t != FREE) {
      double* a = &m.jnt_axis[3 * j];
      double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      if (!(n > 0)) return "joint axis must be non-zero";
      for (int k = 0; k < 3; k++) a[k] /= n;
      if (m.jnt_limited[j] && !(m.jnt_range[2 * j] < m.jnt_range[2 * j + 1])) return "limited joint needs range lo < hi";
    }
  }
  for (int j = 0; j < m.njnt; j++)
    if (m.jnt_type[j] == FREE && (m.parent[m.jnt_body[j]] != 0 || m.body_jntnum[m.jnt_body[j]] != 1))
      return "a free joint must be the only joint of a child of the world";
  // dofs and the dof tree (parent = previous dof of the body, else the last dof of the nearest
  // ancestor body that has dofs)
  m.dof_body.assign(m.nv, 0);
  m.dof_jnt.assign(m.nv, 0);
  m.dof_parent.assign(m.nv, -1);
  std::vector<int> body_lastdof(m.nbody, -1);
  for (int b = 1; b < m.nbody; b++) {
    int last = body_lastdof[m.parent[b]];
    for (int j = m.body_jntadr[b]; j < m.body_jntadr[b] + m.body_jntnum[b]; j++) {
      int n = m.jnt_type[j] == FREE ? 6 : 1;
      for (int k = 0; k < n; k++) {
        int dof = m.jnt_dofadr[j] + k;
        m.dof_body[dof] = b;
        m.dof_jnt[dof] = j;
        m.dof_parent[dof] = last;
        last = dof;
      }
    }
    body_lastdof[b] = last;
  }
  m.body_root.assign(m.nbody, 0);
  for (int b = 1; b < m.nbody; b++) m.body_root[b] = m.parent[b] == 0 ? b : m.body_root[m.parent[b]];
  m.dof_damping.assign(d.dof_damping, d.dof_damping + m.nv);
  m.dof_armature.assign(m.nv, 0.0);
  for (int i = 0; i < m.nv; i++)
    m.dof_armature[i] = d.dof_armature[i] + rotor_armature(d.dof_rotor[3 * i], d.dof_rotor[3 * i + 1], d.dof_rotor[3 * i + 2]);
  // geoms
  m.geom_type.assign(d.geom_type, d.geom_type + d.ngeom);
  m.geom_body.assign(d.geom_body, d.geom_body + d.ngeom);
  m.geom_pos.assign(d.geom_pos, d.geom_pos + 3 * d.ngeom);
  m.geom_quat.assign(d.geom_quat, d.geom_quat + 4 * d.ngeom);
  m.geom_size.assign(d.geom_size, d.geom_size + 3 * d.ngeom);
  m.geom_mass.assign(d.geom_mass, d.geom_mass + d.ngeom);
  for (int g = 0; g < m.ngeom; g++) {
    if (m.geom_type[g] < PLANE || m.geom_type[g] > MESH) return "unknown geom type";
    if (m.geom_body[g] < 0 || m.geom_body[g] >= m.nbody) return "geom_body out of range";
    if (m.geom_type[g] == HFIELD) {
      if (m.geom_body[g] != 0 || m.geom_mass[g] != 0) return "a heightfield must be a massless geom of the world";
      if (d.hfield_nrow < 2 || d.hfield_ncol < 2 || !d.hfield_data) return "a heightfield geom needs a grid of at least 2 x 2";
      if (!(m.geom_size[3 * g] > 0 && m.geom_size[3 * g + 1] > 0 && m.geom_size[3 * g + 2] >= 0))
        return "heightfield size must be (hx > 0, hy > 0, hz >= 0)";
    }
    double* q = &m.geom_quat[4 * g];
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(n > 0)) return "geom_quat must be non-zero";
    for (int k = 0; k < 4; k++) q[k] /= n;
  }
  if (d.hfield_nrow >= 2 && d.hfield_ncol >= 2 && d.hfield_data) {
    m.hf_nrow = d.hfield_nrow;
    m.hf_ncol = d.hfield_ncol;
    m.hfield.assign(d.hfield_data, d.hfield_data + (size_t)d.hfield_nrow * d.hfield_ncol);
    for (double e : m.hfield)
      if (!(e >= 0.0 && e <= 1.0)) return "heightfield elevations must lie in [0, 1]";
  }
  // convex meshes: vertices as given, face planes from the outward triangles, mass properties
  std::vector<double> mvol(d.nmesh), mcom(3 * (size_t)d.nmesh), mI(9 * (size_t)d.nmesh);
  for (int k = 0; k < d.nmesh; k++) {
    Solid sd;
    const int nv = d.mesh_vertnum[k], nf = d.mesh_facenum[k];
    const int* face = d.mesh_face + 3 * (size_t)d.mesh_faceadr[k];
    const std::string err = mesh_solid(d.mesh_vert + 3 * (size_t)d.mesh_vertadr[k], nv, face, nf, sd);
    if (!err.empty()) return err;
    mesh_mass(sd, face, nf, mvol[k], &mcom[3 * k], &mI[9 * k]);
    if (!(mvol[k] > 0)) return "mesh encloses no volume";
    m.meshes.push_back(sd);
  }
  m.geom_meshid.assign(m.ngeom, -1);
  for (int g = 0; g < m.ngeom; g++)
    if (m.geom_type[g] == MESH) {
      if (!d.geom_meshid || d.geom_meshid[g] < 0 || d.geom_meshid[g] >= d.nmesh) return "a mesh geom needs a mesh";
      m.geom_meshid[g] = d.geom_meshid[g];
    }
  // a geom's solid: centre of mass in the body frame and inertia about it in the body axes
  auto geom_solid = [&](int g, double c[3], double Ib[9]) {
    M3<double> R = quat_rot(&m.geom_quat[4 * g]);
    double Il[9] = {0}, off[3] = {0, 0, 0};
    const int mk = m.geom_meshid[g];
    if (mk >= 0) {
      for (int k = 0; k < 3; k++) off[k] = mcom[3 * mk + k];
      for (int k = 0; k < 9; k++) Il[k] = m.geom_mass[g] / mvol[mk] * mI[9 * mk + k];
    } else {
      double Id[3];
      solid_inertia(m.geom_type[g], &m.geom_size[3 * g], m.geom_mass[g], Id);
      for (int k = 0; k < 3; k++) Il[4 * k] = Id[k];
    }
    for (int r = 0; r < 3; r++) {
      c[r] = m.geom_pos[3 * g + r];
      for (int k = 0; k < 3; k++) c[r] += R[3 * r + k] * off[k];
    }
    for (int r = 0; r < 3; r++)
      for (int s2 = 0; s2 < 3; s2++) {
        double v = 0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) v += R[3 * r + a] * Il[3 * a + b] * R[3 * s2 + b];
        Ib[3 * r + s2] = v;
      }
  };
  // mass properties: given, or the union of the body's geoms as uniform solids
  m.mass.assign(m.nbody, 0.0);
  m.ipos.assign(3 * m.nbody, 0.0);
  m.inertia.assign(6 * m.nbody, 0.0);
  for (int b = 1; b < m.nbody; b++) {
    if (!d.body_geom_inertia[b]) {
      m.mass[b] = d.body_mass[b];
      for (int k = 0; k < 3; k++) m.ipos[3 * b + k] = d.body_ipos[3 * b + k];
      for (int k = 0; k < 6; k++) m.inertia[6 * b + k] = d.body_inertia[6 * b + k];
      continue;
    }
    double M = 0, c[3] = {0, 0, 0};
    for (int g = 0; g < m.ngeom; g++) {
      if (m.geom_body[g] != b || m.geom_mass[g] <= 0) continue;
      double gc[3], Ib[9];
      geom_solid(g, gc, Ib);
      M += m.geom_mass[g];
      for (int k = 0; k < 3; k++) c[k] += m.geom_mass[g] * gc[k];
    }
    if (M <= 0) continue;
    for (int k = 0; k < 3; k++) c[k] /= M;
    double I[9] = {0};
    for (int g = 0; g < m.ngeom; g++) {
      if (m.geom_body[g] != b || m.geom_mass[g] <= 0) continue;
      if (m.geom_type[g] == PLANE) return "a plane cannot carry mass";
      double gc[3], Ib[9];
      geom_solid(g, gc, Ib);
      double dv[3] = {gc[0] - c[0], gc[1] - c[1], gc[2] - c[2]};
      double dd = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
      for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) I[3 * r + s] += Ib[3 * r + s] + m.geom_mass[g] * ((r == s ? dd : 0.0) - dv[r] * dv[s]);
    }
    m.mass[b] = M;
    for (int k = 0; k < 3; k++) m.ipos[3 * b + k] = c[k];
    double six[6] = {I[0], I[4], I[8], I[1], I[2], I[5]};
    for (int k = 0; k < 6; k++) m.inertia[6 * b + k] = six[k];
  }
  // contact pairs and their static slots
  m.nslot = 0;
  for (int p = 0; p < m.npair; p++) {
    int g1 = d.pair_geom[2 * p], g2 = d.pair_geom[2 * p + 1];
    if (g1 < 0 || g1 >= m.ngeom || g2 < 0 || g2 >= m.ngeom) return "pair geom out of range";
    int n = pair_max_points(m.geom_type[g1], m.geom_type[g2]);
    if (n < 0) return "unsupported pair (geom1's type must not exceed geom2's: plane < sphere < capsule < box; a heightfield pairs as geom1 with spheres, capsules, boxes and meshes; a cylinder pairs with planes; a mesh with planes and heightfields)";
    if (d.pair_condim[p] != 1 && d.pair_condim[p] != 3) return "pair_condim must be 1 or 3";
    m.pair_g1.push_back(g1);
    m.pair_g2.push_back(g2);
    m.pair_condim.push_back(d.pair_condim[p]);
    m.pair_friction.push_back(d.pair_friction[p]);
    m.pair_slotadr.push_back(m.nslot);
    m.pair_nslot.push_back(n);
    m.nslot += n;
  }
  // actuators
  for (int a = 0; a < m.nu; a++) {
    int j = d.act_jnt[a];
    if (j < 0 || j >= m.njnt || m.jnt_type[j] == FREE) return "actuators act on hinge or slide joints";
    if (d.act_type[a] != MOTOR && d.act_type[a] != POSITION) return "unknown actuator type";
  }
  m.act_type.assign(d.act_type, d.act_type + d.nu);
  m.act_jnt.assign(d.act_jnt, d.act_jnt + d.nu);
  m.act_gear.assign(d.act_gear, d.act_gear + d.nu);
  m.act_kp.assign(d.act_kp, d.act_kp + d.nu);
  m.act_kd.assign(d.act_kd, d.act_kd + d.nu);
  m.act_ctrllimited.assign(d.act_ctrllimited, d.act_ctrllimited + d.nu);
  m.act_ctrlrange.assign(d.act_ctrlrange, d.act_ctrlrange + 2 * d.nu);
  m.act_forcelimited.assign(d.nu, 0);
  m.act_forcerange.assign(2 * d.nu, 0.0);
  for (int a = 0; a < d.nu; a++)
    if (d.act_forcelimited && d.act_forcelimited[a]) {
      if (!d.act_forcerange || !(d.act_forcerange[2 * a] <= d.act_forcerange[2 * a + 1]))
        return "act_forcerange must satisfy lo <= hi";
      m.act_forcelimited[a] = 1;
      m.act_forcerange[2 * a] = d.act_forcerange[2 * a];
      m.act_forcerange[2 * a + 1] = d.act_forcerange[2 * a + 1];
    }
  // options
  if (!(d.timestep > 0)) return "timestep must be > 0";
  m.timestep = d.timestep;
  for (int k = 0; k < 3; k++) m.gravity[k] = d.gravity[k];
  m.iterations = d.iterations;
  m.cone = d.cone;
  if (m.cone != PYRAMIDAL && m.cone != ELLIPTIC) return "unknown cone";
  m.impratio = d.impratio;
  if (m.cone == ELLIPTIC && m.impratio != 1.0) return "the elliptic cone is implemented for impratio = 1";
  for (int k = 0; k < 2; k++) m.solref[k] = d.solref[k];
  for (int k = 0; k < 5; k++) m.solimp[k] = d.solimp[k];
  m.margin = d.margin;
  m.max_contacts = d.max_contacts < 0 ? m.nslot : std::min(d.max_contacts, m.nslot);
  m.nlimited = 0;
  for (int j = 0; j < m.njnt; j++)
    if (m.jnt_limited[j] && m.jnt_type[j] != FREE) m.nlimited++;
  m.rows_per_contact = 4;
  m.dof_frictionloss.assign(m.nv, 0.0);
  m.nfric = 0;
  if (d.dof_frictionloss)
    for (int i = 0; i < m.nv; i++) {
      if (!(d.dof_frictionloss[i] >= 0.0)) return "dof_frictionloss must be >= 0";
      m.dof_frictionloss[i] = d.dof_frictionloss[i];
      if (d.dof_frictionloss[i] > 0) m.nfric++;
    }
  m.nrow_max = m.max_contacts * m.rows_per_contact + m.nlimited + m.nfric;
  return "";
}

}  // namespace orc
