// Host-side model compiler: validates a pg_model_desc, derives the tables the step kernel
// needs (levels, child lists, dof tree, packed LDL pattern, contact slots, mass properties,
// options) and packs them into one blob of 32-bit words (layout in pg_internal.h).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {

namespace {

struct Blob {
  std::vector<uint32_t> w;
  int ints(const std::vector<int>& v) {
    int o = (int)w.size();
    for (int x : v) w.push_back((uint32_t)x);
    return o;
  }
  int floats(const std::vector<float>& v) {
    int o = (int)w.size();
    for (float x : v) {
      uint32_t u;
      std::memcpy(&u, &x, 4);
      w.push_back(u);
    }
    return o;
  }
};

// points a primitive pair type can produce (its static slot count); -1: unsupported
int slots_for(int t1, int t2) {
  if (t1 == PG_GEOM_HFIELD)
    return t2 == PG_GEOM_SPHERE ? 1 : (t2 == PG_GEOM_CAPSULE ? 2 : (t2 == PG_GEOM_BOX || t2 == PG_GEOM_MESH ? 4 : -1));
  if (t2 == PG_GEOM_CYLINDER || t2 == PG_GEOM_MESH) return t1 == PG_GEOM_PLANE ? 4 : -1;
  static const int table[4][4] = {
      //            plane sphere capsule box
      /* plane   */ {-1, 1, 2, 4},
      /* sphere  */ {-1, 1, 1, 1},
      /* capsule */ {-1, -1, 1, 2},
      /* box     */ {-1, -1, -1, 4},
  };
  if (t1 < 0 || t1 > 3 || t2 < 0 || t2 > 3) return -1;
  return table[t1][t2];
}

// rotation matrix (row-major) of a quaternion, normalised here
void quat_matrix(const float* qin, double R[9]) {
  double w = qin[0], x = qin[1], y = qin[2], z = qin[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  double xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  R[0] = 1 - 2 * (yy + zz); R[1] = 2 * (xy - wz); R[2] = 2 * (xz + wy);
  R[3] = 2 * (xy + wz); R[4] = 1 - 2 * (xx + zz); R[5] = 2 * (yz - wx);
  R[6] = 2 * (xz - wy); R[7] = 2 * (yz + wx); R[8] = 1 - 2 * (xx + yy);
}

// principal moments of a uniform solid about its centre (geom axes)
void principal_moments(int type, const float* size, double m, double I[3]) {
  const double pi = 3.14159265358979323846;
  I[0] = I[1] = I[2] = 0.0;
  if (type == PG_GEOM_SPHERE) {
    double r = size[0];
    I[0] = I[1] = I[2] = 2.0 / 5.0 * m * r * r;
  } else if (type == PG_GEOM_BOX) {
    double X = 2.0 * size[0], Y = 2.0 * size[1], Z = 2.0 * size[2];
    I[0] = m / 12.0 * (Y * Y + Z * Z);
    I[1] = m / 12.0 * (X * X + Z * Z);
    I[2] = m / 12.0 * (X * X + Y * Y);
  } else if (type == PG_GEOM_CAPSULE) {
    // cylinder of length L plus two hemispherical caps, mass shared by volume
    double r = size[0], L = 2.0 * size[1];
    double v_cyl = pi * r * r * L, v_caps = 4.0 / 3.0 * pi * r * r * r;
    double m_cyl = m * v_cyl / (v_cyl + v_caps), m_cap = 0.5 * m * v_caps / (v_cyl + v_caps);   // per cap
    double cyl_axial = 0.5 * m_cyl * r * r, cyl_trans = m_cyl * (3.0 * r * r + L * L) / 12.0;
    double d = 0.5 * L + 3.0 * r / 8.0;   // cap centroid from the capsule centre
    double cap_axial = 0.4 * m_cap * r * r;
    double cap_trans = m_cap * (83.0 / 320.0) * r * r + m_cap * d * d;
    I[0] = I[1] = cyl_trans + 2.0 * cap_trans;
    I[2] = cyl_axial + 2.0 * cap_axial;
  } else if (type == PG_GEOM_CYLINDER) {
    double r = size[0], L = 2.0 * size[1];
    I[0] = I[1] = m * (3.0 * r * r + L * L) / 12.0;
    I[2] = 0.5 * m * r * r;
  }
}

int align4(int x) { return (x + 3) & ~3; }

// a convex mesh, checked: its outward face planes (n, offset: n . x <= offset inside) and the mass
// properties of the uniform solid hull of unit density (volume, centroid, inertia about the
// centroid in the geom axes), from signed tetrahedra on the origin and each outward triangle
struct MeshProps {
  std::vector<float> plane;   // 4 per face
  double vol = 0, com[3] = {0, 0, 0}, I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
};

int mesh_props(const float* v, int nvert, const int* f, int nface, MeshProps& out) {
  if (nvert < 4 || nface < 4) return set_error(PG_EINVAL, "a mesh needs at least 4 vertices and 4 faces");
  if (nvert > kMaxMeshVert || nface > kMaxMeshFace) return set_error(PG_ECAPACITY, "a mesh exceeds 32 vertices or 64 faces");
  double ext = 0, mid[3] = {0, 0, 0};
  for (int i = 0; i < nvert; i++)
    for (int k = 0; k < 3; k++) {
      if (!std::isfinite(v[3 * i + k])) return set_error(PG_EINVAL, "non-finite mesh vertex");
      ext = std::max(ext, std::fabs((double)v[3 * i + k]));
      mid[k] += v[3 * i + k] / (double)nvert;
    }
  double first[3] = {0, 0, 0}, C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  out.plane.assign(4 * (size_t)nface, 0.f);
  for (int t = 0; t < nface; t++) {
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; k++) {
      const int ia = f[3 * t], ib = f[3 * t + 1], ic = f[3 * t + 2];
      if (ia < 0 || ia >= nvert || ib < 0 || ib >= nvert || ic < 0 || ic >= nvert)
        return set_error(PG_EINVAL, "mesh face index out of range");
      a[k] = v[3 * ia + k]; b[k] = v[3 * ib + k]; c[k] = v[3 * ic + k];
    }
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(nn > 1e-12 * (ext * ext + 1e-30))) return set_error(PG_EINVAL, "degenerate mesh face");
    for (int k = 0; k < 3; k++) n[k] /= nn;
    const double off = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
    // outward: the vertices' mean lies inside, and no vertex lies outside the face's plane
    if (!(n[0] * mid[0] + n[1] * mid[1] + n[2] * mid[2] < off)) return set_error(PG_EINVAL, "mesh face not outward");
    for (int i = 0; i < nvert; i++)
      if (n[0] * v[3 * i] + n[1] * v[3 * i + 1] + n[2] * v[3 * i + 2] - off > 1e-5 * (ext + 1e-30))
        return set_error(PG_EINVAL, "mesh is not convex: a vertex lies outside a face's plane");
    for (int k = 0; k < 3; k++) out.plane[4 * t + k] = (float)n[k];
    out.plane[4 * t + 3] = (float)off;
    // signed tetrahedron (origin, a, b, c): volume, first moment, second moment about the origin
    const double V = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                      a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
    out.vol += V;
    const double sum[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
    for (int k = 0; k < 3; k++) first[k] += V * sum[k] / 4.0;
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++)
        C[r][q] += V / 20.0 * (a[r] * a[q] + b[r] * b[q] + c[r] * c[q] + sum[r] * sum[q]);
  }
  if (!(out.vol > 0)) return set_error(PG_EINVAL, "mesh encloses no volume");
  for (int k = 0; k < 3; k++) out.com[k] = first[k] / out.vol;
  const double tr = C[0][0] + C[1][1] + C[2][2];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) {
      // inertia about the origin, then moved to the centroid (parallel axes)
      const double Io = (r == q ? tr : 0.0) - C[r][q];
      const double c2 = out.com[0] * out.com[0] + out.com[1] * out.com[1] + out.com[2] * out.com[2];
      out.I[r][q] = Io - out.vol * ((r == q ? c2 : 0.0) - out.com[r] * out.com[q]);
    }
  return PG_OK;
}

}  // namespace

int compile_model(const pg_model_desc* d, pg_model* out) {
  if (!d) return set_error(PG_EINVAL, "desc is NULL");
  const int nbody = d->nbody, njnt = d->njnt, ngeom = d->ngeom, npair = d->npair, nu = d->nu;
  if (nbody < 1 || njnt < 0 || ngeom < 0 || npair < 0 || nu < 0) return set_error(PG_EINVAL, "negative counts");
  if (nbody > kMaxBody) return set_error(PG_ECAPACITY, "nbody exceeds the kernel limit (64)");
  if (!d->body_parent || !d->body_pos || !d->body_quat) return set_error(PG_EINVAL, "body arrays missing");
  // ---- tree ----
  std::vector<int> parent(d->body_parent, d->body_parent + nbody);
  parent[0] = -1;
  for (int b = 1; b < nbody; b++)
    if (parent[b] < 0 || parent[b] >= b) return set_error(PG_EINVAL, "body_parent violates level order (parent[i] < i)");
  std::vector<int> root(nbody, 0);
  for (int b = 1; b < nbody; b++) root[b] = parent[b] == 0 ? b : root[parent[b]];
  // ---- joints ----
  std::vector<int> jnt_type(njnt), jnt_body(njnt), qposadr(njnt), dofadr(njnt);
  std::vector<int> body_jntadr(nbody, 0), body_jntnum(nbody, 0);
  std::vector<float> jpos(3 * njnt), jaxis(3 * njnt), jrange(2 * njnt);
  int nq = 0, nv = 0;
  for (int j = 0; j < njnt; j++) {
    int t = d->jnt_type[j], b = d->jnt_body[j];
    if (t != PG_JNT_FREE && t != PG_JNT_HINGE && t != PG_JNT_SLIDE) return set_error(PG_EINVAL, "bad joint type");
    if (b < 1 || b >= nbody) return set_error(PG_EINVAL, "jnt_body out of range");
    if (j > 0 && d->jnt_body[j - 1] > b) return set_error(PG_EINVAL, "joints must be grouped by body, in body order");
    jnt_type[j] = t;
    jnt_body[j] = b;
    if (body_jntnum[b]++ == 0) body_jntadr[b] = j;
    qposadr[j] = nq;
    dofadr[j] = nv;
    nq += t == PG_JNT_FREE ? 7 : 1;
    nv += t == PG_JNT_FREE ? 6 : 1;
    double ax = d->jnt_axis[3 * j], ay = d->jnt_axis[3 * j + 1], az = d->jnt_axis[3 * j + 2];
    double an = std::sqrt(ax * ax + ay * ay + az * az);
    if (t != PG_JNT_FREE && !(an > 0)) return set_error(PG_EINVAL, "zero joint axis");
    if (t == PG_JNT_FREE) an = 1.0;
    jaxis[3 * j] = (float)(ax / an); jaxis[3 * j + 1] = (float)(ay / an); jaxis[3 * j + 2] = (float)(az / an);
    for (int k = 0; k < 3; k++) jpos[3 * j + k] = d->jnt_pos[3 * j + k];
    jrange[2 * j] = d->jnt_range[2 * j];
    jrange[2 * j + 1] = d->jnt_range[2 * j + 1];
    if (d->jnt_limited[j] && t != PG_JNT_FREE && !(jrange[2 * j] < jrange[2 * j + 1]))
      return set_error(PG_EINVAL, "limited joint needs range lo < hi");
  }
  for (int j = 0; j < njnt; j++)
    if (jnt_type[j] == PG_JNT_FREE && (parent[jnt_body[j]] != 0 || body_jntnum[jnt_body[j]] != 1))
      return set_error(PG_EINVAL, "a free joint must be the only joint of a child of the world");
  if (nv > kMaxNv) return set_error(PG_ECAPACITY, "nv exceeds the kernel limit (64)");
  // ---- dof tree: each dof's parent is the previous dof on its body, else the last dof of the
  // nearest ancestor body with dofs ----
  std::vector<int> dof_body(nv), dof_parent(nv, -1), depth(nv, 0);
  std::vector<int> last_dof(nbody, -1);
  std::vector<uint64_t> mask(nbody, 0);
  for (int b = 1; b < nbody; b++) {
    int prev = last_dof[parent[b]];
    mask[b] = mask[parent[b]];
    for (int j = body_jntadr[b]; j < body_jntadr[b] + body_jntnum[b]; j++) {
      int n = jnt_type[j] == PG_JNT_FREE ? 6 : 1;
      for (int k = 0; k < n; k++) {
        int dof = dofadr[j] + k;
        dof_body[dof] = b;
        dof_parent[dof] = prev;
        depth[dof] = prev < 0 ? 0 : depth[prev] + 1;
        mask[b] |= (uint64_t)1 << dof;
        prev = dof;
      }
    }
    last_dof[b] = prev;
  }
  std::vector<int> rowadr(nv), Lcol;
  for (int i = 0; i < nv; i++) {
    rowadr[i] = (int)Lcol.size();
    for (int a = i; a >= 0; a = dof_parent[a]) Lcol.push_back(a);
  }
  const int nL = (int)Lcol.size();
  // ---- convex meshes ----
  const int nmesh = d->nmesh;
  if (nmesh < 0) return set_error(PG_EINVAL, "negative nmesh");
  if (nmesh > 0 && (!d->mesh_vertadr || !d->mesh_vertnum || !d->mesh_vert || !d->mesh_faceadr || !d->mesh_facenum ||
                    !d->mesh_face))
    return set_error(PG_EINVAL, "mesh arrays missing");
  std::vector<MeshProps> mprops(nmesh);
  std::vector<int> mvadr(nmesh), mvnum(nmesh), mfadr(nmesh), mfnum(nmesh);
  std::vector<float> mvert, mplane;
  for (int k = 0; k < nmesh; k++) {
    const int va = d->mesh_vertadr[k], vn = d->mesh_vertnum[k], fa = d->mesh_faceadr[k], fn = d->mesh_facenum[k];
    if (va < 0 || fa < 0) return set_error(PG_EINVAL, "negative mesh address");
    const int rc = mesh_props(d->mesh_vert + 3 * (size_t)va, vn, d->mesh_face + 3 * (size_t)fa, fn, mprops[k]);
    if (rc != PG_OK) return rc;
    mvadr[k] = (int)(mvert.size() / 3); mvnum[k] = vn;
    mfadr[k] = (int)(mplane.size() / 4); mfnum[k] = fn;
    mvert.insert(mvert.end(), d->mesh_vert + 3 * (size_t)va, d->mesh_vert + 3 * ((size_t)va + vn));
    mplane.insert(mplane.end(), mprops[k].plane.begin(), mprops[k].plane.end());
  }
  std::vector<int> gmesh(ngeom, -1);
  for (int g = 0; g < ngeom; g++)
    if (d->geom_type[g] == PG_GEOM_MESH) {
      if (!d->geom_meshid || d->geom_meshid[g] < 0 || d->geom_meshid[g] >= nmesh)
        return set_error(PG_EINVAL, "a mesh geom needs a valid geom_meshid");
      gmesh[g] = d->geom_meshid[g];
    }
  // a geom's solid: its centre of mass in the body frame and its inertia about it in the geom axes
  auto geom_solid = [&](int g, double com[3], double Il[3][3]) {
    for (int a = 0; a < 3; a++)
      for (int c = 0; c < 3; c++) Il[a][c] = 0.0;
    double R[9];
    quat_matrix(d->geom_quat + 4 * g, R);
    const double m = d->geom_mass[g];
    double off[3] = {0, 0, 0};
    if (gmesh[g] >= 0) {
      const MeshProps& mp = mprops[gmesh[g]];
      for (int k = 0; k < 3; k++) off[k] = mp.com[k];
      for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) Il[a][c] = m / mp.vol * mp.I[a][c];
    } else {
      double Ip[3];
      principal_moments(d->geom_type[g], d->geom_size + 3 * g, m, Ip);
      for (int a = 0; a < 3; a++) Il[a][a] = Ip[a];
    }
    for (int k = 0; k < 3; k++) com[k] = d->geom_pos[3 * g + k] + R[3 * k] * off[0] + R[3 * k + 1] * off[1] + R[3 * k + 2] * off[2];
  };
  // ---- mass properties ----
  std::vector<float> mass(nbody, 0.f), ipos(3 * nbody, 0.f), inertia(6 * nbody, 0.f);
  for (int b = 1; b < nbody; b++) {
    if (!(d->body_geom_inertia && d->body_geom_inertia[b])) {
      mass[b] = d->body_mass[b];
      for (int k = 0; k < 3; k++) ipos[3 * b + k] = d->body_ipos[3 * b + k];
      for (int k = 0; k < 6; k++) inertia[6 * b + k] = d->body_inertia[6 * b + k];
      continue;
    }
    double M = 0, com[3] = {0, 0, 0};
    for (int g = 0; g < ngeom; g++)
      if (d->geom_body[g] == b && d->geom_mass[g] > 0) {
        double gc[3], Il[3][3];
        geom_solid(g, gc, Il);
        M += d->geom_mass[g];
        for (int k = 0; k < 3; k++) com[k] += d->geom_mass[g] * gc[k];
      }
    if (!(M > 0)) continue;
    for (int k = 0; k < 3; k++) com[k] /= M;
    double I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int g = 0; g < ngeom; g++) {
      if (d->geom_body[g] != b || !(d->geom_mass[g] > 0)) continue;
      if (d->geom_type[g] == PG_GEOM_PLANE) return set_error(PG_EINVAL, "a plane geom cannot carry mass");
      double R[9], gc[3], Il[3][3];
      quat_matrix(d->geom_quat + 4 * g, R);
      geom_solid(g, gc, Il);
      double r[3];
      for (int k = 0; k < 3; k++) r[k] = gc[k] - com[k];
      double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) {
          double rot = 0.0;   // R Il R^T
          for (int u = 0; u < 3; u++)
            for (int w = 0; w < 3; w++) rot += R[3 * a + u] * Il[u][w] * R[3 * c + w];
          double shift = d->geom_mass[g] * ((a == c ? r2 : 0.0) - r[a] * r[c]);
          I[a][c] += rot + shift;
        }
    }
    mass[b] = (float)M;
    for (int k = 0; k < 3; k++) ipos[3 * b + k] = (float)com[k];
    inertia[6 * b + 0] = (float)I[0][0]; inertia[6 * b + 1] = (float)I[1][1]; inertia[6 * b + 2] = (float)I[2][2];
    inertia[6 * b + 3] = (float)I[0][1]; inertia[6 * b + 4] = (float)I[0][2]; inertia[6 * b + 5] = (float)I[1][2];
  }
  // ---- dofs ----
  std::vector<float> damping(nv), armature(nv);
  for (int i = 0; i < nv; i++) {
    damping[i] = d->dof_damping ? d->dof_damping[i] : 0.f;
    double arm = d->dof_armature ? d->dof_armature[i] : 0.0;
    if (d->dof_rotor) {
      double kg = d->dof_rotor[3 * i], mr = d->dof_rotor[3 * i + 1], rr = d->dof_rotor[3 * i + 2];
      double Ir = 0.5 * mr * rr * rr;   // uniform rotor disc
      arm += kg * kg * Ir;               // reflected through the gearbox
    }
    armature[i] = (float)arm;
  }
  // ---- geoms and pairs ----
  std::vector<int> gtype(d->geom_type, d->geom_type + ngeom), gbody(d->geom_body, d->geom_body + ngeom);
  std::vector<float> gpos(d->geom_pos, d->geom_pos + 3 * ngeom), gquat(4 * ngeom), gsize(d->geom_size, d->geom_size + 3 * ngeom);
  for (int g = 0; g < ngeom; g++) {
    if (gtype[g] < PG_GEOM_PLANE || gtype[g] > PG_GEOM_MESH) return set_error(PG_EINVAL, "bad geom type");
    if (gbody[g] < 0 || gbody[g] >= nbody) return set_error(PG_EINVAL, "geom_body out of range");
    if (gtype[g] == PG_GEOM_HFIELD) {
      if (gbody[g] != 0 || d->geom_mass[g] != 0.f) return set_error(PG_EINVAL, "a heightfield must be a massless geom of the world");
      if (d->hfield_nrow < 2 || d->hfield_ncol < 2 || !d->hfield_data)
        return set_error(PG_EINVAL, "a heightfield geom needs hfield_data of at least 2 x 2 elevations");
      if (!(gsize[3 * g] > 0.f && gsize[3 * g + 1] > 0.f && gsize[3 * g + 2] >= 0.f))
        return set_error(PG_EINVAL, "heightfield size must be (hx > 0, hy > 0, hz >= 0)");
    }
    double q[4], n = 0;
    for (int k = 0; k < 4; k++) { q[k] = d->geom_quat[4 * g + k]; n += q[k] * q[k]; }
    n = std::sqrt(n);
    if (!(n > 0)) return set_error(PG_EINVAL, "zero geom quaternion");
    for (int k = 0; k < 4; k++) gquat[4 * g + k] = (float)(q[k] / n);
  }
  std::vector<float> hfield;
  if (d->hfield_data && d->hfield_nrow >= 2 && d->hfield_ncol >= 2) {
    if ((int64_t)d->hfield_nrow * d->hfield_ncol > (1 << 24)) return set_error(PG_ECAPACITY, "heightfield larger than 2^24 samples");
    hfield.assign(d->hfield_data, d->hfield_data + (size_t)d->hfield_nrow * d->hfield_ncol);
    for (float e : hfield)
      if (!(e >= 0.f && e <= 1.f)) return set_error(PG_EINVAL, "heightfield elevations must lie in [0, 1]");
  }
  std::vector<int> pg1(npair), pg2(npair), pcondim(npair), pslotadr(npair), pnslot(npair);
  std::vector<float> pfric(npair);
  int nslot = 0;
  for (int p = 0; p < npair; p++) {
    int a = d->pair_geom[2 * p], b = d->pair_geom[2 * p + 1];
    if (a < 0 || a >= ngeom || b < 0 || b >= ngeom) return set_error(PG_EINVAL, "pair geom out of range");
    int n = slots_for(gtype[a], gtype[b]);
    if (n < 0) return set_error(PG_EUNSUPPORTED, "unsupported pair: type(geom1) must not exceed type(geom2) (plane<sphere<capsule<box), plane-plane unsupported; a heightfield pairs as geom1 with spheres, capsules, boxes and meshes; a cylinder pairs as geom2 with a plane; a mesh as geom2 with a plane or a heightfield");
    if (d->pair_condim[p] != 1 && d->pair_condim[p] != 3) return set_error(PG_EUNSUPPORTED, "pair_condim must be 1 or 3");
    pg1[p] = a; pg2[p] = b; pcondim[p] = d->pair_condim[p]; pfric[p] = d->pair_friction[p];
    pslotadr[p] = nslot; pnslot[p] = n;
    nslot += n;
  }
  if (nslot > kMaxSlot) return set_error(PG_ECAPACITY, "candidate contact slots exceed the kernel limit (64)");
  // ---- actuators ----
  std::vector<int> atype(nu), adof(nu), aqadr(nu), aclim(nu), aflim(nu, 0);
  std::vector<float> agear(nu), akp(nu), akd(nu), arange(2 * nu), afrange(2 * nu, 0.f);
  for (int a = 0; a < nu; a++) {
    int j = d->act_jnt[a];
    if (j < 0 || j >= njnt || jnt_type[j] == PG_JNT_FREE) return set_error(PG_EINVAL, "actuators drive hinge or slide joints");
    if (d->act_type[a] != PG_ACT_MOTOR && d->act_type[a] != PG_ACT_POSITION) return set_error(PG_EINVAL, "bad actuator type");
    atype[a] = d->act_type[a]; adof[a] = dofadr[j]; aqadr[a] = qposadr[j]; aclim[a] = d->act_ctrllimited[a];
    agear[a] = d->act_gear[a]; akp[a] = d->act_kp[a]; akd[a] = d->act_kd[a];
    arange[2 * a] = d->act_ctrlrange[2 * a]; arange[2 * a + 1] = d->act_ctrlrange[2 * a + 1];
    if (d->act_forcelimited && d->act_forcelimited[a]) {
      if (!d->act_forcerange) return set_error(PG_EINVAL, "act_forcelimited needs act_forcerange");
      const float lo = d->act_forcerange[2 * a], hi = d->act_forcerange[2 * a + 1];
      if (!(lo <= hi)) return set_error(PG_EINVAL, "act_forcerange must satisfy lo <= hi");
      aflim[a] = 1; afrange[2 * a] = lo; afrange[2 * a + 1] = hi;
    }
  }
  std::vector<int> limit_jnt;
  for (int j = 0; j < njnt; j++)
    if (d->jnt_limited[j] && jnt_type[j] != PG_JNT_FREE) limit_jnt.push_back(j);
  // ---- pair columns: the dofs whose contact-Jacobian column can be non-zero, i.e. the dofs on
  // exactly one of the two bodies' chains (shared ancestors cancel), sorted deepest first, with
  // sign +1 for geom2's side and -1 for geom1's.  When every pair's columns form one chain the
  // Newton Hessian keeps M's ancestor pattern and is factorised like M. ----
  std::vector<int> pcoladr(npair), pncol(npair), col_dof, col_sign, slot_pair(std::max(nslot, 1), 0);
  int tree_hessian = 1, ncol_max = 1;
  for (int p = 0; p < npair; p++) {
    const int b1 = gbody[pg1[p]], b2 = gbody[pg2[p]];
    pcoladr[p] = (int)col_dof.size();
    for (int dof = nv - 1; dof >= 0; dof--) {
      const bool in1 = (mask[b1] >> dof) & 1u, in2 = (mask[b2] >> dof) & 1u;
      if (in1 == in2) continue;
      col_dof.push_back(dof);
      col_sign.push_back(in2 ? 1 : -1);
    }
    pncol[p] = (int)col_dof.size() - pcoladr[p];
    ncol_max = std::max(ncol_max, pncol[p]);
    for (int a = pcoladr[p] + 1; a < (int)col_dof.size(); a++) {
      // each column must be the parent dof of the previous one (one chain, consecutive depths:
      // column b of column a's row then sits b - a entries into that packed row)
      if (dof_parent[col_dof[a - 1]] != col_dof[a]) tree_hessian = 0;
    }
    for (int s = pslotadr[p]; s < pslotadr[p] + pnslot[p]; s++) slot_pair[s] = p;
  }
  std::vector<int> root_freeadr(nbody, -1);
  for (int j = 0; j < njnt; j++)
    if (jnt_type[j] == PG_JNT_FREE) root_freeadr[jnt_body[j]] = qposadr[j];
  // ---- options ----
  if (!(d->timestep > 0)) return set_error(PG_EINVAL, "timestep must be > 0");
  if (d->iterations < 1) return set_error(PG_EINVAL, "iterations must be >= 1");
  if (d->cone != PG_CONE_PYRAMIDAL && d->cone != PG_CONE_ELLIPTIC) return set_error(PG_EINVAL, "unknown cone");
  if (d->cone == PG_CONE_ELLIPTIC && d->impratio != 1.f)
    return set_error(PG_EUNSUPPORTED, "the elliptic cone is implemented for impratio = 1");
  int max_contacts = d->max_contacts < 0 ? nslot : std::min(d->max_contacts, nslot);
  // joint friction loss: one two-sided row per dof with a positive loss, after the limit rows
  std::vector<int> fric_dof;
  std::vector<float> fric_F;
  if (d->dof_frictionloss)
    for (int i = 0; i < nv; i++) {
      const float F = d->dof_frictionloss[i];
      if (!(F >= 0.f) || !std::isfinite(F)) return set_error(PG_EINVAL, "dof_frictionloss must be finite and >= 0");
      if (F > 0.f) { fric_dof.push_back(i); fric_F.push_back(F); }
    }
  int nrow_max = 4 * max_contacts + (int)limit_jnt.size() + (int)fric_dof.size();
  if (nrow_max > kMaxRow) return set_error(PG_ECAPACITY, "constraint rows exceed the kernel limit (128)");

  ModelHdr h;
  std::memset(&h, 0, sizeof(h));
  h.nbody = nbody; h.njnt = njnt; h.nq = nq; h.nv = nv; h.nu = nu; h.ngeom = ngeom; h.npair = npair;
  h.nslot = nslot; h.nrow_max = nrow_max; h.max_contacts = max_contacts; h.nlimited = (int)limit_jnt.size();
  h.nL = nL; h.cap = d->iterations; h.cone = d->cone; h.tree_hessian = tree_hessian; h.ncol_max = ncol_max;
  h.h = d->timestep;
  h.substeps = std::max(d->substeps, 1);
  h.hf_nrow = hfield.empty() ? 0 : d->hfield_nrow;
  h.hf_ncol = hfield.empty() ? 0 : d->hfield_ncol;
  for (int k = 0; k < 3; k++) h.grav[k] = d->gravity[k];
  {
    double tc = std::max((double)d->solref[0], 2.0 * (double)d->timestep), zeta = d->solref[1], dmax = d->solimp[1];
    h.kref = (float)(1.0 / (dmax * dmax * tc * tc * zeta * zeta));
    h.bref = (float)(2.0 / (dmax * tc));
  }
  for (int k = 0; k < 5; k++) h.solimp[k] = d->solimp[k];
  h.imp_mid_inv = (float)(1.0 / std::pow((double)d->solimp[3], (double)d->solimp[4] - 1.0));
  h.imp_tail_inv = (float)(1.0 / std::pow(1.0 - (double)d->solimp[3], (double)d->solimp[4] - 1.0));
  h.margin = d->margin;

  Blob B;
  B.w.assign(kHdrWords, 0u);
  std::vector<float> bpos(d->body_pos, d->body_pos + 3 * nbody), bquat(4 * nbody);
  for (int b = 0; b < nbody; b++) {
    double n = 0;
    for (int k = 0; k < 4; k++) n += (double)d->body_quat[4 * b + k] * d->body_quat[4 * b + k];
    n = std::sqrt(n);
    if (!(n > 0)) return set_error(PG_EINVAL, "zero body quaternion");
    for (int k = 0; k < 4; k++) bquat[4 * b + k] = (float)(d->body_quat[4 * b + k] / n);
  }
  h.o_body_parent = B.ints(parent); h.o_body_root = B.ints(root);
  h.o_body_jntadr = B.ints(body_jntadr); h.o_body_jntnum = B.ints(body_jntnum);
  h.o_body_pos = B.floats(bpos); h.o_body_quat = B.floats(bquat); h.o_body_mass = B.floats(mass);
  h.o_body_ipos = B.floats(ipos); h.o_body_inertia = B.floats(inertia); h.o_root_freeadr = B.ints(root_freeadr);
  h.o_jnt_type = B.ints(jnt_type); h.o_jnt_qposadr = B.ints(qposadr); h.o_jnt_dofadr = B.ints(dofadr);
  h.o_jnt_pos = B.floats(jpos); h.o_jnt_axis = B.floats(jaxis); h.o_jnt_range = B.floats(jrange);
  h.o_dof_body = B.ints(dof_body); h.o_dof_depth = B.ints(depth); h.o_dof_rowadr = B.ints(rowadr);
  h.o_dof_damping = B.floats(damping); h.o_dof_armature = B.floats(armature); h.o_Lcol = B.ints(Lcol);
  h.o_geom_type = B.ints(gtype); h.o_geom_body = B.ints(gbody); h.o_geom_pos = B.floats(gpos);
  h.o_geom_quat = B.floats(gquat); h.o_geom_size = B.floats(gsize);
  h.o_pair_g1 = B.ints(pg1); h.o_pair_g2 = B.ints(pg2); h.o_pair_friction = B.floats(pfric);
  h.o_pair_condim = B.ints(pcondim); h.o_pair_slotadr = B.ints(pslotadr); h.o_pair_nslot = B.ints(pnslot);
  h.o_pair_coladr = B.ints(pcoladr); h.o_pair_ncol = B.ints(pncol); h.o_col_dof = B.ints(col_dof);
  h.o_col_sign = B.ints(col_sign); h.o_slot_pair = B.ints(slot_pair);
  h.o_act_type = B.ints(atype); h.o_act_dof = B.ints(adof); h.o_act_qposadr = B.ints(aqadr);
  h.o_act_gear = B.floats(agear); h.o_act_kp = B.floats(akp); h.o_act_kd = B.floats(akd);
  h.o_act_ctrllimited = B.ints(aclim); h.o_act_range = B.floats(arange);
  h.o_act_forcelimited = B.ints(aflim); h.o_act_forcerange = B.floats(afrange);
  h.dr_com = 2;
  h.dr_arm = 2 + 3 * nbody;
  h.dr_cal = 2 + 3 * nbody + nv;
  h.dr_kp = h.dr_cal + nu;
  h.dr_kd = h.dr_kp + nu;
  h.dr_mass = h.dr_kd + nu;
  h.dr_fric = h.dr_mass + nbody;
  h.nrand = h.dr_fric + nv;
  h.o_limit_jnt = B.ints(limit_jnt);
  h.nfric = (int)fric_dof.size();
  h.o_fric_dof = B.ints(fric_dof); h.o_fric_F = B.floats(fric_F);
  h.nmesh = nmesh;
  h.o_mesh_vertadr = B.ints(mvadr); h.o_mesh_vertnum = B.ints(mvnum); h.o_mesh_vert = B.floats(mvert);
  h.o_mesh_faceadr = B.ints(mfadr); h.o_mesh_facenum = B.ints(mfnum); h.o_mesh_plane = B.floats(mplane);
  h.o_geom_meshid = B.ints(gmesh);
  while (B.w.size() % 4) B.w.push_back(0u);
  h.words = (int)B.w.size();

  // ---- per-env workspace: buffers with the phase interval in which they are live, packed
  // first-fit.  Phases: 0 state, 1 kinematics, 2 RNEA, 3 CRBA, 4 LDL, 5 smooth acceleration,
  // 6 collision, 7 Jacobians, 8 row parameters, 9 Newton, 10 integration / diagnostics. ----
  struct Buf { int* off; int size; int birth, death; };
  const int R = std::max(nrow_max, 1), C = std::max(max_contacts, 1);
  const int Hsize = tree_hessian ? 0 : nv * nv;
  std::vector<Buf> bufs = {
      {&h.w_qpos, nq, 0, 10}, {&h.w_qvel, nv, 0, 10}, {&h.w_warm, nv, 0, 10},
      {&h.w_xpos, 3 * nbody, 1, 7}, {&h.w_xquat, 4 * nbody, 1, 7}, {&h.w_cdof, 6 * nv, 1, 7},
      {&h.w_cinert, 10 * nbody, 1, 3}, {&h.w_cvel, 6 * nbody, 2, 2}, {&h.w_cacc, 6 * nbody, 2, 2},
      {&h.w_cfrc, 6 * nbody, 2, 2}, {&h.w_bias, nv, 2, 5}, {&h.w_M, nL, 3, 9}, {&h.w_L, nL, 4, 9},
      {&h.w_a0, nv, 5, 9}, {&h.w_Dinv, nv, 5, 8}, {&h.w_con, kConFloats * C, 6, 10}, {&h.w_J, 3 * ncol_max * C, 7, 10},
      {&h.w_gcol, ncol_max * C, 7, 10}, {&h.w_lsgn, std::max((int)limit_jnt.size(), 1), 7, 10},
      {&h.w_gmu, C, 8, 10}, {&h.w_gcond, C, 8, 10},
      {&h.w_z, 3 * nv, 8, 8}, {&h.w_rr, R, 8, 10}, {&h.w_rv, R, 8, 10},
      {&h.w_Ahat, R, 8, 10}, {&h.w_imp, R, 8, 10}, {&h.w_aref, R, 8, 10}, {&h.w_rD, R, 8, 10},
      {&h.w_jar, R, 9, 10}, {&h.w_Jp, R, 9, 9}, {&h.w_bp, R, 9, 9}, {&h.w_a, nv, 9, 10}, {&h.w_g, nv, 9, 9}, {&h.w_p, nv, 9, 9},
      {&h.w_t, nv, 9, 9}, {&h.w_H, Hsize, 9, 9}};
  std::vector<std::array<int, 4>> placed;   // offset, size, birth, death
  int ws = 0;
  for (Buf& b : bufs) {
    int off = 0;
    bool moved = true;
    while (moved) {
      moved = false;
      for (auto& q : placed) {
        const bool overlap_t = !(b.death < q[2] || q[3] < b.birth);
        const bool overlap_s = off < q[0] + q[1] && q[0] < off + b.size;
        if (overlap_t && overlap_s) { off = q[0] + q[1]; moved = true; }
      }
    }
    *b.off = off;
    placed.push_back({off, b.size, b.birth, b.death});
    ws = std::max(ws, off + b.size);
  }
  h.ws_floats = std::max(ws, 1);
  // ---- adjoint layout: the buffers of the reverse sweep's substep, packed by lifetime like the
  // forward's.  Phases: 0 the running state adjoint (across substeps), 1 forward recompute,
  // 2 integration reverse and lambda = H^-1 abar, 3 forces and constraint rows, 4 CRBA,
  // 5 composite-to-own inertias and RNEA, 6 inertia wrenches, 7 inward sweep. ----
  {
    ModelHdr& g = out->hdr_adj;
    g = h;
    const int RA = std::max(nrow_max, 1), CA = std::max(max_contacts, 1);
    struct ABuf { int* off; int size; int birth, death; };
    std::vector<ABuf> ab = {
        {&g.b_q, nq, 0, 7}, {&g.b_v, nv, 0, 7},
        {&g.w_qpos, nq, 1, 7}, {&g.w_qvel, nv, 1, 5}, {&g.w_a, nv, 1, 3},
        {&g.w_xpos, 3 * nbody, 1, 7}, {&g.w_xquat, 4 * nbody, 1, 7}, {&g.w_cdof, 6 * nv, 1, 7},
        {&g.w_cinert, 10 * nbody, 1, 4}, {&g.w_ci0, 10 * nbody, 1, 5},
        {&g.w_cvel, 6 * nbody, 1, 5}, {&g.w_cacc, 6 * nbody, 1, 5}, {&g.w_cfrc, 6 * nbody, 1, 5},
        {&g.w_M, nL, 1, 2}, {&g.w_L, nL, 1, 3},
        {&g.w_con, kConFloats * CA, 1, 3}, {&g.w_J, 3 * ncol_max * CA, 1, 3}, {&g.w_gcol, ncol_max * CA, 1, 3},
        {&g.w_lsgn, std::max((int)limit_jnt.size(), 1), 1, 3}, {&g.w_gmu, CA, 1, 3}, {&g.w_gcond, CA, 1, 3},
        {&g.w_rr, RA, 1, 3}, {&g.w_Ahat, RA, 1, 3}, {&g.w_imp, RA, 1, 3}, {&g.w_rD, RA, 1, 3},
        {&g.w_jar, RA, 1, 3}, {&g.w_Jp, RA, 1, 3},
        // used by the forward recompute only
        {&g.w_warm, nv, 1, 1}, {&g.w_bias, nv, 1, 1}, {&g.w_a0, nv, 1, 1}, {&g.w_Dinv, nv, 1, 1},
        {&g.w_z, 3 * nv, 1, 1}, {&g.w_rv, RA, 1, 1}, {&g.w_aref, RA, 1, 1}, {&g.w_g, nv, 1, 1},
        {&g.w_p, nv, 1, 1}, {&g.w_t, nv, 1, 1}, {&g.w_H, tree_hessian ? 0 : nv * nv, 1, 1}, {&g.w_bp, RA, 1, 1},
        // the reverse sweep's own
        {&g.w_HL, nL, 2, 2}, {&g.b_a, nv, 2, 3}, {&g.b_bias, nv, 3, 5}, {&g.b_M, nL, 3, 4},
        {&g.b_cdof, 6 * nv, 3, 7}, {&g.b_I, 10 * nbody, 3, 6}, {&g.b_wr, 6 * nbody, 3, 7}, {&g.b_w, 3 * nv, 3, 3},
        {&g.b_vel, 6 * nbody, 5, 5}, {&g.b_acc, 6 * nbody, 5, 5}, {&g.b_frc, 6 * nbody, 5, 5}};
    std::vector<std::array<int, 4>> put;
    int top = 0;
    for (ABuf& b : ab) {
      int off = 0;
      bool moved = true;
      while (moved) {
        moved = false;
        for (auto& q : put) {
          const bool overlap_t = !(b.death < q[2] || q[3] < b.birth);
          const bool overlap_s = off < q[0] + q[1] && q[0] < off + b.size;
          if (overlap_t && overlap_s) { off = q[0] + q[1]; moved = true; }
        }
      }
      *b.off = off;
      put.push_back({off, b.size, b.birth, b.death});
      top = std::max(top, off + b.size);
    }
    g.ws_adj_floats = std::max(top, 1);
    // scope of the hand-written adjoint: contacts only between a world-fixed plane or heightfield
    // (geom1) and a sphere, capsule, box or (on a plane) cylinder, which keeps the Newton Hessian
    // on the mass matrix's pattern
    bool ok = true;
    for (int p = 0; p < npair; p++) {
      const int g1 = d->pair_geom[2 * p], g2 = d->pair_geom[2 * p + 1];
      const bool ground = d->geom_type[g1] == PG_GEOM_PLANE || d->geom_type[g1] == PG_GEOM_HFIELD;
      if (!ground || d->geom_body[g1] != 0 || d->geom_type[g2] == PG_GEOM_PLANE || d->geom_type[g2] == PG_GEOM_MESH ||
          (d->geom_type[g1] == PG_GEOM_HFIELD && (d->geom_type[g2] == PG_GEOM_CYLINDER || d->geom_type[g2] == PG_GEOM_BOX)))
        ok = false;
    }
    if (npair > 0 && !tree_hessian) ok = false;
    if (d->cone == PG_CONE_ELLIPTIC) ok = false;
    g.adj_ok = ok ? 1 : 0;
    h.adj_ok = g.adj_ok;
    h.ws_adj_floats = g.ws_adj_floats;
  }
  if ((size_t)4 * h.ws_floats > (size_t)kMaxSmem) return set_error(PG_ECAPACITY, "one environment's workspace exceeds shared memory");
  // environments per warp (soa): the largest power of two <= 32 whose warp of workspaces fits in
  // shared memory.  A batch may run the model narrower (pg_batch_compile).
  h.soa = 32;
  while (h.soa > 1 && (size_t)4 * h.soa * h.ws_floats > (size_t)kMaxSmem) h.soa /= 2;
  // ---- debug record layout ----
  int q = 0;
  auto dbg = [&](int n) { int r = q; q += n; return r; };
  h.dbg_xpos = dbg(3 * nbody); h.dbg_xmat = dbg(9 * nbody); h.dbg_xcom = dbg(3 * nbody); h.dbg_M = dbg(nv * nv);
  h.dbg_bias = dbg(nv); h.dbg_passive = dbg(nv); h.dbg_act = dbg(nv); h.dbg_a0 = dbg(nv); h.dbg_con = dbg(14 * nslot);
  h.dbg_nrow = dbg(1); h.dbg_rows = dbg(nrow_max * (nv + 7)); h.dbg_qacc = dbg(nv); h.dbg_iter = dbg(1);
  h.dbg_status = dbg(1); h.dbg_qpos = dbg(nq); h.dbg_qvel = dbg(nv);
  h.debug_floats = q;

  out->hdr_adj.debug_floats = h.debug_floats;
  std::memcpy(B.w.data(), &h, sizeof(h));
  out->hdr = h;
  out->blob_adj = B.w;
  std::memcpy(out->blob_adj.data(), &out->hdr_adj, sizeof(h));
  out->blob = std::move(B.w);
  out->hfield = std::move(hfield);
  return PG_OK;
}

}  // namespace pg
