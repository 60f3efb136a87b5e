// FP64 oracle -- TEST INFRASTRUCTURE ONLY.  Model description and the derived tables
// the oracle needs (addresses, dof tree, mass properties, contact slots).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "orc_math.hpp"

namespace orc {

enum { FREE = 0, HINGE = 1, SLIDE = 2 };
enum { PLANE = 0, SPHERE = 1, CAPSULE = 2, BOX = 3, HFIELD = 4, CYLINDER = 5, MESH = 6 };
enum { MOTOR = 0, POSITION = 1 };
enum { PYRAMIDAL = 0, ELLIPTIC = 1 };

// status bits (per environment, OR-accumulated)
enum : uint32_t { ST_NAN = 1u, ST_NOT_CONVERGED = 2u, ST_CAPACITY = 4u, ST_WARM_RESET = 8u };

// Raw description handed in through the C API (plain arrays, values already rounded to
// float32 and widened).  Mirrors the flat kinematic-tree arrays of the input generator.
struct Desc {
  int nbody, njnt, ngeom, npair, nu;
  const int* body_parent; const double* body_pos; const double* body_quat; const double* body_mass;
  const double* body_ipos; const double* body_inertia; const int* body_geom_inertia;
  const int* jnt_type; const int* jnt_body; const double* jnt_pos; const double* jnt_axis;
  const int* jnt_limited; const double* jnt_range;
  const double* dof_damping; const double* dof_armature; const double* dof_rotor;
  const int* geom_type; const int* geom_body; const double* geom_pos; const double* geom_quat;
  const double* geom_size; const double* geom_mass;
  const int* pair_geom; const double* pair_friction; const int* pair_condim;
  const int* act_type; const int* act_jnt; const double* act_gear; const double* act_kp; const double* act_kd;
  const int* act_ctrllimited; const double* act_ctrlrange;
  double timestep; const double* gravity; int iterations; int cone; double impratio;
  const double* solref; const double* solimp; double margin; int max_contacts;
  int hfield_nrow, hfield_ncol; const double* hfield_data;   // the model's heightfield (elevations)
  const int* act_forcelimited; const double* act_forcerange;  // actuator torque limits (NULL: none)
  const double* dof_frictionloss;                               // [nv] joint friction loss (NULL: none)
  int nmesh;                                                    // convex meshes (MESH geoms)
  const int* mesh_vertadr; const int* mesh_vertnum; const double* mesh_vert;
  const int* mesh_faceadr; const int* mesh_facenum; const int* mesh_face;
  const int* geom_meshid;
};

// A convex solid for the collision routines: its vertices and outward face planes
// (n . x <= offset inside) in its own frame.  A box is 8 corners (corner i has +h on axis k when
// bit k of i is set) and 6 faces in the order -x, +x, -y, +y, -z, +z.
struct Solid {
  std::vector<double> vert;    // 3 per vertex
  std::vector<double> plane;   // 4 per face: outward unit normal, offset
  int nv() const { return (int)vert.size() / 3; }
  int nf() const { return (int)plane.size() / 4; }
};

// A heightfield grid: elevations e in [0, 1], row i at y = -hy + 2 hy i / (nrow - 1), column j at
// x = -hx + 2 hx j / (ncol - 1) of the geom frame; the surface height is hz e (size = hx, hy, hz).
struct HField {
  int nrow = 0, ncol = 0;
  const double* e = nullptr;
};

// The solid of a convex mesh: its vertices and the outward planes of its triangles (counter-
// clockwise seen from outside); an error message when a vertex lies outside a face's plane.
std::string mesh_solid(const double* vert, int nv, const int* face, int nf, Solid& sd);

struct Model {
  int nbody = 0, njnt = 0, nq = 0, nv = 0, ngeom = 0, npair = 0, nu = 0;
  std::vector<int> parent, body_jntadr, body_jntnum, body_root;
  std::vector<double> body_pos, body_quat;
  // mass properties in the body frame: mass, COM, full inertia about the COM (xx,yy,zz,xy,xz,yz)
  std::vector<double> mass, ipos, inertia;
  std::vector<int> jnt_type, jnt_body, jnt_qposadr, jnt_dofadr, jnt_limited;
  std::vector<double> jnt_pos, jnt_axis, jnt_range;
  std::vector<int> dof_body, dof_jnt, dof_parent;
  std::vector<double> dof_damping, dof_armature;
  std::vector<int> geom_type, geom_body;
  std::vector<double> geom_pos, geom_quat, geom_size, geom_mass;
  std::vector<int> pair_g1, pair_g2, pair_condim, pair_slotadr, pair_nslot;
  std::vector<double> pair_friction;
  int nslot = 0;
  std::vector<int> act_type, act_jnt, act_ctrllimited;
  std::vector<double> act_gear, act_kp, act_kd, act_ctrlrange;
  std::vector<int> act_forcelimited;
  std::vector<double> act_forcerange;
  double timestep = 0.01, impratio = 1.0, margin = 0.0;
  double gravity[3] = {0, 0, -9.81};
  double solref[2] = {0.02, 1.0};
  double solimp[5] = {0.9, 0.95, 0.001, 0.5, 2.0};
  int iterations = 4, cone = PYRAMIDAL, max_contacts = 0;
  int nlimited = 0;   // joints with limits (each contributes at most one active row)
  std::vector<double> dof_frictionloss;   // per dof; > 0 adds a friction-loss row
  int nfric = 0;
  int rows_per_contact = 4;
  int nrow_max = 0;
  int hf_nrow = 0, hf_ncol = 0;
  std::vector<double> hfield;
  HField hf() const { return HField{hf_nrow, hf_ncol, hfield.empty() ? nullptr : hfield.data()}; }
  std::vector<Solid> meshes;        // each mesh's vertices and the face planes of its triangles
  std::vector<int> geom_meshid;     // a MESH geom's mesh, else -1
};

// Contact points a primitive pair can produce (the static slot count of the pair).
inline int pair_max_points(int t1, int t2) {
  if (t1 == PLANE && t2 == SPHERE) return 1;
  if (t1 == PLANE && t2 == CAPSULE) return 2;
  if (t1 == PLANE && t2 == BOX) return 4;
  if (t1 == SPHERE && t2 == SPHERE) return 1;
  if (t1 == SPHERE && t2 == CAPSULE) return 1;
  if (t1 == CAPSULE && t2 == CAPSULE) return 1;
  if (t1 == SPHERE && t2 == BOX) return 1;
  if (t1 == CAPSULE && t2 == BOX) return 2;
  if (t1 == BOX && t2 == BOX) return 4;
  if (t1 == HFIELD && t2 == SPHERE) return 1;
  if (t1 == HFIELD && t2 == CAPSULE) return 2;
  if (t1 == PLANE && t2 == CYLINDER) return 4;
  if (t1 == PLANE && t2 == MESH) return 4;
  if (t1 == HFIELD && (t2 == BOX || t2 == MESH)) return 4;
  return -1;
}

// Inertia of a uniform solid about its own centre, in its own axes (diagonal), at mass m.
// Box: full edge lengths 2h.  Capsule: radius r, cylinder half-length hl along z, mass split
// between the cylinder and the two hemispheres by volume; a hemisphere's centroid lies 3r/8
// from its flat face (parallel-axis theorem).  Cylinder: radius r, half-length hl along z.
inline void solid_inertia(int type, const double* size, double m, double out[3]) {
  const double PI = 3.14159265358979323846;
  if (type == SPHERE) {
    double r = size[0], I = 0.4 * m * r * r;
    out[0] = out[1] = out[2] = I;
  } else if (type == BOX) {
    double a = 2 * size[0], b = 2 * size[1], c = 2 * size[2];
    out[0] = m * (b * b + c * c) / 12.0;
    out[1] = m * (a * a + c * c) / 12.0;
    out[2] = m * (a * a + b * b) / 12.0;
  } else if (type == CAPSULE) {
    double r = size[0], L = 2 * size[1];
    double vc = PI * r * r * L, vs = 4.0 / 3.0 * PI * r * r * r;
    double mc = m * vc / (vc + vs), ms = m * vs / (vc + vs);
    double axial = mc * r * r / 2 + 0.4 * ms * r * r;
    double perp = mc * (r * r / 4 + L * L / 12) + ms * (0.4 * r * r + L * L / 4 + 3.0 / 8.0 * L * r);
    out[0] = out[1] = perp;
    out[2] = axial;
  } else if (type == CYLINDER) {
    double r = size[0], L = 2 * size[1];
    out[0] = out[1] = m * (3 * r * r + L * L) / 12.0;
    out[2] = m * r * r / 2;
  } else {
    out[0] = out[1] = out[2] = 0;
  }
}

// Reflected rotor inertia I_a = k_g^2 * I_r with I_r = m_r r_r^2 / 2 (App. C.2.2).
inline double rotor_armature(double kg, double mr, double rr) { return kg * kg * 0.5 * mr * rr * rr; }

// Build the oracle model; returns an empty string on success, else the reason.
std::string compile_model(const Desc& d, Model& m);

}  // namespace orc
