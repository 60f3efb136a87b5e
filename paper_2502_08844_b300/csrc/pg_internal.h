// Internal layout shared by the host model compiler and the step kernel.
//
// A compiled model is one flat blob of 32-bit words: a fixed header (counts, options and the
// word offsets of every table) followed by the tables.  Each thread block copies its model's
// blob into shared memory once and reads every table from there.  The blob also records the
// per-environment shared-memory workspace layout (float offsets), computed on the host.
#pragma once
#include <stdint.h>

namespace pg {

// compiled kernel limits
constexpr int kMaxNv = 64;       // ancestor-dof masks are 64-bit
constexpr int kMaxBody = 64;
constexpr int kMaxSlot = 64;
constexpr int kMaxRow = 128;     // active-set masks are 4 x 32 bits

struct ModelHdr {
  // counts
  int nbody, njnt, nq, nv, nu, ngeom, npair, nslot, nrow_max, max_contacts, nlimited, nlevel, nL;
  int cap, cone;
  // options (float32)
  float h, grav[3], kref, bref, solimp[5], margin;
  // table offsets (words from the blob start)
  int o_body_parent, o_body_root, o_body_jntadr, o_body_jntnum, o_body_pos, o_body_quat, o_body_mass,
      o_body_ipos, o_body_inertia, o_body_dofmask, o_level_start, o_level_body, o_child_start, o_child;
  int o_jnt_type, o_jnt_qposadr, o_jnt_dofadr, o_jnt_pos, o_jnt_axis, o_jnt_range;
  int o_dof_body, o_dof_depth, o_dof_rowadr, o_dof_damping, o_dof_armature, o_Lcol;
  int o_geom_type, o_geom_body, o_geom_pos, o_geom_quat, o_geom_size;
  int o_pair_g1, o_pair_g2, o_pair_friction, o_pair_condim, o_pair_slotadr, o_pair_nslot;
  int o_act_type, o_act_dof, o_act_qposadr, o_act_gear, o_act_kp, o_act_kd, o_act_ctrllimited, o_act_range;
  int o_limit_jnt;
  int words;   // total blob size
  // per-env workspace layout (float offsets from the env's workspace base)
  int ws_floats;
  int w_qpos, w_qvel, w_warm, w_ctrl;
  int w_M, w_L, w_D, w_bias, w_passive, w_act, w_a0, w_vtmp, w_con;
  // union 1: kinematics (until the rows are built) / Newton + row solves (afterwards)
  int w_xpos, w_xquat, w_xmat, w_xipos, w_janchor, w_jaxis, w_gpos, w_gmat, w_cdof, w_cinert;
  int w_H, w_a, w_g, w_p, w_Mp, w_Z;
  // union 2: dynamics temporaries (CRBA / RNEA) / constraint rows
  int w_crb, w_cvel, w_cacc, w_cfrc, w_F;
  int w_J, w_rr, w_rv, w_aref, w_rD, w_Ahat, w_imp, w_jar, w_Jp, w_force, w_rowslot;
  int debug_floats;
  int dbg_xpos, dbg_xmat, dbg_xcom, dbg_M, dbg_bias, dbg_passive, dbg_act, dbg_a0, dbg_con, dbg_nrow, dbg_rows,
      dbg_qacc, dbg_iter, dbg_status, dbg_qpos, dbg_qvel;
};

constexpr int kHdrWords = (int)(sizeof(ModelHdr) / 4);
static_assert(sizeof(ModelHdr) % 4 == 0, "header must be whole words");

// one thread block's work: `count` consecutive envs starting at `env0` of model `model`
struct Tile {
  int model;
  int env0;
  int count;
  int pad;
};

}  // namespace pg
