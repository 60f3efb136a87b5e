// Internal layout shared by the host model compiler and the step kernel.
//
// A compiled model is one flat blob of 32-bit words: a fixed header (counts, options, the word
// offsets of every table and the per-environment workspace layout) followed by the tables.
// The blobs of a batch's models travel to the step kernel as a read-only kernel parameter; all
// threads of a warp step different environments of the same model, so every table read is a
// uniform (broadcast) read that never aliases the workspace.
//
// Per-environment workspaces are structure-of-arrays across the 32 lanes of a warp: element i
// of lane l lives at [i * 32 + l], so lanes never conflict on a shared-memory bank whatever
// element each of them touches.  The host assigns every buffer an interval of the substep's
// phases and packs buffers whose intervals do not overlap into the same space.
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif
#include "pg.h"

namespace pg {

// compiled kernel limits
constexpr int kMaxNv = 64;
constexpr int kMaxBody = 64;
constexpr int kMaxSlot = 64;
constexpr int kMaxRow = 128;     // active-set masks are 4 x 32 bits per environment
constexpr int kMaxEnvsPerCta = 256;
constexpr int kMaxSmem = 232448;       // 227 KB opt-in shared memory per block
constexpr int kMaxModels = 8;          // models per batch (their blobs travel as a kernel parameter)
constexpr int kMaxParamWords = 7168;   // 28 KB of blob words in the kernel's parameter space
constexpr int kMaxMeshVert = 32;       // vertices of a convex mesh
constexpr int kMaxMeshFace = 64;       // faces (triangles) of a convex mesh

struct ModelHdr {
  // counts
  int nbody, njnt, nq, nv, nu, ngeom, npair, nslot, nrow_max, max_contacts, nlimited, nL;
  int cap, cone, tree_hessian, ncol_max, soa, substeps;
  int hf_nrow, hf_ncol;   // the heightfield grid (its elevations live in device memory, not the blob)
  // options (float32)
  float h, grav[3], kref, bref, solimp[5], margin;
  float imp_mid_inv, imp_tail_inv;   // 1 / mid^(p-1) and 1 / (1 - mid)^(p-1) of the impedance
  // table offsets (words from the blob start)
  int o_body_parent, o_body_root, o_body_jntadr, o_body_jntnum, o_body_pos, o_body_quat, o_body_mass,
      o_body_ipos, o_body_inertia, o_root_freeadr;
  int o_jnt_type, o_jnt_qposadr, o_jnt_dofadr, o_jnt_pos, o_jnt_axis, o_jnt_range;
  int o_dof_body, o_dof_depth, o_dof_rowadr, o_dof_damping, o_dof_armature, o_Lcol;
  int o_geom_type, o_geom_body, o_geom_pos, o_geom_quat, o_geom_size;
  int o_pair_g1, o_pair_g2, o_pair_friction, o_pair_condim, o_pair_slotadr, o_pair_nslot, o_pair_coladr,
      o_pair_ncol, o_col_dof, o_col_sign, o_slot_pair;
  int o_act_type, o_act_dof, o_act_qposadr, o_act_gear, o_act_kp, o_act_kd, o_act_ctrllimited, o_act_range;
  int o_act_forcelimited, o_act_forcerange;
  int nrand;          // rows of the per-environment parameters of pg_step_dr
  int dr_com, dr_arm, dr_cal;   // their first rows: COM offsets, armature, calibration offsets,
  int dr_kp, dr_kd, dr_mass, dr_fric;   // PD gain scales, link mass scales, friction-loss scales
  int o_limit_jnt;
  int nfric, o_fric_dof, o_fric_F;   // friction-loss rows: their dofs and force bounds
  int nmesh, o_mesh_vertadr, o_mesh_vertnum, o_mesh_vert, o_mesh_faceadr, o_mesh_facenum, o_mesh_plane,
      o_geom_meshid;                 // convex meshes: vertices (3 floats) and outward face planes
                                     // (n, offset: 4 floats) per mesh; each geom's mesh or -1
  int words;   // total blob size
  // per-environment workspace layout (element offsets, see above)
  int ws_floats;
  int w_qpos, w_qvel, w_warm;
  int w_xpos, w_xquat, w_cdof, w_cinert, w_cvel, w_cacc, w_cfrc, w_bias;
  int w_M, w_L, w_a0, w_con, w_J, w_z;
  int w_gcol, w_gmu, w_gcond, w_lsgn, w_rr, w_rv, w_Ahat, w_imp, w_aref, w_rD, w_jar, w_Jp;
  int w_a, w_g, w_p, w_t, w_H, w_Dinv, w_bp;
  // adjoint workspace (the reverse sweep): every forward buffer above gets its own space (no
  // sharing between phases), plus the own body inertias `ci0` (CRBA overwrites w_cinert with
  // composites), the Hessian factor `HL` and the adjoint buffers b_*.  Valid only in the adjoint
  // copy of the header; adj_ok = 0 when the model is outside the adjoint's scope.
  int adj_ok, ws_adj_floats;
  int w_ci0, w_HL;
  int b_q, b_v, b_a, b_bias, b_M, b_cdof, b_I, b_vel, b_acc, b_frc, b_wr, b_w;
  int debug_floats;
  int dbg_xpos, dbg_xmat, dbg_xcom, dbg_M, dbg_bias, dbg_passive, dbg_act, dbg_a0, dbg_con, dbg_nrow, dbg_rows,
      dbg_qacc, dbg_iter, dbg_status, dbg_qpos, dbg_qvel;
};

constexpr int kHdrWords = (int)(sizeof(ModelHdr) / 4);
static_assert(sizeof(ModelHdr) % 4 == 0, "header must be whole words");

// per active contact in the workspace: slot, dist, pos[3], n[3], feature (the capsule endpoint or
// box corner a plane contact comes from; 0 otherwise)
constexpr int kConFloats = 9;

// A locomotion task (pg_env_step) as the step kernel reads it: the action mapping, the feet
// and the reward table's parameters, in kernel-parameter space beside the model blobs.
struct EnvTask {
  int mode, nu, nfeet, episode_length;
  int base_qpos, base_dof;          // the free joint's qpos and dof addresses
  float scale, contact_height, clearance, sig_v, sig_w, air_min, air_max;
  float weight[PG_NTERMS];
  float q_default[kMaxNv];
  int foot_body[PG_MAX_FEET];
  int foot_lastdof[PG_MAX_FEET];    // last dof of the chain that moves the foot's body
  float foot_pos[3 * PG_MAX_FEET];  // sphere centre in its body's frame
  float foot_r[PG_MAX_FEET];
};

// the task's per-call arrays ([rows][ld] device memory, see pg_env_step)
struct EnvArgs {
  float* state;            // q_des [nu] | previous action [nu] | air time [nfeet] | contact [nfeet] | step [1]
  const float* actions;    // [nu]
  const float* cmd;        // [3]
  const float* qpos0;      // [nq] reset state
  const float* qvel0;      // [nv]
  float* obs;              // [12 + 3 nu]
  float* reward;           // [1]
  float* done;             // [1]
  float* truncated;        // [1]
  float* terms;            // [PG_NTERMS] or NULL
  EnvTask task;
};

// The branch-parallel step kernel's arguments (see branch_body.cuh): batch state and controls in
// the [coord][ld] layout of pg_state; the n environments from env0 (one model's part of a batch).
struct BranchArgs {
  float* qpos;
  float* qvel;
  float* warm;
  uint32_t* status;
  uint32_t* stats;       // optional solver counters [3][ld], or NULL
  const float* ctrl;
  int64_t ld, env0, n;
  int n_substeps;
  float* out_force;      // optional [out_nslot][3][ld] contact forces of the last substep, or NULL
  int32_t* out_ncon;     // optional [ld] active contacts of the last substep, or NULL
  int out_nslot;
  const float* hfield;   // the model's heightfield elevations (device), or NULL
  const float* dr;       // per-environment parameters [nrand][ld] (pg_step_dr), in the DR variant
  float* tape;           // optional substep record for the adjoint, or NULL: for substep s, rows
  int tape_rows, tape_nq, tape_nv;   // qpos [0, nq), qvel at tape_nq, warm start at tape_nq +
                                     // tape_nv, the solver's acceleration at tape_nq + 2 tape_nv
};

// one thread block's work: `count` consecutive envs starting at `env0` of model `model`
struct Tile {
  int model;
  int env0;
  int count;
  int pad;
};

}  // namespace pg
