/*
 * pg.h -- C ABI of the B300-native batched physics step.
 *
 * The library advances thousands of independent copies of articulated rigid-body models
 * ("environments") by one control step per call, entirely on the GPU: forward kinematics,
 * composite-rigid-body mass matrix with a tree-sparse LDL^T factorisation, recursive
 * Newton-Euler bias forces, primitive-geom collision, contact/limit Jacobians, a per-env
 * convex soft-contact Newton solve with an exact line search and a fixed iteration cap,
 * PD / motor actuation and semi-implicit Euler.  This is the physics step under the
 * training loop of MuJoCo Playground (arXiv 2502.08844): its environments run the MJX
 * physics step on thousands of envs on one device (Sec. 1), with static pair lists whose
 * cost follows the number of possible contacts (Limitations), per-task solver caps
 * ("iterations", Table dm_control_envs), PD position control (eq. pd_mapping, App. B.2.1),
 * reflected rotor inertia (App. C.2.2) and physics substeps per control decision
 * (App. "Bottlenecks in Pixels-based Training": 10 substeps of 5 ms per 20 Hz decision).
 *
 * Conventions
 *   - Every function returns PG_OK (0) or a negative status; pg_last_error() then gives a
 *     human-readable reason (thread-local, valid until the next call on the same thread).
 *   - Argument errors are detected synchronously, before any work is queued.  Numerical
 *     trouble inside an environment never traps: it sets bits of that env's status word.
 *   - Device work is queued on the caller's stream and is asynchronous.
 *   - Ownership: the caller owns every state, control, output and gradient buffer (for
 *     example torch tensors); the library owns models, batches and their device copies,
 *     all allocated at compile time.  pg_step allocates nothing.
 *   - A batch holds per-batch staging buffers and scratch: issue the calls that use one batch
 *     from one host thread at a time.
 *   - Batch state is structure-of-arrays: coordinate-major [coord][ld] float32 device
 *     arrays, env e of coordinate c at c*ld + e, with n <= ld (ld is the row pitch in
 *     elements).  In a mixed batch every array has max-over-models rows.
 */
#ifndef PG_H_
#define PG_H_

#ifdef __CUDACC_RTC__   /* the library's runtime kernel compiler: no system headers */
typedef unsigned long size_t;
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------------- */
#define PG_OK 0
#define PG_EINVAL (-1)        /* bad argument, bad array, level order violated          */
#define PG_ENOMEM (-2)        /* device or host allocation failed                       */
#define PG_ECUDA (-3)         /* a CUDA runtime call failed                             */
#define PG_EUNSUPPORTED (-4)  /* pair type, cone type or size beyond the kernel limits   */
#define PG_ECAPACITY (-5)     /* too many bodies/dofs/rows for the compiled kernels      */

/* ---- per-environment status bits (OR-accumulated until pg_reset) ------------------ */
#define PG_STATUS_NAN 1u            /* non-finite qacc / qvel / qpos                     */
#define PG_STATUS_NOT_CONVERGED 2u  /* Newton reached its cap before exact termination   */
#define PG_STATUS_CAPACITY 4u       /* more active contacts than max_contacts (extra     */
                                    /* contacts dropped in slot order)                   */
#define PG_STATUS_WARM_RESET 8u     /* non-finite warm start replaced by the smooth acc. */

/* ---- type codes ------------------------------------------------------------------- */
enum { PG_JNT_FREE = 0, PG_JNT_HINGE = 1, PG_JNT_SLIDE = 2 };
enum { PG_GEOM_PLANE = 0, PG_GEOM_SPHERE = 1, PG_GEOM_CAPSULE = 2, PG_GEOM_BOX = 3, PG_GEOM_HFIELD = 4,
       PG_GEOM_CYLINDER = 5, PG_GEOM_MESH = 6 };
enum { PG_ACT_MOTOR = 0, PG_ACT_POSITION = 1 };
enum { PG_CONE_PYRAMIDAL = 0, PG_CONE_ELLIPTIC = 1 };

/*
 * Model description: flat kinematic-tree arrays in level order (host memory, caller-owned,
 * read only during pg_model_compile).  Body 0 is the world; parent[i] < i.  Joints are
 * grouped by body in body order; a free joint is the only joint of a child of the world.
 * Lengths: nbody, njnt, ngeom, npair, nu, and nv = sum of dofs (free 6, hinge/slide 1).
 *   body_pos[3], body_quat[4]     frame of the body in its parent at q = 0, quat (w,x,y,z)
 *   body_mass, body_ipos[3], body_inertia[6] (xx,yy,zz,xy,xz,yz about the COM, body axes),
 *   body_geom_inertia              1: derive mass, COM and inertia from the body's geoms as
 *                                  uniform solids of geom_mass (box: 2*size edges; capsule:
 *                                  radius size[0], cylinder half-length size[1] along z;
 *                                  cylinder: radius size[0], half-length size[1] along z)
 *   jnt_pos[3], jnt_axis[3]        anchor and axis in the body frame; jnt_range[2] (lo < hi)
 *   dof_rotor[3]                   (gear ratio k_g, rotor mass m_r, radius r_r): armature
 *                                  k_g^2 m_r r_r^2 / 2 is added to dof_armature (App. C.2.2)
 *   pair_geom[2]                   candidate pair (geom1, geom2), type(geom1) <= type(geom2)
 *                                  in plane < sphere < capsule < box; the normal points from
 *                                  geom1 to geom2.  Static list: no broadphase.
 *                                  A heightfield (PG_GEOM_HFIELD, a massless geom of the world)
 *                                  pairs as geom1 with spheres (1 point) and capsules (2: its end
 *                                  spheres); see hfield_data below.
 *                                  A cylinder (PG_GEOM_CYLINDER) pairs as geom2 with a plane (4
 *                                  points: the deepest rim point of each cap and two more rim
 *                                  points of the lower cap, 120 degrees either side).
 *                                  A heightfield also pairs as geom1 with boxes and convex meshes,
 *                                  and a convex mesh (PG_GEOM_MESH) as geom2 with a plane (4 points
 *                                  each; see the mesh fields below).
 *   pair_condim                    1 (frictionless) or 3 (pyramidal cone, 4 edge rows)
 *   act_jnt                        hinge or slide joint driven by the actuator
 *   solref = (timeconst, dampratio); solimp = (d0, dwidth, width, mid, power)
 *   iterations                     Newton iteration cap (>= 1); max_contacts: cap on active
 *                                  contacts per env (< 0: number of candidate slots)
 */
typedef struct pg_model_desc {
  int nbody, njnt, ngeom, npair, nu;
  const int* body_parent; const float* body_pos; const float* body_quat; const float* body_mass;
  const float* body_ipos; const float* body_inertia; const int* body_geom_inertia;
  const int* jnt_type; const int* jnt_body; const float* jnt_pos; const float* jnt_axis;
  const int* jnt_limited; const float* jnt_range;
  const float* dof_damping; const float* dof_armature; const float* dof_rotor;
  const int* geom_type; const int* geom_body; const float* geom_pos; const float* geom_quat;
  const float* geom_size; const float* geom_mass;
  const int* pair_geom; const float* pair_friction; const int* pair_condim;
  const int* act_type; const int* act_jnt; const float* act_gear; const float* act_kp; const float* act_kd;
  const int* act_ctrllimited; const float* act_ctrlrange;
  float timestep; const float* gravity; int iterations; int cone; float impratio;
  const float* solref; const float* solimp; float margin; int max_contacts;
  int substeps;   /* the model's own physics substeps per control step (used by pg_step when
                     n_substeps == 0, e.g. in a mixed batch); values < 1 mean 1 */
  /* The model's heightfield, used by its PG_GEOM_HFIELD geoms (rough terrain, App. B
   * "Finetuning"): hfield_nrow x hfield_ncol (each >= 2) elevations in [0, 1], row-major; row i
   * lies at y = -hy + 2 hy i / (nrow - 1) and column j at x = -hx + 2 hx j / (ncol - 1) of the
   * geom frame, at height hz * elevation, with geom_size = (hx, hy, hz).  Each grid cell is split
   * along its (i, j)-(i+1, j+1) diagonal into two triangles.  A sphere's contact is the closest
   * point of the triangles within its radius (in the grid's xy), or, when its centre is below the
   * triangle under it, the depth along that triangle's normal; off the grid there is no contact.
   * Unused (0, 0, NULL) without heightfield geoms. */
  int hfield_nrow, hfield_ncol;
  const float* hfield_data;
  /* Actuator torque limits (the 8 Nm bounds of the hand, App. C): where act_forcelimited[a] is
   * non-zero the actuator's force is clipped to act_forcerange[2a .. 2a+1].  NULL: no limits. */
  const int* act_forcelimited;
  const float* act_forcerange;
  /* Joint friction loss (the hand's friction loss, App. C): [nv], NULL for none.  Each dof with
   * a positive loss F gets a two-sided constraint row (Jacobian e_d, reference acceleration
   * -b qvel_d) whose soft cost is the Huber function of its residual x with regulariser
   * R = 1 / D: D x^2 / 2 while |x| <= R F, F |x| - R F^2 / 2 outside, so its force stays in
   * [-F, F].  With either cone. */
  const float* dof_frictionloss;
  /* Convex meshes (PG_GEOM_MESH: rigid shapes beyond the primitives, as convex hulls; the
   * heightfield's box pairs serve box feet on App. B.2.5's rough terrain): mesh k has mesh_vertnum[k] vertices, mesh_vert[3 (mesh_vertadr[k] + i) + 0..2] in the
   * geom frame, and mesh_facenum[k] triangles, mesh_face[3 (mesh_faceadr[k] + f) + 0..2] (indices
   * into the mesh's own vertices, counter-clockwise seen from outside), that bound the convex
   * hull of those vertices.  geom_meshid[g] is the mesh of a mesh geom (ignored for other types).
   * A mesh geom's mass properties (body_geom_inertia) are those of a uniform solid hull of mass
   * geom_mass.  Contacts (4 slots a pair):
   *   plane against mesh: the 4 deepest vertices (ties: lower index), kept in vertex order, each
   *     at its distance to the plane along the plane's normal;
   *   heightfield against box or mesh: the candidates are the solid's vertices over the grid, at
   *     their signed distance to the plane of the triangle under them (that triangle's upward
   *     normal), then the grid vertices inside the solid, at the depth of the nearest face
   *     (normal: minus that face's outward normal; ties: lower face index), in row-major order;
   *     the 4 deepest candidates (ties: candidate order) are kept in candidate order.
   * Each contact point lies midway between the two surfaces.  At most 32 vertices and 64 faces
   * a mesh.  PG_EINVAL when a face is not outward or a vertex lies outside a face's plane.
   * Unused (0, NULL) without mesh geoms. */
  int nmesh;
  const int* mesh_vertadr; const int* mesh_vertnum; const float* mesh_vert;
  const int* mesh_faceadr; const int* mesh_facenum; const int* mesh_face;
  const int* geom_meshid;
} pg_model_desc;

typedef struct pg_model pg_model;   /* opaque, library-owned */
typedef struct pg_batch pg_batch;   /* opaque, library-owned */

typedef struct pg_model_sizes {
  int nq, nv, nu, nbody, njnt, ngeom, npair;
  int nslot;          /* candidate contact slots (sum over pairs of the pair's max points) */
  int nrow_max;       /* max constraint rows per env (4 per contact + 1 per limited joint) */
  int max_contacts;
  int workspace_bytes;  /* per-env shared-memory workspace of the step kernel            */
  int debug_floats;     /* length of the record written by pg_debug_substep              */
  int adjoint_workspace_bytes;  /* per-env workspace of pg_step_vjp; 0 when the model is
                                   outside the adjoint's scope (see pg_step_vjp)          */
  int nparam;           /* nbody + nv + nu: rows of the per-env parameter gradient        */
  int nrand;            /* 2 + 4 nbody + 2 nv + 3 nu: rows of pg_step_dr's per-env parameters */
} pg_model_sizes;

/* Caller-owned batch state (device pointers, [coord][ld] float32; status [n] uint32). */
typedef struct pg_state {
  float* qpos;        /* [nq_max][ld] */
  float* qvel;        /* [nv_max][ld] */
  float* qacc_warm;   /* [nv_max][ld]; warm start of the Newton solve, zeroed by pg_reset */
  uint32_t* status;   /* [n] status bits                                                   */
  int64_t n;          /* number of environments                                            */
  int64_t ld;         /* row pitch in elements (>= n)                                      */
  uint32_t* stats;    /* optional [3][ld] solver counters, NULL = off: per env and substep
                         += Newton iterations, += constraint rows, += rows * iterations      */
} pg_state;

/* ---- locomotion task around the step (pg_env_step) ---------------------------------- */
enum { PG_ACTION_ABSOLUTE = 0, PG_ACTION_RELATIVE = 1 };
/* Reward terms of the locomotion reward table (App. B, "Reward and Termination"), in the order
 * of pg_task_desc.weight and of pg_env_step's optional terms output.  Each is the table's
 * expression without its coefficient k (the coefficient is the weight):
 *   LIN_VEL      exp(-|cmd_xy - v_xy|^2 / sigma_lin_vel), v in the base frame
 *   ANG_VEL      exp(-(cmd_wz - w_z)^2 / sigma_ang_vel), w in the base frame
 *   AIR_TIME     sum over feet of clip((T_air - air_time_min) * C_touchdown, 0,
 *                air_time_max - air_time_min), C_touchdown = 1 on the step a foot lands
 *   CLEARANCE    sum over feet of (p_fz - clearance_height)^2 * |v_f,xy|^0.5
 *   SLIP         sum over feet of C_f |v_f,xy|^2, C_f = 1 while the foot touches the ground
 *   ORIENTATION  |g_xy|^2 of the gravity direction in the base frame
 *   TORQUE       |tau|^2 of the PD actuator torques at the step's final state
 *   JOINT_POS    |q - q_default|^2 over the actuated joints
 *   ACTION_RATE  |a_t - a_{t-1}|^2
 *   ENERGY       sum over actuated joints of |qdot_j tau_j|
 *   POSE         exp(-|q - q_default|^2)
 *   TERMINATION  1 when the episode terminated on this step (not when truncated)
 *   STAND_STILL  |cmd_xy| (as printed in the table)
 *   LIN_Z        v_z^2, base frame
 *   ANG_XY       w_x^2 + w_y^2, base frame
 * The reward is max(sum_i weight_i term_i, 0) (the table's weighted sum, clipped at zero). */
enum {
  PG_R_LIN_VEL = 0, PG_R_ANG_VEL, PG_R_AIR_TIME, PG_R_CLEARANCE, PG_R_SLIP, PG_R_ORIENTATION, PG_R_TORQUE,
  PG_R_JOINT_POS, PG_R_ACTION_RATE, PG_R_ENERGY, PG_R_POSE, PG_R_TERMINATION, PG_R_STAND_STILL, PG_R_LIN_Z,
  PG_R_ANG_XY, PG_NTERMS
};
#define PG_MAX_FEET 8

#ifndef __CUDACC_RTC__   /* host API (not seen by the run-time kernel compiler) */

/* Validate a description and build the library's model (host tables and a device copy).
 * Errors: PG_EINVAL (malformed tree or arrays), PG_EUNSUPPORTED (pair/cone type),
 * PG_ECAPACITY (beyond the kernel's compiled limits: nv <= 64, nbody <= 64, slots <= 64,
 * rows <= 128), PG_ECUDA / PG_ENOMEM. */
int pg_model_compile(const pg_model_desc* desc, pg_model** out);
int pg_model_info(const pg_model* model, pg_model_sizes* out);
void pg_model_free(pg_model* model);

/* Batch of environments: counts[k] consecutive envs of models[k], in that order.  The
 * models must outlive the batch.  envs_per_cta (>= 1, or 0 for the default) sets how many
 * environments share a thread block of the thread-per-environment kernels (one thread each;
 * the default is one wave: about n / SMs per block) and, when not 0, of the branch-parallel
 * kernel's barrier launch (envs_per_cta / (32 / lanes per environment) warps a block, 1 to 8;
 * its default is one wave).  With envs_per_cta 0 the thread-per-environment kernels hold each
 * model's environments in warps of its widest width (pg_batch_kernel's envs_per_warp), unless
 * they need more than one wave at that width: then at the width whose block holds the most of them
 * (fewer waves, more schedulers busy, less divergence; no change to the arithmetic).  Allocates
 * the batch's device tables and nothing else; the scratch of pg_step_vjp is reserved by
 * pg_batch_reserve_vjp (or by the first pg_step_vjp call that needs it). */
int pg_batch_compile(const pg_model* const* models, const int64_t* counts, int nmodels, int envs_per_cta,
                     pg_batch** out);
int pg_batch_info(const pg_batch* batch, int64_t* n_envs, int* nq_max, int* nv_max, int* nu_max);
void pg_batch_free(pg_batch* batch);

/* Compile, at run time, step kernels specialised to the batch's model and use them for every
 * following pg_step / pg_step_host of this batch. Same as pg_batch_specialize_ex(batch,
 * PG_SPEC_BRANCH).
 *
 * What changes. The specialised kernel takes the model's header, tables and workspace stride as
 * constants, which the generic kernel reads at run time. The arithmetic is the same source in
 * the same order; the compiler may regroup an FMA where a constant folds, so results agree with
 * the generic kernel's to rounding (not bit for bit).
 *
 * How. The kernel is compiled with NVRTC (libnvrtc.so.13, loaded on first use) for sm_103a and
 * cached per process and on disk ($PG_KERNEL_CACHE, else ~/.cache/paper_2502_08844_b300/kernels);
 * cubins that pg_model_precompile wrote into kernel_cache/ beside the library file are used too.
 * A first compile takes seconds, so call this before any stream capture and outside timed
 * regions.
 *
 * Scope. For a single-model batch the specialised build covers the step, pg_step_dr, the
 * environment step (pg_env_step) and, for models inside the adjoint's scope, the tape replay and
 * reverse sweep of pg_step_vjp; the debug kernel stays generic. For a mixed batch pg_step runs
 * one specialised kernel per model over that model's environments (one kernel holding every
 * model's body measured slower: blocks of different models on one SM evict each other's code from
 * the instruction cache), one launch after the other on the caller's stream (launched
 * concurrently on forked streams they measured slower).  The batch's other kernels stay generic.
 *
 * Errors. PG_EUNSUPPORTED (NVRTC missing or failing, with its log in pg_last_error; the batch
 * then keeps the generic kernel), PG_ECUDA. */
int pg_batch_specialize(pg_batch* batch);

/* pg_batch_specialize with options. flags:
 *   PG_SPEC_BRANCH  for a single-model batch whose model qualifies, pg_step and pg_step_host run
 *                   the branch-parallel kernel (in a mixed batch, each qualifying model's part): one thread per (environment, branch), where the
 *                   branches are the chains of hinge/slide bodies hanging from the model's trunk
 *                   (a quadruped's legs, a humanoid's legs and arms) and the trunk's work is shared
 *                   through warp shuffles. It computes the same step (Sec. 3, "Environment": the
 *                   physics step of MJX) with the mass matrix and the Newton Hessian factorised as
 *                   block arrowheads (branches first, the trunk's Schur complement last), so results
 *                   agree with the other kernels to FP32 rounding. A model qualifies when it has
 *                   2 to 8 branches, each contact pair touches at most one branch, at most one
 *                   actuator drives each dof, the cone is pyramidal, its pairs are primitives up to
 *                   boxes (a heightfield as geom1 included), it has no joint friction loss, and its
 *                   candidate contact points fit max_contacts; pg_batch_kernel reports why one does
 *                   not. Variants of it also run pg_step_dr (per-environment parameters), the
 *                   physics of pg_env_step (without parameters; the task's targets and its reward
 *                   to observation run as launches of the specialised kernel either side), and the
 *                   adjoint's tape replay (a model inside the adjoint's scope); a variant that
 *                   the compiler fits far worse than the plain kernel (pg_batch_kernel's branch_dr,
 *                   branch_tape report which run) is left out, and its caller keeps the
 *                   thread-per-environment kernel.  The adjoint's reverse sweep keeps the
 *                   thread-per-environment kernel.
 *   0               the thread-per-environment specialised kernels only.
 *   PG_SPEC_BRANCH_WARP  see below.
 * Errors as pg_batch_specialize; flags other than these: PG_EINVAL. */
#define PG_SPEC_BRANCH 1u
/* How the branch-parallel kernel is launched.  By default as one wave of blocks of up to 8 warps
 * (the warps per SM the batch needs) whose warps start every substep together (a barrier per
 * substep): the substep is a long straight-line program, bound by fetching its own instructions,
 * and warps that run it close together share those fetches (each substep then waits for the
 * block's slowest Newton solve).  PG_SPEC_BRANCH_WARP (implies PG_SPEC_BRANCH): blocks of one warp
 * and no barrier. */
#define PG_SPEC_BRANCH_WARP 2u
int pg_batch_specialize_ex(pg_batch* batch, unsigned flags);

/* Which kernel pg_step runs for the batch. */
enum { PG_KERNEL_GENERIC = 0, PG_KERNEL_SPECIALISED = 1, PG_KERNEL_SPECIALISED_PARTS = 2, PG_KERNEL_BRANCH = 3 };
typedef struct {
  int kernel;          /* PG_KERNEL_*                                                              */
  int lanes_per_env;   /* threads per environment (1, or the branch kernel's lane group)           */
  int branches;        /* branches of the model (branch kernel), else 0                            */
  char reason[160];    /* why the branch kernel is not used (empty when it is or was not asked)    */
  int branch_parts;    /* mixed batch: models whose part runs the branch-parallel kernel          */
  int sync;            /* branch kernel launched with a barrier per substep (the default)        */
  int branch_dr;       /* pg_step_dr runs the branch kernel's per-environment-parameter variant   */
  int branch_tape;     /* the adjoint's forward recording runs the branch kernel's tape variant    */
  int envs_per_warp;   /* thread-per-environment kernels: environments per warp of the first model */
} pg_kernel_info;
int pg_batch_kernel(const pg_batch* batch, pg_kernel_info* out);
/* Whether a model qualifies for the branch-parallel kernel (host only, no device work): out->kernel
 * is PG_KERNEL_BRANCH with its lane group and branch count, else PG_KERNEL_SPECIALISED with the
 * reason.  With the environment variable PG_BRANCH_SOURCE set to a path, the kernel source
 * generated for the model is written there (a developer aid). */
int pg_model_branch_plan(const pg_model* model, pg_kernel_info* out);

/* Compile ahead of time, with NVRTC and without any device work, the cubins that
 * pg_batch_specialize_ex(batch, flags) needs for `count` environments of `model` in a batch
 * compiled with envs_per_cta: the specialised thread-per-environment kernels at the width
 * pg_batch_compile takes on `sms` multiprocessors (0: 148, a B300's), and with PG_SPEC_BRANCH or
 * PG_SPEC_BRANCH_WARP the branch-parallel kernel when the model qualifies.  They go to the
 * directory `dir` (NULL or "": the disk cache that pg_batch_specialize writes), named by the same
 * key pg_batch_specialize looks them up by (the generated source, the NVRTC version and the
 * library's embedded kernel headers); a cubin already there is not compiled again.
 * pg_batch_specialize also reads kernel_cache/ beside the library file, so cubins compiled there
 * when the library is built spare its first calls the compile (seconds to a minute per model);
 * the kernels are the same either way.  Host only; may be called from several threads at once.
 * envs_per_warp, when not NULL, receives the thread-per-environment kernels' width; with
 * PG_PRECOMPILE_WIDTH_ONLY in flags nothing is compiled.  The paper has no counterpart: this is a
 * build step of the run-time specialisation.
 * Errors: PG_EINVAL (NULL model, negative count or sms, envs_per_cta outside 0..256, unknown
 * flags), PG_EUNSUPPORTED (NVRTC missing or failing, with its log in pg_last_error). */
#define PG_PRECOMPILE_WIDTH_ONLY 4u
int pg_model_precompile(const pg_model* model, int64_t count, int envs_per_cta, int sms, unsigned flags,
                        const char* dir, int* envs_per_warp);

/* Reset the envs whose env_mask_dev[e] != 0 (all envs when env_mask_dev is NULL): copy
 * qpos0/qvel0 ([coord][ld], same layout as the state), zero qacc_warm and status. */
int pg_reset(const pg_batch* batch, pg_state* state, const uint8_t* env_mask_dev, const float* qpos0_dev,
             const float* qvel0_dev, void* stream);

/* One control step (the environment's step of Sec. 3, "Environment": the physics advanced by
 * n_substeps substeps at the model's timestep with the controls held): n_substeps physics
 * substeps with the controls ctrl_dev ([nu_max][ld]) held (zero-order hold); n_substeps == 0
 * runs each model's own `substeps` (a mixed batch whose models run different rates).  Every
 * environment integrates with its own model's timestep.  Advances qpos, qvel, qacc_warm and ORs
 * status bits in place.  After the call qacc_warm holds the last substep's acceleration. */
int pg_step(const pg_batch* batch, pg_state* state, const float* ctrl_dev, int n_substeps, void* stream);

/* Optional outputs of pg_step_ex, all caller-owned device buffers (NULL: not written).
 *   contact_force  [nslot][3][ld] float32, nslot = pg_batch_nslot(): for each candidate contact
 *                  slot of the environment's model (its pairs in order, each with its static
 *                  number of points), the force of the last substep's solve in the contact's
 *                  frame (normal, t1, t2 of R14): a pyramid's edge forces D_e max(0, aref_e - J_e a)
 *                  summed back into the frame (f_n = sum_e f_e, f_t1 = mu (f_0 - f_1), f_t2 =
 *                  mu (f_2 - f_3)), an elliptic contact's minus the gradient of its cone cost; 0
 *                  for a slot without an active contact (and for slots beyond the model's own).
 *   ncon           [ld] int32: the last substep's active contacts. */
typedef struct pg_step_out {
  float* contact_force;
  int32_t* ncon;
} pg_step_out;

/* pg_step with optional outputs (out may be NULL: exactly pg_step).  Every kernel writes them:
 * the generic, the model-specialised, the branch-parallel and a mixed batch's parts. */
int pg_step_ex(const pg_batch* batch, pg_state* state, const float* ctrl_dev, int n_substeps, const pg_step_out* out,
               void* stream);

/* Candidate contact slots of the batch's models (the largest): the rows of pg_step_out's
 * contact_force. */
int pg_batch_nslot(const pg_batch* batch);

/* pg_step with per-environment physical parameters (domain randomisation, App. B "Domain
 * Randomization": ground friction, payload mass, link centres of mass, reflected inertia, joint
 * calibration offsets; App. C.2 adds PD gains, link masses and motor friction).  params_dev is
 * [nrand_max][ld] float32 (caller-owned), per environment:
 *   row 0                      friction scale: every pair's friction is multiplied by it;
 *   row 1                      payload: a point mass added at the centre of mass of body 1 (the
 *                              base of a floating robot), so body 1's mass grows and its
 *                              inertia about its centre of mass is unchanged;
 *   rows 2 .. 2 + 3 nbody      centre-of-mass offset (x, y, z, body frame) of each body, its
 *                              inertia about the centre of mass unchanged;
 *   next nv rows               armature added to each dof;
 *   next nu rows               calibration offset of each actuator: a PD actuator acts as if
 *                              its target were ctrl + offset (a motor ignores it);
 *   next nu rows               kp scale s: a PD actuator's kp becomes kp (1 + s);
 *   next nu rows               kd scale s: its kd becomes kd (1 + s);
 *   next nbody rows            link mass scale s: body b's mass and its inertia about its centre
 *                              of mass become (1 + s) times theirs (before body 1's payload);
 *   next nv rows               friction-loss scale s: a dof's friction loss F becomes F (1 + s)
 *                              (a dof compiled without friction loss keeps none).
 * nrand = 2 + 4 nbody + 2 nv + 3 nu.  An all-zero block except row 0 = 1 is the nominal model.
 * In a mixed batch each environment reads the rows of its own model's layout.  The adjoint
 * (pg_step_vjp) differentiates the nominal model only.  Errors as pg_step, and PG_EINVAL for a
 * NULL params_dev. */
int pg_step_dr(const pg_batch* batch, pg_state* state, const float* ctrl_dev, const float* params_dev, int n_substeps,
               void* stream);

/* Diagnostics: one substep of environment `env` only (the others are untouched), writing
 * every intermediate to out_dev (debug_floats floats, device memory) in this order:
 * xpos[nbody][3] xmat[nbody][9] xcom[nbody][3] M[nv][nv] bias[nv] passive[nv] actuator[nv]
 * a0[nv] contacts[nslot][14] (active, dist, pos3, n3, t1 3, t2 3) nrow rows[nrow_max][nv+7]
 * (J[nv], r, v, aref, D, Ahat, imp, force) qacc[nv] iterations status qpos_next[nq]
 * qvel_next[nv].  The env's state is advanced as by one substep of pg_step. */
int pg_debug_substep(const pg_batch* batch, pg_state* state, const float* ctrl_dev, int64_t env, float* out_dev,
                     void* stream);

/* Host-buffer convenience path: copy ctrl_host ([nu_max][ld] floats, pinned recommended)
 * to a library-owned device buffer, run pg_step, copy qpos/qvel back to qpos_host/qvel_host
 * ([coord][ld]).  Returns after queuing; synchronise the stream before reading the host
 * outputs.  The device buffer is allocated on the first call and grown (after synchronising the
 * device) when a later call needs more. */
int pg_step_host(pg_batch* batch, pg_state* state, const float* ctrl_host, float* qpos_host, float* qvel_host,
                 int n_substeps, void* stream);

/* n_steps control steps with host inputs and outputs, the transfers overlapped with the
 * computation: step t reads ctrl_host + t [nu_max][ld] and leaves its resulting state in
 * qpos_host + t [nq_max][ld] and qvel_host + t [nv_max][ld] (all pinned host memory for the
 * overlap).  Step t + 1's controls upload while step t computes, and step t's state (snapshotted
 * on the device) downloads while step t + 1 computes, on two library-owned streams ordered by
 * events against `stream`.  The state advances as by n_steps pg_step calls with the same kernels.
 * Returns after queuing; the host outputs are complete when `stream` is synchronised.  Allocates
 * its double buffers (two control rows, two state snapshots) on first use or when the batch's
 * sizes outgrow them (after synchronising the device, so that no earlier call still uses the old
 * ones).  Calls on one batch share these buffers: issue them on one stream, or synchronise between
 * calls on different streams.  n_steps = 0 does nothing (the buffers may then be NULL).  Errors as
 * pg_step_host, and PG_EINVAL for n_steps < 0. */
int pg_rollout_host(pg_batch* batch, pg_state* state, const float* ctrl_host, float* qpos_host, float* qvel_host,
                    int n_steps, int n_substeps, void* stream);

/* Reverse-mode sweep (vector-Jacobian product) of n_steps consecutive control steps.
 *
 * The paper reports no gradients. This is the library's adjoint of the step above. It is a
 * hand-written reverse sweep: the smooth dynamics (kinematics, CRBA, RNEA, actuation,
 * semi-implicit Euler) are differentiated directly, and the convex contact solve implicitly at
 * the solver's final iterate with the active set held fixed.
 *
 * Procedure. The call replays the steps forward from `ckpt`, on library-owned scratch,
 * recording every substep's start state and acceleration. It then sweeps back from the last
 * step to the first.
 *
 * Arguments (device memory, [coord][ld] float32, ld = ckpt->ld):
 *   ckpt          state at the start of the first step: qpos, qvel, qacc_warm. Read only;
 *                 status and stats are ignored.
 *   ctrl_dev      [n_steps][nu_max][ld] controls of the steps.
 *   g_qpos_dev    [n_steps][nq_max][ld] cotangent (dLoss/d) of the qpos after each step, or NULL.
 *   g_qvel_dev    [n_steps][nv_max][ld] the same for qvel, or NULL.
 *   adj_qpos_dev  [nq_max][ld] in/out. In: the adjoint of the state after the last step,
 *                 added to that step's cotangent. Out: the adjoint of ckpt's qpos.
 *   adj_qvel_dev  [nv_max][ld] the same for qvel.
 *   g_ctrl_dev    [n_steps][nu_max][ld] out: dLoss/dctrl.
 *   g_param_dev   [nparam_max][ld], ACCUMULATED (+=): per environment, the gradient with
 *                 respect to its model's body masses [nbody] (a body's rotational inertia
 *                 scales with its mass), then dof damping [nv], then actuator kp [nu].
 *
 * Gradients are not taken with respect to the warm start. The solver's result does not depend
 * on it at convergence.
 *
 * Scope. Every model of the batch needs adjoint_workspace_bytes > 0. That means:
 *   * any joints and actuators;
 *   * joint limits;
 *   * contacts only between a world-fixed plane or heightfield (geom1) and spheres, capsules or
 *     boxes, and between a world-fixed plane and cylinders.  On a heightfield's edges and
 *     vertices the contact normal turns with the state, and on a cylinder the rim points turn
 *     with its axis; the reverse sweep follows both.
 * A force clipped at its actuator's torque limit, and a friction-loss row's force at its bound,
 * are constant: nothing flows back through them.
 * Otherwise the call returns PG_EUNSUPPORTED.
 *
 * Scratch and errors.
 *   * Scratch, about n_steps * substeps * (nq + 3 nv) floats per env (plus the adjoint
 *     workspace when 8 environments' workspaces do not fit in one block's 227 KB of shared
 *     memory), is library-owned: reserve it up front with pg_batch_reserve_vjp, after which
 *     calls within the reserved sizes allocate nothing. A call that needs more than is reserved
 *     grows it: it synchronises the device (earlier calls' queued work may still use the old
 *     scratch), frees the old and allocates the new, so make such a call before any stream
 *     capture.
 *   * Calls on the same batch share the scratch: calls that overlap on the GPU race.
 *   * Errors: PG_EINVAL for NULL or inconsistent arguments, PG_EUNSUPPORTED,
 *     PG_ENOMEM / PG_ECUDA. */
/* Reserve pg_step_vjp's scratch for calls of up to n_steps control steps of n_substeps substeps
 * (0: each model's own) on states of row pitch ld, so that those calls allocate nothing.
 * Errors: PG_EINVAL, PG_EUNSUPPORTED (a model outside the adjoint's scope), PG_ECUDA. */
int pg_batch_reserve_vjp(pg_batch* batch, int n_steps, int n_substeps, int64_t ld);

int pg_step_vjp(pg_batch* batch, const pg_state* ckpt, const float* ctrl_dev, int n_steps, int n_substeps,
                const float* g_qpos_dev, const float* g_qvel_dev, float* adj_qpos_dev, float* adj_qvel_dev,
                float* g_ctrl_dev, float* g_param_dev, void* stream);

/* pg_step_vjp without allocation: the same arguments, results and scope as pg_step_vjp, with
 * the scratch in a fixed array of 4194304 floats (16 MiB) inside the library, not allocated.
 * The paper has no counterpart; this exists for callers that must not allocate device memory
 * during the call, e.g. one whose device memory is all held by its own pool, or a latency-bound
 * loop where cudaMalloc / cudaFree would synchronise the device.
 *   * A call that needs more scratch (n_steps, environments, substeps) returns PG_ECAPACITY
 *     before any GPU work.
 *   * Every call on a device shares the array, so calls that overlap on the GPU race.
 *   * The first call on a device looks up the array's address and may load the library's device
 *     code. Make it before any stream capture. */
int pg_step_vjp_noalloc(pg_batch* batch, const pg_state* ckpt, const float* ctrl_dev, int n_steps, int n_substeps,
                        const float* g_qpos_dev, const float* g_qvel_dev, float* adj_qpos_dev, float* adj_qvel_dev,
                        float* g_ctrl_dev, float* g_param_dev, void* stream);

/* ---- locomotion task (the steps either side of the physics in the training loop) ----
 *
 * A task wraps one model's step with the environment logic of the paper's locomotion tasks
 * (App. B, "Observation and Action" and "Reward and Termination"): the action-to-target
 * mapping, the observation, the reward table, termination when the robot turns over, and
 * automatic reset.  pg_env_step runs all of it inside the step kernel's launch, before and
 * after the physics substeps.
 *
 * Task description (host memory, caller-owned, read only during pg_task_compile):
 *   action_mode      PG_ACTION_ABSOLUTE: q_des = q_default + action_scale * a_t (joystick
 *                    tasks); PG_ACTION_RELATIVE: q_des = q_des_prev + action_scale * a_t.
 *                    q_des is clipped to each actuator's ctrlrange when it is limited, and
 *                    is the PD target of the step (eq. pd_mapping).
 *   q_default        [nu] default joint targets (also the reset value of q_des).
 *   nfeet, foot_geom [nfeet] (<= PG_MAX_FEET) sphere geoms at the feet. A foot's height is its
 *                    sphere's lowest point above the world plane z = 0; it touches the ground
 *                    while that height is below contact_height.
 *   clearance_height desired swing height of the feet (p_des_z of the clearance term).
 *   sigma_lin_vel, sigma_ang_vel, air_time_min, air_time_max: reward parameters.
 *   weight           [PG_NTERMS] weights of the reward terms (see the PG_R_* list).
 *   episode_length   control steps after which an episode is truncated (>= 1).
 * The model must have a free joint on body 1 (the base) and only PD position actuators on
 * hinge or slide joints.
 * Errors: PG_EINVAL (malformed description), PG_EUNSUPPORTED (model outside that shape). */
typedef struct pg_task_desc {
  int action_mode;
  float action_scale;
  const float* q_default;
  int nfeet;
  const int* foot_geom;
  float contact_height, clearance_height;
  float sigma_lin_vel, sigma_ang_vel, air_time_min, air_time_max;
  float weight[PG_NTERMS];
  int episode_length;
} pg_task_desc;

typedef struct pg_task pg_task;   /* opaque, library-owned */

typedef struct pg_task_sizes {
  int nobs;         /* observation rows: 3 gravity + 3 linear + 3 angular velocity (base
                       frame) + nu joint positions (q - q_default) + nu joint velocities +
                       nu previous action + 3 command = 12 + 3 nu                         */
  int nterms;       /* PG_NTERMS                                                          */
  int state_rows;   /* rows of the per-env task state: q_des [nu], previous action [nu],
                       foot air time [nfeet], foot contact [nfeet], episode step [1]       */
} pg_task_sizes;

int pg_task_compile(const pg_model* model, const pg_task_desc* desc, pg_task** out);
int pg_task_info(const pg_task* task, pg_task_sizes* out);
void pg_task_free(pg_task* task);

/* Start every environment of the batch on its initial state: state <- (qpos0, qvel0), warm
 * start and status zeroed; task state: q_des <- q_default, previous action, air time, contact
 * and episode step <- 0; obs <- the observation of the initial state with command cmd.
 * Arguments (device memory, [rows][ld]): task_state [state_rows], qpos0 [nq], qvel0 [nv],
 * cmd [3] (vx, vy, wz), obs [nobs].  The batch must hold the task's model only.
 * Errors: PG_EINVAL, PG_EUNSUPPORTED (another model in the batch), PG_ECUDA. */
int pg_env_reset(const pg_batch* batch, const pg_task* task, pg_state* state, float* task_state_dev,
                 const float* qpos0_dev, const float* qvel0_dev, const float* cmd_dev, float* obs_dev, void* stream);

/* One environment step of every env, in one kernel launch:
 *   1. q_des from the actions a_t ([nu][ld], in [-1, 1] by convention) by action_mode;
 *   2. n_substeps physics substeps with q_des as the PD targets (as pg_step);
 *   3. on the final state: the reward terms, the reward, termination (the base's z axis points
 *      below the horizon, or a non-finite state) and truncation (episode_length reached);
 *   4. environments that are done start over from (qpos0, qvel0) as in pg_env_reset;
 *   5. obs of every env's current state (after any reset), with the action just applied as
 *      the previous action (zero after a reset).
 * Outputs ([rows][ld] device memory): obs [nobs], reward [1], done [1] (1 when the episode
 * ended on this step: terminated or truncated), truncated [1] (1 when it ended by
 * episode_length only), terms [PG_NTERMS] (unweighted reward terms, or NULL).
 * reward, done, truncated and terms describe the transition; obs describes the state the next
 * action acts on.  params_dev (optional, NULL for none): per-environment physical parameters in
 * pg_step_dr's layout, used by the physics and the PD torques of the reward terms.  Errors as
 * pg_env_reset. */
int pg_env_step(const pg_batch* batch, const pg_task* task, pg_state* state, float* task_state_dev,
                const float* action_dev, const float* cmd_dev, const float* qpos0_dev, const float* qvel0_dev,
                int n_substeps, float* obs_dev, float* reward_dev, float* done_dev, float* truncated_dev,
                float* terms_dev, const float* params_dev, void* stream);

/* ---- batch ray-traced pixel observations -------------------------------------------------
 *
 * The paper pairs the batched physics with batch rendering for pixel-based policies (Sec. 5,
 * Madrona batch renderer: 64 x 64 cartpole frames).  pg_render ray-traces one image per
 * environment from the batch state, on the GPU:
 *   * a pinhole camera shared by the batch (world position, look-at point, up vector, vertical
 *     field of view in degrees, width x height pixels); pixel (x, y) has y = 0 at the top and
 *     its ray passes through the pixel's centre;
 *   * every drawn geom of the model at the environment's current pose (forward kinematics of
 *     qpos): planes (infinite, both faces), spheres, capsules and boxes; heightfields are not
 *     drawn;
 *   * Lambertian shading under one directional light: colour = albedo * (ambient + diffuse *
 *     (n . l) * lit), l = -light_dir normalised, lit = 1 when n . l > 0 and a shadow ray from the
 *     hit point towards the light meets no drawn geom; rays that hit nothing get the background.
 * Output (device memory, caller-owned): format PG_PIXELS_U8: uint8 [n][height][width][3],
 * round(255 * clip(colour, 0, 1)); PG_PIXELS_F32: float32 [n][height][width][3] unclipped.
 * hits_dev (optional, int32 [n][height][width]): 0 for the background, else (geom + 1) plus
 * 65536 when no direct light reaches the point (lit = 0).
 * Scope: single-model batches; ngeom <= 64; width, height in 1 .. 1024.  Errors: PG_EINVAL,
 * PG_EUNSUPPORTED (a mixed batch), PG_ECAPACITY, PG_ECUDA. */
enum { PG_PIXELS_U8 = 0, PG_PIXELS_F32 = 1 };

typedef struct pg_render_desc {
  float cam_pos[3], cam_lookat[3], cam_up[3];
  float fovy_deg;
  int width, height;
  float light_dir[3];     /* direction the light travels                                  */
  float ambient, diffuse;
  float background[3];
  const float* geom_rgb;  /* [ngeom][3] albedo; a geom whose first component is < 0 is not
                             drawn (and casts no shadow)                                    */
  /* Per-environment visual randomisation (each NULL for none; device memory, [3][ld] with the
   * state's ld): env_cam_offset moves the camera's position (its look-at point stays, so the view
   * direction turns with it); env_light_dir replaces light_dir; env_tint multiplies every colour
   * of the image, background included (colour and brightness randomisation). */
  const float* env_cam_offset;
  const float* env_light_dir;
  const float* env_tint;
} pg_render_desc;

int pg_render(const pg_batch* batch, const pg_state* state, const pg_render_desc* desc, int format, void* pixels_dev,
              int32_t* hits_dev, void* stream);

const char* pg_last_error(void);

#endif  /* __CUDACC_RTC__ */

#ifdef __cplusplus
}
#endif
#endif /* PG_H_ */
