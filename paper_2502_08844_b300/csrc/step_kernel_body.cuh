// The step kernel's body and its argument block, shared by the library's compiled kernels
// (step_kernels.cuh) and by the model-specialised kernels it compiles at run time (NVRTC, see
// specialize.cpp).  The including unit sets PG_WITH_ELLIPTIC; PG_SPEC (run-time compilation)
// takes model SPEC_M of the batch from the constant SpecModel<SPEC_M> (its blob and SoA width,
// defined by the generated source) instead of the kernel argument, so the compiler folds every
// header field, table entry and workspace offset.
#pragma once
#include "env_device.cuh"

namespace pg {
namespace {

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
struct StepArgs {
  const Tile* tiles;
  float* qpos;
  float* qvel;
  float* warm;
  uint32_t* status;
  uint32_t* stats;
  const float* ctrl;
  int64_t ld;
  int n_substeps;
  float* dbg;
  Tile dbg_tile;
  float* tape;                        // optional record of every substep (see TAPE below)
  int tape_rows, tape_nq, tape_nv;    // rows per substep entry; the batch's nq_max, nv_max
  int model_off[kMaxModels];          // word offset of each model's blob in `blob`
  const float* hfield[kMaxModels];    // each model's heightfield elevations (device), or NULL
  const float* dr;                    // per-environment parameters (pg_step_dr), or NULL
  EnvArgs env;                        // the locomotion task of an environment step (ENV below)
  float* out_force;                   // optional [nslot][3][ld] contact forces of the last substep (pg_step_ex)
  int32_t* out_ncon;                  // optional [ld] active contacts of the last substep
  int out_nslot;                      // candidate contact slots of the batch's models (the rows of out_force)
  int env_phase;                      // ENV: 0 the whole environment step, 1 the joint targets only,
                                      // 2 the step's end only (reward to observation; the substeps
                                      // ran in another kernel)
  uint32_t blob[kMaxParamWords];      // the batch's model blobs (header + tables)
};
static_assert(sizeof(StepArgs) <= 32764, "the step's argument block must fit the kernel parameter space");

// One thread per environment; a block steps the `count` consecutive environments of its tile.
// TAPE: also record, for every substep s, the state it starts from and the acceleration the
// solver returns, at tape[(s * tape_rows + row) * ld + env] with rows qpos [0, nq), qvel from
// tape_nq, the warm start from tape_nq + tape_nv and the acceleration from tape_nq + 2 tape_nv
// (the adjoint replays the substeps from this record).
// ENV: an environment step of the locomotion task A.env: the joint targets from the actions
// before the substeps (they are the PD targets), and after them the reward, termination,
// automatic reset and observation (env_device.cuh).

// DR: per-environment parameters (A.dr, pg_step_dr); the environment step (ENV) reads them when
// A.dr is set; otherwise the context's parameter pointer is a compile-time NULL and every
// parameter branch folds away.
template <bool DEBUG, bool TAPE, int SPEC_M = 0, bool ENV = false, bool DR = false>
__device__ __forceinline__ void step_body(const StepArgs& A) {
  extern __shared__ __align__(16) float smem[];
  const Tile tile = DEBUG ? A.dbg_tile : A.tiles[blockIdx.x];
#ifdef PG_SPEC
  const uint32_t* blob = SpecModel<SPEC_M>::blob();
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(blob);
  constexpr int S = SpecModel<SPEC_M>::soa;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#else
  const uint32_t* blob = A.blob + A.model_off[tile.model];
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(blob);
  const int S = h.soa, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#endif

  if (lane >= S) return;
  const int t = warp * S + lane;   // environment within the tile
  if (t >= tile.count) return;
  const int64_t env = tile.env0 + t;
  float* w = smem + warp * (S * h.ws_floats) + lane;
  Ctx c{h, S, reinterpret_cast<const int*>(blob), reinterpret_cast<const float*>(blob), w, ENV ? A.env.state : A.ctrl,
        A.ld, env, A.hfield[tile.model], (DR || ENV) ? A.dr : nullptr};
  if (ENV && A.env_phase != 2) env_targets(c, A.env);
  if (ENV && A.env_phase == 1) return;
  for (int k = 0; k < h.nq; k++) W(qpos, k) = A.qpos[k * A.ld + env];
  uint32_t status = 0;
  bool warm_bad = false;
  for (int k = 0; k < h.nv; k++) {
    W(qvel, k) = A.qvel[k * A.ld + env];
    const float wv = A.warm[k * A.ld + env];
    warm_bad = warm_bad || !isfinite(wv);
    W(warm, k) = wv;
  }
  if (warm_bad) {   // a non-finite warm start is replaced by zeros (flagged)
    status |= PG_STATUS_WARM_RESET;
    for (int k = 0; k < h.nv; k++) W(warm, k) = 0.f;
  }
  uint32_t cnt[3] = {0u, 0u, 0u};
  const int nsub_model = A.n_substeps > 0 ? A.n_substeps : h.substeps;
  const int nsub = DEBUG ? 1 : (ENV && A.env_phase == 2 ? 0 : nsub_model);
  int nc = 0;
  for (int s = 0; s < nsub; s++) {
    float* tp = TAPE ? A.tape + (int64_t)s * A.tape_rows * A.ld + env : nullptr;
    if (TAPE) {
      for (int k = 0; k < h.nq; k++) tp[k * A.ld] = W(qpos, k);
      for (int k = 0; k < h.nv; k++) {
        tp[(A.tape_nq + k) * A.ld] = W(qvel, k);
        tp[(A.tape_nq + A.tape_nv + k) * A.ld] = W(warm, k);
      }
    }
    nc = substep<DEBUG>(c, status, A.dbg, cnt);
    if (TAPE)
      for (int k = 0; k < h.nv; k++) tp[(A.tape_nq + 2 * A.tape_nv + k) * A.ld] = W(warm, k);
  }
  if (!DEBUG && !TAPE && !ENV) {   // the optional outputs of pg_step_ex (the last substep's contacts)
    if (A.out_force) contact_forces_out(c, nc, A.out_force, A.out_nslot);
    if (A.out_ncon) A.out_ncon[env] = nc;
  }
  for (int k = 0; k < h.nq; k++) A.qpos[k * A.ld + env] = W(qpos, k);
  for (int k = 0; k < h.nv; k++) {
    A.qvel[k * A.ld + env] = W(qvel, k);
    A.warm[k * A.ld + env] = W(warm, k);
  }
  if (status) A.status[env] |= status;
  if (A.stats)
    for (int k = 0; k < 3; k++) A.stats[k * A.ld + env] += cnt[k];
  if (ENV) env_finish(c, A.env, (float)nsub_model * h.h, A.qpos, A.qvel, A.warm, A.status);
}

}  // namespace
}  // namespace pg
