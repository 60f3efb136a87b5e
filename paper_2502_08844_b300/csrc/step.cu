// Fused batched physics step for sm_103a: one thread per environment.
//
// A thread block holds up to 256 environments of one model (a tile); each warp steps 32 of them
// in lockstep through the same generic loops over the model's tables, which sit in shared
// memory and are read as broadcasts.  Every environment's working set (state, kinematics,
// packed mass matrix and its LDL^T factor, contacts, constraint rows, Newton vectors) lives in
// a structure-of-arrays shared-memory workspace, element i of lane l at [32 i + l], so no two
// lanes ever hit the same bank.  All substeps of a control step run on chip; state is read
// once and written once, coalesced across environments.  FP32 CUDA-core arithmetic throughout
// (the per-environment matrices are small and not a dense contraction, so no tensor cores).
//
// Per substep: kinematics (frames, motion subspaces cdof and spatial inertias about each tree's
// reference point o) -> RNEA bias forces -> CRBA mass matrix (packed on the ancestor pattern)
// -> tree-sparse LDL^T and a0 = M^-1 (tau - c) -> collision over the static pair list ->
// contact / joint-limit rows with exact Ahat = (J M^-1 J^T)_rr -> Newton on the convex
// soft-constraint cost (Hessian on M's pattern when every pair lies on one kinematic chain,
// dense otherwise; exact line search) -> semi-implicit Euler.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "pg_host.h"
#include "pg_internal.h"
#define PG_WITH_ELLIPTIC 0
#define PG_STEP_NS pyramidal
#include "step_kernels.cuh"

namespace pg {
namespace {

__global__ void reset_kernel(float* qpos, float* qvel, float* warm, uint32_t* status, int64_t ld, int64_t n,
                             const uint8_t* mask, const float* qpos0, const float* qvel0, int nq_max, int nv_max) {
  const int64_t env = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (env >= n) return;
  if (mask && !mask[env]) return;
  for (int c = 0; c < nq_max; c++) qpos[c * ld + env] = qpos0[c * ld + env];
  for (int c = 0; c < nv_max; c++) {
    qvel[c * ld + env] = qvel0[c * ld + env];
    warm[c * ld + env] = 0.f;
  }
  status[env] = 0u;
}

// a new episode for every environment of a single-model batch, and its first observation
struct EnvResetArgs {
  float* qpos;
  float* qvel;
  float* warm;
  uint32_t* status;
  int64_t ld, n;
  EnvArgs env;
  uint32_t blob[kMaxParamWords];   // the model's blob (the actuators' addresses)
};
static_assert(sizeof(EnvResetArgs) <= 32764, "the reset's argument block must fit the kernel parameter space");

__global__ void env_reset_kernel(const __grid_constant__ EnvResetArgs A) {
  const int64_t env = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (env >= A.n) return;
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(A.blob);
  Ctx c{h, 0, reinterpret_cast<const int*>(A.blob), reinterpret_cast<const float*>(A.blob), nullptr, nullptr, A.ld, env};
  env_restart(c, A.env, A.qpos, A.qvel, A.warm, A.status);
  env_observe(c, A.env.task, A.qpos, A.qvel, nullptr, A.env.cmd, A.env.obs);
}

}  // namespace

// a batch with an elliptic-cone model runs the kernels compiled with the elliptic cone; all
// other batches the ones without it
cudaError_t configure_step_kernels(size_t smem_bytes) {
  cudaError_t e = pyramidal::configure(smem_bytes);
  if (e != cudaSuccess) return e;
  return elliptic::configure(smem_bytes);
}

cudaError_t launch_step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                        const float* dr, const pg_step_out* out) {
  if (b->branch_kernel && !dr) return launch_branch(b, s, ctrl, n_substeps, st, out);
  if (b->branch_kernel_dr && dr && !out) return launch_branch_dr(b, s, ctrl, dr, n_substeps, st);
  if (b->spec_kernel) return pyramidal::step_spec(b, s, ctrl, n_substeps, st, dr, out);
  if (!b->spec_parts.empty() && !dr) return pyramidal::step_spec_parts(b, s, ctrl, n_substeps, st, out);
  return b->has_elliptic ? elliptic::step(b, s, ctrl, n_substeps, st, dr, out)
                         : pyramidal::step(b, s, ctrl, n_substeps, st, dr, out);
}

cudaError_t launch_step_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                             int tape_rows, cudaStream_t st) {
  if (b->branch_kernel_tape) return launch_branch_tape(b, s, ctrl, n_substeps, tape, tape_rows, st);
  if (b->spec_kernel_tape) return pyramidal::step_spec_tape(b, s, ctrl, n_substeps, tape, tape_rows, st);
  return b->has_elliptic ? elliptic::step_tape(b, s, ctrl, n_substeps, tape, tape_rows, st)
                         : pyramidal::step_tape(b, s, ctrl, n_substeps, tape, tape_rows, st);
}

cudaError_t launch_env_step(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps, cudaStream_t st,
                            const float* dr) {
  if (b->branch_kernel && b->spec_kernel_env && !dr) {
    // the joint targets, the substeps on the branch-parallel kernel (its controls are the task
    // state's target rows), then the step's end: three launches
    cudaError_t e = pyramidal::step_spec_env(b, s, E, n_substeps, st, nullptr, 1);
    if (e == cudaSuccess) e = launch_branch(b, s, E.state, n_substeps, st);
    if (e == cudaSuccess) e = pyramidal::step_spec_env(b, s, E, n_substeps, st, nullptr, 2);
    return e;
  }
  if (b->spec_kernel_env) return pyramidal::step_spec_env(b, s, E, n_substeps, st, dr);
  return b->has_elliptic ? elliptic::step_env(b, s, E, n_substeps, st, dr)
                         : pyramidal::step_env(b, s, E, n_substeps, st, dr);
}

cudaError_t launch_env_reset(const pg_batch* b, const pg_state* s, const EnvArgs& E, cudaStream_t st) {
  if (s->n == 0) return cudaSuccess;
  static thread_local EnvResetArgs A;
  A.qpos = s->qpos; A.qvel = s->qvel; A.warm = s->qacc_warm; A.status = s->status;
  A.ld = s->ld; A.n = s->n; A.env = E;
  std::memcpy(A.blob, b->blob_host.data(), std::min(b->blob_host.size(), (size_t)kMaxParamWords) * sizeof(uint32_t));
  const int threads = 128;
  env_reset_kernel<<<(unsigned)((s->n + threads - 1) / threads), threads, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_debug(const pg_batch* b, const pg_state* s, const float* ctrl, int64_t env, float* out, cudaStream_t st) {
  return b->has_elliptic ? elliptic::debug(b, s, ctrl, env, out, st) : pyramidal::debug(b, s, ctrl, env, out, st);
}

cudaError_t launch_reset(const pg_batch* b, const pg_state* s, const uint8_t* mask, const float* qpos0, const float* qvel0,
                         cudaStream_t st) {
  if (s->n == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)((s->n + threads - 1) / threads);
  reset_kernel<<<blocks, threads, 0, st>>>(s->qpos, s->qvel, s->qacc_warm, s->status, s->ld, s->n, mask, qpos0, qvel0,
                                           b->nq_max, b->nv_max);
  return cudaGetLastError();
}

}  // namespace pg
