// The step kernels (production, solver-tape and single-environment debug variants) and their
// launchers, compiled once per friction-cone configuration: the including translation unit sets
// PG_WITH_ELLIPTIC (0: pyramidal and frictionless contacts only, no elliptic code in the hot
// loops; 1: the elliptic cone as well) and PG_STEP_NS, the namespace of its launchers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstring>

#include "pg_host.h"
#include "pg_internal.h"
#include "step_kernel_body.cuh"

namespace pg {
namespace {

template <bool DEBUG, bool TAPE, bool ENV = false, bool DR = false>
__global__ void __launch_bounds__(kMaxEnvsPerCta) step_kernel(const __grid_constant__ StepArgs A) {
  step_body<DEBUG, TAPE, 0, ENV, DR>(A);
}

}  // namespace

namespace PG_STEP_NS {

cudaError_t configure(size_t smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(step_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<false, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

static void make_args(StepArgs& A, const pg_batch* b, const pg_state* s, const float* ctrl) {
  A.tiles = b->d_tiles;
  A.qpos = s->qpos;
  A.qvel = s->qvel;
  A.warm = s->qacc_warm;
  A.status = s->status;
  A.stats = s->stats;
  A.ctrl = ctrl;
  A.ld = s->ld;
  A.n_substeps = 1;
  A.dbg = nullptr;
  A.dbg_tile = Tile{0, 0, 0, 0};
  A.tape = nullptr;
  A.tape_rows = A.tape_nq = A.tape_nv = 0;
  A.env.state = nullptr;
  A.dr = nullptr;
  A.out_force = nullptr;
  A.out_ncon = nullptr;
  A.out_nslot = 0;
  A.env_phase = 0;
  for (int k = 0; k < kMaxModels; k++) A.model_off[k] = k < (int)b->blob_off.size() ? b->blob_off[k] : 0;
  for (int k = 0; k < kMaxModels; k++) A.hfield[k] = b->hfield_ptr[k];
  std::memcpy(A.blob, b->blob_host.data(), b->blob_host.size() * sizeof(uint32_t));
}

static void set_out(StepArgs& A, const pg_batch* b, const pg_step_out* out) {
  if (!out) return;
  A.out_force = out->contact_force;
  A.out_ncon = out->ncon;
  A.out_nslot = b->nslot_max;
}

cudaError_t step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                 const float* dr, const pg_step_out* out) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  A.dr = dr;
  set_out(A, b, out);
  if (dr) step_kernel<false, false, false, true><<<b->ntiles, b->threads, b->smem_bytes, st>>>(A);
  else step_kernel<false, false><<<b->ntiles, b->threads, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

// the batch's model-specialised kernel (same argument block)
cudaError_t step_spec(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                      const float* dr, const pg_step_out* out) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  A.dr = dr;
  set_out(A, b, out);
  void* params[] = {&A};
  return cudaLaunchKernel((const void*)(dr ? b->spec_kernel_dr : b->spec_kernel), dim3(b->ntiles), dim3(b->threads),
                          params, b->smem_bytes, st);
}

cudaError_t step_spec_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                           int tape_rows, cudaStream_t st) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  A.tape = tape;
  A.tape_rows = tape_rows;
  A.tape_nq = b->nq_max;
  A.tape_nv = b->nv_max;
  void* params[] = {&A};
  return cudaLaunchKernel((const void*)b->spec_kernel_tape, dim3(b->ntiles), dim3(b->threads), params, b->smem_bytes, st);
}

cudaError_t step_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                             int tape_rows, cudaStream_t st) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  A.tape = tape;
  A.tape_rows = tape_rows;
  A.tape_nq = b->nq_max;
  A.tape_nv = b->nv_max;
  step_kernel<false, true><<<b->ntiles, b->threads, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

// a mixed batch's specialised step: each model's kernel over its own tiles, back to back
cudaError_t step_spec_parts(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                            const pg_step_out* out) {
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  set_out(A, b, out);
  for (const pg_batch::SpecPart& part : b->spec_parts) {
    if (part.branch) {   // the model's branch-parallel kernel over its environments
      cudaError_t e = launch_branch_range(part.branch, part.branch_sync, part.branch_lanes, part.env0, part.count, s, ctrl,
                                          n_substeps, st, out, b->nslot_max, nullptr, 0, 0, 0, b->envs_per_cta_req,
                                          b->hfield_ptr[part.model]);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (part.ntiles == 0) continue;
    A.tiles = b->d_tiles + part.tile0;
    void* params[] = {&A};
    cudaError_t e = cudaLaunchKernel((const void*)part.kernel, dim3(part.ntiles), dim3(part.threads), params, part.smem, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// an environment step of the locomotion task E (generic kernel, or the batch's specialised one)
cudaError_t step_env(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps, cudaStream_t st,
                     const float* dr, int phase) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, nullptr);
  A.n_substeps = n_substeps;
  A.env = E;
  A.dr = dr;
  A.env_phase = phase;
  step_kernel<false, false, true><<<b->ntiles, b->threads, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

cudaError_t step_spec_env(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps, cudaStream_t st,
                          const float* dr, int phase) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, nullptr);
  A.n_substeps = n_substeps;
  A.env = E;
  A.dr = dr;
  A.env_phase = phase;
  void* params[] = {&A};
  return cudaLaunchKernel((const void*)b->spec_kernel_env, dim3(b->ntiles), dim3(b->threads), params, b->smem_bytes, st);
}

cudaError_t debug(const pg_batch* b, const pg_state* s, const float* ctrl, int64_t env, float* out, cudaStream_t st) {
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  int model = 0;
  for (size_t k = 0; k < b->models.size(); k++)
    if (env >= b->env_off[k] && env < b->env_off[k] + b->counts[k]) model = (int)k;
  A.dbg = out;
  A.dbg_tile = Tile{model, (int)env, 1, 0};
  step_kernel<true, false><<<1, 32, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

}  // namespace PG_STEP_NS
}  // namespace pg
