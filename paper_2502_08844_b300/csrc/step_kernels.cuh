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
#include "step_device.cuh"

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
  uint32_t blob[kMaxParamWords];      // the batch's model blobs (header + tables)
};

// One thread per environment; a block steps the `count` consecutive environments of its tile.
// TAPE: also record, for every substep s, the state it starts from and the acceleration the
// solver returns, at tape[(s * tape_rows + row) * ld + env] with rows qpos [0, nq), qvel from
// tape_nq, the warm start from tape_nq + tape_nv and the acceleration from tape_nq + 2 tape_nv
// (the adjoint replays the substeps from this record).
template <bool DEBUG, bool TAPE>
__global__ void __launch_bounds__(kMaxEnvsPerCta) step_kernel(const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(16) float smem[];
  const Tile tile = DEBUG ? A.dbg_tile : A.tiles[blockIdx.x];
  const uint32_t* blob = A.blob + A.model_off[tile.model];
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(blob);
  const int S = h.soa, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane >= S) return;
  const int t = warp * S + lane;   // environment within the tile
  if (t >= tile.count) return;
  const int64_t env = tile.env0 + t;
  float* w = smem + warp * (S * h.ws_floats) + lane;
  Ctx c{h, S, reinterpret_cast<const int*>(blob), reinterpret_cast<const float*>(blob), w, A.ctrl, A.ld, env};
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
  const int nsub = DEBUG ? 1 : (A.n_substeps > 0 ? A.n_substeps : h.substeps);
  for (int s = 0; s < nsub; s++) {
    float* tp = TAPE ? A.tape + (int64_t)s * A.tape_rows * A.ld + env : nullptr;
    if (TAPE) {
      for (int k = 0; k < h.nq; k++) tp[k * A.ld] = W(qpos, k);
      for (int k = 0; k < h.nv; k++) {
        tp[(A.tape_nq + k) * A.ld] = W(qvel, k);
        tp[(A.tape_nq + A.tape_nv + k) * A.ld] = W(warm, k);
      }
    }
    substep<DEBUG>(c, status, A.dbg, cnt);
    if (TAPE)
      for (int k = 0; k < h.nv; k++) tp[(A.tape_nq + 2 * A.tape_nv + k) * A.ld] = W(warm, k);
  }
  for (int k = 0; k < h.nq; k++) A.qpos[k * A.ld + env] = W(qpos, k);
  for (int k = 0; k < h.nv; k++) {
    A.qvel[k * A.ld + env] = W(qvel, k);
    A.warm[k * A.ld + env] = W(warm, k);
  }
  if (status) A.status[env] |= status;
  if (A.stats)
    for (int k = 0; k < 3; k++) A.stats[k * A.ld + env] += cnt[k];
}

}  // namespace

namespace PG_STEP_NS {

cudaError_t configure(size_t smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(step_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
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
  for (int k = 0; k < kMaxModels; k++) A.model_off[k] = k < (int)b->blob_off.size() ? b->blob_off[k] : 0;
  std::memcpy(A.blob, b->blob_host.data(), b->blob_host.size() * sizeof(uint32_t));
}

cudaError_t step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st) {
  if (b->ntiles == 0) return cudaSuccess;
  static thread_local StepArgs A;
  make_args(A, b, s, ctrl);
  A.n_substeps = n_substeps;
  step_kernel<false, false><<<b->ntiles, b->threads, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
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
