// pg_step_vjp_noalloc: the reverse sweep of pg_step_vjp on a fixed, statically allocated scratch
// array instead of library-allocated scratch.
//
// Who needs it. pg_step_vjp allocates its scratch with cudaMalloc on its first call and grows
// it when a later call needs more. Some callers must not allocate device memory during a call:
//   * a training loop that has given all device memory to its own pooled allocator, where a
//     cudaMalloc can fail;
//   * a latency-bound control loop, where a cudaMalloc or cudaFree is an implicit device-wide
//     synchronisation.
// This entry point calls no cudaMalloc, cudaFree or other allocating routine. Its scratch is the
// file-scope array below.
//
// Cost and limits.
//   * The array takes kNoAllocScratchFloats floats (16 MiB) of device memory on every device
//     where this module is loaded.
//   * A call whose scratch would exceed it is rejected with PG_ECAPACITY before any GPU work.
//   * Every call shares the one array. Calls that overlap on the GPU (different streams, or
//     different host threads on one device) race on it and corrupt each other's results.
//   * The first call on a device looks up the array's device address (cudaGetSymbolAddress).
//     With lazy module loading that also loads this module. Make the first call on each device
//     before any stream capture.
//
// Zeroing. The replayed state is copied in from the checkpoint on every call, and the tape and
// adjoint workspaces are written before they are read. The replay's status words are the only
// part that must start at zero, and every call clears them itself (cudaMemsetAsync).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {
namespace {

constexpr size_t kNoAllocScratchFloats = (size_t)4 << 20;   // 4 Mi floats = 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// the scratch's device address on the current device (looked up once per device)
int scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(PG_EUNSUPPORTED, "device index beyond the no-alloc set-up table");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    float* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(PG_ECUDA, std::string("cudaGetSymbolAddress (no-alloc scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" int pg_step_vjp_noalloc(pg_batch* b, const pg_state* ck, const float* ctrl, int n_steps, int n_substeps,
                                   const float* g_qpos, const float* g_qvel, float* adj_qpos, float* adj_qvel,
                                   float* g_ctrl, float* g_param, void* stream) {
  if (!b || !ck) return set_error(PG_EINVAL, "NULL batch or checkpoint");
  if (ck->n != b->n) return set_error(PG_EINVAL, "ckpt.n differs from the batch's environment count");
  if (ck->ld < ck->n) return set_error(PG_EINVAL, "ckpt.ld must be >= ckpt.n");
  if (n_steps < 1) return set_error(PG_EINVAL, "n_steps must be >= 1");
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (b->n == 0) return PG_OK;
  if (!ck->qpos || !ck->qvel || !ck->qacc_warm) return set_error(PG_EINVAL, "NULL checkpoint array");
  if ((b->nu_max > 0 && (!ctrl || !g_ctrl)) || !adj_qpos || !adj_qvel || !g_param)
    return set_error(PG_EINVAL, "NULL argument");
  int sub_max = 1, ws_max = 1;
  for (const pg_model* m : b->models) {
    if (!m->hdr.adj_ok) return set_error(PG_EUNSUPPORTED, "a model of the batch is outside the adjoint's scope");
    sub_max = std::max(sub_max, n_substeps > 0 ? n_substeps : std::max(m->hdr.substeps, 1));
    ws_max = std::max(ws_max, m->hdr_adj.ws_adj_floats);
  }
  const int64_t ld = ck->ld;
  const int nq = b->nq_max, nv = b->nv_max, nu = std::max(b->nu_max, 1);
  const int tape_rows = nq + 3 * nv;
  const size_t state_f = (size_t)(nq + 2 * nv + 1) * ld;
  const size_t tape_step = (size_t)sub_max * tape_rows * ld;
  const size_t ws_f = vjp_smem_soa(ws_max) > 0 ? 0 : (size_t)ws_max * ld;   // 0: in shared memory
  // reject before any size product can overflow: each factor is bounded by the scratch size
  if (state_f > kNoAllocScratchFloats || ws_f > kNoAllocScratchFloats || tape_step > kNoAllocScratchFloats ||
      (size_t)n_steps > kNoAllocScratchFloats / tape_step ||
      state_f + ws_f + (size_t)n_steps * tape_step > kNoAllocScratchFloats)
    return set_error(PG_ECAPACITY,
                     "pg_step_vjp_noalloc: this call needs more than the fixed scratch of 4194304 floats (16 MiB); "
                     "use fewer steps per call or fewer environments, or pg_step_vjp");
  float* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != PG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  float* sq = base;
  float* sv = sq + (size_t)nq * ld;
  float* sw = sv + (size_t)nv * ld;
  uint32_t* sstat = reinterpret_cast<uint32_t*>(sw + (size_t)nv * ld);
  float* tape = base + state_f;
  float* ws = tape + (size_t)n_steps * tape_step;
  pg_state s{sq, sv, sw, sstat, ck->n, ld, nullptr};
  cudaError_t e;
  if ((e = cudaMemcpyAsync(sq, ck->qpos, (size_t)nq * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sv, ck->qvel, (size_t)nv * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sw, ck->qacc_warm, (size_t)nv * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(sstat, 0, (size_t)ld * 4, st)) != cudaSuccess)
    return set_error(PG_ECUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
  for (int t = 0; t < n_steps; t++) {
    const float* u = b->nu_max > 0 ? ctrl + (size_t)t * nu * ld : nullptr;
    if ((e = launch_step_tape(b, &s, u, n_substeps, tape + t * tape_step, tape_rows, st)) != cudaSuccess)
      return set_error(PG_ECUDA, std::string("replay launch: ") + cudaGetErrorString(e));
  }
  for (int t = n_steps - 1; t >= 0; t--) {
    const float* u = b->nu_max > 0 ? ctrl + (size_t)t * nu * ld : nullptr;
    if ((e = launch_vjp_step(b, tape + t * tape_step, tape_rows, u, g_qpos ? g_qpos + (size_t)t * nq * ld : nullptr,
                             g_qvel ? g_qvel + (size_t)t * nv * ld : nullptr, adj_qpos, adj_qvel,
                             b->nu_max > 0 ? g_ctrl + (size_t)t * nu * ld : nullptr, g_param, ws, ld, n_substeps, st)) !=
        cudaSuccess)
      return set_error(PG_ECUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
  }
  return PG_OK;
}
