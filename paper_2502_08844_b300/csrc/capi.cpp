// C ABI entry points (declared in include/pg.h): argument checks, batch / tile construction,
// device copies of the model blobs, kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {

static thread_local std::string g_error;

int set_error(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

static int cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? PG_ENOMEM : PG_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// Environments per warp of the thread-per-environment kernels for `count` environments of model m
// (envs_per_cta as pg_batch_compile takes it; sms multiprocessors).  The model's widest width,
// unless its environments need more than one wave of blocks at that width: then the width whose
// block holds the most environments (the widest among equals).  A large workspace limits an SM to
// a few environments; held as one wide warp they run on one of its four schedulers with their
// branches serialised, while narrower warps hold more of them, fill more schedulers and diverge
// less (8192 hands: 16 environments an SM as one warp, or 20 as five warps of 4, 35 % faster with
// the elliptic cone).  When every environment fits in one wave anyway, extra warps only contend
// for the instruction cache (2048 humanoids run 19 % slower at 8 than at 16 a warp).  The width
// changes no arithmetic.
int thread_soa(const pg_model* m, int64_t count, int envs_per_cta, int sms) {
  const int ws = m->hdr.ws_floats;
  // environments a block holds at soa environments per warp (shared memory; at most 8 warps)
  auto block_envs = [&](int soa) {
    return (int)std::min<size_t>((size_t)kMaxSmem / ((size_t)4 * soa * ws), kMaxEnvsPerCta / 32) * soa;
  };
  int soa = m->hdr.soa;
  if (!envs_per_cta && count > (int64_t)sms * block_envs(soa)) {
    int most = block_envs(soa);
    for (int s = soa / 2; s >= 1; s /= 2)
      if (block_envs(s) > most) {
        most = block_envs(s);
        soa = s;
      }
  }
  return soa;
}
}  // namespace pg

using namespace pg;

extern "C" {

const char* pg_last_error(void) { return g_error.c_str(); }

int pg_model_compile(const pg_model_desc* desc, pg_model** out) {
  if (!out) return set_error(PG_EINVAL, "out is NULL");
  *out = nullptr;
  pg_model* m = new (std::nothrow) pg_model();
  if (!m) return set_error(PG_ENOMEM, "host allocation failed");
  int rc = compile_model(desc, m);
  if (rc != PG_OK) {
    delete m;
    return rc;
  }
  *out = m;
  g_error.clear();
  return PG_OK;
}

int pg_model_info(const pg_model* m, pg_model_sizes* out) {
  if (!m || !out) return set_error(PG_EINVAL, "NULL argument");
  const ModelHdr& h = m->hdr;
  out->nq = h.nq; out->nv = h.nv; out->nu = h.nu; out->nbody = h.nbody; out->njnt = h.njnt; out->ngeom = h.ngeom;
  out->npair = h.npair; out->nslot = h.nslot; out->nrow_max = h.nrow_max; out->max_contacts = h.max_contacts;
  out->workspace_bytes = 4 * h.ws_floats;
  out->debug_floats = h.debug_floats;
  out->adjoint_workspace_bytes = h.adj_ok ? 4 * h.ws_adj_floats : 0;
  out->nparam = h.nbody + h.nv + h.nu;
  out->nrand = h.nrand;
  return PG_OK;
}

void pg_model_free(pg_model* m) {
  if (!m) return;
  if (m->d_blob) cudaFree(m->d_blob);
  delete m;
}

static void free_host_stage(pg_batch::HostStage& h) {
  for (int k = 0; k < 2; k++) {
    if (h.ctrl[k]) cudaFree(h.ctrl[k]);
    if (h.snap[k]) cudaFree(h.snap[k]);
    for (cudaEvent_t ev : {h.in_done[k], h.ctrl_free[k], h.snap_done[k], h.snap_free[k]})
      if (ev) cudaEventDestroy(ev);
  }
  if (h.start) cudaEventDestroy(h.start);
  if (h.in) cudaStreamDestroy(h.in);
  if (h.out) cudaStreamDestroy(h.out);
  h = pg_batch::HostStage();
}

void pg_batch_free(pg_batch* b) {
  if (!b) return;
  if (b->d_blobs) cudaFree(b->d_blobs);
  if (b->d_blob_off) cudaFree(b->d_blob_off);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_hfields) cudaFree(b->d_hfields);
  if (b->d_ctrl_stage) cudaFree(b->d_ctrl_stage);
  free_host_stage(b->host_stage);
  if (b->d_vjp) cudaFree(b->d_vjp);
  if (b->spec_lib) cudaLibraryUnload(b->spec_lib);
  if (b->branch_lib) cudaLibraryUnload(b->branch_lib);
  for (const pg_batch::SpecPart& part : b->spec_parts) {
    cudaLibraryUnload(part.lib);
    if (part.branch_lib) cudaLibraryUnload(part.branch_lib);
  }
  delete b;
}

int pg_batch_compile(const pg_model* const* models, const int64_t* counts, int nmodels, int envs_per_cta, pg_batch** out) {
  if (!out) return set_error(PG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!models || !counts || nmodels < 1) return set_error(PG_EINVAL, "need at least one model");
  pg_batch* b = new (std::nothrow) pg_batch();
  if (!b) return set_error(PG_ENOMEM, "host allocation failed");
  for (int k = 0; k < nmodels; k++) {
    if (!models[k]) { delete b; return set_error(PG_EINVAL, "NULL model in batch"); }
    if (counts[k] < 0) { delete b; return set_error(PG_EINVAL, "negative env count"); }
    b->models.push_back(models[k]);
    b->counts.push_back(counts[k]);
    b->env_off.push_back(b->n);
    b->n += counts[k];
    const ModelHdr& h = models[k]->hdr;
    b->nq_max = std::max(b->nq_max, h.nq);
    b->nv_max = std::max(b->nv_max, h.nv);
    b->nslot_max = std::max(b->nslot_max, h.nslot);
    b->nu_max = std::max(b->nu_max, h.nu);
    b->max_ws_floats = std::max(b->max_ws_floats, h.ws_floats);
    b->max_blob_words = std::max(b->max_blob_words, h.words);
    b->max_debug = std::max(b->max_debug, h.debug_floats);
    b->has_elliptic = b->has_elliptic || h.cone == PG_CONE_ELLIPTIC;
    b->blob_off.push_back(0);
  }
  if (b->n > (int64_t)1 << 31) { delete b; return set_error(PG_EINVAL, "too many environments"); }
  if (envs_per_cta < 0 || envs_per_cta > kMaxEnvsPerCta) { delete b; return set_error(PG_EINVAL, "envs_per_cta must be 0 (auto) or 1..256"); }
  b->envs_per_cta_req = envs_per_cta;
  // environments per block: enough blocks to give every SM work in one wave, as many envs per
  // block as shared memory allows.  Each warp holds `soa` environments of its model.
  int sms = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // each model's blocks use as many warps as fit its own per-warp workspace; the launch
  // reserves the largest block footprint
  size_t smem = 0;
  int nwarps_max = 1;
  for (int k = 0; k < nmodels; k++) {
    const int ws = models[k]->hdr.ws_floats;
    const int soa = thread_soa(models[k], counts[k], envs_per_cta, sms);
    b->soa.push_back(soa);
    const size_t per_warp = (size_t)4 * soa * ws;
    const int warps_fit = (int)std::min<size_t>((size_t)kMaxSmem / per_warp, kMaxEnvsPerCta / 32);
    const int cap = warps_fit * soa;
    if (envs_per_cta && envs_per_cta > cap) { delete b; return set_error(PG_ECAPACITY, "envs_per_cta exceeds shared memory for these models"); }
    int e = envs_per_cta ? envs_per_cta : (int)std::max<int64_t>(1, (counts[k] + sms - 1) / sms);
    e = std::min(e, cap);
    b->envs_per_cta.push_back(e);
    const int nw = (e + soa - 1) / soa;
    nwarps_max = std::max(nwarps_max, nw);
    smem = std::max(smem, (size_t)nw * per_warp);
  }
  b->threads = 32 * nwarps_max;
  b->smem_bytes = smem;
  std::vector<uint32_t> all;
  for (int k = 0; k < nmodels; k++) {
    b->blob_off[k] = (int)all.size();
    all.insert(all.end(), models[k]->blob.begin(), models[k]->blob.end());
    all[b->blob_off[k] + offsetof(ModelHdr, soa) / 4] = (uint32_t)b->soa[k];   // this batch's width
  }
  if ((int)all.size() > kMaxParamWords) { delete b; return set_error(PG_ECAPACITY, "the batch's model tables exceed the 28 KB kernel-parameter budget"); }
  b->blob_host = all;
  for (int k = 0; k < nmodels; k++) b->blob_host_adj.insert(b->blob_host_adj.end(), models[k]->blob_adj.begin(), models[k]->blob_adj.end());
  for (int k = 0; k < nmodels; k++) {
    const int e = b->envs_per_cta[k];
    for (int64_t e0 = 0; e0 < counts[k]; e0 += e)
      b->tiles.push_back(Tile{k, (int)(b->env_off[k] + e0), (int)std::min<int64_t>(e, counts[k] - e0), 0});
  }
  // heaviest models' tiles first (blocks start roughly in index order): a per-environment cost
  // proxy of the model's workspace size
  std::stable_sort(b->tiles.begin(), b->tiles.end(), [&](const Tile& x, const Tile& y) {
    return models[x.model]->hdr.ws_floats > models[y.model]->hdr.ws_floats;
  });
  b->ntiles = (int)b->tiles.size();
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_blobs, all.size() * 4)) != cudaSuccess) { pg_batch_free(b); return cuda_error(e, "cudaMalloc"); }
  if ((e = cudaMalloc(&b->d_blob_off, nmodels * sizeof(int))) != cudaSuccess) { pg_batch_free(b); return cuda_error(e, "cudaMalloc"); }
  if (b->ntiles && (e = cudaMalloc(&b->d_tiles, b->tiles.size() * sizeof(Tile))) != cudaSuccess) { pg_batch_free(b); return cuda_error(e, "cudaMalloc"); }
  if ((e = cudaMemcpy(b->d_blobs, all.data(), all.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_blob_off, b->blob_off.data(), nmodels * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (b->ntiles && (e = cudaMemcpy(b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice)) != cudaSuccess)) {
    pg_batch_free(b);
    return cuda_error(e, "cudaMemcpy");
  }
  // the models' heightfields, one device copy per model that has one
  size_t hf_total = 0;
  for (int k = 0; k < nmodels; k++) hf_total += models[k]->hfield.size();
  if (hf_total) {
    if ((e = cudaMalloc(&b->d_hfields, hf_total * sizeof(float))) != cudaSuccess) { pg_batch_free(b); return cuda_error(e, "cudaMalloc"); }
    size_t off = 0;
    for (int k = 0; k < nmodels; k++) {
      const std::vector<float>& hf = models[k]->hfield;
      if (hf.empty()) continue;
      if ((e = cudaMemcpy(b->d_hfields + off, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
        pg_batch_free(b);
        return cuda_error(e, "cudaMemcpy");
      }
      b->hfield_ptr[k] = b->d_hfields + off;
      off += hf.size();
    }
  }
  if ((e = configure_step_kernels(b->smem_bytes)) != cudaSuccess) { pg_batch_free(b); return cuda_error(e, "cudaFuncSetAttribute"); }
  *out = b;
  g_error.clear();
  return PG_OK;
}

int pg_batch_info(const pg_batch* b, int64_t* n_envs, int* nq_max, int* nv_max, int* nu_max) {
  if (!b) return set_error(PG_EINVAL, "batch is NULL");
  if (n_envs) *n_envs = b->n;
  if (nq_max) *nq_max = b->nq_max;
  if (nv_max) *nv_max = b->nv_max;
  if (nu_max) *nu_max = b->nu_max;
  return PG_OK;
}

static int check_state(const pg_batch* b, const pg_state* s) {
  if (!b || !s) return set_error(PG_EINVAL, "NULL batch or state");
  if (s->n != b->n) return set_error(PG_EINVAL, "state.n differs from the batch's environment count");
  if (s->ld < s->n) return set_error(PG_EINVAL, "state.ld must be >= state.n");
  if (b->n > 0 && (!s->qpos || !s->qvel || !s->qacc_warm || !s->status)) return set_error(PG_EINVAL, "NULL state array");
  return PG_OK;
}

int pg_reset(const pg_batch* b, pg_state* s, const uint8_t* mask, const float* qpos0, const float* qvel0, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (b->n > 0 && (!qpos0 || !qvel0)) return set_error(PG_EINVAL, "NULL qpos0 / qvel0");
  cudaError_t e = launch_reset(b, s, mask, qpos0, qvel0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "reset launch");
  return PG_OK;
}

int pg_step(const pg_batch* b, pg_state* s, const float* ctrl, int n_substeps, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (b->n > 0 && b->nu_max > 0 && !ctrl) return set_error(PG_EINVAL, "NULL ctrl");
  cudaError_t e = launch_step(b, s, ctrl, n_substeps, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "step launch");
  return PG_OK;
}

int pg_step_ex(const pg_batch* b, pg_state* s, const float* ctrl, int n_substeps, const pg_step_out* out, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (b->n > 0 && b->nu_max > 0 && !ctrl) return set_error(PG_EINVAL, "NULL ctrl");
  cudaError_t e = launch_step(b, s, ctrl, n_substeps, (cudaStream_t)stream, nullptr,
                              out && (out->contact_force || out->ncon) ? out : nullptr);
  if (e != cudaSuccess) return cuda_error(e, "step launch");
  return PG_OK;
}

int pg_batch_nslot(const pg_batch* b) { return b ? b->nslot_max : 0; }

int pg_step_dr(const pg_batch* b, pg_state* s, const float* ctrl, const float* params, int n_substeps, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (b->n > 0 && b->nu_max > 0 && !ctrl) return set_error(PG_EINVAL, "NULL ctrl");
  if (b->n > 0 && !params) return set_error(PG_EINVAL, "NULL params");
  cudaError_t e = launch_step(b, s, ctrl, n_substeps, (cudaStream_t)stream, params);
  if (e != cudaSuccess) return cuda_error(e, "step launch");
  return PG_OK;
}

int pg_debug_substep(const pg_batch* b, pg_state* s, const float* ctrl, int64_t env, float* out, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (env < 0 || env >= b->n) return set_error(PG_EINVAL, "env out of range");
  if (!out) return set_error(PG_EINVAL, "NULL out");
  if (b->nu_max > 0 && !ctrl) return set_error(PG_EINVAL, "NULL ctrl");
  cudaError_t e = launch_debug(b, s, ctrl, env, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "debug launch");
  return PG_OK;
}

int pg_step_host(pg_batch* b, pg_state* s, const float* ctrl_host, float* qpos_host, float* qvel_host, int n_substeps,
                 void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if ((b->nu_max > 0 && !ctrl_host) || !qpos_host || !qvel_host) return set_error(PG_EINVAL, "NULL host buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = (size_t)std::max(b->nu_max, 1) * (size_t)s->ld;
  if (b->ctrl_stage_floats < need) {
    if (b->d_ctrl_stage) {   // an earlier call's queued upload and launch may still use it
      cudaDeviceSynchronize();
      cudaFree(b->d_ctrl_stage);
    }
    b->d_ctrl_stage = nullptr;
    b->ctrl_stage_floats = 0;
    cudaError_t e = cudaMalloc(&b->d_ctrl_stage, need * sizeof(float));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (control staging)");
    b->ctrl_stage_floats = need;
  }
  cudaError_t e;
  if (b->nu_max > 0 &&
      (e = cudaMemcpyAsync(b->d_ctrl_stage, ctrl_host, (size_t)b->nu_max * s->ld * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_error(e, "control upload");
  if ((e = launch_step(b, s, b->d_ctrl_stage, n_substeps, st)) != cudaSuccess) return cuda_error(e, "step launch");
  if ((e = cudaMemcpyAsync(qpos_host, s->qpos, (size_t)b->nq_max * s->ld * sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_error(e, "qpos download");
  if ((e = cudaMemcpyAsync(qvel_host, s->qvel, (size_t)b->nv_max * s->ld * sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_error(e, "qvel download");
  return PG_OK;
}

// pg_rollout_host's staging for control buffers of ctrl_f floats and snapshots of snap_f floats
static int host_stage(pg_batch* b, size_t ctrl_f, size_t snap_f) {
  pg_batch::HostStage& h = b->host_stage;
  if (h.in && h.ctrl_floats >= ctrl_f && h.snap_floats >= snap_f) return PG_OK;
  // larger buffers: an earlier rollout's copies and launches (on its caller's stream too) may still
  // read the old ones, so they finish before the old buffers are freed
  if (h.in) cudaDeviceSynchronize();
  free_host_stage(h);
  cudaError_t e = cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    for (cudaEvent_t* ev : {&h.in_done[k], &h.ctrl_free[k], &h.snap_done[k], &h.snap_free[k]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&h.ctrl[k], ctrl_f * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h.snap[k], snap_f * sizeof(float));
  }
  if (e != cudaSuccess) {
    free_host_stage(h);
    return cuda_error(e, "rollout staging");
  }
  h.ctrl_floats = ctrl_f;
  h.snap_floats = snap_f;
  return PG_OK;
}

int pg_rollout_host(pg_batch* b, pg_state* s, const float* ctrl_host, float* qpos_host, float* qvel_host, int n_steps,
                    int n_substeps, void* stream) {
  int rc = check_state(b, s);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (n_steps < 0) return set_error(PG_EINVAL, "n_steps must be >= 0");
  if (n_steps == 0) return PG_OK;   // nothing to read or write: the buffers may be NULL
  if ((b->nu_max > 0 && !ctrl_host) || !qpos_host || !qvel_host) return set_error(PG_EINVAL, "NULL host buffer");
  const size_t cf = (size_t)b->nu_max * s->ld, qf = (size_t)b->nq_max * s->ld, vf = (size_t)b->nv_max * s->ld;
  if ((rc = host_stage(b, std::max<size_t>(cf, 1), qf + vf)) != PG_OK) return rc;
  pg_batch::HostStage& h = b->host_stage;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(h.start, st);   // the staging streams start after the caller's queued work
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h.in, h.start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h.out, h.start, 0);
  for (int t = 0; t < n_steps && e == cudaSuccess; t++) {
    const int k = t & 1;
    // upload step t's controls once the launch of step t - 2 (which read this buffer) has run
    if (t >= 2) e = cudaStreamWaitEvent(h.in, h.ctrl_free[k], 0);
    if (e == cudaSuccess && cf)
      e = cudaMemcpyAsync(h.ctrl[k], ctrl_host + (size_t)t * cf, cf * sizeof(float), cudaMemcpyHostToDevice, h.in);
    if (e == cudaSuccess) e = cudaEventRecord(h.in_done[k], h.in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h.in_done[k], 0);
    if (e == cudaSuccess) e = launch_step(b, s, h.ctrl[k], n_substeps, st);
    if (e == cudaSuccess) e = cudaEventRecord(h.ctrl_free[k], st);
    // snapshot the state once the download of step t - 2 has left this buffer, then download
    // it on the other stream while the next step computes
    if (e == cudaSuccess && t >= 2) e = cudaStreamWaitEvent(st, h.snap_free[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.snap[k], s->qpos, qf * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.snap[k] + qf, s->qvel, vf * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(h.snap_done[k], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.out, h.snap_done[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(qpos_host + (size_t)t * qf, h.snap[k], qf * sizeof(float), cudaMemcpyDeviceToHost, h.out);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(qvel_host + (size_t)t * vf, h.snap[k] + qf, vf * sizeof(float), cudaMemcpyDeviceToHost, h.out);
    if (e == cudaSuccess) e = cudaEventRecord(h.snap_free[k], h.out);
  }
  // the caller's stream completes only after the last downloads
  for (int k = 0; k < std::min(n_steps, 2) && e == cudaSuccess; k++) e = cudaStreamWaitEvent(st, h.snap_free[k], 0);
  if (e != cudaSuccess) return cuda_error(e, "rollout");
  return PG_OK;
}

// the scratch of a pg_step_vjp call: the replayed state (qpos | qvel | warm | status), the substep
// tape, and the reverse sweep's workspace when a block of it does not fit in shared memory
static int vjp_scratch(const pg_batch* b, int n_steps, int n_substeps, int64_t ld, size_t& state_f, size_t& tape_f,
                       size_t& need, int& sub_max) {
  sub_max = 1;
  int ws_max = 1;
  for (const pg_model* m : b->models) {
    if (!m->hdr.adj_ok) return set_error(PG_EUNSUPPORTED, "a model of the batch is outside the adjoint's scope");
    sub_max = std::max(sub_max, n_substeps > 0 ? n_substeps : std::max(m->hdr.substeps, 1));
    ws_max = std::max(ws_max, m->hdr_adj.ws_adj_floats);
  }
  const int nq = b->nq_max, nv = b->nv_max;
  state_f = (size_t)(nq + 2 * nv + 1) * ld;
  tape_f = (size_t)n_steps * sub_max * (nq + 3 * nv) * ld;
  const size_t ws_f = vjp_smem_soa(ws_max) > 0 ? 0 : (size_t)ws_max * ld;
  need = state_f + tape_f + ws_f;
  return PG_OK;
}

static int grow_vjp(pg_batch* b, size_t need) {
  if (b->vjp_floats >= need) return PG_OK;
  if (b->d_vjp) {   // an earlier call's queued replay and sweep may still use it
    cudaDeviceSynchronize();
    cudaFree(b->d_vjp);
  }
  b->d_vjp = nullptr;
  b->vjp_floats = 0;
  cudaError_t e = cudaMalloc(&b->d_vjp, need * sizeof(float));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (adjoint scratch)");
  b->vjp_floats = need;
  return PG_OK;
}

int pg_batch_reserve_vjp(pg_batch* b, int n_steps, int n_substeps, int64_t ld) {
  if (!b) return set_error(PG_EINVAL, "NULL batch");
  if (n_steps < 1) return set_error(PG_EINVAL, "n_steps must be >= 1");
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (ld < b->n) return set_error(PG_EINVAL, "ld must be >= the batch's environment count");
  if (b->n == 0) return PG_OK;
  size_t state_f = 0, tape_f = 0, need = 0;
  int sub_max = 1;
  int rc = vjp_scratch(b, n_steps, n_substeps, ld, state_f, tape_f, need, sub_max);
  if (rc != PG_OK) return rc;
  return grow_vjp(b, need);
}

int pg_step_vjp(pg_batch* b, const pg_state* ck, const float* ctrl, int n_steps, int n_substeps, const float* g_qpos,
                const float* g_qvel, float* adj_qpos, float* adj_qvel, float* g_ctrl, float* g_param, void* stream) {
  if (!b || !ck) return set_error(PG_EINVAL, "NULL batch or checkpoint");
  if (ck->n != b->n) return set_error(PG_EINVAL, "ckpt.n differs from the batch's environment count");
  if (ck->ld < ck->n) return set_error(PG_EINVAL, "ckpt.ld must be >= ckpt.n");
  if (n_steps < 1) return set_error(PG_EINVAL, "n_steps must be >= 1");
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: each model's own)");
  if (b->n == 0) return PG_OK;
  if (!ck->qpos || !ck->qvel || !ck->qacc_warm) return set_error(PG_EINVAL, "NULL checkpoint array");
  if ((b->nu_max > 0 && (!ctrl || !g_ctrl)) || !adj_qpos || !adj_qvel || !g_param)
    return set_error(PG_EINVAL, "NULL argument");
  size_t state_f = 0, tape_f = 0, need = 0;
  int sub_max = 1;
  int rc = vjp_scratch(b, n_steps, n_substeps, ck->ld, state_f, tape_f, need, sub_max);
  if (rc != PG_OK) return rc;
  if ((rc = grow_vjp(b, need)) != PG_OK) return rc;
  const int64_t ld = ck->ld;
  const int nq = b->nq_max, nv = b->nv_max, nu = std::max(b->nu_max, 1);
  const int tape_rows = nq + 3 * nv;
  cudaStream_t st = (cudaStream_t)stream;
  float* sq = b->d_vjp;
  float* sv = sq + (size_t)nq * ld;
  float* sw = sv + (size_t)nv * ld;
  uint32_t* sstat = reinterpret_cast<uint32_t*>(sw + (size_t)nv * ld);
  float* tape = b->d_vjp + state_f;
  float* ws = tape + tape_f;
  pg_state s{sq, sv, sw, sstat, ck->n, ld, nullptr};
  cudaError_t e;
  if ((e = cudaMemcpyAsync(sq, ck->qpos, (size_t)nq * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sv, ck->qvel, (size_t)nv * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sw, ck->qacc_warm, (size_t)nv * ld * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(sstat, 0, (size_t)ld * 4, st)) != cudaSuccess)
    return cuda_error(e, "checkpoint copy");
  const size_t tape_step = (size_t)sub_max * tape_rows * ld;
  for (int t = 0; t < n_steps; t++) {
    const float* u = b->nu_max > 0 ? ctrl + (size_t)t * nu * ld : nullptr;
    if ((e = launch_step_tape(b, &s, u, n_substeps, tape + t * tape_step, tape_rows, st)) != cudaSuccess)
      return cuda_error(e, "replay launch");
  }
  for (int t = n_steps - 1; t >= 0; t--) {
    const float* u = b->nu_max > 0 ? ctrl + (size_t)t * nu * ld : nullptr;
    if ((e = launch_vjp_step(b, tape + t * tape_step, tape_rows, u, g_qpos ? g_qpos + (size_t)t * nq * ld : nullptr,
                             g_qvel ? g_qvel + (size_t)t * nv * ld : nullptr, adj_qpos, adj_qvel,
                             b->nu_max > 0 ? g_ctrl + (size_t)t * nu * ld : nullptr, g_param, ws, ld, n_substeps, st)) !=
        cudaSuccess)
      return cuda_error(e, "adjoint launch");
  }
  return PG_OK;
}

}  // extern "C"
