// Host-side internals of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_internal.h"

struct pg_model {
  pg::ModelHdr hdr;
  std::vector<uint32_t> blob;
  pg::ModelHdr hdr_adj;             // the adjoint's header (its workspace layout)
  std::vector<uint32_t> blob_adj;   // the blob with the adjoint's header
  uint32_t* d_blob = nullptr;   // device copy of the blob
  std::vector<float> hfield;    // the heightfield's elevations (empty without one); the batch
                                // holds the device copy
};

struct pg_task {
  const pg_model* model;
  pg::EnvTask task;
  int nobs, state_rows;
};

struct pg_batch {
  std::vector<const pg_model*> models;
  std::vector<int64_t> counts, env_off;
  int64_t n = 0;
  int nq_max = 0, nv_max = 0, nu_max = 0;
  int nslot_max = 0;               // candidate contact slots of the batch's models (pg_step_out rows)
  int threads = 32;                // threads per block (one environment per thread)
  std::vector<int> envs_per_cta;   // per model
  int envs_per_cta_req = 0;        // as requested (0: the default one-wave shapes); the branch-
                                   // parallel launch takes it as environments per block
  int max_ws_floats = 0, max_blob_words = 0, max_debug = 0;
  size_t smem_bytes = 0;
  uint32_t* d_blobs = nullptr;     // all models' blobs, concatenated
  int* d_blob_off = nullptr;       // word offset of each model's blob
  pg::Tile* d_tiles = nullptr;
  float* d_hfields = nullptr;                      // the models' heightfields, concatenated
  const float* hfield_ptr[pg::kMaxModels] = {};    // each model's grid in d_hfields (NULL: none)
  int ntiles = 0;
  std::vector<int> blob_off;
  std::vector<uint32_t> blob_host;   // all models' blobs, concatenated (passed as a kernel parameter)
  std::vector<pg::Tile> tiles;
  std::vector<uint32_t> blob_host_adj;   // the same with the adjoint headers
  bool has_elliptic = false;             // a model uses the elliptic cone (selects the kernels)
  // model-specialised step kernel compiled at run time (pg_batch_specialize), else NULL
  cudaLibrary_t spec_lib = nullptr;
  cudaKernel_t spec_kernel = nullptr;
  cudaKernel_t spec_kernel_tape = nullptr;   // the same with the substep tape (adjoint replay)
  cudaKernel_t spec_kernel_vjp = nullptr;    // the adjoint's reverse sweep (NULL outside its scope)
  cudaKernel_t spec_kernel_env = nullptr;    // the environment step of a locomotion task
  cudaKernel_t spec_kernel_dr = nullptr;     // the step with per-environment parameters
  // a mixed batch's specialised step: one kernel per model over that model's (contiguous) tiles
  struct SpecPart {
    cudaLibrary_t lib;
    cudaKernel_t kernel;
    int tile0, ntiles, threads;
    size_t smem;
    // the model's branch-parallel kernel over its environments [env0, env0 + count), or NULL
    cudaLibrary_t branch_lib;
    cudaKernel_t branch;
    cudaKernel_t branch_sync;
    int branch_lanes;
    int64_t env0, count;
    int model;   // the part's model in the batch
  };
  std::vector<SpecPart> spec_parts;
  std::vector<int> soa;   // each model's environments per warp in this batch (its header's soa in blob_host)
  // the branch-parallel step kernel (pg_batch_specialize_ex with PG_SPEC_BRANCH), else NULL
  cudaLibrary_t branch_lib = nullptr;
  cudaKernel_t branch_kernel = nullptr;
  cudaKernel_t branch_kernel_sync = nullptr;   // the same with a barrier per substep (the default launch)
  cudaKernel_t branch_kernel_tape = nullptr;   // the barrier launch recording the adjoint's substep tape
  cudaKernel_t branch_kernel_dr = nullptr;     // the barrier launch with per-environment parameters
  int branch_lanes = 0, branch_count = 0;
  std::string branch_why;   // why a requested branch kernel is not used
  // staging buffer of the host-buffer path (allocated on its first use)
  float* d_ctrl_stage = nullptr;
  size_t ctrl_stage_floats = 0;
  // pg_rollout_host's double-buffered staging: two control buffers and two state snapshots, an
  // upload and a download stream, and the events that order them against the step launches
  struct HostStage {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, in_done[2] = {nullptr, nullptr}, ctrl_free[2] = {nullptr, nullptr},
                snap_done[2] = {nullptr, nullptr}, snap_free[2] = {nullptr, nullptr};
    float* ctrl[2] = {nullptr, nullptr};
    float* snap[2] = {nullptr, nullptr};
    size_t ctrl_floats = 0, snap_floats = 0;
  } host_stage;
  // scratch of pg_step_vjp (allocated on its first use, grown when a call needs more): the
  // replayed state, the substep tape and the adjoint workspaces
  float* d_vjp = nullptr;
  size_t vjp_floats = 0;
};

namespace pg {

int set_error(int code, const std::string& msg);

// Run f once per device (the current one), under a lock, before any caller on that device goes
// on: kernel attributes are set before the first launch that needs them, whatever the threads.
template <class F>
void once_per_device(std::mutex& mu, unsigned long long& done, F&& f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { f(); return; }
  const unsigned long long bit = 1ull << dev;
  std::lock_guard<std::mutex> lock(mu);
  if (done & bit) return;
  f();
  done |= bit;
}
int compile_model(const pg_model_desc* d, pg_model* out);
// capi.cpp: environments per warp of the thread-per-environment kernels (pg_batch_compile's rule)
int thread_soa(const pg_model* m, int64_t count, int envs_per_cta, int sms);
// branch.cpp: the branch-parallel kernel's plan and generated source for a model
int branch_plan(const pg_model* m, std::string& src, std::string& why, int& lanes_per_env, int& threads,
                int& branches);
cudaError_t launch_branch(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                          const pg_step_out* out = nullptr);
cudaError_t launch_branch_range(cudaKernel_t k, cudaKernel_t k_sync, int lanes, int64_t env0, int64_t count,
                                const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                                const pg_step_out* out = nullptr, int nslot = 0, float* tape = nullptr,
                                int tape_rows = 0, int tape_nq = 0, int tape_nv = 0, int envs_per_block = 0,
                                const float* hfield = nullptr, const float* dr = nullptr);
// the branch-parallel step with per-environment parameters (pg_step_dr's layout)
cudaError_t launch_branch_dr(const pg_batch* b, const pg_state* s, const float* ctrl, const float* dr, int n_substeps,
                             cudaStream_t st);
// the branch-parallel step recording the adjoint's substep tape (layout of launch_step_tape)
cudaError_t launch_branch_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                               int tape_rows, cudaStream_t st);

// kernel launchers (step.cu)
cudaError_t launch_step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                        const float* dr = nullptr, const pg_step_out* out = nullptr);
cudaError_t launch_debug(const pg_batch* b, const pg_state* s, const float* ctrl, int64_t env, float* out,
                         cudaStream_t st);
cudaError_t launch_reset(const pg_batch* b, const pg_state* s, const uint8_t* mask, const float* qpos0,
                         const float* qvel0, cudaStream_t st);
cudaError_t configure_step_kernels(size_t smem_bytes);
// environment step and reset of a locomotion task (step.cu)
cudaError_t launch_env_step(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps, cudaStream_t st,
                            const float* dr = nullptr);
cudaError_t launch_env_reset(const pg_batch* b, const pg_state* s, const EnvArgs& E, cudaStream_t st);
cudaError_t launch_step_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                             int tape_rows, cudaStream_t st);
// the kernels of step_kernels.cuh, compiled without (step.cu) and with (step_elliptic.cu) the
// elliptic cone
#define PG_DECLARE_STEP_KERNELS(NS)                                                                               \
  namespace NS {                                                                                                 \
  cudaError_t configure(size_t smem_bytes);                                                                      \
  cudaError_t step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,     \
                   const float* dr = nullptr, const pg_step_out* out = nullptr);                                 \
  cudaError_t step_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,     \
                        int tape_rows, cudaStream_t st);                                                         \
  cudaError_t debug(const pg_batch* b, const pg_state* s, const float* ctrl, int64_t env, float* out,            \
                    cudaStream_t st);                                                                            \
  cudaError_t step_spec(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,\
                        const float* dr = nullptr, const pg_step_out* out = nullptr);                            \
  cudaError_t step_spec_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,\
                             int tape_rows, cudaStream_t st);                                                   \
  cudaError_t step_env(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps, cudaStream_t st,   \
                       const float* dr = nullptr, int phase = 0);                                               \
  cudaError_t step_spec_env(const pg_batch* b, const pg_state* s, const EnvArgs& E, int n_substeps,            \
                            cudaStream_t st, const float* dr = nullptr, int phase = 0);                        \
  cudaError_t step_spec_parts(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps,          \
                              cudaStream_t st, const pg_step_out* out = nullptr);                              \
  }
PG_DECLARE_STEP_KERNELS(pyramidal)
PG_DECLARE_STEP_KERNELS(elliptic)
#undef PG_DECLARE_STEP_KERNELS
// adjoint.cu
// Environments per block of the reverse sweep with its workspace (ws_adj_floats floats per
// environment) in shared memory: the widest of kVjpSoa, kVjpSoa/2, ... 8 whose block fits in one
// SM's opt-in shared memory, or 0 when not even 8 fit (the workspace then lives in global memory).
constexpr int kVjpSoa = 16;
inline int vjp_smem_soa(int ws_adj_floats) {
  for (int s = kVjpSoa; s >= 8; s /= 2)
    if ((size_t)4 * s * ws_adj_floats <= (size_t)kMaxSmem) return s;
  return 0;
}

cudaError_t launch_vjp_step(const pg_batch* b, const float* tape, int tape_rows, const float* ctrl, const float* gq,
                            const float* gv, float* adj_q, float* adj_v, float* g_ctrl, float* g_params, float* ws,
                            int64_t ld, int n_substeps, cudaStream_t st);

}  // namespace pg
