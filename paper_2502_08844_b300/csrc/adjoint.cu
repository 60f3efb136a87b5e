// The adjoint's kernel (generic build) and its launcher; the device code is in adjoint_body.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "pg_host.h"
#include "pg_internal.h"
#define PG_WITH_ELLIPTIC 0   // the adjoint covers pyramidal and frictionless contacts
#include "adjoint_body.cuh"

namespace pg {
namespace {

template <bool SMEM>
__global__ void __launch_bounds__(64) vjp_kernel(const __grid_constant__ VjpArgs A) { vjp_body<0, SMEM>(A); }

}  // namespace

cudaError_t launch_vjp_step(const pg_batch* b, const float* tape, int tape_rows, const float* ctrl, const float* gq,
                            const float* gv, float* adj_q, float* adj_v, float* g_ctrl, float* g_params, float* ws,
                            int64_t ld, int n_substeps, cudaStream_t st) {
  if (b->n == 0) return cudaSuccess;
  static thread_local VjpArgs A;
  A.tape = tape; A.ctrl = ctrl; A.gq = gq; A.gv = gv; A.adj_q = adj_q; A.adj_v = adj_v; A.g_ctrl = g_ctrl;
  A.g_params = g_params; A.ws = ws; A.ld = ld; A.n = b->n; A.tape_rows = tape_rows; A.nq_max = b->nq_max;
  A.nv_max = b->nv_max; A.n_substeps = n_substeps; A.nmodels = (int)b->models.size();
  for (int k = 0; k < kMaxModels; k++) {
    A.env_end[k] = k < A.nmodels ? b->env_off[k] + b->counts[k] : b->n;
    A.model_off[k] = k < A.nmodels ? b->blob_off[k] : 0;
    A.hfield[k] = b->hfield_ptr[k];
  }
  std::memcpy(A.blob, b->blob_host_adj.data(), b->blob_host_adj.size() * sizeof(uint32_t));
  // the widest shared-memory block every model's workspace fits in (0: global memory)
  int ws_max = 1;
  for (const pg_model* m : b->models) ws_max = std::max(ws_max, m->hdr_adj.ws_adj_floats);
  A.soa = vjp_smem_soa(ws_max);
  // a shared-memory block holds soa environments; the global-memory form runs one warp of
  // consecutive environments (128-byte aligned workspace accesses)
  const int threads = A.soa > 0 ? A.soa : 32;
  const unsigned blocks = (unsigned)((b->n + threads - 1) / threads);
  const size_t smem = (size_t)4 * A.soa * ws_max;
  if (b->spec_kernel_vjp) {   // the batch's model-specialised build (pg_batch_specialize)
    void* params[] = {&A};
    return cudaLaunchKernel((const void*)b->spec_kernel_vjp, dim3(blocks), dim3(threads), params, smem, st);
  }
  static std::mutex mu;
  static unsigned long long configured = 0;
  once_per_device(mu, configured, [] {
    cudaFuncSetAttribute(vjp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    // no shared memory in the global-memory form: the SM's unified cache goes to L1
    cudaFuncSetAttribute(vjp_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  });
  if (A.soa > 0) vjp_kernel<true><<<blocks, threads, smem, st>>>(A);
  else vjp_kernel<false><<<blocks, threads, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace pg
