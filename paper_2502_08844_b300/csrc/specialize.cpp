// Model-specialised step kernels, compiled at run time.
//
// Why: the library's compiled kernel reads the model at run time. That covers the header fields
// and tables (kernel-parameter loads) and the structure-of-arrays stride of the workspace. About
// 40 % of its instructions are this addressing arithmetic and table reads. Compiling the same
// kernel body with the model's blob as a constant array turns all of it into immediates.
//
// How: pg_batch_specialize generates a small source that defines the model's blob and includes
// the kernel body headers, which are embedded in this library at build time. It
// compiles that source with NVRTC (loaded with dlopen on first use) for sm_103a, loads the
// cubin with cudaLibraryLoadData, and from then on pg_step launches that kernel for the batch.
// The arithmetic is the same source in the same order, so results equal the generic kernel's.
//
// Cache: compiled cubins are kept per process and on disk, keyed by a hash of the generated
// source and the NVRTC version. The disk cache is $PG_KERNEL_CACHE or
// ~/.cache/paper_2502_08844_b300/kernels.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {

// the kernel sources embedded at build time (generated by build.py)
extern const int kEmbeddedCount;
extern const char* const kEmbeddedNames[];
extern const char* const kEmbeddedTexts[];

namespace {

// ---- NVRTC, resolved at run time ----
typedef int (*nvrtcCreateProgram_t)(void**, const char*, const char*, int, const char* const*, const char* const*);
typedef int (*nvrtcCompileProgram_t)(void*, int, const char* const*);
typedef int (*nvrtcGetSize_t)(void*, size_t*);
typedef int (*nvrtcGetData_t)(void*, char*);
typedef int (*nvrtcDestroyProgram_t)(void**);
typedef int (*nvrtcVersion_t)(int*, int*);

struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcCreateProgram_t create = nullptr;
  nvrtcCompileProgram_t compile = nullptr;
  nvrtcGetSize_t log_size = nullptr, cubin_size = nullptr;
  nvrtcGetData_t log = nullptr, cubin = nullptr;
  nvrtcDestroyProgram_t destroy = nullptr;
  int major = 0, minor = 0;
};

std::mutex g_mutex;
std::map<uint64_t, std::vector<char>> g_cubins;

Nvrtc load_nvrtc() {
  Nvrtc n;
  const char* names[] = {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"};
  void* h = nullptr;
  for (const char* nm : names)
    if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) { n.why = "NVRTC (libnvrtc.so.13) not found"; return n; }
  n.create = (nvrtcCreateProgram_t)dlsym(h, "nvrtcCreateProgram");
  n.compile = (nvrtcCompileProgram_t)dlsym(h, "nvrtcCompileProgram");
  n.log_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetProgramLogSize");
  n.log = (nvrtcGetData_t)dlsym(h, "nvrtcGetProgramLog");
  n.cubin_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetCUBINSize");
  n.cubin = (nvrtcGetData_t)dlsym(h, "nvrtcGetCUBIN");
  n.destroy = (nvrtcDestroyProgram_t)dlsym(h, "nvrtcDestroyProgram");
  nvrtcVersion_t ver = (nvrtcVersion_t)dlsym(h, "nvrtcVersion");
  if (!n.create || !n.compile || !n.log_size || !n.log || !n.cubin_size || !n.cubin || !n.destroy || !ver) {
    n.why = "NVRTC lacks an expected entry point";
    return n;
  }
  ver(&n.major, &n.minor);
  n.ok = true;
  return n;
}

// NVRTC, loaded on first use (a function-local static: initialised once, thread-safe)
const Nvrtc& nvrtc() {
  static const Nvrtc n = load_nvrtc();
  return n;
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char ch : s) { h ^= ch; h *= 1099511628211ull; }
  return h;
}

std::string cache_dir() {
  if (const char* d = getenv("PG_KERNEL_CACHE")) return d;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/paper_2502_08844_b300/kernels";
}

// Cubins compiled ahead of time (pg_model_precompile) into kernel_cache/ beside the library file,
// read only; empty when the library's path is unknown.
const std::string& shipped_cache_dir() {
  static const std::string dir = [] {
    Dl_info info{};
    if (!dladdr((const void*)&shipped_cache_dir, &info) || !info.dli_fname) return std::string();
    const std::string lib = info.dli_fname;
    const size_t slash = lib.rfind('/');
    return (slash == std::string::npos ? std::string(".") : lib.substr(0, slash)) + "/kernel_cache";
  }();
  return dir;
}

void mkdirs(const std::string& path) {
  std::string cur;
  for (size_t i = 0; i < path.size(); i++) {
    cur += path[i];
    if (path[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
  }
  mkdir(path.c_str(), 0755);
}

bool read_file(const std::string& p, std::vector<char>& out) {
  FILE* f = fopen(p.c_str(), "rb");
  if (!f) return false;
  fseek(f, 0, SEEK_END);
  long n = ftell(f);
  fseek(f, 0, SEEK_SET);
  out.resize(n > 0 ? (size_t)n : 0);
  bool ok = n > 0 && fread(out.data(), 1, (size_t)n, f) == (size_t)n;
  fclose(f);
  return ok;
}

void write_file(const std::string& p, const std::vector<char>& data) {
  // a temporary name of this process and call, renamed into place: concurrent writers of one
  // cubin (threads or processes) never see each other's partial file
  static std::atomic<unsigned> serial{0};
  const std::string tmp = p + ".tmp" + std::to_string((long)getpid()) + "." + std::to_string(serial++);
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
  fclose(f);
  if (ok) rename(tmp.c_str(), p.c_str());
  else remove(tmp.c_str());
}

// The generated translation unit: the model's blob as a constant array with the batch's SoA width
// soa (SpecModel<0>, and the header's soa word), then the kernel body and the kernel.
std::string spec_source(const pg_model* m, int soa) {
  std::string s;
  std::vector<uint32_t> blob = m->blob;
  blob[offsetof(ModelHdr, soa) / 4] = (uint32_t)soa;
  s += "#define PG_WITH_ELLIPTIC " + std::string(m->hdr.cone == PG_CONE_ELLIPTIC ? "1" : "0") + "\n";
  s += "#define PG_SPEC 1\n#include \"pg_internal.h\"\nnamespace pg {\ntemplate <int M> struct SpecModel;\n";
  // in the constant bank: reads at compile-time indices fold away, the rest are uniform
  // constant-cache loads (every thread steps the same model)
  s += "__constant__ const uint32_t kSpecBlob[" + std::to_string(blob.size()) + "] __attribute__((aligned(16))) = {";
  for (size_t i = 0; i < blob.size(); i++) {
    if (i % 16 == 0) s += "\n";
    s += std::to_string(blob[i]) + "u,";
  }
  s += "\n};\n";
  const bool adj = m->hdr.adj_ok && m->hdr.cone != PG_CONE_ELLIPTIC;
  if (adj) {   // the same tables with the adjoint's header (its workspace layout)
    s += "__constant__ const uint32_t kSpecBlobAdj[" + std::to_string(m->blob_adj.size()) +
         "] __attribute__((aligned(16))) = {";
    for (size_t i = 0; i < m->blob_adj.size(); i++) {
      if (i % 16 == 0) s += "\n";
      s += std::to_string(m->blob_adj[i]) + "u,";
    }
    s += "\n};\n";
  }
  s += "template <> struct SpecModel<0> {\n  static constexpr int soa = " + std::to_string(soa) +
       ";\n  __device__ static const uint32_t* blob() { return kSpecBlob; }\n";
  if (adj)
    s += "  static constexpr int vjp_soa = " + std::to_string(vjp_smem_soa(m->hdr_adj.ws_adj_floats)) +
         ";\n  __device__ static const uint32_t* blob_adj() { return kSpecBlobAdj; }\n";
  s += "};\n}  // namespace pg\n#include \"step_kernel_body.cuh\"\n";
  const std::string lb = "__launch_bounds__(" + std::to_string(kMaxEnvsPerCta) + ")";
  s += "extern \"C\" __global__ void " + lb + " pg_step_spec(const __grid_constant__ pg::StepArgs A) { pg::step_body<false, false, 0>(A); }\n";
  s += "extern \"C\" __global__ void " + lb + " pg_step_spec_tape(const __grid_constant__ pg::StepArgs A) { pg::step_body<false, true, 0>(A); }\n";
  s += "extern \"C\" __global__ void " + lb + " pg_env_step_spec(const __grid_constant__ pg::StepArgs A) { pg::step_body<false, false, 0, true>(A); }\n";
  s += "extern \"C\" __global__ void " + lb + " pg_step_spec_dr(const __grid_constant__ pg::StepArgs A) { pg::step_body<false, false, 0, false, true>(A); }\n";
  if (adj)
    s += "#include \"adjoint_body.cuh\"\nextern \"C\" __global__ void __launch_bounds__(64) pg_vjp_spec(const __grid_constant__ pg::VjpArgs A) { pg::vjp_body<0, " + std::string(vjp_smem_soa(m->hdr_adj.ws_adj_floats) > 0 ? "true" : "false") + ">(A); }\n";
  return s;
}

// NVRTC: the cubin of a generated source for sm_103a
int nvrtc_compile(const std::string& src, const char* name, std::vector<char>& cubin) {
  const Nvrtc& n = nvrtc();
  void* prog = nullptr;
  if (n.create(&prog, src.c_str(), name, kEmbeddedCount, kEmbeddedTexts, kEmbeddedNames) != 0)
    return set_error(PG_EUNSUPPORTED, "pg_batch_specialize: nvrtcCreateProgram failed");
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
  const int rc = n.compile(prog, 3, opts);
  if (rc != 0) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    n.destroy(&prog);
    return set_error(PG_EUNSUPPORTED, "pg_batch_specialize: NVRTC compilation failed: " + log.substr(0, 2000));
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  cubin.assign(cs, 0);
  n.cubin(prog, cubin.data());
  n.destroy(&prog);
  return PG_OK;
}

// Compile (or find in the caches) the cubin of a generated source.  The caches, in order: this
// process's, the writable disk cache, the cubins shipped beside the library; a miss compiles and
// writes the disk cache.  With out_dir (pg_model_precompile): compile into out_dir unless the
// cubin is there already, and leave `cubin` empty.
int compile_source(const std::string& src, const char* name, std::vector<char>& cubin,
                   const std::string* out_dir = nullptr) {
  const Nvrtc& n = nvrtc();
  if (!n.ok) return set_error(PG_EUNSUPPORTED, "pg_batch_specialize: " + n.why);
  std::string key_src = src + "|nvrtc " + std::to_string(n.major) + "." + std::to_string(n.minor) + "|sm_103a";
  for (int i = 0; i < kEmbeddedCount; i++) key_src += kEmbeddedTexts[i];
  const uint64_t key = fnv1a(key_src);
  char fname[32];
  snprintf(fname, sizeof(fname), "%016llx.cubin", (unsigned long long)key);
  if (out_dir) {
    const std::string path = *out_dir + "/" + fname;
    struct stat st{};
    if (stat(path.c_str(), &st) == 0 && st.st_size > 0) return PG_OK;
    std::vector<char> bin;
    const int rc = nvrtc_compile(src, name, bin);
    if (rc != PG_OK) return rc;
    mkdirs(*out_dir);
    write_file(path, bin);
    return PG_OK;
  }
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_cubins.find(key);
    if (it != g_cubins.end()) { cubin = it->second; return PG_OK; }
  }
  const std::string dir = cache_dir(), path = dir + "/" + fname;
  const std::string& shipped = shipped_cache_dir();
  if (!read_file(path, cubin) && (shipped.empty() || !read_file(shipped + "/" + fname, cubin))) {
    const int rc = nvrtc_compile(src, name, cubin);
    if (rc != PG_OK) return rc;
    mkdirs(dir);
    write_file(path, cubin);
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  g_cubins[key] = cubin;
  return PG_OK;
}

int compile_cubin(const pg_model* m, int soa, std::vector<char>& cubin) {
  return compile_source(spec_source(m, soa), "pg_step_spec.cu", cubin);
}

// the branch-parallel kernel of a model, when it qualifies: lib and kernel set (else NULL, with the
// reason in why)
int compile_branch(const pg_model* m, bool warp_blocks, cudaLibrary_t& lib, cudaKernel_t& kernel,
                   cudaKernel_t& kernel_sync, int& lanes, int& branches, std::string& why,
                   cudaKernel_t* kernel_tape = nullptr, cudaKernel_t* kernel_dr = nullptr) {
  lib = nullptr;
  kernel = nullptr;
  kernel_sync = nullptr;
  if (kernel_tape) *kernel_tape = nullptr;
  if (kernel_dr) *kernel_dr = nullptr;
  std::string src;
  int threads = 0;
  if (branch_plan(m, src, why, lanes, threads, branches) != PG_OK) return PG_OK;
  std::vector<char> cubin;
  int rc = compile_source(src, "pg_step_branch.cu", cubin);
  if (rc != PG_OK) return rc;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e));
  e = cudaLibraryGetKernel(&kernel, lib, "pg_step_branch");
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&kernel_sync, lib, "pg_step_branch_sync");
  if (e == cudaSuccess && kernel_tape) e = cudaLibraryGetKernel(kernel_tape, lib, "pg_step_branch_tape");
  if (e == cudaSuccess && kernel_dr) e = cudaLibraryGetKernel(kernel_dr, lib, "pg_step_branch_dr");
  // a variant that the compiler fitted far worse than the plain barrier kernel (ptxas has fallen
  // back to 32 registers and a large stack frame for some of the humanoid's variants) is not used:
  // its callers keep the thread-per-environment kernels
  if (e == cudaSuccess && kernel_sync) {
    cudaFuncAttributes base{}, var{};
    if (cudaFuncGetAttributes(&base, (const void*)kernel_sync) == cudaSuccess)
      for (cudaKernel_t* v : {kernel_tape, kernel_dr})
        if (v && *v && cudaFuncGetAttributes(&var, (const void*)*v) == cudaSuccess &&
            (var.numRegs < base.numRegs / 2 || var.localSizeBytes > 2 * base.localSizeBytes + 1024))
          *v = nullptr;
    cudaGetLastError();
  }
  if (warp_blocks) kernel_sync = nullptr;   // pg_step launches blocks of one warp, no barrier
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    lib = nullptr;
    kernel = nullptr;
    kernel_sync = nullptr;
    if (kernel_tape) *kernel_tape = nullptr;
    if (kernel_dr) *kernel_dr = nullptr;
    return set_error(PG_ECUDA, std::string("branch kernel set-up: ") + cudaGetErrorString(e));
  }
  why.clear();
  return PG_OK;
}

// the branch-parallel kernel of a single-model batch, when its model qualifies (else the reason
// goes to b->branch_why and the batch keeps its other kernels)
int specialize_branch(pg_batch* b, bool warp_blocks) {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t k = nullptr, ks = nullptr, kt = nullptr, kd = nullptr;
  int lanes = 0, branches = 0;
  const int rc = compile_branch(b->models[0], warp_blocks, lib, k, ks, lanes, branches, b->branch_why,
                                b->models[0]->hdr.adj_ok ? &kt : nullptr, &kd);
  if (rc != PG_OK || !k) return rc;
  b->branch_lib = lib;
  b->branch_kernel = k;
  b->branch_kernel_sync = ks;
  b->branch_kernel_tape = kt;
  b->branch_kernel_dr = kd;
  b->branch_lanes = lanes;
  b->branch_count = branches;
  return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

// A mixed batch: one specialised step kernel per model, each launched over that model's tiles
// (the batch's tiles are grouped by model).  One kernel holding every model's body behind a switch
// measured slower than the generic kernel: blocks of different models share an SM and their large
// specialised bodies evict each other from the instruction cache.  Launched one model after the
// other, each kernel runs alone.  The tape, adjoint, environment and debug kernels stay generic.
// With PG_SPEC_BRANCH every model that qualifies runs its branch-parallel kernel over its own
// environments instead.
static int specialize_parts(pg_batch* b, unsigned flags) {
  std::vector<pg_batch::SpecPart> parts;
  auto fail = [&](int rc) {
    for (const pg_batch::SpecPart& p : parts) {
      cudaLibraryUnload(p.lib);
      if (p.branch_lib) cudaLibraryUnload(p.branch_lib);
    }
    return rc;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  for (int k = 0; k < (int)b->models.size(); k++) {
    const pg_model* m = b->models[k];
    pg_batch::SpecPart part{};
    part.tile0 = -1;
    for (int t = 0; t < b->ntiles; t++)
      if (b->tiles[t].model == k) {
        if (part.tile0 < 0) part.tile0 = t;
        else if (t != part.tile0 + part.ntiles) return fail(set_error(PG_EINVAL, "a model's tiles are not contiguous"));
        part.ntiles++;
      }
    if (part.tile0 < 0) part.tile0 = 0;
    const int soa = b->soa[k], nw = (b->envs_per_cta[k] + soa - 1) / soa;
    part.threads = 32 * nw;
    part.smem = (size_t)4 * nw * soa * m->hdr.ws_floats;
    std::vector<char> cubin;
    int rc = compile_cubin(m, soa, cubin);
    if (rc != PG_OK) return fail(rc);
    e = cudaLibraryLoadData(&part.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return fail(set_error(PG_ECUDA, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e)));
    parts.push_back(part);
    e = cudaLibraryGetKernel(&parts.back().kernel, part.lib, "pg_step_spec");
    if (e == cudaSuccess)
      e = cudaKernelSetAttributeForDevice(parts.back().kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)part.smem, dev);
    if (e != cudaSuccess) return fail(set_error(PG_ECUDA, std::string("specialised kernel set-up: ") + cudaGetErrorString(e)));
    parts.back().env0 = b->env_off[k];
    parts.back().count = b->counts[k];
    parts.back().model = k;
    if (flags & PG_SPEC_BRANCH) {
      int branches = 0;
      std::string why;
      rc = compile_branch(m, (flags & PG_SPEC_BRANCH_WARP) != 0, parts.back().branch_lib, parts.back().branch,
                          parts.back().branch_sync, parts.back().branch_lanes, branches, why);
      if (rc != PG_OK) return fail(rc);
    }
  }
  b->spec_parts = parts;
  return PG_OK;
}

extern "C" int pg_batch_specialize(pg_batch* b) { return pg_batch_specialize_ex(b, PG_SPEC_BRANCH); }

extern "C" int pg_batch_kernel(const pg_batch* b, pg_kernel_info* out) {
  if (!b || !out) return set_error(PG_EINVAL, "batch or out is NULL");
  std::memset(out, 0, sizeof(*out));
  out->lanes_per_env = 1;
  out->envs_per_warp = b->soa.empty() ? 0 : b->soa[0];
  if (b->branch_kernel) {
    out->kernel = PG_KERNEL_BRANCH;
    out->lanes_per_env = b->branch_lanes;
    out->branches = b->branch_count;
    out->sync = b->branch_kernel_sync != nullptr;
    out->branch_dr = b->branch_kernel_dr != nullptr;
    out->branch_tape = b->branch_kernel_tape != nullptr;
  } else if (b->spec_kernel) {
    out->kernel = PG_KERNEL_SPECIALISED;
  } else if (!b->spec_parts.empty()) {
    out->kernel = PG_KERNEL_SPECIALISED_PARTS;
    for (const pg_batch::SpecPart& p : b->spec_parts) out->branch_parts += p.branch ? 1 : 0;
  }
  snprintf(out->reason, sizeof(out->reason), "%s", b->branch_why.c_str());
  return PG_OK;
}

extern "C" int pg_model_branch_plan(const pg_model* m, pg_kernel_info* out) {
  if (!m || !out) return set_error(PG_EINVAL, "model or out is NULL");
  std::memset(out, 0, sizeof(*out));
  std::string src, why;
  int lanes = 0, threads = 0, branches = 0;
  if (branch_plan(m, src, why, lanes, threads, branches) != PG_OK) {
    out->kernel = PG_KERNEL_SPECIALISED;
    out->lanes_per_env = 1;
    snprintf(out->reason, sizeof(out->reason), "%s", why.c_str());
    return PG_OK;
  }
  out->kernel = PG_KERNEL_BRANCH;
  out->lanes_per_env = lanes;
  out->branches = branches;
  if (const char* dump = getenv("PG_BRANCH_SOURCE")) {
    FILE* f = fopen(dump, "w");
    if (f) { fwrite(src.data(), 1, src.size(), f); fclose(f); }
  }
  return PG_OK;
}

extern "C" int pg_model_precompile(const pg_model* m, int64_t count, int envs_per_cta, int sms, unsigned flags,
                                   const char* dir, int* envs_per_warp) {
  if (!m) return set_error(PG_EINVAL, "model is NULL");
  if (count < 0 || sms < 0) return set_error(PG_EINVAL, "negative env count or SM count");
  if (envs_per_cta < 0 || envs_per_cta > kMaxEnvsPerCta) return set_error(PG_EINVAL, "envs_per_cta must be 0 (auto) or 1..256");
  if (flags & ~(PG_SPEC_BRANCH | PG_SPEC_BRANCH_WARP | PG_PRECOMPILE_WIDTH_ONLY))
    return set_error(PG_EINVAL, "unknown pg_model_precompile flags");
  const int soa = thread_soa(m, count, envs_per_cta, sms ? sms : 148);
  if (envs_per_warp) *envs_per_warp = soa;
  if (flags & PG_PRECOMPILE_WIDTH_ONLY) return PG_OK;
  const std::string out = dir && *dir ? std::string(dir) : cache_dir();
  std::vector<char> unused;
  int rc = compile_source(spec_source(m, soa), "pg_step_spec.cu", unused, &out);
  if (rc != PG_OK || !(flags & (PG_SPEC_BRANCH | PG_SPEC_BRANCH_WARP))) return rc;
  std::string src, why;
  int lanes = 0, threads = 0, branches = 0;
  if (branch_plan(m, src, why, lanes, threads, branches) != PG_OK) return PG_OK;   // does not qualify
  return compile_source(src, "pg_step_branch.cu", unused, &out);
}

extern "C" int pg_batch_specialize_ex(pg_batch* b, unsigned flags) {
  if (!b) return set_error(PG_EINVAL, "batch is NULL");
  if (flags & ~(PG_SPEC_BRANCH | PG_SPEC_BRANCH_WARP)) return set_error(PG_EINVAL, "unknown pg_batch_specialize_ex flags");
  if (flags & PG_SPEC_BRANCH_WARP) flags |= PG_SPEC_BRANCH;
  if (b->models.size() != 1) return b->spec_parts.empty() ? specialize_parts(b, flags) : PG_OK;
  if ((flags & PG_SPEC_BRANCH) && !b->branch_kernel) {
    const int rc = specialize_branch(b, (flags & PG_SPEC_BRANCH_WARP) != 0);
    if (rc != PG_OK) return rc;
  }
  if (b->spec_kernel) return PG_OK;
  std::vector<char> cubin;
  int rc = compile_cubin(b->models[0], b->soa[0], cubin);
  if (rc != PG_OK) return rc;
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e));
  cudaKernel_t k = nullptr, kt = nullptr, kv = nullptr, ke = nullptr, kd = nullptr;
  e = cudaLibraryGetKernel(&k, lib, "pg_step_spec");
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&kt, lib, "pg_step_spec_tape");
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&ke, lib, "pg_env_step_spec");
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&kd, lib, "pg_step_spec_dr");
  if (e == cudaSuccess && b->models[0]->hdr.adj_ok && b->models[0]->hdr.cone != PG_CONE_ELLIPTIC)
    e = cudaLibraryGetKernel(&kv, lib, "pg_vjp_spec");
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes, dev);
  if (e == cudaSuccess)
    e = cudaKernelSetAttributeForDevice(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes, dev);
  if (e == cudaSuccess)
    e = cudaKernelSetAttributeForDevice(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes, dev);
  if (e == cudaSuccess)
    e = cudaKernelSetAttributeForDevice(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes, dev);
  if (e == cudaSuccess && kv) {
    if (vjp_smem_soa(b->models[0]->hdr_adj.ws_adj_floats) > 0)   // workspace in shared memory
      e = cudaKernelSetAttributeForDevice(kv, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem, dev);
    else   // workspace in global memory: all of the unified cache to L1
      e = cudaKernelSetAttributeForDevice(kv, cudaFuncAttributePreferredSharedMemoryCarveout, 0, dev);
  }
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    return set_error(PG_ECUDA, std::string("specialised kernel set-up: ") + cudaGetErrorString(e));
  }
  b->spec_lib = lib;
  b->spec_kernel = k;
  b->spec_kernel_tape = kt;
  b->spec_kernel_vjp = kv;
  b->spec_kernel_env = ke;
  b->spec_kernel_dr = kd;
  return PG_OK;
}
