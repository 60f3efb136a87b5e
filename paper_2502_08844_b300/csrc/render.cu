// Batch ray tracer for pixel observations (pg_render).  The paper pairs the batched physics with
// a CUDA batch ray tracer for vision-based policies (Sec. 5, "Batch Rendering with Madrona"); this
// is the library's own: one thread block per environment.  Its first thread runs the
// environment's forward kinematics (the step's device code) into shared memory and writes every
// geom's world frame there; then the block's threads trace the image's pixels, each a primary
// ray against every drawn geom (closest hit, first geom on ties) and, on a hit whose surface faces
// the light, one shadow ray towards it against the other geoms.  Lambertian shading with an
// ambient term.  A scene holds a handful of primitives, so every ray tests them all (a
// bounding-volume hierarchy pays only well above the 64 geoms this kernel takes); capsules and
// boxes are tested only by rays that meet their bounding spheres.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"
#define PG_WITH_ELLIPTIC 0
#include "step_device.cuh"

namespace pg {
namespace {

constexpr int kMaxRenderGeoms = 64;
constexpr float kRayEps = 1e-5f;      // smallest accepted hit distance
constexpr float kShadowLift = 1e-4f;  // shadow rays start this far off the surface, along its normal
constexpr float kMiss = 3.0e38f;

struct RenderArgs {
  const float* qpos;
  int64_t ld, n;
  int width, height, format;
  float cam[3], fwd[3], right[3], up[3];   // right and up scaled by the image-plane half extents
  float light[3];                           // unit vector towards the light
  float ambient, diffuse, bg[3];
  float rgb[3 * kMaxRenderGeoms];
  float lookat[3], upv[3];                  // for per-environment camera positions
  float tan_half, aspect;
  const float* env_cam;                     // [3][ld] per-environment camera offsets, or NULL
  const float* env_light;                   // [3][ld] per-environment light directions, or NULL
  const float* env_tint;                    // [3][ld] per-environment colour multipliers, or NULL
  void* pixels;
  int32_t* hits;
  uint32_t blob[kMaxParamWords];
};
static_assert(sizeof(RenderArgs) <= 32764, "the renderer's argument block must fit the kernel parameter space");

// one geom's world frame: origin, rotation (row-major), size, type
struct GeomFrame {
  float x[3], R[9], s[3];
  float bound2;   // squared radius of a sphere about x holding the shape (slightly enlarged)
  int type;
};

// the ray o + t d (t > 0) misses the ball |y - x|^2 <= r2 around a shape; conservative (a ray that
// starts inside the ball, or meets it, is never pruned), so pruning changes no result
__device__ __forceinline__ bool misses_bound(float3 o, float3 d, float3 x, float r2) {
  const float3 oc = o - x;
  const float b = dot3(oc, d), cc = dot3(oc, oc) - r2;
  return cc > 0.f && (b > 0.f || b * b < cc);
}

__device__ __forceinline__ float3 ld3s(const float* p) { return make_float3(p[0], p[1], p[2]); }

// plane through x with normal nz (both faces): the facing normal at the hit
__device__ __forceinline__ float ray_plane(float3 o, float3 d, float3 x, float3 nz, float3& n) {
  const float den = dot3(nz, d);
  if (fabsf(den) < 1e-12f) return kMiss;
  const float t = dot3(nz, x - o) / den;
  if (!(t > kRayEps)) return kMiss;
  n = den < 0.f ? nz : nz * -1.f;
  return t;
}

// sphere (c, r): the nearer root beyond kRayEps
__device__ __forceinline__ float ray_sphere(float3 o, float3 d, float3 c, float r, float3& n) {
  const float3 oc = o - c;
  const float b = dot3(oc, d), cc = dot3(oc, oc) - r * r;
  const float disc = b * b - cc;
  if (disc < 0.f) return kMiss;
  const float sq = sqrtf(disc);
  float t = -b - sq;
  if (!(t > kRayEps)) t = -b + sq;
  if (!(t > kRayEps)) return kMiss;
  n = (o + d * t - c) * (1.f / r);
  return t;
}

// capsule (frame x, R; radius r, half-length h along its z): the cylinder's side within |z| <= h
// and the two end spheres, nearest first
__device__ float ray_capsule(float3 o, float3 d, float3 x, const float* R, float r, float h, float3& n) {
  const float3 lo = mat_tmul(R, o - x), ld = mat_tmul(R, d);
  float best = kMiss;
  float3 nl = make_float3(0.f, 0.f, 1.f);
  const float a = ld.x * ld.x + ld.y * ld.y;
  if (a > 1e-12f) {
    const float b = lo.x * ld.x + lo.y * ld.y, c = lo.x * lo.x + lo.y * lo.y - r * r;
    const float disc = b * b - a * c;
    if (disc >= 0.f) {
      const float sq = sqrtf(disc);
      for (int k = 0; k < 2; k++) {
        const float t = (-b + (k ? sq : -sq)) / a;
        const float z = lo.z + t * ld.z;
        if (t > kRayEps && t < best && fabsf(z) <= h) {
          best = t;
          nl = make_float3((lo.x + t * ld.x) / r, (lo.y + t * ld.y) / r, 0.f);
        }
      }
    }
  }
  for (int e = 0; e < 2; e++) {
    float3 ns;
    const float t = ray_sphere(lo, ld, make_float3(0.f, 0.f, e ? h : -h), r, ns);
    if (t < best) { best = t; nl = ns; }
  }
  if (best < kMiss) n = mat_mul(R, nl);
  return best;
}

// cylinder (frame x, R; radius r, half-length h along z): the side's roots within |z| <= h and the
// two caps' discs, nearest first; the outward normal
__device__ float ray_cylinder(float3 o, float3 d, float3 x, const float* R, float r, float h, float3& n) {
  const float3 lo = mat_tmul(R, o - x), ld = mat_tmul(R, d);
  float best = kMiss;
  float3 nl = make_float3(0.f, 0.f, 1.f);
  const float a = ld.x * ld.x + ld.y * ld.y;
  if (a > 1e-12f) {
    const float b = lo.x * ld.x + lo.y * ld.y, c = lo.x * lo.x + lo.y * lo.y - r * r;
    const float disc = b * b - a * c;
    if (disc >= 0.f) {
      const float sq = sqrtf(disc);
      for (int k = 0; k < 2; k++) {
        const float t = (-b + (k ? sq : -sq)) / a;
        const float z = lo.z + t * ld.z;
        if (t > kRayEps && t < best && fabsf(z) <= h) {
          best = t;
          nl = make_float3((lo.x + t * ld.x) / r, (lo.y + t * ld.y) / r, 0.f);
        }
      }
    }
  }
  if (fabsf(ld.z) > 1e-12f) {
    for (int e = 0; e < 2; e++) {
      const float zc = e ? h : -h;
      const float t = (zc - lo.z) / ld.z;
      const float px = lo.x + t * ld.x, py = lo.y + t * ld.y;
      if (t > kRayEps && t < best && px * px + py * py <= r * r) {
        best = t;
        nl = make_float3(0.f, 0.f, e ? 1.f : -1.f);
      }
    }
  }
  if (best < kMiss) n = mat_mul(R, nl);
  return best;
}

// box (frame x, R; half-sizes hs): slabs; the entering face's outward normal
__device__ float ray_box(float3 o, float3 d, float3 x, const float* R, float3 hs, float3& n) {
  const float3 lo = mat_tmul(R, o - x), ld = mat_tmul(R, d);
  const float O[3] = {lo.x, lo.y, lo.z}, D[3] = {ld.x, ld.y, ld.z}, H[3] = {hs.x, hs.y, hs.z};
  float tn = -kMiss, tf = kMiss;
  int an = 0, af = 0;
  float sn = 1.f, sf = 1.f;
  for (int k = 0; k < 3; k++) {
    if (fabsf(D[k]) < 1e-12f) {
      if (fabsf(O[k]) > H[k]) return kMiss;
      continue;
    }
    const float inv = 1.f / D[k];
    float t1 = (-H[k] - O[k]) * inv, t2 = (H[k] - O[k]) * inv;
    float s1 = -1.f, s2 = 1.f;   // the face each root lies on
    if (t1 > t2) {
      const float tt = t1; t1 = t2; t2 = tt;
      s1 = 1.f; s2 = -1.f;
    }
    if (t1 > tn) { tn = t1; an = k; sn = s1; }
    if (t2 < tf) { tf = t2; af = k; sf = s2; }
  }
  if (tn > tf || !(tf > kRayEps)) return kMiss;
  const bool inside = !(tn > kRayEps);
  const float t = inside ? tf : tn;
  const int ax = inside ? af : an;
  const float sg = inside ? sf : sn;
  const float3 nl = make_float3(ax == 0 ? sg : 0.f, ax == 1 ? sg : 0.f, ax == 2 ? sg : 0.f);
  n = mat_mul(R, nl);
  return t;
}

__device__ float ray_geom(const GeomFrame& g, float3 o, float3 d, float3& n) {
  const float3 x = ld3s(g.x);
  if (g.type == PG_GEOM_CAPSULE || g.type == PG_GEOM_BOX || g.type == PG_GEOM_CYLINDER) {
    if (misses_bound(o, d, x, g.bound2)) return kMiss;
  }
  switch (g.type) {
    case PG_GEOM_PLANE: return ray_plane(o, d, x, mat_col(g.R, 2), n);
    case PG_GEOM_SPHERE: return ray_sphere(o, d, x, g.s[0], n);
    case PG_GEOM_CAPSULE: return ray_capsule(o, d, x, g.R, g.s[0], g.s[1], n);
    case PG_GEOM_BOX: return ray_box(o, d, x, g.R, ld3s(g.s), n);
    case PG_GEOM_CYLINDER: return ray_cylinder(o, d, x, g.R, g.s[0], g.s[1], n);
    default: return kMiss;
  }
}

// VDR: per-environment visual randomisation (camera offsets, light directions, tints); a separate
// variant, so that the plain kernel carries none of its registers
template <bool VDR>
__global__ void __launch_bounds__(256) render_kernel(const __grid_constant__ RenderArgs A) {
  extern __shared__ __align__(16) float ws[];
  __shared__ GeomFrame frames[kMaxRenderGeoms];
  const int64_t env = blockIdx.x;
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(A.blob);
  const int ng = h.ngeom;
  if (threadIdx.x == 0) {
    Ctx c{h, 1, reinterpret_cast<const int*>(A.blob), reinterpret_cast<const float*>(A.blob), ws, nullptr, A.ld, env};
    for (int k = 0; k < h.nq; k++) W(qpos, k) = A.qpos[k * A.ld + env];
    kinematics<false>(c);
    for (int g = 0; g < ng; g++) {
      float3 bx;
      Quat bq;
      body_frame(c, MI(geom_body, g), bx, bq);
      const float3 x = bx + qrot(bq, T3(&MF(geom_pos, 3 * g)));
      GeomFrame& f = frames[g];
      f.x[0] = x.x; f.x[1] = x.y; f.x[2] = x.z;
      qmat(qnormalize(qmul(bq, Quat{MF(geom_quat, 4 * g), MF(geom_quat, 4 * g + 1), MF(geom_quat, 4 * g + 2),
                                    MF(geom_quat, 4 * g + 3)})), f.R);
      for (int k = 0; k < 3; k++) f.s[k] = MF(geom_size, 3 * g + k);
      f.type = A.rgb[3 * g] < 0.f ? -1 : MI(geom_type, g);   // hidden geoms and heightfields: not drawn
      const float br = f.type == PG_GEOM_CAPSULE ? f.s[0] + f.s[1]
                                                 : sqrtf(f.s[0] * f.s[0] + f.s[1] * f.s[1] + f.s[2] * f.s[2]);
      f.bound2 = br * br * 1.0002f + 1e-8f;
    }
  }
  __syncthreads();
  float3 cam = ld3s(A.cam), fwd = ld3s(A.fwd), right = ld3s(A.right), up = ld3s(A.up), light = ld3s(A.light);
  float tint[3] = {1.f, 1.f, 1.f};
  if (VDR && A.env_cam) {   // this environment's camera: moved, still looking at the same point
    cam = cam + make_float3(A.env_cam[env], A.env_cam[A.ld + env], A.env_cam[2 * A.ld + env]);
    fwd = ld3s(A.lookat) - cam;
    fwd = fwd * rsqrtf(dot3(fwd, fwd));
    float3 r = cross3(fwd, ld3s(A.upv));
    r = r * rsqrtf(dot3(r, r));
    up = cross3(r, fwd) * A.tan_half;
    right = r * (A.tan_half * A.aspect);
  }
  if (VDR && A.env_light) {
    light = make_float3(A.env_light[env], A.env_light[A.ld + env], A.env_light[2 * A.ld + env]) * -1.f;
    light = light * rsqrtf(dot3(light, light));
  }
  if (VDR && A.env_tint)
    for (int k = 0; k < 3; k++) tint[k] = A.env_tint[k * A.ld + env];
  const int W_ = A.width, H_ = A.height, np = W_ * H_;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int px = p % W_, py = p / W_;
    const float sx = 2.f * ((float)px + 0.5f) / (float)W_ - 1.f, sy = 1.f - 2.f * ((float)py + 0.5f) / (float)H_;
    float3 d = fwd + right * sx + up * sy;
    d = d * rsqrtf(dot3(d, d));
    float best = kMiss;
    int hit = -1;
    float3 n = make_float3(0.f, 0.f, 1.f);
    for (int g = 0; g < ng; g++) {
      float3 ng_;
      const float t = ray_geom(frames[g], cam, d, ng_);
      if (t < best) { best = t; hit = g; n = ng_; }
    }
    float col[3] = {A.bg[0], A.bg[1], A.bg[2]};
    int32_t code = 0;
    if (hit >= 0) {
      // direct light reaches the point when its surface faces the light and no other geom blocks
      // the shadow ray; every drawn geom is convex or a plane, so the one hit cannot block a ray
      // that leaves its lit side (the ray stays beyond the surface's tangent plane)
      const float nl = dot3(n, light);
      bool lit = nl > 0.f;
      const float3 q = cam + d * best + n * kShadowLift;
      for (int g = 0; g < ng && lit; g++) {
        float3 dummy;
        if (g != hit && ray_geom(frames[g], q, light, dummy) < kMiss) lit = false;
      }
      const float shade = A.ambient + (lit ? A.diffuse * nl : 0.f);
      for (int k = 0; k < 3; k++) col[k] = A.rgb[3 * hit + k] * shade;
      code = (hit + 1) + (lit ? 0 : 65536);
    }
    if (VDR)
      for (int k = 0; k < 3; k++) col[k] *= tint[k];
    const int64_t pix = env * (int64_t)np + p;
    if (A.format == PG_PIXELS_U8) {
      uint8_t* o = static_cast<uint8_t*>(A.pixels) + 3 * pix;
      for (int k = 0; k < 3; k++) o[k] = (uint8_t)fminf(fmaxf(rintf(255.f * col[k]), 0.f), 255.f);
    } else {
      float* o = static_cast<float*>(A.pixels) + 3 * pix;
      for (int k = 0; k < 3; k++) o[k] = col[k];
    }
    if (A.hits) A.hits[pix] = code;
  }
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" int pg_render(const pg_batch* b, const pg_state* s, const pg_render_desc* d, int format, void* pixels,
                         int32_t* hits, void* stream) {
  if (!b || !s || !d) return set_error(PG_EINVAL, "NULL batch, state or description");
  if (b->models.size() != 1) return set_error(PG_EUNSUPPORTED, "pg_render takes a single-model batch");
  if (s->n != b->n || s->ld < s->n) return set_error(PG_EINVAL, "state does not match the batch");
  if (format != PG_PIXELS_U8 && format != PG_PIXELS_F32) return set_error(PG_EINVAL, "format must be PG_PIXELS_U8 or PG_PIXELS_F32");
  if (d->width < 1 || d->width > 1024 || d->height < 1 || d->height > 1024)
    return set_error(PG_EINVAL, "width and height must lie in 1 .. 1024");
  if (!(d->fovy_deg > 0.f && d->fovy_deg < 180.f)) return set_error(PG_EINVAL, "fovy_deg must lie in (0, 180)");
  if (!d->geom_rgb) return set_error(PG_EINVAL, "NULL geom_rgb");
  const pg_model* m = b->models[0];
  if (m->hdr.ngeom > kMaxRenderGeoms) return set_error(PG_ECAPACITY, "pg_render draws at most 64 geoms");
  if (b->n == 0) return PG_OK;
  if (!pixels || !s->qpos) return set_error(PG_EINVAL, "NULL pixels or qpos");
  // camera basis (double), then the image-plane half extents folded into right / up
  double P[3], F[3], U[3], L[3];
  for (int k = 0; k < 3; k++) { P[k] = d->cam_pos[k]; F[k] = d->cam_lookat[k] - d->cam_pos[k]; U[k] = d->cam_up[k]; L[k] = -d->light_dir[k]; }
  auto norm = [](double* v) {
    const double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(l > 0)) return false;
    for (int k = 0; k < 3; k++) v[k] /= l;
    return true;
  };
  if (!norm(F) || !norm(L)) return set_error(PG_EINVAL, "camera look-at and light direction must be non-zero");
  double Rt[3] = {F[1] * U[2] - F[2] * U[1], F[2] * U[0] - F[0] * U[2], F[0] * U[1] - F[1] * U[0]};
  if (!norm(Rt)) return set_error(PG_EINVAL, "camera up must not be parallel to the view direction");
  double Up[3] = {Rt[1] * F[2] - Rt[2] * F[1], Rt[2] * F[0] - Rt[0] * F[2], Rt[0] * F[1] - Rt[1] * F[0]};
  const double th = std::tan(0.5 * d->fovy_deg * 3.14159265358979323846 / 180.0), asp = (double)d->width / d->height;
  static thread_local RenderArgs A;
  A.qpos = s->qpos; A.ld = s->ld; A.n = s->n;
  A.width = d->width; A.height = d->height; A.format = format;
  for (int k = 0; k < 3; k++) {
    A.cam[k] = (float)P[k]; A.fwd[k] = (float)F[k]; A.right[k] = (float)(Rt[k] * th * asp); A.up[k] = (float)(Up[k] * th);
    A.light[k] = (float)L[k]; A.bg[k] = d->background[k];
  }
  A.ambient = d->ambient; A.diffuse = d->diffuse;
  for (int k = 0; k < 3; k++) { A.lookat[k] = d->cam_lookat[k]; A.upv[k] = d->cam_up[k]; }
  A.tan_half = (float)th;
  A.aspect = (float)asp;
  A.env_cam = d->env_cam_offset; A.env_light = d->env_light_dir; A.env_tint = d->env_tint;
  for (int g = 0; g < m->hdr.ngeom; g++)
    for (int k = 0; k < 3; k++) A.rgb[3 * g + k] = d->geom_rgb[3 * g + k];
  A.pixels = pixels; A.hits = hits;
  std::memcpy(A.blob, m->blob.data(), std::min(m->blob.size(), (size_t)kMaxParamWords) * sizeof(uint32_t));
  const size_t smem = (size_t)4 * m->hdr.ws_floats;
  static std::mutex mu;
  static unsigned long long configured = 0;
  once_per_device(mu, configured, [] {
    cudaFuncSetAttribute(render_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem - 8192);
    cudaFuncSetAttribute(render_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem - 8192);
  });
  if (A.env_cam || A.env_light || A.env_tint)
    render_kernel<true><<<(unsigned)b->n, 256, smem, (cudaStream_t)stream>>>(A);
  else
    render_kernel<false><<<(unsigned)b->n, 256, smem, (cudaStream_t)stream>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("render launch: ") + cudaGetErrorString(e));
  return PG_OK;
}
