// Device functions of the physics step: vector and quaternion algebra, collision primitives and
// every phase of one substep for one environment (a thread), over a structure-of-arrays
// workspace (element i of environment l at w[i * S + l], S the structure-of-arrays width).
// Included by the step kernels and by the adjoint kernels; everything lives in an anonymous
// namespace, one copy per translation unit.
#pragma once
// PG_WITH_ELLIPTIC (0 or 1), set by the including translation unit, says whether its kernels
// handle the elliptic friction cone; with 0 every elliptic branch is compiled out of the loops.
#ifndef PG_WITH_ELLIPTIC
#error "define PG_WITH_ELLIPTIC (0 or 1) before including step_device.cuh"
#endif
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#endif

#include "pg.h"
#include "pg_internal.h"

// PG_SPEC_UNROLL: in a model-specialised build (PG_SPEC, trip counts and tables are constants)
// the tree factorisation, solve and product loops are unrolled completely, so every workspace
// address is a constant and the compiler schedules the loads freely; elsewhere it is empty.
#ifdef PG_SPEC
#define PG_SPEC_UNROLL _Pragma("unroll")
#else
#define PG_SPEC_UNROLL
#endif

namespace pg {
namespace {


// ---------------------------------------------------------------------------------------
// small vector algebra
// ---------------------------------------------------------------------------------------
struct Quat {
  float w, x, y, z;
};

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 ld3(const float* p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ void st3(float* p, float3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
__device__ __forceinline__ Quat ldq(const float* p) { return Quat{p[0], p[1], p[2], p[3]}; }
__device__ __forceinline__ void stq(float* p, Quat q) { p[0] = q.w; p[1] = q.x; p[2] = q.y; p[3] = q.z; }

__device__ __forceinline__ Quat qmul(Quat a, Quat b) {
  return Quat{a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
              a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ Quat qnormalize(Quat q) {
  float s = rsqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return Quat{q.w * s, q.x * s, q.y * s, q.z * s};
}
// rotate v by the unit quaternion q: v + 2 w (u x v) + 2 u x (u x v)
__device__ __forceinline__ float3 qrot(Quat q, float3 v) {
  float3 u = make_float3(q.x, q.y, q.z);
  float3 t = cross3(u, v) * 2.0f;
  return v + t * q.w + cross3(u, t);
}
__device__ __forceinline__ void qmat(Quat q, float* R) {
  float xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z, xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
  float wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
  R[0] = 1 - 2 * (yy + zz); R[1] = 2 * (xy - wz); R[2] = 2 * (xz + wy);
  R[3] = 2 * (xy + wz); R[4] = 1 - 2 * (xx + zz); R[5] = 2 * (yz - wx);
  R[6] = 2 * (xz - wy); R[7] = 2 * (yz + wx); R[8] = 1 - 2 * (xx + yy);
}
__device__ __forceinline__ float3 mat_col(const float* R, int k) { return make_float3(R[k], R[3 + k], R[6 + k]); }
__device__ __forceinline__ float3 mat_mul(const float* R, float3 v) {
  return make_float3(R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
                     R[6] * v.x + R[7] * v.y + R[8] * v.z);
}
__device__ __forceinline__ float3 mat_tmul(const float* R, float3 v) {   // R^T v
  return make_float3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
                     R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

// ---------------------------------------------------------------------------------------
// collision primitives (per thread)
// ---------------------------------------------------------------------------------------
struct Con {
  float dist;
  float3 pos, n;
  int feat = 0;   // capsule endpoint / box corner index of a plane contact
};

__device__ Con sphere_sphere(float3 c1, float r1, float3 c2, float r2) {
  Con k;
  const float3 d = c2 - c1;
  const float L = sqrtf(dot3(d, d));
  k.n = L > 1e-12f ? d * (1.f / L) : make_float3(0.f, 0.f, 1.f);
  k.dist = L - r1 - r2;
  k.pos = ((c1 + k.n * r1) + (c2 - k.n * r2)) * 0.5f;
  return k;
}

__device__ Con plane_sphere(float3 p0, float3 nz, float3 c, float r) {
  Con k;
  const float hgt = dot3(nz, c - p0);
  k.n = nz;
  k.dist = hgt - r;
  k.pos = c - nz * (r + 0.5f * k.dist);
  return k;
}

// sphere (geom1) vs box (geom2): clamped closest point outside, least-penetration face inside
__device__ Con sphere_box(float3 c, float r, float3 bp, const float* bR, float3 hs) {
  Con k;
  const float3 p = mat_tmul(bR, c - bp);
  const float hh[3] = {hs.x, hs.y, hs.z};
  const float pp[3] = {p.x, p.y, p.z};
  float q[3];
  bool inside = true;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    q[i] = fminf(fmaxf(pp[i], -hh[i]), hh[i]);
    if (pp[i] > hh[i] || pp[i] < -hh[i]) inside = false;
  }
  float3 out_dir, surf;
  if (!inside) {
    const float3 dl = make_float3(pp[0] - q[0], pp[1] - q[1], pp[2] - q[2]);
    const float L = sqrtf(dot3(dl, dl));
    out_dir = mat_mul(bR, dl * (1.f / L));
    surf = make_float3(q[0], q[1], q[2]);
    k.dist = L - r;
  } else {
    int kb = 0;
    float best = hh[0] - fabsf(pp[0]);
#pragma unroll
    for (int i = 1; i < 3; i++) {
      const float s = hh[i] - fabsf(pp[i]);
      if (s < best) { best = s; kb = i; }
    }
    const float sg = pp[kb] >= 0.f ? 1.f : -1.f;
    float ev[3] = {0.f, 0.f, 0.f};
    ev[kb] = sg;
    out_dir = mat_mul(bR, make_float3(ev[0], ev[1], ev[2]));
    float sf[3] = {pp[0], pp[1], pp[2]};
    sf[kb] = sg * hh[kb];
    surf = make_float3(sf[0], sf[1], sf[2]);
    k.dist = -(hh[kb] - sg * pp[kb]) - r;
  }
  k.n = out_dir * -1.f;
  k.pos = ((bp + mat_mul(bR, surf)) + (c + k.n * r)) * 0.5f;
  return k;
}

// closest points of c1 + u a1 (|u| <= h1) and c2 + v a2 (|v| <= h2)
__device__ void seg_seg(float3 c1, float3 a1, float h1, float3 c2, float3 a2, float h2, float& u, float& v) {
  const float3 r = c1 - c2;
  const float b = dot3(a1, a2), c = dot3(a1, r), f = dot3(a2, r);
  const float den = 1.f - b * b;
  u = den > 1e-10f ? fminf(fmaxf((b * f - c) / den, -h1), h1) : 0.f;
  v = fminf(fmaxf(b * u + f, -h2), h2);
  u = fminf(fmaxf(b * v - c, -h1), h1);
}

// box-box: separating axes (3 + 3 face normals, 9 edge products), face axes preferred within a
// relative tolerance, face case by clipping the incident face against the reference face's
// side planes, edge case by the closest points of the supporting edges.  Returns the count.
__device__ int box_box(float3 pA, const float* RA, float3 hA3, float3 pB, const float* RB, float3 hB3, Con* out) {
  const float hA[3] = {hA3.x, hA3.y, hA3.z}, hB[3] = {hB3.x, hB3.y, hB3.z};
  float3 A[3], B[3];
#pragma unroll
  for (int k = 0; k < 3; k++) { A[k] = mat_col(RA, k); B[k] = mat_col(RB, k); }
  const float3 dc = pB - pA;
  float best_ov[3] = {0.f, 0.f, 0.f};
  int best_ax[3] = {-1, -1, -1};
  float3 axes_best[3];
  for (int k = 0; k < 15; k++) {
    float3 L;
    if (k < 3) L = A[k];
    else if (k < 6) L = B[k - 3];
    else {
      L = cross3(A[(k - 6) / 3], B[(k - 6) % 3]);
      const float n = sqrtf(dot3(L, L));
      if (!(n > 1e-6f)) continue;
      L = L * (1.f / n);
    }
    float rA = 0.f, rB = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      rA += hA[i] * fabsf(dot3(L, A[i]));
      rB += hB[i] * fabsf(dot3(L, B[i]));
    }
    const float ov = rA + rB - fabsf(dot3(L, dc));
    if (ov < 0.f) return 0;
    const int grp = k < 3 ? 0 : (k < 6 ? 1 : 2);
    if (best_ax[grp] < 0 || ov < best_ov[grp]) { best_ov[grp] = ov; best_ax[grp] = k; axes_best[grp] = L; }
  }
  int g = 0;
  if (best_ov[1] < best_ov[0] - 1e-5f * (1.f + best_ov[0])) g = 1;
  if (best_ax[2] >= 0 && best_ov[2] < best_ov[g] - 1e-5f * (1.f + best_ov[g])) g = 2;
  const float depth = best_ov[g];
  const int best = best_ax[g];
  float3 n = axes_best[g];
  if (dot3(n, dc) < 0.f) n = n * -1.f;
  if (g == 2) {
    const int i = (best - 6) / 3, j = (best - 6) % 3;
    float3 ea = pA, eb = pB;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (k != i) ea = ea + A[k] * (dot3(n, A[k]) >= 0.f ? hA[k] : -hA[k]);
      if (k != j) eb = eb + B[k] * (dot3(n, B[k]) >= 0.f ? -hB[k] : hB[k]);
    }
    float u, v;
    seg_seg(ea, A[i], hA[i], eb, B[j], hB[j], u, v);
    out[0].n = n;
    out[0].dist = -depth;
    out[0].pos = ((ea + A[i] * u) + (eb + B[j] * v)) * 0.5f;
    return 1;
  }
  const bool refA = g == 0;
  const float3 pR = refA ? pA : pB, pI = refA ? pB : pA;
  const float3* AR = refA ? A : B;
  const float3* AI = refA ? B : A;
  const float* hR = refA ? hA : hB;
  const float* hI = refA ? hB : hA;
  const int kr = refA ? best : best - 3;
  const float3 nref = refA ? n : n * -1.f;
  int fk = 0;
  float fs = 1.f, bd = 2.f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float dd = dot3(AI[k], nref);
    if (dd < bd) { bd = dd; fk = k; fs = 1.f; }
    if (-dd < bd) { bd = -dd; fk = k; fs = -1.f; }
  }
  const int ku = (fk + 1) % 3, kv = (fk + 2) % 3;
  float3 poly[8], tmp[8];
  int np = 4;
  const float su[4] = {-1.f, 1.f, 1.f, -1.f}, sv[4] = {-1.f, -1.f, 1.f, 1.f};
#pragma unroll
  for (int c = 0; c < 4; c++) poly[c] = pI + AI[fk] * (fs * hI[fk]) + AI[ku] * (su[c] * hI[ku]) + AI[kv] * (sv[c] * hI[kv]);
  const int ru = (kr + 1) % 3, rv = (kr + 2) % 3;
  for (int pl = 0; pl < 4 && np > 0; pl++) {
    const float3 pn = (pl < 2 ? AR[ru] : AR[rv]) * ((pl % 2 == 0) ? 1.f : -1.f);
    const float ph = pl < 2 ? hR[ru] : hR[rv];
    int no = 0;
    float3 S = poly[np - 1];
    float sS = ph - dot3(S - pR, pn);
    for (int q = 0; q < np; q++) {
      const float3 E = poly[q];
      const float sE = ph - dot3(E - pR, pn);
      if (sE >= 0.f) {
        if (sS < 0.f && no < 8) tmp[no++] = S + (E - S) * (sS / (sS - sE));
        if (no < 8) tmp[no++] = E;
      } else if (sS >= 0.f && no < 8) {
        tmp[no++] = S + (E - S) * (sS / (sS - sE));
      }
      S = E;
      sS = sE;
    }
    np = no;
    for (int q = 0; q < np; q++) poly[q] = tmp[q];
  }
  float dep[8];
  int idx[8], nk = 0;
  for (int q = 0; q < np; q++) {
    dep[q] = hR[kr] - dot3(poly[q] - pR, nref);
    if (dep[q] >= 0.f) idx[nk++] = q;
  }
  if (nk > 4) {
    int keep[4];
    int p0 = idx[0];
    for (int q = 0; q < nk; q++) if (dep[idx[q]] > dep[p0]) p0 = idx[q];
    int p1 = -1; float b1 = -1.f;
    for (int q = 0; q < nk; q++) {
      const int i = idx[q];
      if (i == p0) continue;
      const float3 dd = poly[i] - poly[p0];
      const float dv = sqrtf(dot3(dd, dd));
      if (dv > b1) { b1 = dv; p1 = i; }
    }
    int p2 = -1; float b2 = -1.f;
    for (int q = 0; q < nk; q++) {
      const int i = idx[q];
      if (i == p0 || i == p1) continue;
      const float3 cr = cross3(poly[p1] - poly[p0], poly[i] - poly[p0]);
      const float a = sqrtf(dot3(cr, cr));
      if (a > b2) { b2 = a; p2 = i; }
    }
    int p3 = -1; float b3 = -1.f;
    for (int q = 0; q < nk; q++) {
      const int i = idx[q];
      if (i == p0 || i == p1 || i == p2) continue;
      const float3 c1 = cross3(poly[p1] - poly[p0], poly[i] - poly[p0]);
      const float3 c2 = cross3(poly[p2] - poly[p1], poly[i] - poly[p1]);
      const float3 c3 = cross3(poly[p0] - poly[p2], poly[i] - poly[p2]);
      const float a = sqrtf(dot3(c1, c1)) + sqrtf(dot3(c2, c2)) + sqrtf(dot3(c3, c3));
      if (a > b3) { b3 = a; p3 = i; }
    }
    keep[0] = p0; keep[1] = p1; keep[2] = p2; keep[3] = p3;
    // polygon order
    for (int a = 0; a < 4; a++)
      for (int b = a + 1; b < 4; b++)
        if (keep[b] < keep[a]) { const int t = keep[a]; keep[a] = keep[b]; keep[b] = t; }
    for (int a = 0; a < 4; a++) idx[a] = keep[a];
    nk = 4;
  }
  for (int c = 0; c < nk; c++) {
    const int i = idx[c];
    out[c].n = n;
    out[c].dist = -dep[i];
    out[c].pos = poly[i] + nref * (0.5f * dep[i]);
  }
  return nk;
}

// frame: t1 = normalise(n x e_k) with e_k the world axis of smallest |n_k| (ties: lowest k)
__device__ __forceinline__ void contact_frame(float3 n, float3& t1, float3& t2) {
  const float a0 = fabsf(n.x), a1 = fabsf(n.y), a2 = fabsf(n.z);
  int k = 0;
  if (a1 < a0) k = 1;
  if (a2 < (k == 0 ? a0 : a1)) k = 2;
  const float3 ek = make_float3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f);
  float3 t = cross3(n, ek);
  t1 = t * rsqrtf(dot3(t, t));
  t2 = cross3(n, t1);
}

// ---------------------------------------------------------------------------------------
// per-environment context: model tables in shared memory (broadcast reads), the thread's
// structure-of-arrays workspace (element i at w[32 i]) and its controls in global memory
// ---------------------------------------------------------------------------------------
struct Ctx {
  const ModelHdr& h;
  int S;   // element stride of the structure-of-arrays workspace (environments per warp block)
  const int* __restrict__ I;
  const float* __restrict__ F;
  float* __restrict__ w;
  const float* __restrict__ ctrl;
  int64_t ld;
  int64_t env;
  const float* __restrict__ hf;   // the model's heightfield elevations (device memory), or NULL
  const float* __restrict__ dr;   // per-environment parameters ([nrand][ld], pg_step_dr), or NULL
};


#define MI(name, i) (c.I[c.h.o_##name + (i)])
#define MF(name, i) (c.F[c.h.o_##name + (i)])
#define W(name, i) (c.w[(c.h.w_##name + (i)) * c.S])

__device__ __forceinline__ float3 W3(const Ctx& c, int off) {
  return make_float3(c.w[off * c.S], c.w[(off + 1) * c.S], c.w[(off + 2) * c.S]);
}
__device__ __forceinline__ void S3(const Ctx& c, int off, float3 v) {
  c.w[off * c.S] = v.x; c.w[(off + 1) * c.S] = v.y; c.w[(off + 2) * c.S] = v.z;
}
__device__ __forceinline__ float3 T3(const float* t) { return make_float3(t[0], t[1], t[2]); }

// row k of this environment's parameters (pg_step_dr)
__device__ __forceinline__ float dr_row(const Ctx& c, int k) { return __ldg(c.dr + k * c.ld + c.env); }

// body b's link mass scale 1 + s_b (mass and inertia about the centre of mass), 1 without
// per-environment parameters
__device__ __forceinline__ float mass_scale(const Ctx& c, int b) {
  return c.dr ? 1.f + dr_row(c, c.h.dr_mass + b) : 1.f;
}

// body b's mass and centre of mass (body frame), with this environment's link mass scale, its
// payload on body 1 and its centre-of-mass offsets
__device__ __forceinline__ void body_massprops(const Ctx& c, int b, float& m, float3& ipos) {
  m = MF(body_mass, b);
  ipos = T3(&MF(body_ipos, 3 * b));
  if (c.dr) {
    m *= mass_scale(c, b);
    if (b == 1) m += dr_row(c, 1);
    ipos = ipos + make_float3(dr_row(c, c.h.dr_com + 3 * b), dr_row(c, c.h.dr_com + 3 * b + 1),
                              dr_row(c, c.h.dr_com + 3 * b + 2));
  }
}

// actuator a's force at control u (motor: gear * u; PD: kp (u + calibration - q) - kd qd, the
// gains scaled by this environment's 1 + s), u already clipped to a limited control range, then
// clipped to a limited force range
__device__ __forceinline__ float actuator_force(const Ctx& c, int a, float u) {
  float tau;
  if (MI(act_type, a) == PG_ACT_MOTOR) {
    tau = MF(act_gear, a) * u;
  } else {
    float kp = MF(act_kp, a), kd = MF(act_kd, a);
    if (c.dr) {
      u += dr_row(c, c.h.dr_cal + a);
      kp *= 1.f + dr_row(c, c.h.dr_kp + a);
      kd *= 1.f + dr_row(c, c.h.dr_kd + a);
    }
    tau = kp * (u - W(qpos, MI(act_qposadr, a))) - kd * W(qvel, MI(act_dof, a));
  }
  if (MI(act_forcelimited, a)) tau = fminf(fmaxf(tau, MF(act_forcerange, 2 * a)), MF(act_forcerange, 2 * a + 1));
  return tau;
}

// reference point of body b's tree: the free root's position, else the root's fixed frame origin
__device__ __forceinline__ float3 tree_origin(const Ctx& c, int b) {
  const int r = MI(body_root, b), fa = MI(root_freeadr, r);
  if (fa >= 0) return W3(c, c.h.w_qpos + fa);
  return T3(&MF(body_pos, 3 * r));
}

__device__ __forceinline__ void body_frame(const Ctx& c, int b, float3& x, Quat& q) {
  if (b == 0) {
    x = make_float3(0.f, 0.f, 0.f);
    q = Quat{1.f, 0.f, 0.f, 0.f};
  } else {
    x = W3(c, c.h.w_xpos + 3 * b);
    const int o = c.h.w_xquat + 4 * b;
    q = Quat{c.w[o * c.S], c.w[(o + 1) * c.S], c.w[(o + 2) * c.S], c.w[(o + 3) * c.S]};
  }
}

// ---------------------------------------------------------------------------------------
// kinematics: bodies in level order (parent before child), each from its parent's frame, the
// body offset and its joints (hinge: rotation about the axis through the anchor; slide:
// translation; free: qpos position and normalised quaternion).  On the way: the motion
// subspace of every dof (cdof, angular;linear about the tree's reference point o) and the
// body's spatial inertia about o (Ixx Iyy Izz Ixy Ixz Iyz, m c, m); INERTIA = false skips the
// inertias (frames and motion subspaces only).
// ---------------------------------------------------------------------------------------
template <bool INERTIA = true>
__device__ void kinematics(const Ctx& c) {
  const ModelHdr& h = c.h;
  for (int b = 1; b < h.nbody; b++) {
    float3 x;
    Quat q;
    body_frame(c, MI(body_parent, b), x, q);
    x = x + qrot(q, T3(&MF(body_pos, 3 * b)));
    q = qmul(q, Quat{MF(body_quat, 4 * b), MF(body_quat, 4 * b + 1), MF(body_quat, 4 * b + 2), MF(body_quat, 4 * b + 3)});
    const float3 o = tree_origin(c, b);
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    for (int j = j0; j < j0 + nj; j++) {
      const int type = MI(jnt_type, j), qa = MI(jnt_qposadr, j), d0 = MI(jnt_dofadr, j);
      if (type == PG_JNT_FREE) {
        x = W3(c, h.w_qpos + qa);
        q = qnormalize(Quat{W(qpos, qa + 3), W(qpos, qa + 4), W(qpos, qa + 5), W(qpos, qa + 6)});
        float R[9];
        qmat(q, R);
        for (int k = 0; k < 3; k++) {
          S3(c, h.w_cdof + 6 * (d0 + k), make_float3(0.f, 0.f, 0.f));
          S3(c, h.w_cdof + 6 * (d0 + k) + 3, make_float3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f));
          const float3 ax = mat_col(R, k);
          S3(c, h.w_cdof + 6 * (d0 + 3 + k), ax);
          S3(c, h.w_cdof + 6 * (d0 + 3 + k) + 3, cross3(ax, o - x));
        }
      } else {
        const float3 lp = T3(&MF(jnt_pos, 3 * j)), la = T3(&MF(jnt_axis, 3 * j));
        const float3 anchor = x + qrot(q, lp), axis = qrot(q, la);
        if (type == PG_JNT_HINGE) {
          S3(c, h.w_cdof + 6 * d0, axis);
          S3(c, h.w_cdof + 6 * d0 + 3, cross3(axis, o - anchor));
          float sn, cs;
          sincosf(0.5f * W(qpos, qa), &sn, &cs);
          q = qmul(q, Quat{cs, la.x * sn, la.y * sn, la.z * sn});
          x = anchor - qrot(q, lp);
        } else {
          S3(c, h.w_cdof + 6 * d0, make_float3(0.f, 0.f, 0.f));
          S3(c, h.w_cdof + 6 * d0 + 3, axis);
          x = x + axis * W(qpos, qa);
        }
      }
    }
    q = qnormalize(q);
    S3(c, h.w_xpos + 3 * b, x);
    const int qo = h.w_xquat + 4 * b;
    c.w[qo * c.S] = q.w; c.w[(qo + 1) * c.S] = q.x; c.w[(qo + 2) * c.S] = q.y; c.w[(qo + 3) * c.S] = q.z;
    if (!INERTIA) continue;
    // spatial inertia about o: I_com(world) + m (|c|^2 1 - c c^T), h = m c
    float R[9];
    qmat(q, R);
    float m;
    float3 ip;
    body_massprops(c, b, m, ip);
    const float3 com = x + mat_mul(R, ip);
    const float* In = &MF(body_inertia, 6 * b);
    const float ms = mass_scale(c, b);
    const float Ib[9] = {ms * In[0], ms * In[3], ms * In[4], ms * In[3], ms * In[1],
                         ms * In[5], ms * In[4], ms * In[5], ms * In[2]};
    float T[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int k = 0; k < 3; k++) T[3 * r + k] = R[3 * r] * Ib[k] + R[3 * r + 1] * Ib[3 + k] + R[3 * r + 2] * Ib[6 + k];
    const float3 cc = com - o;
    const float c2 = dot3(cc, cc);
    const int ci = h.w_cinert + 10 * b;
    c.w[(ci + 0) * c.S] = T[0] * R[0] + T[1] * R[1] + T[2] * R[2] + m * (c2 - cc.x * cc.x);
    c.w[(ci + 1) * c.S] = T[3] * R[3] + T[4] * R[4] + T[5] * R[5] + m * (c2 - cc.y * cc.y);
    c.w[(ci + 2) * c.S] = T[6] * R[6] + T[7] * R[7] + T[8] * R[8] + m * (c2 - cc.z * cc.z);
    c.w[(ci + 3) * c.S] = T[0] * R[3] + T[1] * R[4] + T[2] * R[5] - m * cc.x * cc.y;
    c.w[(ci + 4) * c.S] = T[0] * R[6] + T[1] * R[7] + T[2] * R[8] - m * cc.x * cc.z;
    c.w[(ci + 5) * c.S] = T[3] * R[6] + T[4] * R[7] + T[5] * R[8] - m * cc.y * cc.z;
    c.w[(ci + 6) * c.S] = m * cc.x;
    c.w[(ci + 7) * c.S] = m * cc.y;
    c.w[(ci + 8) * c.S] = m * cc.z;
    c.w[(ci + 9) * c.S] = m;
  }
}

// spatial inertia (about o) times a motion vector (w; v)
__device__ __forceinline__ void inert_mul(const Ctx& c, int ci, float3 w, float3 v, float3& fa, float3& fl) {
  const float* q = c.w + ci * c.S;
  const int S = c.S;
  const float i0 = q[0], i1 = q[S], i2 = q[2 * S], i3 = q[3 * S], i4 = q[4 * S], i5 = q[5 * S];
  const float3 hc = make_float3(q[6 * S], q[7 * S], q[8 * S]);
  const float m = q[9 * S];
  fa = make_float3(i0 * w.x + i3 * w.y + i4 * w.z, i3 * w.x + i1 * w.y + i5 * w.z, i4 * w.x + i5 * w.y + i2 * w.z) +
       cross3(hc, v);
  fl = v * m - cross3(hc, w);
}

// ---------------------------------------------------------------------------------------
// RNEA bias forces c(q, qdot): velocities and bias accelerations outward (the world
// accelerates by -gravity), body forces I a + v x* I v accumulated inward, projected on cdof.
// Serial joints of one body act as massless intermediate frames; the free joint's three
// rotations all take the velocity after its translation (their axes move with the body).
// ---------------------------------------------------------------------------------------
__device__ void rnea(const Ctx& c) {
  const ModelHdr& h = c.h;
  for (int b = 1; b < h.nbody; b++) {
    const int p = MI(body_parent, b);
    float3 w, v, aw, av;
    if (p == 0) {
      w = v = aw = make_float3(0.f, 0.f, 0.f);
      av = make_float3(-h.grav[0], -h.grav[1], -h.grav[2]);
    } else {
      w = W3(c, h.w_cvel + 6 * p); v = W3(c, h.w_cvel + 6 * p + 3);
      aw = W3(c, h.w_cacc + 6 * p); av = W3(c, h.w_cacc + 6 * p + 3);
    }
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    for (int j = j0; j < j0 + nj; j++) {
      const int d0 = MI(jnt_dofadr, j);
      float3 dw, dv;
      if (MI(jnt_type, j) == PG_JNT_FREE) {
        v = v + make_float3(W(qvel, d0), W(qvel, d0 + 1), W(qvel, d0 + 2));
        dw = dv = make_float3(0.f, 0.f, 0.f);
        for (int k = 3; k < 6; k++) {
          const float qd = W(qvel, d0 + k);
          dw = dw + W3(c, h.w_cdof + 6 * (d0 + k)) * qd;
          dv = dv + W3(c, h.w_cdof + 6 * (d0 + k) + 3) * qd;
        }
      } else {
        const float qd = W(qvel, d0);
        dw = W3(c, h.w_cdof + 6 * d0) * qd;
        dv = W3(c, h.w_cdof + 6 * d0 + 3) * qd;
      }
      aw = aw + cross3(w, dw);
      av = av + cross3(w, dv) + cross3(v, dw);
      w = w + dw;
      v = v + dv;
    }
    S3(c, h.w_cvel + 6 * b, w); S3(c, h.w_cvel + 6 * b + 3, v);
    S3(c, h.w_cacc + 6 * b, aw); S3(c, h.w_cacc + 6 * b + 3, av);
    float3 fa, fl, ia, il;
    inert_mul(c, h.w_cinert + 10 * b, aw, av, fa, fl);
    inert_mul(c, h.w_cinert + 10 * b, w, v, ia, il);
    S3(c, h.w_cfrc + 6 * b, fa + cross3(w, ia) + cross3(v, il));
    S3(c, h.w_cfrc + 6 * b + 3, fl + cross3(w, il));
  }
  for (int b = h.nbody - 1; b >= 1; b--) {
    const int p = MI(body_parent, b);
    if (p == 0) continue;
    for (int k = 0; k < 6; k++) W(cfrc, 6 * p + k) += W(cfrc, 6 * b + k);
  }
  for (int d = 0; d < h.nv; d++) {
    const int f = h.w_cfrc + 6 * MI(dof_body, d);
    W(bias, d) = dot3(W3(c, h.w_cdof + 6 * d), W3(c, f)) + dot3(W3(c, h.w_cdof + 6 * d + 3), W3(c, f + 3));
  }
}

// ---------------------------------------------------------------------------------------
// CRBA: composite inertias (inward sum, in place), M_ji = cdof_i . (Ic(body j) cdof_j) for i on
// j's dof chain, armature on the diagonal, stored packed (row j: j, parent(j), ...)
// ---------------------------------------------------------------------------------------
__device__ void crba(const Ctx& c) {
  const ModelHdr& h = c.h;
  for (int b = h.nbody - 1; b >= 1; b--) {
    const int p = MI(body_parent, b);
    if (p == 0) continue;
    for (int k = 0; k < 10; k++) W(cinert, 10 * p + k) += W(cinert, 10 * b + k);
  }
  for (int j = 0; j < h.nv; j++) {
    float3 fa, fl;
    inert_mul(c, h.w_cinert + 10 * MI(dof_body, j), W3(c, h.w_cdof + 6 * j), W3(c, h.w_cdof + 6 * j + 3), fa, fl);
    const int r0 = MI(dof_rowadr, j), n = MI(dof_depth, j) + 1;
    for (int t = 0; t < n; t++) {
      const int i = MI(Lcol, r0 + t);
      float v = dot3(W3(c, h.w_cdof + 6 * i), fa) + dot3(W3(c, h.w_cdof + 6 * i + 3), fl);
      if (t == 0) v += MF(dof_armature, j) + (c.dr ? dr_row(c, h.dr_arm + j) : 0.f);
      W(M, r0 + t) = v;
    }
  }
}

// packed tree-sparse factorisation in place: A = L^T D L, L unit lower triangular on the
// ancestor pattern (no fill-in); row k ends as (D_k, L_k,parent(k), ...)
// (The inner loops below move 4 entries at a time: all loads of a chunk first, then the
// arithmetic, then the stores.  Row segments never overlap, so this is the same arithmetic in the
// same order per entry; it lets the shared-memory loads of a chunk overlap instead of waiting
// behind the previous store, which the compiler cannot prove independent.)
__device__ void ldl_factor(const Ctx& c, int A) {
  const ModelHdr& h = c.h;
  const int S = c.S;
  float* a = c.w + A * S;
  PG_SPEC_UNROLL
  for (int k = h.nv - 1; k >= 0; k--) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    const float dinv = __frcp_rn(a[r0 * S]);   // = 1 / pivot, correctly rounded
    PG_SPEC_UNROLL
    for (int t = 1; t <= dk; t++) {
      const int ri = MI(dof_rowadr, MI(Lcol, r0 + t));
      const float lt = a[(r0 + t) * S] * dinv;
      float* dst = a + (ri - t) * S;   // entry s of row k updates entry s - t of row i
      int s = t;
      for (; s + 3 <= dk; s += 4) {
        const float x0 = a[(r0 + s) * S], x1 = a[(r0 + s + 1) * S], x2 = a[(r0 + s + 2) * S], x3 = a[(r0 + s + 3) * S];
        const float y0 = dst[s * S], y1 = dst[(s + 1) * S], y2 = dst[(s + 2) * S], y3 = dst[(s + 3) * S];
        dst[s * S] = y0 - lt * x0;
        dst[(s + 1) * S] = y1 - lt * x1;
        dst[(s + 2) * S] = y2 - lt * x2;
        dst[(s + 3) * S] = y3 - lt * x3;
      }
      for (; s <= dk; s++) dst[s * S] -= lt * a[(r0 + s) * S];
    }
    for (int t = 1; t <= dk; t++) a[(r0 + t) * S] *= dinv;
  }
}

// x <- A^-1 x with the packed factor of A (x: element offset of an nv-vector)
__device__ void ldl_solve(const Ctx& c, int A, int X) {
  const ModelHdr& h = c.h;
  const float* a = c.w + A * c.S;
  float* x = c.w + X * c.S;
  const int S = c.S;
  PG_SPEC_UNROLL
  for (int k = h.nv - 1; k >= 0; k--) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    const float xk = x[k * S];
    int t = 1;
    for (; t + 3 <= dk; t += 4) {
      const int i0 = MI(Lcol, r0 + t), i1 = MI(Lcol, r0 + t + 1), i2 = MI(Lcol, r0 + t + 2), i3 = MI(Lcol, r0 + t + 3);
      const float a0 = a[(r0 + t) * S], a1 = a[(r0 + t + 1) * S], a2 = a[(r0 + t + 2) * S], a3 = a[(r0 + t + 3) * S];
      const float y0 = x[i0 * S], y1 = x[i1 * S], y2 = x[i2 * S], y3 = x[i3 * S];
      x[i0 * S] = y0 - a0 * xk;
      x[i1 * S] = y1 - a1 * xk;
      x[i2 * S] = y2 - a2 * xk;
      x[i3 * S] = y3 - a3 * xk;
    }
    for (; t <= dk; t++) x[MI(Lcol, r0 + t) * S] -= a[(r0 + t) * S] * xk;
  }
  for (int k = 0; k < h.nv; k++) x[k * S] /= a[MI(dof_rowadr, k) * S];
  PG_SPEC_UNROLL
  for (int k = 0; k < h.nv; k++) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    float s = x[k * S];
    int t = 1;
    for (; t + 3 <= dk; t += 4) {
      const float a0 = a[(r0 + t) * S], a1 = a[(r0 + t + 1) * S], a2 = a[(r0 + t + 2) * S], a3 = a[(r0 + t + 3) * S];
      const float y0 = x[MI(Lcol, r0 + t) * S], y1 = x[MI(Lcol, r0 + t + 1) * S], y2 = x[MI(Lcol, r0 + t + 2) * S],
                  y3 = x[MI(Lcol, r0 + t + 3) * S];
      s -= a0 * y0;
      s -= a1 * y1;
      s -= a2 * y2;
      s -= a3 * y3;
    }
    for (; t <= dk; t++) s -= a[(r0 + t) * S] * x[MI(Lcol, r0 + t) * S];
    x[k * S] = s;
  }
}

// y = M x with M stored packed symmetric (x, y: element offsets of nv-vectors)
__device__ void sym_mul(const Ctx& c, int Mo, int X, int Y) {
  const ModelHdr& h = c.h;
  const float* m = c.w + Mo * c.S;
  const float* x = c.w + X * c.S;
  float* y = c.w + Y * c.S;
  const int S = c.S;
  for (int j = 0; j < h.nv; j++) y[j * S] = 0.f;
  PG_SPEC_UNROLL
  for (int j = 0; j < h.nv; j++) {
    const int r0 = MI(dof_rowadr, j), dj = MI(dof_depth, j);
    const float xj = x[j * S];
    float yj = m[r0 * S] * xj;
    int t = 1;
    for (; t + 3 <= dj; t += 4) {   // chunks of 4: loads first (see ldl_factor)
      const int i0 = MI(Lcol, r0 + t), i1 = MI(Lcol, r0 + t + 1), i2 = MI(Lcol, r0 + t + 2), i3 = MI(Lcol, r0 + t + 3);
      const float m0 = m[(r0 + t) * S], m1 = m[(r0 + t + 1) * S], m2 = m[(r0 + t + 2) * S], m3 = m[(r0 + t + 3) * S];
      const float x0 = x[i0 * S], x1 = x[i1 * S], x2 = x[i2 * S], x3 = x[i3 * S];
      const float y0 = y[i0 * S], y1 = y[i1 * S], y2 = y[i2 * S], y3 = y[i3 * S];
      yj = fmaf(m0, x0, yj);
      yj = fmaf(m1, x1, yj);
      yj = fmaf(m2, x2, yj);
      yj = fmaf(m3, x3, yj);
      y[i0 * S] = fmaf(m0, xj, y0);
      y[i1 * S] = fmaf(m1, xj, y1);
      y[i2 * S] = fmaf(m2, xj, y2);
      y[i3 * S] = fmaf(m3, xj, y3);
    }
    for (; t <= dj; t++) {
      const int i = MI(Lcol, r0 + t);
      const float mji = m[(r0 + t) * S];
      yj = fmaf(mji, x[i * S], yj);
      y[i * S] = fmaf(mji, xj, y[i * S]);
    }
    y[j * S] += yj;
  }
}

// passive (joint damping) and actuator forces (motor: gear * clamp(u); PD: kp (u - q) - kd qd),
// then a0 = M^-1 (tau - c)
template <bool DEBUG>
__device__ void smooth_acc(const Ctx& c, float* dbg) {
  const ModelHdr& h = c.h;
  for (int d = 0; d < h.nv; d++) {
    const float pas = -MF(dof_damping, d) * W(qvel, d);
    W(a0, d) = pas - W(bias, d);
    if (DEBUG) { dbg[h.dbg_passive + d] = pas; dbg[h.dbg_act + d] = 0.f; dbg[h.dbg_bias + d] = W(bias, d); }
  }
  for (int a = 0; a < h.nu; a++) {
    const int d = MI(act_dof, a);
    float u = c.ctrl[a * c.ld + c.env];
    if (MI(act_ctrllimited, a)) u = fminf(fmaxf(u, MF(act_range, 2 * a)), MF(act_range, 2 * a + 1));
    const float tau = actuator_force(c, a, u);
    W(a0, d) += tau;
    if (DEBUG) dbg[h.dbg_act + d] += tau;
  }
  for (int k = 0; k < h.nL; k++) W(L, k) = W(M, k);
  ldl_factor(c, h.w_L);
  ldl_solve(c, h.w_L, h.w_a0);
  for (int k = 0; k < h.nv; k++) W(Dinv, k) = 1.f / W(L, MI(dof_rowadr, k));   // for the row parameters
}
// ---------------------------------------------------------------------------------------
// heightfield: the grid's triangulation, cell (i, j) split along its (i, j)-(i+1, j+1) diagonal
// into triangle 0 = (v00, v01, v11) and triangle 1 = (v00, v11, v10)
// ---------------------------------------------------------------------------------------
struct HGrid {
  const float* e;
  int nrow, ncol;
  float hx, hy, hz, dx, dy;
};

__device__ __forceinline__ float3 hg_vertex(const HGrid& g, int i, int j) {
  return make_float3(fmaf((float)j, g.dx, -g.hx), fmaf((float)i, g.dy, -g.hy), g.hz * __ldg(g.e + i * g.ncol + j));
}

__device__ __forceinline__ void hg_triangle(const HGrid& g, int i, int j, int t, float3 v[3]) {
  v[0] = hg_vertex(g, i, j);
  v[1] = t == 0 ? hg_vertex(g, i, j + 1) : hg_vertex(g, i + 1, j + 1);
  v[2] = t == 0 ? hg_vertex(g, i + 1, j + 1) : hg_vertex(g, i + 1, j);
}

__device__ __forceinline__ int hg_cell(float u, float d, int n) {
  return min(max((int)floorf(u / d), 0), n - 2);
}

// the terrain feature a closest point lies on (reported for the adjoint): 0 a triangle's face
// (the contact normal is that triangle's, constant in the state), 1 the inside of an edge of
// unit direction u, 2 a vertex
struct HFeature {
  int kind;
  float3 u;
};

// closest point to p on triangle v: its projection onto the plane when the barycentric weights
// are all >= 0, else the nearest of the edges' clamped projections (first edge on ties); FEAT
// also reports its feature in *f
template <bool FEAT = false>
__device__ float3 closest_on_triangle(float3 p, const float3 v[3], HFeature* f = nullptr) {
  const float3 n = cross3(v[1] - v[0], v[2] - v[0]);
  const float inn = 1.f / dot3(n, n);
  const float3 q = p - n * (dot3(n, p - v[0]) * inn);
  const float w0 = dot3(cross3(v[2] - v[1], q - v[1]), n) * inn;
  const float w1 = dot3(cross3(v[0] - v[2], q - v[2]), n) * inn;
  if (w0 >= 0.f && w1 >= 0.f && w0 + w1 <= 1.f) {
    if (FEAT) f->kind = 0;
    return q;
  }
  float3 best = v[0];
  float bd = 3.4e38f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float3 a = v[k], ab = v[(k + 1) % 3] - a;
    const float t = fminf(fmaxf(dot3(p - a, ab) / dot3(ab, ab), 0.f), 1.f);
    const float3 cp = a + ab * t;
    const float3 dd = p - cp;
    const float d2 = dot3(dd, dd);
    if (d2 < bd) {
      bd = d2;
      best = cp;
      if (FEAT) {
        f->kind = t > 0.f && t < 1.f ? 1 : 2;
        f->u = ab * rsqrtf(dot3(ab, ab));
      }
    }
  }
  return best;
}

// Heightfield (geom1 at x1, R1, size (hx, hy, hz)) against a sphere (cw, r):
//   * centre off the grid's xy footprint: no contact;
//   * centre on or below the triangle under it: depth s - r along that triangle's upward normal
//     (s: the centre's signed distance to its plane);
//   * otherwise the closest point q of the triangles in the cells meeting the square of
//     half-width r around the centre (first in row, column, triangle order on ties):
//     normal (c - q)/|c - q|, dist = |c - q| - r.
// The point is midway between the sphere's deepest point and the surface.  FEAT also reports
// the terrain feature of the contact in *f (its edge direction in the grid frame).
template <bool FEAT = false>
__device__ Con hfield_sphere(const HGrid& g, float3 x1, const float* R1, float3 cw, float r, HFeature* f = nullptr) {
  Con out;
  out.feat = 0;
  if (FEAT) f->kind = 0;
  const float3 c = mat_tmul(R1, cw - x1);
  if (!(c.x >= -g.hx && c.x <= g.hx && c.y >= -g.hy && c.y <= g.hy)) {
    out.dist = 1e30f;
    out.n = mat_col(R1, 2);
    out.pos = cw;
    return out;
  }
  const int i = hg_cell(c.y + g.hy, g.dy, g.nrow), j = hg_cell(c.x + g.hx, g.dx, g.ncol);
  const float fu = (c.x + g.hx) / g.dx - (float)j, fv = (c.y + g.hy) / g.dy - (float)i;
  float3 tri[3];
  hg_triangle(g, i, j, fu >= fv ? 0 : 1, tri);
  float3 nt = cross3(tri[1] - tri[0], tri[2] - tri[0]);
  nt = nt * rsqrtf(dot3(nt, nt));
  const float sd = dot3(nt, c - tri[0]);
  float3 nl;
  float d;
  if (sd <= 0.f) {
    nl = nt;
    d = sd;
  } else {
    const int i0 = hg_cell(c.y - r + g.hy, g.dy, g.nrow), i1 = hg_cell(c.y + r + g.hy, g.dy, g.nrow);
    const int j0 = hg_cell(c.x - r + g.hx, g.dx, g.ncol), j1 = hg_cell(c.x + r + g.hx, g.dx, g.ncol);
    float best = 3.4e38f;
    float3 q = c;
    for (int a = i0; a <= i1; a++)
      for (int b = j0; b <= j1; b++)
        for (int t = 0; t < 2; t++) {
          hg_triangle(g, a, b, t, tri);
          HFeature ft{0, make_float3(0.f, 0.f, 0.f)};
          const float3 p = closest_on_triangle<FEAT>(c, tri, &ft);
          const float3 e = c - p;
          const float d2 = dot3(e, e);
          if (d2 < best) {
            best = d2;
            q = p;
            if (FEAT) *f = ft;
          }
        }
    const float3 e = c - q;
    d = sqrtf(dot3(e, e));
    nl = e * (1.f / d);
  }
  out.n = mat_mul(R1, nl);
  out.dist = d - r;
  out.pos = cw - out.n * (r + 0.5f * out.dist);
  return out;
}

// ---------------------------------------------------------------------------------------
// convex solids (a box or a convex mesh) against a plane or the heightfield
// ---------------------------------------------------------------------------------------
// A convex solid in its geom frame: a box (8 corners, corner i at (+-hs.x, +-hs.y, +-hs.z) with
// bit 0, 1, 2 of i choosing +; 6 faces -x, +x, -y, +y, -z, +z) or a mesh of the model (its
// vertices and outward face planes n . p <= offset).
struct Solid {
  int nv, nf;
  float3 hs;
  const float* vert;    // mesh vertices, 3 per vertex (NULL: a box)
  const float* plane;   // mesh face planes, 4 per face
};

__device__ __forceinline__ float3 solid_vertex(const Solid& sd, int i) {
  if (!sd.vert)
    return make_float3((i & 1) ? sd.hs.x : -sd.hs.x, (i & 2) ? sd.hs.y : -sd.hs.y, (i & 4) ? sd.hs.z : -sd.hs.z);
  return make_float3(sd.vert[3 * i], sd.vert[3 * i + 1], sd.vert[3 * i + 2]);
}

// signed distance of the local point p to face f's plane (positive outside); n: its outward normal
__device__ __forceinline__ float solid_face(const Solid& sd, int f, float3 p, float3& n) {
  if (!sd.vert) {
    const float sg = (f & 1) ? 1.f : -1.f;
    const int ax = f >> 1;
    n = make_float3(ax == 0 ? sg : 0.f, ax == 1 ? sg : 0.f, ax == 2 ? sg : 0.f);
    const float pc = ax == 0 ? p.x : (ax == 1 ? p.y : p.z), hc = ax == 0 ? sd.hs.x : (ax == 1 ? sd.hs.y : sd.hs.z);
    return sg * pc - hc;
  }
  n = make_float3(sd.plane[4 * f], sd.plane[4 * f + 1], sd.plane[4 * f + 2]);
  return dot3(n, p) - sd.plane[4 * f + 3];
}

// the 4 deepest of candidates offered in order (ties: the earlier offered), kept in offer order
struct Deepest4 {
  Con k[4];
  int ord[4];
  int n = 0;
  __device__ __forceinline__ void offer(const Con& c, int o) {
    if (n < 4) {
      k[n] = c;
      ord[n] = o;
      n++;
      return;
    }
    int w = 0;   // the shallowest kept (ties: the later offered)
#pragma unroll
    for (int i = 1; i < 4; i++)
      if (k[i].dist > k[w].dist || (k[i].dist == k[w].dist && ord[i] > ord[w])) w = i;
    if (c.dist < k[w].dist) {
      k[w] = c;
      ord[w] = o;
    }
  }
  // into out[0 .. n) in offer order; returns n
  __device__ __forceinline__ int take(Con out[4]) {
    for (int i = 0; i < n; i++) {
      int b = -1;
      for (int j = 0; j < n; j++)
        if (ord[j] >= 0 && (b < 0 || ord[j] < ord[b])) b = j;
      out[i] = k[b];
      out[i].feat = ord[b];
      ord[b] = -1;
    }
    return n;
  }
};

// plane (x1, normal nz) against a convex solid at (x2, R2): every vertex at its distance to the
// plane; the 4 deepest (ties: lower index) in vertex order, each midway between vertex and plane
__device__ int plane_solid(float3 x1, float3 nz, float3 x2, const float* R2, const Solid& sd, Con out[4]) {
  Deepest4 top;
  for (int i = 0; i < sd.nv; i++) {
    const float3 w = x2 + mat_mul(R2, solid_vertex(sd, i));
    Con c;
    c.n = nz;
    c.dist = dot3(nz, w - x1);
    c.pos = w - nz * (0.5f * c.dist);
    top.offer(c, i);
  }
  return top.take(out);
}

// the upward unit normal of the grid triangle under the grid-frame point p (inside the grid's
// footprint) and one of its vertices
__device__ __forceinline__ void hg_under(const HGrid& g, float3 p, float3& nt, float3& v0) {
  const int i = hg_cell(p.y + g.hy, g.dy, g.nrow), j = hg_cell(p.x + g.hx, g.dx, g.ncol);
  const float fu = (p.x + g.hx) / g.dx - (float)j, fv = (p.y + g.hy) / g.dy - (float)i;
  float3 tri[3];
  hg_triangle(g, i, j, fu >= fv ? 0 : 1, tri);
  nt = cross3(tri[1] - tri[0], tri[2] - tri[0]);
  nt = nt * rsqrtf(dot3(nt, nt));
  v0 = tri[0];
}

// Heightfield (geom1 at x1, R1) against a convex solid (geom2 at x2, R2).  Candidates, in order:
//   * each vertex over the grid's footprint, at its signed distance to the plane of the triangle
//     under it along that triangle's upward normal;
//   * each grid vertex strictly inside the solid (row-major), at the depth of the nearest face
//     (ties: lower face index), its normal minus that face's outward normal.
// The 4 deepest (ties: candidate order) are kept in candidate order, each midway between the two
// surfaces.  Returns how many there are.
__device__ int hfield_solid(const HGrid& g, float3 x1, const float* R1, float3 x2, const float* R2, const Solid& sd,
                            Con out[4]) {
  Deepest4 top;
  float xlo = 3.4e38f, xhi = -3.4e38f, ylo = 3.4e38f, yhi = -3.4e38f;
  for (int i = 0; i < sd.nv; i++) {
    const float3 w = x2 + mat_mul(R2, solid_vertex(sd, i));
    const float3 p = mat_tmul(R1, w - x1);
    xlo = fminf(xlo, p.x); xhi = fmaxf(xhi, p.x); ylo = fminf(ylo, p.y); yhi = fmaxf(yhi, p.y);
    if (!(p.x >= -g.hx && p.x <= g.hx && p.y >= -g.hy && p.y <= g.hy)) continue;
    float3 nt, v0;
    hg_under(g, p, nt, v0);
    Con c;
    c.dist = dot3(nt, p - v0);
    c.n = mat_mul(R1, nt);
    c.pos = x1 + mat_mul(R1, p - nt * (0.5f * c.dist));
    top.offer(c, i);
  }
  // the grid vertices under the solid's bounding rectangle (clamped to the grid)
  const int i0 = max(0, (int)ceilf((ylo + g.hy) / g.dy)), i1 = min(g.nrow - 1, (int)floorf((yhi + g.hy) / g.dy));
  const int j0 = max(0, (int)ceilf((xlo + g.hx) / g.dx)), j1 = min(g.ncol - 1, (int)floorf((xhi + g.hx) / g.dx));
  for (int a = i0; a <= i1; a++)
    for (int b = j0; b <= j1; b++) {
      const float3 qw = x1 + mat_mul(R1, hg_vertex(g, a, b));
      const float3 ql = mat_tmul(R2, qw - x2);
      float best = -3.4e38f;
      float3 bn = make_float3(0.f, 0.f, 1.f);
      for (int f = 0; f < sd.nf; f++) {
        float3 n;
        const float sdist = solid_face(sd, f, ql, n);
        if (sdist > best) {
          best = sdist;
          bn = n;
        }
      }
      if (!(best < 0.f)) continue;
      const float3 nw = mat_mul(R2, bn);
      Con c;
      c.dist = best;
      c.n = nw * -1.f;
      c.pos = qw - nw * (0.5f * best);
      top.offer(c, sd.nv + a * g.ncol + b);
    }
  return top.take(out);
}

// ---------------------------------------------------------------------------------------
// collision over the static pair list; active contacts (dist < margin) are kept in slot order
// up to max_contacts as (slot, dist, pos, n)
// ---------------------------------------------------------------------------------------
template <bool DEBUG>
__device__ int collide(const Ctx& c, uint32_t& status, float* dbg) {
  const ModelHdr& h = c.h;
  int nc = 0;
  for (int p = 0; p < h.npair; p++) {
    const int g1 = MI(pair_g1, p), g2 = MI(pair_g2, p);
    const int t1 = MI(geom_type, g1), t2 = MI(geom_type, g2);
    float3 x1, x2;
    float R1[9], R2[9];
    {
      float3 bx;
      Quat bq;
      body_frame(c, MI(geom_body, g1), bx, bq);
      x1 = bx + qrot(bq, T3(&MF(geom_pos, 3 * g1)));
      qmat(qnormalize(qmul(bq, Quat{MF(geom_quat, 4 * g1), MF(geom_quat, 4 * g1 + 1), MF(geom_quat, 4 * g1 + 2),
                                    MF(geom_quat, 4 * g1 + 3)})), R1);
      body_frame(c, MI(geom_body, g2), bx, bq);
      x2 = bx + qrot(bq, T3(&MF(geom_pos, 3 * g2)));
      qmat(qnormalize(qmul(bq, Quat{MF(geom_quat, 4 * g2), MF(geom_quat, 4 * g2 + 1), MF(geom_quat, 4 * g2 + 2),
                                    MF(geom_quat, 4 * g2 + 3)})), R2);
    }
    const float *s1 = &MF(geom_size, 3 * g1), *s2 = &MF(geom_size, 3 * g2);
    const int s0 = MI(pair_slotadr, p), ns = MI(pair_nslot, p);
    Con k[4];
    int valid = ns;
    for (int i = 0; i < 4; i++) { k[i].dist = 1.f; k[i].pos = x1; k[i].n = make_float3(0.f, 0.f, 1.f); }
    // a box or a convex mesh as a solid (vertices and face planes)
    Solid sd{8, 6, make_float3(s2[0], s2[1], s2[2]), nullptr, nullptr};
    if (t2 == PG_GEOM_MESH) {
      const int mk = MI(geom_meshid, g2);
      sd.nv = MI(mesh_vertnum, mk);
      sd.nf = MI(mesh_facenum, mk);
      sd.vert = &MF(mesh_vert, 3 * MI(mesh_vertadr, mk));
      sd.plane = &MF(mesh_plane, 4 * MI(mesh_faceadr, mk));
    }
    if (t1 == PG_GEOM_HFIELD) {
      // a sphere; a capsule meets the terrain at its two end spheres; a box or mesh as a solid
      const HGrid g{c.hf, h.hf_nrow, h.hf_ncol, s1[0], s1[1], s1[2], 2.f * s1[0] / (float)(h.hf_ncol - 1),
                    2.f * s1[1] / (float)(h.hf_nrow - 1)};
      if (t2 == PG_GEOM_BOX || t2 == PG_GEOM_MESH) {
        valid = hfield_solid(g, x1, R1, x2, R2, sd, k);
      } else if (t2 == PG_GEOM_SPHERE) {
        k[0] = hfield_sphere(g, x1, R1, x2, s2[0]);
      } else {
        const float3 a = mat_col(R2, 2);
        k[0] = hfield_sphere(g, x1, R1, x2 - a * s2[1], s2[0]);
        k[1] = hfield_sphere(g, x1, R1, x2 + a * s2[1], s2[0]);
        k[1].feat = 1;
      }
    } else if (t1 == PG_GEOM_PLANE) {
      const float3 nz = mat_col(R1, 2);
      if (t2 == PG_GEOM_SPHERE) {
        k[0] = plane_sphere(x1, nz, x2, s2[0]);
      } else if (t2 == PG_GEOM_CAPSULE) {
        const float3 a = mat_col(R2, 2);
        k[0] = plane_sphere(x1, nz, x2 - a * s2[1], s2[0]);
        k[1] = plane_sphere(x1, nz, x2 + a * s2[1], s2[0]);
        k[1].feat = 1;
      } else if (t2 == PG_GEOM_MESH) {
        valid = plane_solid(x1, nz, x2, R2, sd, k);
      } else if (t2 == PG_GEOM_CYLINDER) {
        // the deepest rim point of each cap (along e, the radius on which the rim falls fastest;
        // the cylinder's x axis when its axis is within 1e-4 of the normal), then two more rim
        // points of the lower cap 120 degrees either side of the first
        const float3 a = mat_col(R2, 2);
        const float s = dot3(nz, a);
        const float3 perp = nz - a * s;
        const float pl = sqrtf(dot3(perp, perp));
        const float3 e = pl < 1e-4f ? mat_col(R2, 0) : perp * (-1.f / pl);
        const float3 b = cross3(a, e);
        const float3 off = a * (s >= 0.f ? -s2[1] : s2[1]);
        const float3 clo = x2 + off, chi = x2 - off;
        const float r = s2[0];
        const float3 p[4] = {clo + e * r, chi + e * r, clo + (e * -0.5f + b * 0.8660254f) * r,
                             clo + (e * -0.5f - b * 0.8660254f) * r};
#pragma unroll
        for (int i = 0; i < 4; i++) {
          k[i].n = nz;
          k[i].dist = dot3(nz, p[i] - x1);
          k[i].pos = p[i] - nz * (0.5f * k[i].dist);
          k[i].feat = i;
        }
      } else {
        float dd[8];
        float3 cp[8];
        for (int v = 0; v < 8; v++) {
          const float3 l = make_float3((v & 1) ? s2[0] : -s2[0], (v & 2) ? s2[1] : -s2[1], (v & 4) ? s2[2] : -s2[2]);
          cp[v] = x2 + mat_mul(R2, l);
          dd[v] = dot3(nz, cp[v] - x1);
        }
        // the 4 deepest corners (ties: lower index), kept in corner order
        unsigned chosen = 0;
        for (int r = 0; r < 4; r++) {
          int bi = -1;
          for (int v = 0; v < 8; v++)
            if (!((chosen >> v) & 1u) && (bi < 0 || dd[v] < dd[bi])) bi = v;
          chosen |= 1u << bi;
        }
        int i = 0;
        for (int v = 0; v < 8; v++)
          if ((chosen >> v) & 1u) {
            k[i].n = nz;
            k[i].dist = dd[v];
            k[i].pos = cp[v] - nz * (0.5f * dd[v]);
            k[i].feat = v;
            i++;
          }
      }
    } else if (t1 == PG_GEOM_SPHERE) {
      if (t2 == PG_GEOM_SPHERE) {
        k[0] = sphere_sphere(x1, s1[0], x2, s2[0]);
      } else if (t2 == PG_GEOM_CAPSULE) {
        const float3 a = mat_col(R2, 2);
        const float t = fminf(fmaxf(dot3(x1 - x2, a), -s2[1]), s2[1]);
        k[0] = sphere_sphere(x1, s1[0], x2 + a * t, s2[0]);
      } else {
        k[0] = sphere_box(x1, s1[0], x2, R2, make_float3(s2[0], s2[1], s2[2]));
      }
    } else if (t1 == PG_GEOM_CAPSULE) {
      const float3 a1 = mat_col(R1, 2);
      if (t2 == PG_GEOM_CAPSULE) {
        const float3 a2 = mat_col(R2, 2);
        float u, v;
        seg_seg(x1, a1, s1[1], x2, a2, s2[1], u, v);
        k[0] = sphere_sphere(x1 + a1 * u, s1[0], x2 + a2 * v, s2[0]);
      } else {
        const float3 hb = make_float3(s2[0], s2[1], s2[2]);
        k[0] = sphere_box(x1 - a1 * s1[1], s1[0], x2, R2, hb);
        k[1] = sphere_box(x1 + a1 * s1[1], s1[0], x2, R2, hb);
      }
    } else {
      valid = box_box(x1, R1, make_float3(s1[0], s1[1], s1[2]), x2, R2, make_float3(s2[0], s2[1], s2[2]), k);
    }
    for (int i = 0; i < ns; i++) {
      const bool act = i < valid && k[i].dist < h.margin;
      if (DEBUG) {
        float3 tv1, tv2;
        contact_frame(k[i].n, tv1, tv2);
        float* o = dbg + h.dbg_con + 14 * (s0 + i);
        o[0] = 0.f;
        o[1] = i < valid ? k[i].dist : 1.f;
        o[2] = k[i].pos.x; o[3] = k[i].pos.y; o[4] = k[i].pos.z;
        o[5] = k[i].n.x; o[6] = k[i].n.y; o[7] = k[i].n.z;
        o[8] = tv1.x; o[9] = tv1.y; o[10] = tv1.z;
        o[11] = tv2.x; o[12] = tv2.y; o[13] = tv2.z;
        if (act && nc < h.max_contacts) o[0] = 1.f;
      }
      if (!act) continue;
      if (nc >= h.max_contacts) { status |= PG_STATUS_CAPACITY; continue; }
      const int o = h.w_con + kConFloats * nc;
      c.w[o * c.S] = (float)(s0 + i);
      c.w[(o + 1) * c.S] = k[i].dist;
      S3(c, o + 2, k[i].pos);
      S3(c, o + 5, k[i].n);
      c.w[(o + 8) * c.S] = (float)k[i].feat;
      nc++;
    }
  }
  return nc;
}

// ---------------------------------------------------------------------------------------
// constraint rows, laid out identically in every environment (static shapes):
//   rows 4k .. 4k+3 belong to the k-th active contact (k < max_contacts): edges n+mu t1,
//   n-mu t1, n+mu t2, n-mu t2 of the pyramid (a condim-1 contact uses edge 0 = n only);
//   rows 4 max_contacts + l belong to the l-th limited joint.
// A row that does not exist in this environment has D = 0 and is never active.  The k-th
// contact's Jacobian rows (n, t1, t2) are stored over its pair's columns, padded to ncol_max
// (padding columns are zero and point at the first column).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int con_pair(const Ctx& c, int k) {
  return MI(slot_pair, (int)c.w[(c.h.w_con + kConFloats * k) * c.S]);
}

__device__ void build_rows(const Ctx& c, int nc) {
  const ModelHdr& h = c.h;
  const int NC = h.ncol_max;
  for (int k = 0; k < h.max_contacts; k++) {
    float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    if (k >= nc) {
      for (int a = 0; a < NC; a++) { J[a * c.S] = 0.f; J[(NC + a) * c.S] = 0.f; J[(2 * NC + a) * c.S] = 0.f; gc[a * c.S] = 0.f; }
      continue;
    }
    const int p = con_pair(c, k);
    const int co = h.w_con + kConFloats * k;
    const float3 pos = W3(c, co + 2), n = W3(c, co + 5);
    float3 t1, t2;
    contact_frame(n, t1, t2);
    const int b1 = MI(geom_body, MI(pair_g1, p)), b2 = MI(geom_body, MI(pair_g2, p));
    const float3 o1 = tree_origin(c, b1), o2 = tree_origin(c, b2);
    const int ca = MI(pair_coladr, p), ncol = MI(pair_ncol, p);
    for (int a = 0; a < NC; a++) {
      if (a < ncol) {
        const int d = MI(col_dof, ca + a), sg = MI(col_sign, ca + a);
        const float3 cw = W3(c, h.w_cdof + 6 * d), cl = W3(c, h.w_cdof + 6 * d + 3);
        const float3 jac = (cl + cross3(cw, pos - (sg > 0 ? o2 : o1))) * (float)sg;
        J[a * c.S] = dot3(n, jac);
        J[(NC + a) * c.S] = dot3(t1, jac);
        J[(2 * NC + a) * c.S] = dot3(t2, jac);
        gc[a * c.S] = __int_as_float(d);
      } else {
        J[a * c.S] = 0.f; J[(NC + a) * c.S] = 0.f; J[(2 * NC + a) * c.S] = 0.f;
        gc[a * c.S] = __int_as_float(ncol > 0 ? MI(col_dof, ca) : 0);
      }
    }
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int j = MI(limit_jnt, li);
    const float q = W(qpos, MI(jnt_qposadr, j));
    float sgn = 0.f;
    if (q - MF(jnt_range, 2 * j) < h.margin) sgn = 1.f;
    else if (MF(jnt_range, 2 * j + 1) - q < h.margin) sgn = -1.f;
    W(lsgn, li) = sgn;
  }
}

__device__ __forceinline__ float edge_value(float mu, int e, float dn, float d1, float d2) {
  const float dt = e < 2 ? d1 : d2;
  return (e & 1) ? dn - mu * dt : dn + mu * dt;
}

// the 4 rows of a contact group: pyramid edges, or (n, t1, t2, -) of an elliptic contact
__device__ __forceinline__ float row_value(bool ell, float mu, int e, float dn, float d1, float d2) {
  if (ell) return e == 0 ? dn : (e == 1 ? d1 : (e == 2 ? d2 : 0.f));
  return edge_value(mu, e, dn, d1, d2);
}

__device__ __forceinline__ bool elliptic_group(const Ctx& c, int k) {
  return PG_WITH_ELLIPTIC && c.h.cone == PG_CONE_ELLIPTIC && W(gcond, k) == 3.f;
}

// Elliptic contact with residual x = (xn, x1, x2), friction mu and D: the soft cost is D/2 times
// the squared distance from x to the dual cone {xn >= mu |xt|}.  Zones: 0 inside (no cost),
// 2 inside the polar cone (mu xn + |xt| <= 0: the full quadratic), 1 between (distance to the
// boundary: D (xn - mu |xt|)^2 / (2 (1 + mu^2))).
__device__ __forceinline__ int cone_zone(float xn, float x1, float x2, float mu) {
  const float t = sqrtf(x1 * x1 + x2 * x2);
  if (xn >= mu * t) return 0;
  if (mu * xn + t <= 0.f) return 2;
  return 1;
}
__device__ __forceinline__ float cone_cost(float xn, float x1, float x2, float mu, float D) {
  const int z = cone_zone(xn, x1, x2, mu);
  if (z == 0) return 0.f;
  if (z == 2) return 0.5f * D * (xn * xn + x1 * x1 + x2 * x2);
  const float ph = xn - mu * sqrtf(x1 * x1 + x2 * x2);
  return 0.5f * D * ph * ph / (1.f + mu * mu);
}
// gradient g and Hessian B = (B00 B01 B02 B11 B12 B22) of the elliptic cost
__device__ __forceinline__ void cone_derivs(float xn, float x1, float x2, float mu, float D, float g[3], float B[6]) {
  const int z = cone_zone(xn, x1, x2, mu);
  if (z == 0) {
    g[0] = g[1] = g[2] = 0.f;
    B[0] = B[1] = B[2] = B[3] = B[4] = B[5] = 0.f;
    return;
  }
  if (z == 2) {
    g[0] = D * xn; g[1] = D * x1; g[2] = D * x2;
    B[0] = D; B[1] = 0.f; B[2] = 0.f; B[3] = D; B[4] = 0.f; B[5] = D;
    return;
  }
  const float t = sqrtf(x1 * x1 + x2 * x2), u1 = x1 / t, u2 = x2 / t;
  const float ph = xn - mu * t, k = D / (1.f + mu * mu);
  const float d1 = -mu * u1, d2 = -mu * u2, q = k * ph * mu / t;   // q: phi times the curvature term
  g[0] = k * ph; g[1] = k * ph * d1; g[2] = k * ph * d2;
  B[0] = k;
  B[1] = k * d1;
  B[2] = k * d2;
  B[3] = k * d1 * d1 - q * (1.f - u1 * u1);
  B[4] = k * d1 * d2 + q * u1 * u2;
  B[5] = k * d2 * d2 - q * (1.f - u2 * u2);
}

// J_r . x for every row into the element buffer OUT (rows of absent contacts give 0)
__device__ void rows_dot(const Ctx& c, int X, int OUT) {
  const ModelHdr& h = c.h;
  const int NC = h.ncol_max, MC = h.max_contacts;
  const float* x = c.w + X * c.S;
  for (int k = 0; k < MC; k++) {
    const float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    const float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    float dn = 0.f, d1 = 0.f, d2 = 0.f;
    for (int a = 0; a < NC; a++) {
      const float xa = x[__float_as_int(gc[a * c.S]) * c.S];
      dn = fmaf(J[a * c.S], xa, dn);
      d1 = fmaf(J[(NC + a) * c.S], xa, d1);
      d2 = fmaf(J[(2 * NC + a) * c.S], xa, d2);
    }
    const float mu = W(gmu, k);
    const bool ell = elliptic_group(c, k);
    for (int e = 0; e < 4; e++) c.w[(OUT + 4 * k + e) * c.S] = row_value(ell, mu, e, dn, d1, d2);
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int d = MI(jnt_dofadr, MI(limit_jnt, li));
    c.w[(OUT + 4 * MC + li) * c.S] = W(lsgn, li) * x[d * c.S];
  }
  for (int k = 0; k < h.nfric; k++) c.w[(OUT + 4 * MC + h.nlimited + k) * c.S] = x[MI(fric_dof, k) * c.S];
}

// first friction-loss row (rows 4 max_contacts + nlimited + k, k < nfric: the dof fric_dof[k])
__device__ __forceinline__ int fric_row0(const ModelHdr& h) { return 4 * h.max_contacts + h.nlimited; }
// friction-loss row k's force bound F, scaled by this environment's 1 + s of its dof
__device__ __forceinline__ float fric_bound(const Ctx& c, int k) {
  const float F = MF(fric_F, k);
  return c.dr ? F * (1.f + dr_row(c, c.h.dr_fric + MI(fric_dof, k))) : F;
}

// impedance d(r) from solimp = (d0, dwidth, width, mid, power)
// (x^p by a multiplication for the usual power 2; the mid-point powers come from the header)
__device__ __forceinline__ float ipow(float x, float p) { return p == 2.f ? x * x : powf(x, p); }
__device__ __forceinline__ float impedance(const ModelHdr& h, float pos) {
  const float d0 = h.solimp[0], d1 = h.solimp[1], width = h.solimp[2], mid = h.solimp[3], pw = h.solimp[4];
  const float x = fminf(fabsf(pos) / width, 1.f);
  float y;
  if (x >= 1.f) y = 1.f;
  else if (x <= mid) y = ipow(x, pw) * h.imp_mid_inv;
  else y = 1.f - ipow(1.f - x, pw) * h.imp_tail_inv;
  return d0 + y * (d1 - d0);
}

// row r from its position, impedance d and Ahat; a row that does not exist gets D = 0
__device__ __forceinline__ void set_row(const Ctx& c, int r, bool valid, float pos, float d, float A) {
  const ModelHdr& h = c.h;
  W(rr, r) = pos;
  W(Ahat, r) = A;
  if (!valid) {
    W(imp, r) = 0.f;
    W(aref, r) = 0.f;
    W(rD, r) = 0.f;
    return;
  }
  W(imp, r) = d;
  W(aref, r) = -h.bref * W(rv, r) - h.kref * d * pos;
  W(rD, r) = d / ((1.f - d) * A);
}

// z <- L^-T z along the chain that starts at dof c0 (z is zero off that chain), or over all dofs
// when the model's pairs do not lie on single chains
__device__ __forceinline__ void ltsolve_chain(const Ctx& c, float* z, int c0) {
  const ModelHdr& h = c.h;
  const float* L = c.w + h.w_L * c.S;
  if (h.tree_hessian) {
    const int rc = MI(dof_rowadr, c0), n = MI(dof_depth, c0);
    for (int t = 0; t <= n; t++) {
      const int k = MI(Lcol, rc + t);
      const float zk = z[k * c.S];
      const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
      for (int s = 1; s <= dk; s++) z[MI(Lcol, r0 + s) * c.S] -= L[(r0 + s) * c.S] * zk;
    }
  } else {
    for (int k = h.nv - 1; k >= 0; k--) {
      const float zk = z[k * c.S];
      const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
      for (int s = 1; s <= dk; s++) z[MI(Lcol, r0 + s) * c.S] -= L[(r0 + s) * c.S] * zk;
    }
  }
}

// z_s <- L^-T z_s for the ns (1 or 3) vectors of one contact along the chain that starts at dof c0,
// all three in the same pass (three independent update chains; the chain's indices and L entries
// are loaded once)
__device__ __forceinline__ void ltsolve_chain3(const Ctx& c, float* z0, float* z1, float* z2, int ns, int c0) {
  const ModelHdr& h = c.h;
  const int S = c.S;
  const float* L = c.w + h.w_L * S;
  const int rc = MI(dof_rowadr, c0), n = MI(dof_depth, c0);
  for (int t = 0; t <= n; t++) {
    const int k = MI(Lcol, rc + t);
    const float a0 = z0[k * S], a1 = ns == 3 ? z1[k * S] : 0.f, a2 = ns == 3 ? z2[k * S] : 0.f;
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    for (int s = 1; s <= dk; s++) {
      const int i = MI(Lcol, r0 + s);
      const float l = L[(r0 + s) * S];
      const float y0 = z0[i * S];
      if (ns == 3) {
        const float y1 = z1[i * S], y2 = z2[i * S];
        z1[i * S] = y1 - l * a1;
        z2[i * S] = y2 - l * a2;
      }
      z0[i * S] = y0 - l * a0;
    }
  }
}

// (M^-1)_dd = sum_k z_k^2 / D_k with z = L^-T e_d, supported on d's chain (the factor of M in L)
__device__ float minv_diag(const Ctx& c, int d) {
  const ModelHdr& h = c.h;
  const float* L = c.w + h.w_L * c.S;
  float* z = c.w + h.w_z * c.S;
  for (int i = 0; i < h.nv; i++) z[i * c.S] = 0.f;
  z[d * c.S] = 1.f;
  const int rc = MI(dof_rowadr, d), n = MI(dof_depth, d);
  float A = 0.f;
  for (int t = 0; t <= n; t++) {
    const int k = MI(Lcol, rc + t);
    const float zk = z[k * c.S];
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    for (int s = 1; s <= dk; s++) z[MI(Lcol, r0 + s) * c.S] -= L[(r0 + s) * c.S] * zk;
    A = fmaf(zk * zk, W(Dinv, k), A);
  }
  return A;
}

// per row: position, velocity, exact Ahat = (J M^-1 J^T)_rr = sum_k z_k z_k / D_k with
// z = L^-T J_r^T (for a pyramid from the n / t1 / t2 solves: Ahat = A_nn +- 2 mu A_nk + mu^2 A_kk),
// impedance, aref = -b v - k d r, D = d / ((1 - d) Ahat) (0 for absent rows)
__device__ void row_params(const Ctx& c, int nc) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, NC = h.ncol_max, MC = h.max_contacts;
  for (int k = 0; k < MC; k++) {
    const bool valid = k < nc;
    const int p = valid ? con_pair(c, k) : 0;
    W(gmu, k) = valid && MI(pair_condim, p) == 3 ? MF(pair_friction, p) * (c.dr ? dr_row(c, 0) : 1.f) : 0.f;
    W(gcond, k) = valid ? (float)MI(pair_condim, p) : 0.f;
  }
  rows_dot(c, h.w_qvel, h.w_rv);
  for (int k = 0; k < MC; k++) {
    const bool valid = k < nc;
    const float mu = W(gmu, k), dist = valid ? W(con, kConFloats * k + 1) : 0.f;
    const bool pyr = W(gcond, k) == 3.f;
    const float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    const float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    float Ann = 1.f, An1 = 0.f, An2 = 0.f, A11 = 1.f, A22 = 1.f, d = 0.f;
    if (valid) {
      d = impedance(h, dist);   // one impedance for all rows of the contact
      const int c0 = __float_as_int(gc[0]);
      const int ns = pyr && !(PG_WITH_ELLIPTIC && c.h.cone == PG_CONE_ELLIPTIC) ? 3 : 1;   // pyramids need t1, t2
      if (h.tree_hessian) {
        // the pair's columns are its chain (distinct dofs), the support of z: no other entry is read
        const int nck = MI(pair_ncol, con_pair(c, k));
        for (int s = 0; s < ns; s++) {
          float* z = c.w + (h.w_z + s * nv) * c.S;
          for (int a = 0; a < nck; a++) z[__float_as_int(gc[a * c.S]) * c.S] = J[(s * NC + a) * c.S];
        }
        ltsolve_chain3(c, c.w + h.w_z * c.S, c.w + (h.w_z + nv) * c.S, c.w + (h.w_z + 2 * nv) * c.S, ns, c0);
      } else {
        for (int s = 0; s < ns; s++) {
          float* z = c.w + (h.w_z + s * nv) * c.S;
          for (int i = 0; i < nv; i++) z[i * c.S] = 0.f;
          for (int a = 0; a < NC; a++) z[__float_as_int(gc[a * c.S]) * c.S] += J[(s * NC + a) * c.S];
          ltsolve_chain(c, z, c0);
        }
      }
      Ann = An1 = An2 = A11 = A22 = 0.f;
      // z is supported on the pair's chain (its columns) when pairs lie on single chains
      const int nsum = h.tree_hessian ? MI(pair_ncol, con_pair(c, k)) : nv;
      for (int q = 0; q < nsum; q++) {
        const int i = h.tree_hessian ? __float_as_int(gc[q * c.S]) : q;
        const float dinv = W(Dinv, i);
        const float zn = W(z, i);
        Ann = fmaf(zn * zn, dinv, Ann);
        if (ns == 3) {
          const float z1 = W(z, nv + i), z2 = W(z, 2 * nv + i);
          An1 = fmaf(zn * z1, dinv, An1);
          An2 = fmaf(zn * z2, dinv, An2);
          A11 = fmaf(z1 * z1, dinv, A11);
          A22 = fmaf(z2 * z2, dinv, A22);
        }
      }
    }
    if (pyr && PG_WITH_ELLIPTIC && c.h.cone == PG_CONE_ELLIPTIC) {
      // normal row: impedance from the depth; the tangent rows share its impedance, Ahat and D
      // (impratio 1) at zero position, so their reference acceleration is -b v
      set_row(c, 4 * k + 0, valid, dist, d, Ann);
      for (int e = 1; e < 3; e++) {
        const int r = 4 * k + e;
        W(rr, r) = 0.f;
        W(Ahat, r) = W(Ahat, 4 * k);
        W(imp, r) = W(imp, 4 * k);
        W(aref, r) = valid ? -h.bref * W(rv, r) : 0.f;
        W(rD, r) = W(rD, 4 * k);
      }
      set_row(c, 4 * k + 3, false, dist, d, 1.f);
    } else if (pyr) {
      set_row(c, 4 * k + 0, valid, dist, d, Ann + 2.f * mu * An1 + mu * mu * A11);
      set_row(c, 4 * k + 1, valid, dist, d, Ann - 2.f * mu * An1 + mu * mu * A11);
      set_row(c, 4 * k + 2, valid, dist, d, Ann + 2.f * mu * An2 + mu * mu * A22);
      set_row(c, 4 * k + 3, valid, dist, d, Ann - 2.f * mu * An2 + mu * mu * A22);
    } else {
      set_row(c, 4 * k + 0, valid, dist, d, Ann);
      for (int e = 1; e < 4; e++) set_row(c, 4 * k + e, false, dist, d, 1.f);
    }
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int j = MI(limit_jnt, li), d = MI(jnt_dofadr, j);
    const float sgn = W(lsgn, li);
    const float q = W(qpos, MI(jnt_qposadr, j));
    const float pos = sgn < 0.f ? MF(jnt_range, 2 * j + 1) - q : q - MF(jnt_range, 2 * j);
    const float A = sgn != 0.f ? minv_diag(c, d) : 1.f;
    set_row(c, 4 * MC + li, sgn != 0.f, pos, sgn != 0.f ? impedance(h, pos) : 0.f, A);
  }
  // friction loss: at zero position (reference acceleration -b v), impedance d(0)
  for (int k = 0; k < h.nfric; k++) set_row(c, fric_row0(h) + k, true, 0.f, impedance(h, 0.f), minv_diag(c, MI(fric_dof, k)));
}

// ---------------------------------------------------------------------------------------
// Newton solve of  min_a f(a) = 1/2 (a-a0)^T M (a-a0) + sum_r 1/2 D_r min(0, J_r a - aref_r)^2
// ---------------------------------------------------------------------------------------
__device__ float cost_of(const Ctx& c, int X) {
  const ModelHdr& h = c.h;
  for (int k = 0; k < h.nv; k++) W(t, k) = c.w[(X + k) * c.S] - W(a0, k);
  sym_mul(c, h.w_M, h.w_t, h.w_g);
  float f = 0.f;
  for (int k = 0; k < h.nv; k++) f = fmaf(0.5f * W(t, k), W(g, k), f);
  rows_dot(c, X, h.w_jar);
  for (int r = 0; r < h.nrow_max; r++) {
    if (r < 4 * h.max_contacts && elliptic_group(c, r >> 2)) {
      if ((r & 3) == 0 && W(rD, r) > 0.f)
        f += cone_cost(W(jar, r) - W(aref, r), W(jar, r + 1) - W(aref, r + 1), W(jar, r + 2) - W(aref, r + 2),
                       W(gmu, r >> 2), W(rD, r));
      continue;
    }
    const float jar = W(jar, r) - W(aref, r);
    if (r >= fric_row0(h)) {   // friction loss: Huber cost with the band |x| <= F / D
      const float D = W(rD, r), F = fric_bound(c, r - fric_row0(h)), rf = F / D;
      f += fabsf(jar) <= rf ? 0.5f * D * jar * jar : F * fabsf(jar) - 0.5f * F * rf;
      continue;
    }
    if (jar < 0.f) f = fmaf(0.5f * W(rD, r) * jar, jar, f);
  }
  return f;
}

__device__ __forceinline__ bool bit(const unsigned act[4], int r) { return (act[r >> 5] >> (r & 31)) & 1u; }

// jar = J a - aref for every row; the active set holds the existing rows with jar < 0, and the
// friction-loss rows inside their band; `side` (optional) marks the friction-loss rows beyond it
// on the positive side
__device__ void residuals(const Ctx& c, unsigned act[4], unsigned* side = nullptr) {
  const ModelHdr& h = c.h;
  rows_dot(c, h.w_a, h.w_jar);
  act[0] = act[1] = act[2] = act[3] = 0u;
  if (side) side[0] = side[1] = side[2] = side[3] = 0u;
  for (int r = 0; r < h.nrow_max; r++) W(jar, r) = W(jar, r) - W(aref, r);
  for (int r = 0; r < h.nrow_max; r++) {
    if (r >= fric_row0(h)) {
      const float x = W(jar, r), rf = fric_bound(c, r - fric_row0(h)) / W(rD, r);
      if (fabsf(x) <= rf) act[r >> 5] |= 1u << (r & 31);
      else if (side && x > 0.f) side[r >> 5] |= 1u << (r & 31);
      continue;
    }
    if (r < 4 * h.max_contacts && elliptic_group(c, r >> 2)) {
      // an elliptic contact's zone on its first two bits: not free / full
      if ((r & 3) == 0 && W(rD, r) > 0.f) {
        const int z = cone_zone(W(jar, r), W(jar, r + 1), W(jar, r + 2), W(gmu, r >> 2));
        if (z != 0) act[r >> 5] |= 1u << (r & 31);
        if (z == 2) act[(r + 1) >> 5] |= 1u << ((r + 1) & 31);
      }
      continue;
    }
    if (W(jar, r) < 0.f && W(rD, r) > 0.f) act[r >> 5] |= 1u << (r & 31);
  }
}

// g = M (a - a0) + J_A^T D_A jar_A, H = M + J_A^T D_A J_A (packed on the tree pattern in the
// L buffer, or dense lower triangle), factorised; p = -H^-1 g.  `zero`: g is exactly zero.
__device__ bool newton_direction(const Ctx& c, const unsigned act[4], bool& zero) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, nL = h.nL, NC = h.ncol_max, MC = h.max_contacts;
  const bool tree = h.tree_hessian != 0;
  for (int k = 0; k < nv; k++) W(t, k) = W(a, k) - W(a0, k);
  sym_mul(c, h.w_M, h.w_t, h.w_g);
  if (tree) {
    for (int k = 0; k < nL; k++) W(L, k) = W(M, k);
  } else {
    for (int i = 0; i < nv * nv; i++) W(H, i) = 0.f;
    for (int j = 0; j < nv; j++) {
      const int r0 = MI(dof_rowadr, j), dj = MI(dof_depth, j);
      for (int t = 0; t <= dj; t++) W(H, j * nv + MI(Lcol, r0 + t)) = W(M, r0 + t);
    }
  }
  for (int k = 0; k < MC; k++) {
    const float mu = W(gmu, k);
    // gradient (gn, g1, g2) and Hessian block (Sn c1 c2 / s1 c12 / s2) in the (n, t1, t2) basis:
    // the active pyramid edges summed, or the elliptic cost's derivatives
    float Sn = 0.f, c1 = 0.f, c2 = 0.f, s1 = 0.f, s2 = 0.f, c12 = 0.f, gn = 0.f, g1 = 0.f, g2 = 0.f;
    if (elliptic_group(c, k)) {
      const int r = 4 * k;
      if (!bit(act, r)) continue;
      float gg[3], B[6];
      cone_derivs(W(jar, r), W(jar, r + 1), W(jar, r + 2), mu, W(rD, r), gg, B);
      gn = gg[0]; g1 = gg[1]; g2 = gg[2];
      Sn = B[0]; c1 = B[1]; c2 = B[2]; s1 = B[3]; c12 = B[4]; s2 = B[5];
    } else {
      for (int e = 0; e < 4; e++) {
        const int r = 4 * k + e;
        const float D = bit(act, r) ? W(rD, r) : 0.f, DJ = D * W(jar, r);
        const float sg = (e & 1) ? -mu : mu;
        Sn += D;
        gn += DJ;
        if (e < 2) { c1 += sg * D; s1 += mu * mu * D; g1 += sg * DJ; }
        else { c2 += sg * D; s2 += mu * mu * D; g2 += sg * DJ; }
      }
    }
    if (Sn == 0.f) continue;
    const float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    const float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    const int nck = MI(pair_ncol, con_pair(c, k));   // the pair's real columns (the rest is zero padding)
    for (int a = 0; a < nck; a++) {
      const int da = __float_as_int(gc[a * c.S]);
      const float na = J[a * c.S], ta = J[(NC + a) * c.S], ua = J[(2 * NC + a) * c.S];
      W(g, da) += gn * na + g1 * ta + g2 * ua;
      const float hn = Sn * na + c1 * ta + c2 * ua;
      const float ht = c1 * na + s1 * ta + c12 * ua;
      const float hu = c2 * na + c12 * ta + s2 * ua;
      const int ra = MI(dof_rowadr, da);
      if (tree) {
        // the columns are a chain of consecutive parents (checked by the model compiler): column b
        // updates entry b - a of row da's packed segment, four at a time with the loads first
        float* Lr = c.w + (h.w_L + ra) * c.S;
        int b = a;
        for (; b + 3 < nck; b += 4) {
          float v[4], l[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            v[q] = hn * J[(b + q) * c.S] + ht * J[(NC + b + q) * c.S] + hu * J[(2 * NC + b + q) * c.S];
            l[q] = Lr[(b + q - a) * c.S];
          }
#pragma unroll
          for (int q = 0; q < 4; q++) Lr[(b + q - a) * c.S] = l[q] + v[q];
        }
        for (; b < nck; b++) Lr[(b - a) * c.S] += hn * J[b * c.S] + ht * J[(NC + b) * c.S] + hu * J[(2 * NC + b) * c.S];
      } else {
        for (int b = a; b < nck; b++) {
          const int db = __float_as_int(gc[b * c.S]);
          const float v = hn * J[b * c.S] + ht * J[(NC + b) * c.S] + hu * J[(2 * NC + b) * c.S];
          W(H, (da > db ? da * nv + db : db * nv + da)) += v;
        }
      }
    }
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int r = 4 * MC + li, d = MI(jnt_dofadr, MI(limit_jnt, li));
    const float D = bit(act, r) ? W(rD, r) : 0.f;
    W(g, d) += W(lsgn, li) * D * W(jar, r);
    if (tree) W(L, MI(dof_rowadr, d)) += D;
    else W(H, d * nv + d) += D;
  }
  for (int k = 0; k < h.nfric; k++) {   // friction loss: quadratic in its band, the bound +-F beyond
    const int r = fric_row0(h) + k, d = MI(fric_dof, k);
    const float x = W(jar, r);
    if (bit(act, r)) {
      const float D = W(rD, r);
      W(g, d) += D * x;
      if (tree) W(L, MI(dof_rowadr, d)) += D;
      else W(H, d * nv + d) += D;
    } else {
      W(g, d) += x > 0.f ? fric_bound(c, k) : -fric_bound(c, k);
    }
  }
  bool nz = false;
  for (int k = 0; k < nv; k++) { W(p, k) = -W(g, k); nz = nz || W(g, k) != 0.f; }
  zero = !nz;
  if (zero) return false;
  if (tree) {
    ldl_factor(c, h.w_L);
    for (int k = 0; k < nv; k++)
      if (!(W(L, MI(dof_rowadr, k)) > 0.f)) return false;
    ldl_solve(c, h.w_L, h.w_p);
    return true;
  }
  for (int j = 0; j < nv; j++) {
    float s = W(H, j * nv + j);
    for (int k = 0; k < j; k++) s -= W(H, j * nv + k) * W(H, j * nv + k);
    if (!(s > 0.f)) return false;
    const float djj = sqrtf(s), inv = 1.f / djj;
    W(H, j * nv + j) = djj;
    for (int i = j + 1; i < nv; i++) {
      float t = W(H, i * nv + j);
      for (int k = 0; k < j; k++) t -= W(H, i * nv + k) * W(H, j * nv + k);
      W(H, i * nv + j) = t * inv;
    }
  }
  for (int i = 0; i < nv; i++) {
    float s = W(p, i);
    for (int k = 0; k < i; k++) s -= W(H, i * nv + k) * W(p, k);
    W(p, i) = s / W(H, i * nv + i);
  }
  for (int i = nv - 1; i >= 0; i--) {
    float s = W(p, i);
    for (int k = i + 1; k < nv; k++) s -= W(H, k * nv + i) * W(p, k);
    W(p, i) = s / W(H, i * nv + i);
  }
  return true;
}

// Exact minimiser of phi(alpha) = f(a + alpha p) (convex, piecewise quadratic): start from the
// active set just after alpha = 0 and walk the breakpoints alpha_r = -jar_r / Jp_r in increasing
// order (each next one found by a scan), toggling the rows that cross, until the root of the
// current linear piece of phi' lies before the next breakpoint.
__device__ float line_search(const Ctx& c) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, R = h.nrow_max;
  sym_mul(c, h.w_M, h.w_p, h.w_g);   // g <- M p
  float qt = 0.f, lt = 0.f;
  for (int k = 0; k < nv; k++) {
    qt = fmaf(W(p, k), W(g, k), qt);
    lt = fmaf(W(t, k), W(g, k), lt);   // t = a - a0
  }
  rows_dot(c, h.w_p, h.w_Jp);
  unsigned on[4] = {0u, 0u, 0u, 0u};
  const float none = -__int_as_float(0x7f800000);   // -inf: no breakpoint
  const int R0 = fric_row0(h);
  for (int r = 0; r < R0; r++) {
    const float D = W(rD, r), jp = W(Jp, r), jr = W(jar, r);
    if (D > 0.f && (jr < 0.f || (jr == 0.f && jp < 0.f))) {
      on[r >> 5] |= 1u << (r & 31);
      qt = fmaf(D * jp, jp, qt);
      lt = fmaf(D * jp, jr, lt);
    }
    W(bp, r) = D > 0.f && jp != 0.f ? -jr / jp : none;   // the row's breakpoint, once
  }
  // friction-loss rows: quadratic inside the band |x| <= F / D, slope +-F Jp beyond it; the next
  // band edge the motion reaches is the row's breakpoint (the far edge once inside)
  for (int r = R0; r < R; r++) {
    const float D = W(rD, r), jp = W(Jp, r), jr = W(jar, r), F = fric_bound(c, r - R0), rf = F / D;
    const bool mid = (jr > -rf && jr < rf) || (jr == rf && jp <= 0.f) || (jr == -rf && jp >= 0.f);
    if (mid) {
      on[r >> 5] |= 1u << (r & 31);
      qt = fmaf(D * jp, jp, qt);
      lt = fmaf(D * jp, jr, lt);
      W(bp, r) = jp > 0.f ? (rf - jr) / jp : (jp < 0.f ? (-rf - jr) / jp : none);
    } else {
      lt = fmaf(jr > 0.f ? F : -F, jp, lt);
      W(bp, r) = (jr > 0.f && jp < 0.f) ? (rf - jr) / jp : ((jr < 0.f && jp > 0.f) ? (-rf - jr) / jp : none);
    }
  }
  float alpha = 0.f;
  for (int step = 0; step <= R; step++) {
    const float root = qt > 0.f ? -lt / qt : alpha;
    float next = __int_as_float(0x7f800000);   // +inf
    for (int r = 0; r < R; r++) {
      const float br = W(bp, r);
      if (br > alpha && br < next) next = br;
    }
    if (root <= next) return root;
    alpha = next;
    for (int r = 0; r < R; r++) {
      if (W(bp, r) != next) continue;
      const float D = W(rD, r), jp = W(Jp, r);
      const float sg = bit(on, r) ? -1.f : 1.f;
      if (r >= R0) {
        // a friction-loss row at a band edge: entering the band from the side it came from, or
        // leaving it towards the side the motion leads to
        const float F = fric_bound(c, r - R0), s = jp > 0.f ? 1.f : -1.f;
        if (sg > 0.f) {   // entering: drop the slope -s F Jp, add the quadratic, next the far edge
          lt = fmaf(s * F, jp, lt);
          W(bp, r) = (s * F / D - W(jar, r)) / jp;
        } else {          // leaving: drop the quadratic (below), add the slope s F Jp
          lt = fmaf(s * F, jp, lt);
          W(bp, r) = none;
        }
      }
      on[r >> 5] ^= 1u << (r & 31);
      qt = fmaf(sg * D * jp, jp, qt);
      lt = fmaf(sg * D * jp, W(jar, r), lt);
    }
  }
  return qt > 0.f ? -lt / qt : alpha;
}

// Line search when elliptic contacts make phi(alpha) = f(a + alpha p) convex but not piecewise
// quadratic (friction-loss rows add their Huber terms): bracket the root of phi' (phi'(0) < 0;
// alpha doubled from 1 until phi' >= 0), then safeguarded Newton steps on phi' (bisection whenever
// the Newton point leaves the bracket) until the bracket or |phi'| is at FP32 rounding level.
__device__ float line_search_smooth(const Ctx& c) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, R = h.nrow_max, MC = h.max_contacts;
  sym_mul(c, h.w_M, h.w_p, h.w_g);   // g <- M p
  float qt = 0.f, lt = 0.f;
  for (int k = 0; k < nv; k++) {
    qt = fmaf(W(p, k), W(g, k), qt);
    lt = fmaf(W(t, k), W(g, k), lt);   // t = a - a0
  }
  rows_dot(c, h.w_p, h.w_Jp);
  auto deriv = [&](float al, float& d2) {
    float d1 = fmaf(al, qt, lt);
    d2 = qt;
    for (int r = 0; r < R; r++) {
      if (!(W(rD, r) > 0.f)) continue;
      if (r < 4 * MC && elliptic_group(c, r >> 2)) {
        if ((r & 3) != 0) continue;
        const float y0 = W(Jp, r), y1 = W(Jp, r + 1), y2 = W(Jp, r + 2);
        float gg[3], B[6];
        cone_derivs(fmaf(al, y0, W(jar, r)), fmaf(al, y1, W(jar, r + 1)), fmaf(al, y2, W(jar, r + 2)), W(gmu, r >> 2),
                    W(rD, r), gg, B);
        d1 += gg[0] * y0 + gg[1] * y1 + gg[2] * y2;
        d2 += B[0] * y0 * y0 + B[3] * y1 * y1 + B[5] * y2 * y2 + 2.f * (B[1] * y0 * y1 + B[2] * y0 * y2 + B[4] * y1 * y2);
        continue;
      }
      const float jp = W(Jp, r), x = fmaf(al, jp, W(jar, r));
      if (r >= fric_row0(h)) {   // friction loss: D x inside the band |x| <= F / D, the bound +-F beyond
        const float F = fric_bound(c, r - fric_row0(h));
        if (fabsf(x) <= F / W(rD, r)) {
          d1 = fmaf(W(rD, r) * x, jp, d1);
          d2 = fmaf(W(rD, r) * jp, jp, d2);
        } else {
          d1 = fmaf(x > 0.f ? F : -F, jp, d1);
        }
        continue;
      }
      if (x < 0.f) {
        d1 = fmaf(W(rD, r) * x, jp, d1);
        d2 = fmaf(W(rD, r) * jp, jp, d2);
      }
    }
    return d1;
  };
  float d2;
  const float g0 = deriv(0.f, d2);
  if (!(g0 < 0.f)) return 0.f;
  float lo = 0.f, hi = 1.f;
  for (int k = 0; k < 60 && deriv(hi, d2) < 0.f; k++) { lo = hi; hi *= 2.f; }
  float al = lo;
  float glo = deriv(lo, d2);
  for (int it = 0; it < 40; it++) {
    float cand = al - glo / d2;
    if (!(cand > lo && cand < hi)) cand = 0.5f * (lo + hi);
    float d2c;
    const float gc = deriv(cand, d2c);
    if (gc < 0.f) lo = cand;
    else hi = cand;
    al = cand;
    glo = gc;
    d2 = d2c;
    if (hi - lo <= 1e-6f * hi || fabsf(gc) <= 1e-6f * fabsf(g0)) break;
  }
  return al;
}

// any elliptic contact in this environment's rows
__device__ __forceinline__ bool has_elliptic(const Ctx& c) {
  if (!PG_WITH_ELLIPTIC || c.h.cone != PG_CONE_ELLIPTIC) return false;
  bool any = false;
  for (int k = 0; k < c.h.max_contacts; k++) any = any || (elliptic_group(c, k) && W(rD, 4 * k) > 0.f);
  return any;
}

// Newton's method with exact termination: stop at the cap or when the active set after the
// step equals the one the Hessian was built from.  Warm start: qacc_warm if f(warm) < f(a0).
// With elliptic contacts the step is exact only when none is on its cone's boundary zone;
// otherwise it stops when f no longer decreases.
__device__ int newton(const Ctx& c, bool& converged) {
  const ModelHdr& h = c.h;
  const int nv = h.nv;
  converged = false;
  const float fw = cost_of(c, h.w_warm), f0 = cost_of(c, h.w_a0);
  const bool use_warm = fw < f0;
  float f_cur = use_warm ? fw : f0;
  for (int k = 0; k < nv; k++) W(a, k) = use_warm ? W(warm, k) : W(a0, k);
  const bool ell = has_elliptic(c);
  unsigned act[4], side[4];
  residuals(c, act, side);
  int it = 0;
  while (it < h.cap) {
    bool zero = false;
    const bool ok = newton_direction(c, act, zero);
    it++;
    if (zero) { converged = true; break; }
    if (!ok) break;
    const float alpha = ell ? line_search_smooth(c) : line_search(c);
    for (int k = 0; k < nv; k++) W(a, k) = fmaf(alpha, W(p, k), W(a, k));
    const float f_new = ell ? cost_of(c, h.w_a) : 0.f;   // (before the residuals: cost_of reuses jar)
    unsigned act2[4], side2[4];
    residuals(c, act2, side2);
    const bool same = act2[0] == act[0] && act2[1] == act[1] && act2[2] == act[2] && act2[3] == act[3] &&
                      side2[0] == side[0] && side2[1] == side[1] && side2[2] == side[2] && side2[3] == side[3];
    for (int k = 0; k < 4; k++) { act[k] = act2[k]; side[k] = side2[k]; }
    if (!ell) {
      if (same) { converged = true; break; }
      continue;
    }
    bool middle = false;
    for (int k = 0; k < h.max_contacts; k++)
      middle = middle || (elliptic_group(c, k) && W(rD, 4 * k) > 0.f && bit(act, 4 * k) && !bit(act, 4 * k + 1));
    if ((same && !middle) || !(f_new < f_cur)) { converged = true; break; }
    f_cur = f_new;
  }
  return it;
}

// The contact forces of the substep just solved (its nc active contacts), each in its contact's
// frame (normal, t1, t2), into out[(slot * 3 + k) * ld + env] for every candidate slot < nslot (0 for
// a slot without an active contact): a pyramid's edge forces D_e max(0, aref_e - J_e a) summed back
// into the frame (f_n = sum f_e, f_t1 = mu (f_0 - f_1), f_t2 = mu (f_2 - f_3)); an elliptic contact's
// force minus the gradient of its cone cost.
__device__ void contact_forces_out(const Ctx& c, int nc, float* out, int nslot) {
  const ModelHdr& h = c.h;
  for (int s = 0; s < nslot; s++)
    for (int k = 0; k < 3; k++) out[(s * 3 + k) * c.ld + c.env] = 0.f;
  rows_dot(c, h.w_a, h.w_jar);
  for (int k = 0; k < nc; k++) {
    const int slot = (int)W(con, kConFloats * k);
    float f[3] = {0.f, 0.f, 0.f};
    if (elliptic_group(c, k)) {
      const int r = 4 * k;
      if (W(rD, r) > 0.f) {
        float gg[3], B[6];
        cone_derivs(W(jar, r) - W(aref, r), W(jar, r + 1) - W(aref, r + 1), W(jar, r + 2) - W(aref, r + 2), W(gmu, k),
                    W(rD, r), gg, B);
        f[0] = -gg[0]; f[1] = -gg[1]; f[2] = -gg[2];
      }
    } else {
      float fe[4];
      for (int e = 0; e < 4; e++) {
        const int r = 4 * k + e;
        const float x = W(jar, r) - W(aref, r);
        fe[e] = W(rD, r) > 0.f && x < 0.f ? -W(rD, r) * x : 0.f;
      }
      const float mu = W(gmu, k);
      f[0] = fe[0] + fe[1] + fe[2] + fe[3];
      f[1] = mu * (fe[0] - fe[1]);
      f[2] = mu * (fe[2] - fe[3]);
    }
    if (slot >= 0 && slot < nslot)
      for (int q = 0; q < 3; q++) out[(slot * 3 + q) * c.ld + c.env] = f[q];
  }
}

// ---------------------------------------------------------------------------------------
// one substep; returns its active contacts
// ---------------------------------------------------------------------------------------
template <bool DEBUG>
__device__ int substep(const Ctx& c, uint32_t& status, float* dbg, uint32_t cnt[3]) {
  const ModelHdr& h = c.h;
  const int nv = h.nv;
  kinematics(c);
  if (DEBUG) {
    for (int b = 0; b < h.nbody; b++) {
      float3 x;
      Quat q;
      body_frame(c, b, x, q);
      float R[9];
      qmat(q, R);
      float mb;
      float3 ip;
      if (b) body_massprops(c, b, mb, ip);
      const float3 com = b ? x + mat_mul(R, ip) : make_float3(0.f, 0.f, 0.f);
      dbg[h.dbg_xpos + 3 * b] = x.x; dbg[h.dbg_xpos + 3 * b + 1] = x.y; dbg[h.dbg_xpos + 3 * b + 2] = x.z;
      dbg[h.dbg_xcom + 3 * b] = com.x; dbg[h.dbg_xcom + 3 * b + 1] = com.y; dbg[h.dbg_xcom + 3 * b + 2] = com.z;
      for (int k = 0; k < 9; k++) dbg[h.dbg_xmat + 9 * b + k] = R[k];
    }
  }
  rnea(c);
  crba(c);
  if (DEBUG) {
    for (int i = 0; i < nv * nv; i++) dbg[h.dbg_M + i] = 0.f;
    for (int j = 0; j < nv; j++) {
      const int r0 = MI(dof_rowadr, j), dj = MI(dof_depth, j);
      for (int t = 0; t <= dj; t++) {
        const int i = MI(Lcol, r0 + t);
        dbg[h.dbg_M + j * nv + i] = W(M, r0 + t);
        dbg[h.dbg_M + i * nv + j] = W(M, r0 + t);
      }
    }
  }
  smooth_acc<DEBUG>(c, dbg);
  if (DEBUG)
    for (int k = 0; k < nv; k++) dbg[h.dbg_a0 + k] = W(a0, k);
  const int nc = collide<DEBUG>(c, status, dbg);
  build_rows(c, nc);
  row_params(c, nc);
  int nrow = 0;   // rows that exist in this environment
  for (int r = 0; r < h.nrow_max; r++) nrow += W(rD, r) > 0.f ? 1 : 0;
  int iters = 0;
  bool conv = true;
  if (nrow == 0) {
    for (int k = 0; k < nv; k++) W(a, k) = W(a0, k);
  } else {
    iters = newton(c, conv);
    if (!conv) status |= PG_STATUS_NOT_CONVERGED;
  }
  cnt[0] += (uint32_t)iters;
  cnt[1] += (uint32_t)nrow;
  cnt[2] += (uint32_t)(nrow * iters);
  if (DEBUG) {
    // rows in the oracle's order: existing contact rows, then existing limit rows
    rows_dot(c, h.w_a, h.w_jar);
    int o_r = 0;
    for (int r = 0; r < h.nrow_max; r++) {
      if (!(W(rD, r) > 0.f)) continue;
      float* o = dbg + h.dbg_rows + (o_r++) * (nv + 7);
      for (int k = 0; k < nv; k++) o[k] = 0.f;
      if (r < 4 * h.max_contacts) {
        const int k = r >> 2, e = r & 3;
        const float mu = W(gmu, k);
        const float* J = c.w + (h.w_J + 3 * h.ncol_max * k) * c.S;
        const float* gc = c.w + (h.w_gcol + h.ncol_max * k) * c.S;
        const bool ell = elliptic_group(c, k);
        for (int a = 0; a < h.ncol_max; a++)
          o[__float_as_int(gc[a * c.S])] += W(gcond, k) == 3.f
              ? row_value(ell, mu, e, J[a * c.S], J[(h.ncol_max + a) * c.S], J[(2 * h.ncol_max + a) * c.S])
              : J[a * c.S];
      } else if (r < fric_row0(h)) {
        const int li = r - 4 * h.max_contacts, d = MI(jnt_dofadr, MI(limit_jnt, li));
        o[d] = W(lsgn, li);
      } else {
        o[MI(fric_dof, r - fric_row0(h))] = 1.f;
      }
      o[nv] = W(rr, r); o[nv + 1] = W(rv, r); o[nv + 2] = W(aref, r); o[nv + 3] = W(rD, r);
      o[nv + 4] = W(Ahat, r); o[nv + 5] = W(imp, r);
      const float jar = W(jar, r) - W(aref, r);
      o[nv + 6] = jar < 0.f ? -W(rD, r) * jar : 0.f;
      if (r >= fric_row0(h)) {   // friction loss: -D x inside the band, the bound beyond
        const float F = fric_bound(c, r - fric_row0(h));
        o[nv + 6] = fabsf(jar) <= F / W(rD, r) ? -W(rD, r) * jar : (jar > 0.f ? -F : F);
      }
      if (r < 4 * h.max_contacts && elliptic_group(c, r >> 2)) {   // force = -grad of the cone cost
        const int r0 = r & ~3;
        float gg[3], B[6];
        cone_derivs(W(jar, r0) - W(aref, r0), W(jar, r0 + 1) - W(aref, r0 + 1), W(jar, r0 + 2) - W(aref, r0 + 2),
                    W(gmu, r >> 2), W(rD, r0), gg, B);
        o[nv + 6] = -gg[r & 3];
      }
    }
    dbg[h.dbg_nrow] = (float)nrow;
    dbg[h.dbg_iter] = (float)iters;
  }
  // semi-implicit Euler
  bool bad = false;
  for (int d = 0; d < nv; d++) {
    const float acc = W(a, d);
    W(qvel, d) = fmaf(h.h, acc, W(qvel, d));
    W(warm, d) = acc;
    bad = bad || !isfinite(acc) || !isfinite(W(qvel, d));
    if (DEBUG) dbg[h.dbg_qacc + d] = acc;
  }
  for (int j = 0; j < h.njnt; j++) {
    const int qa = MI(jnt_qposadr, j), da = MI(jnt_dofadr, j);
    if (MI(jnt_type, j) == PG_JNT_FREE) {
      for (int k = 0; k < 3; k++) W(qpos, qa + k) = fmaf(h.h, W(qvel, da + k), W(qpos, qa + k));
      const float3 w = make_float3(W(qvel, da + 3), W(qvel, da + 4), W(qvel, da + 5));
      const float wn = sqrtf(dot3(w, w));
      Quat q{W(qpos, qa + 3), W(qpos, qa + 4), W(qpos, qa + 5), W(qpos, qa + 6)};
      if (wn > 0.f) {
        float sn, cs;
        sincosf(0.5f * h.h * wn, &sn, &cs);
        const float s = sn / wn;
        q = qmul(q, Quat{cs, w.x * s, w.y * s, w.z * s});
      }
      q = qnormalize(q);
      W(qpos, qa + 3) = q.w; W(qpos, qa + 4) = q.x; W(qpos, qa + 5) = q.y; W(qpos, qa + 6) = q.z;
      for (int k = 0; k < 7; k++) bad = bad || !isfinite(W(qpos, qa + k));
    } else {
      W(qpos, qa) = fmaf(h.h, W(qvel, da), W(qpos, qa));
      bad = bad || !isfinite(W(qpos, qa));
    }
  }
  if (bad) status |= PG_STATUS_NAN;
  if (DEBUG) {
    for (int k = 0; k < h.nq; k++) dbg[h.dbg_qpos + k] = W(qpos, k);
    for (int k = 0; k < nv; k++) dbg[h.dbg_qvel + k] = W(qvel, k);
    dbg[h.dbg_status] = (float)status;
  }
  return nc;
}

}  // namespace
}  // namespace pg
