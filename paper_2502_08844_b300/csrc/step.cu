// Fused batched physics step for sm_103a: one warp per environment, one thread block per tile
// of consecutive environments of one model.  The block copies its model blob into shared
// memory, stages its environments' state in a per-warp shared-memory workspace, runs all
// substeps on chip, and writes the state back.  FP32 CUDA-core arithmetic throughout (the
// per-environment matrices are small and not a dense contraction, so no tensor cores).
//
// Per substep (all 32 lanes of a warp cooperate; level-parallel tree sweeps):
//   FK -> body COM / spatial inertia / geom frames / motion subspaces (cdof)
//   -> CRBA (composite inertias, dense symmetric M) -> tree-sparse LDL^T of M
//   -> RNEA bias forces -> passive + actuator forces -> a0 = M^-1 (tau - c)
//   -> collision over the static pair list -> contact / limit rows, Ahat = (J M^-1 J^T)_ii
//   -> Newton on the convex soft-constraint cost (dense H, Cholesky, exact line search)
//   -> semi-implicit Euler.
// Spatial vectors are (angular; linear) in world axes about each tree's reference point
// o = position of the tree's root body (a body whose parent is the world).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pg_host.h"
#include "pg_internal.h"

namespace pg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// spatial inertia (about o, world axes) times a motion vector: ci = (Ixx Iyy Izz Ixy Ixz Iyz, h, m)
__device__ __forceinline__ void inert_mul(const float* ci, float3 w, float3 v, float3& fa, float3& fl) {
  float3 h = make_float3(ci[6], ci[7], ci[8]);
  fa = make_float3(ci[0] * w.x + ci[3] * w.y + ci[4] * w.z, ci[3] * w.x + ci[1] * w.y + ci[5] * w.z,
                   ci[4] * w.x + ci[5] * w.y + ci[2] * w.z) + cross3(h, v);
  fl = v * ci[9] - cross3(h, w);
}

// ---------------------------------------------------------------------------------------
// environment context
// ---------------------------------------------------------------------------------------
struct Env {
  const ModelHdr* h;
  const int* I;
  const float* F;
  float* w;
  int lane;
};

#define MI(name, i) (e.I[e.h->o_##name + (i)])
#define MF(name, i) (e.F[e.h->o_##name + (i)])
#define WS(name) (e.w + e.h->w_##name)

// ---------------------------------------------------------------------------------------
// kinematics
// ---------------------------------------------------------------------------------------
__device__ void fk(const Env& e) {
  const ModelHdr& h = *e.h;
  float *xpos = WS(xpos), *xquat = WS(xquat), *xmat = WS(xmat), *janc = WS(janchor), *jax = WS(jaxis);
  const float* qpos = WS(qpos);
  if (e.lane == 0) {
    st3(xpos, make_float3(0.f, 0.f, 0.f));
    stq(xquat, Quat{1.f, 0.f, 0.f, 0.f});
    float* R = xmat;
    R[0] = 1; R[1] = 0; R[2] = 0; R[3] = 0; R[4] = 1; R[5] = 0; R[6] = 0; R[7] = 0; R[8] = 1;
  }
  __syncwarp();
  for (int L = 1; L < h.nlevel; L++) {
    const int s = MI(level_start, L), t = MI(level_start, L + 1);
    for (int k = s + e.lane; k < t; k += 32) {
      const int b = MI(level_body, k), p = MI(body_parent, b);
      Quat qp = ldq(xquat + 4 * p);
      float3 x = ld3(xpos + 3 * p) + qrot(qp, ld3(&MF(body_pos, 3 * b)));
      Quat q = qmul(qp, ldq(&MF(body_quat, 4 * b)));
      const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
      for (int j = j0; j < j0 + nj; j++) {
        const int type = MI(jnt_type, j), qa = MI(jnt_qposadr, j);
        if (type == PG_JNT_FREE) {
          x = ld3(qpos + qa);
          q = qnormalize(Quat{qpos[qa + 3], qpos[qa + 4], qpos[qa + 5], qpos[qa + 6]});
          st3(janc + 3 * j, x);
          st3(jax + 3 * j, make_float3(0.f, 0.f, 0.f));
        } else {
          const float3 lp = ld3(&MF(jnt_pos, 3 * j)), la = ld3(&MF(jnt_axis, 3 * j));
          const float3 anchor = x + qrot(q, lp), axis = qrot(q, la);
          st3(janc + 3 * j, anchor);
          st3(jax + 3 * j, axis);
          if (type == PG_JNT_HINGE) {
            float sn, cs;
            sincosf(0.5f * qpos[qa], &sn, &cs);
            q = qmul(q, Quat{cs, la.x * sn, la.y * sn, la.z * sn});
            x = anchor - qrot(q, lp);
          } else {
            x = x + axis * qpos[qa];
          }
        }
      }
      q = qnormalize(q);
      st3(xpos + 3 * b, x);
      stq(xquat + 4 * b, q);
      qmat(q, xmat + 9 * b);
    }
    __syncwarp();
  }
}

// COM, spatial inertia about the tree reference point, geom frames and motion subspaces
__device__ void derived(const Env& e) {
  const ModelHdr& h = *e.h;
  const float *xpos = WS(xpos), *xmat = WS(xmat), *xquat = WS(xquat);
  float *xipos = WS(xipos), *cinert = WS(cinert), *gpos = WS(gpos), *gmat = WS(gmat), *cdof = WS(cdof);
  for (int b = 1 + e.lane; b < h.nbody; b += 32) {
    const float* R = xmat + 9 * b;
    const float3 o = ld3(xpos + 3 * MI(body_root, b));
    const float3 com = ld3(xpos + 3 * b) + mat_mul(R, ld3(&MF(body_ipos, 3 * b)));
    st3(xipos + 3 * b, com);
    const float m = MF(body_mass, b);
    const float* In = &MF(body_inertia, 6 * b);
    // I_world = R I_body R^T
    float Ib[9] = {In[0], In[3], In[4], In[3], In[1], In[5], In[4], In[5], In[2]};
    float T[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int c = 0; c < 3; c++) T[3 * r + c] = R[3 * r] * Ib[c] + R[3 * r + 1] * Ib[3 + c] + R[3 * r + 2] * Ib[6 + c];
    float Iw[6];
    Iw[0] = T[0] * R[0] + T[1] * R[1] + T[2] * R[2];
    Iw[1] = T[3] * R[3] + T[4] * R[4] + T[5] * R[5];
    Iw[2] = T[6] * R[6] + T[7] * R[7] + T[8] * R[8];
    Iw[3] = T[0] * R[3] + T[1] * R[4] + T[2] * R[5];
    Iw[4] = T[0] * R[6] + T[1] * R[7] + T[2] * R[8];
    Iw[5] = T[3] * R[6] + T[4] * R[7] + T[5] * R[8];
    const float3 c = com - o;
    const float c2 = dot3(c, c);
    float* ci = cinert + 10 * b;
    ci[0] = Iw[0] + m * (c2 - c.x * c.x);
    ci[1] = Iw[1] + m * (c2 - c.y * c.y);
    ci[2] = Iw[2] + m * (c2 - c.z * c.z);
    ci[3] = Iw[3] - m * c.x * c.y;
    ci[4] = Iw[4] - m * c.x * c.z;
    ci[5] = Iw[5] - m * c.y * c.z;
    ci[6] = m * c.x; ci[7] = m * c.y; ci[8] = m * c.z;
    ci[9] = m;
  }
  for (int g = e.lane; g < h.ngeom; g += 32) {
    const int b = MI(geom_body, g);
    Quat qb = ldq(xquat + 4 * b);
    st3(gpos + 3 * g, ld3(xpos + 3 * b) + qrot(qb, ld3(&MF(geom_pos, 3 * g))));
    qmat(qnormalize(qmul(qb, ldq(&MF(geom_quat, 4 * g)))), gmat + 9 * g);
  }
  for (int d = e.lane; d < h.nv; d += 32) {
    const int b = MI(dof_body, d);
    const float3 o = ld3(xpos + 3 * MI(body_root, b));
    // the joint owning this dof: the last joint of b whose dofadr <= d
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    int j = j0;
    for (int jj = j0; jj < j0 + nj; jj++)
      if (MI(jnt_dofadr, jj) <= d) j = jj;
    const int type = MI(jnt_type, j);
    float3 ang, lin;
    if (type == PG_JNT_FREE) {
      const int k = d - MI(jnt_dofadr, j);
      if (k < 3) {
        ang = make_float3(0.f, 0.f, 0.f);
        lin = make_float3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f);
      } else {
        ang = mat_col(xmat + 9 * b, k - 3);
        lin = cross3(ang, o - ld3(xpos + 3 * b));
      }
    } else if (type == PG_JNT_HINGE) {
      ang = ld3(WS(jaxis) + 3 * j);
      lin = cross3(ang, o - ld3(WS(janchor) + 3 * j));
    } else {
      ang = make_float3(0.f, 0.f, 0.f);
      lin = ld3(WS(jaxis) + 3 * j);
    }
    st3(cdof + 6 * d, ang);
    st3(cdof + 6 * d + 3, lin);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// CRBA: composite inertias (backward level sweep), M_ji = cdof_i . (Ic(body j) cdof_j) for i on
// j's dof chain; armature on the diagonal.  Dense symmetric M plus the packed copy that the
// LDL factorisation works on (row j: j, parent(j), grandparent(j), ...).
// ---------------------------------------------------------------------------------------
__device__ void crba(const Env& e) {
  const ModelHdr& h = *e.h;
  float *crb = WS(crb), *Fv = WS(F), *M = WS(M), *Lp = WS(L);
  const float *cinert = WS(cinert), *cdof = WS(cdof);
  for (int i = e.lane; i < 10 * h.nbody; i += 32) crb[i] = cinert[i];
  for (int i = e.lane; i < h.nv * h.nv; i += 32) M[i] = 0.f;
  __syncwarp();
  for (int L = h.nlevel - 2; L >= 1; L--) {
    const int s = MI(level_start, L), t = MI(level_start, L + 1);
    for (int k = s + e.lane; k < t; k += 32) {
      const int p = MI(level_body, k);
      float acc[10];
#pragma unroll
      for (int i = 0; i < 10; i++) acc[i] = crb[10 * p + i];
      for (int c = MI(child_start, p); c < MI(child_start, p + 1); c++) {
        const int ch = MI(child, c);
#pragma unroll
        for (int i = 0; i < 10; i++) acc[i] += crb[10 * ch + i];
      }
#pragma unroll
      for (int i = 0; i < 10; i++) crb[10 * p + i] = acc[i];
    }
    __syncwarp();
  }
  for (int d = e.lane; d < h.nv; d += 32) {
    float3 fa, fl;
    inert_mul(crb + 10 * MI(dof_body, d), ld3(cdof + 6 * d), ld3(cdof + 6 * d + 3), fa, fl);
    st3(Fv + 6 * d, fa);
    st3(Fv + 6 * d + 3, fl);
  }
  __syncwarp();
  const int nv = h.nv;
  for (int j = e.lane; j < nv; j += 32) {
    const float3 fa = ld3(Fv + 6 * j), fl = ld3(Fv + 6 * j + 3);
    const int r0 = MI(dof_rowadr, j), n = MI(dof_depth, j) + 1;
    for (int t = 0; t < n; t++) {
      const int i = MI(Lcol, r0 + t);
      float v = dot3(ld3(cdof + 6 * i), fa) + dot3(ld3(cdof + 6 * i + 3), fl);
      if (t == 0) v += MF(dof_armature, j);
      M[j * nv + i] = v;
      M[i * nv + j] = v;
      Lp[r0 + t] = v;
    }
  }
  __syncwarp();
}

// In-place tree-sparse factorisation M = L^T D L (L unit lower triangular on the ancestor
// pattern, no fill-in): for k = nv-1 .. 0, with d = D_k = M_kk, the entries of row k become
// L_ki = M_ki / d and every ancestor pair (i, j) of k (j on i's chain) is updated
// M_ij -= L_ki M_kj.  Lane t handles the t-th ancestor row of k.
__device__ void ldl_factor(const Env& e) {
  const ModelHdr& h = *e.h;
  float *Lp = WS(L), *D = WS(D), *tmp = WS(vtmp);
  for (int k = h.nv - 1; k >= 0; k--) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    const float diag = Lp[r0];
    for (int t = e.lane + 1; t <= dk; t += 32) {
      const float lkt = Lp[r0 + t] / diag;
      tmp[t] = lkt;
      const int i = MI(Lcol, r0 + t), ri = MI(dof_rowadr, i);
      for (int s = t; s <= dk; s++) Lp[ri + (s - t)] -= lkt * Lp[r0 + s];
    }
    __syncwarp();
    for (int t = e.lane + 1; t <= dk; t += 32) Lp[r0 + t] = tmp[t];
    if (e.lane == 0) D[k] = diag;
    __syncwarp();
  }
}

// x <- M^-1 x with the packed factor (one lane; x in shared memory)
__device__ void ldl_solve_lane(const Env& e, float* x) {
  const ModelHdr& h = *e.h;
  const float *Lp = WS(L), *D = WS(D);
  for (int k = h.nv - 1; k >= 0; k--) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    const float xk = x[k];
    for (int t = 1; t <= dk; t++) x[MI(Lcol, r0 + t)] -= Lp[r0 + t] * xk;
  }
  for (int k = 0; k < h.nv; k++) x[k] /= D[k];
  for (int k = 0; k < h.nv; k++) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    float s = x[k];
    for (int t = 1; t <= dk; t++) s -= Lp[r0 + t] * x[MI(Lcol, r0 + t)];
    x[k] = s;
  }
}

// ---------------------------------------------------------------------------------------
// RNEA bias forces c(q, qdot): velocities and bias accelerations outward (the world
// accelerates by -gravity), body forces I a + v x* I v, accumulated inward, projected on cdof.
// Serial joints on one body are a chain of massless frames; a free joint's three rotational
// dofs all use the velocity after its translation (their axes move with the body).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cross_motion(float3 w, float3 v, float3 a, float3 b, float3& ra, float3& rl) {
  ra = cross3(w, a);
  rl = cross3(w, b) + cross3(v, a);
}

__device__ void rnea(const Env& e) {
  const ModelHdr& h = *e.h;
  float *cvel = WS(cvel), *cacc = WS(cacc), *cfrc = WS(cfrc), *bias = WS(bias);
  const float *cdof = WS(cdof), *cinert = WS(cinert), *qvel = WS(qvel);
  if (e.lane == 0) {
    for (int i = 0; i < 6; i++) cvel[i] = 0.f;
    cacc[0] = cacc[1] = cacc[2] = 0.f;
    cacc[3] = -h.grav[0]; cacc[4] = -h.grav[1]; cacc[5] = -h.grav[2];
  }
  __syncwarp();
  for (int L = 1; L < h.nlevel; L++) {
    const int s = MI(level_start, L), t = MI(level_start, L + 1);
    for (int k = s + e.lane; k < t; k += 32) {
      const int b = MI(level_body, k), p = MI(body_parent, b);
      float3 w = ld3(cvel + 6 * p), v = ld3(cvel + 6 * p + 3), aw = ld3(cacc + 6 * p), av = ld3(cacc + 6 * p + 3);
      const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
      for (int j = j0; j < j0 + nj; j++) {
        const int d0 = MI(jnt_dofadr, j);
        if (MI(jnt_type, j) == PG_JNT_FREE) {
          v = v + make_float3(qvel[d0], qvel[d0 + 1], qvel[d0 + 2]);   // world-axis translation
          float3 dw = make_float3(0.f, 0.f, 0.f), dv = dw;
          for (int k3 = 3; k3 < 6; k3++) {
            dw = dw + ld3(cdof + 6 * (d0 + k3)) * qvel[d0 + k3];
            dv = dv + ld3(cdof + 6 * (d0 + k3) + 3) * qvel[d0 + k3];
          }
          float3 ra, rl;
          cross_motion(w, v, dw, dv, ra, rl);
          aw = aw + ra; av = av + rl;
          w = w + dw; v = v + dv;
        } else {
          const float qd = qvel[d0];
          const float3 dw = ld3(cdof + 6 * d0) * qd, dv = ld3(cdof + 6 * d0 + 3) * qd;
          float3 ra, rl;
          cross_motion(w, v, dw, dv, ra, rl);
          aw = aw + ra; av = av + rl;
          w = w + dw; v = v + dv;
        }
      }
      st3(cvel + 6 * b, w); st3(cvel + 6 * b + 3, v);
      st3(cacc + 6 * b, aw); st3(cacc + 6 * b + 3, av);
      // f = I a + v x* (I v)
      float3 fa, fl, ia, il;
      inert_mul(cinert + 10 * b, aw, av, fa, fl);
      inert_mul(cinert + 10 * b, w, v, ia, il);
      fa = fa + cross3(w, ia) + cross3(v, il);
      fl = fl + cross3(w, il);
      st3(cfrc + 6 * b, fa); st3(cfrc + 6 * b + 3, fl);
    }
    __syncwarp();
  }
  for (int L = h.nlevel - 2; L >= 1; L--) {
    const int s = MI(level_start, L), t = MI(level_start, L + 1);
    for (int k = s + e.lane; k < t; k += 32) {
      const int p = MI(level_body, k);
      float acc[6];
#pragma unroll
      for (int i = 0; i < 6; i++) acc[i] = cfrc[6 * p + i];
      for (int c = MI(child_start, p); c < MI(child_start, p + 1); c++) {
        const int ch = MI(child, c);
#pragma unroll
        for (int i = 0; i < 6; i++) acc[i] += cfrc[6 * ch + i];
      }
#pragma unroll
      for (int i = 0; i < 6; i++) cfrc[6 * p + i] = acc[i];
    }
    __syncwarp();
  }
  for (int d = e.lane; d < h.nv; d += 32) {
    const float* f = cfrc + 6 * MI(dof_body, d);
    bias[d] = dot3(ld3(cdof + 6 * d), ld3(f)) + dot3(ld3(cdof + 6 * d + 3), ld3(f + 3));
  }
  __syncwarp();
}

// passive (joint damping) and actuator forces (motor: gear * clamp(u); position / PD:
// kp (u - q) - kd qdot), then the unconstrained acceleration a0 = M^-1 (tau - c)
__device__ void smooth_acc(const Env& e) {
  const ModelHdr& h = *e.h;
  float *passive = WS(passive), *act = WS(act), *a0 = WS(a0);
  const float *qvel = WS(qvel), *qpos = WS(qpos), *ctrl = WS(ctrl), *bias = WS(bias);
  for (int d = e.lane; d < h.nv; d += 32) {
    passive[d] = -MF(dof_damping, d) * qvel[d];
    float tau = 0.f;
    for (int a = 0; a < h.nu; a++) {
      if (MI(act_dof, a) != d) continue;
      float u = ctrl[a];
      if (MI(act_ctrllimited, a)) u = fminf(fmaxf(u, MF(act_range, 2 * a)), MF(act_range, 2 * a + 1));
      if (MI(act_type, a) == PG_ACT_MOTOR) tau += MF(act_gear, a) * u;
      else tau += MF(act_kp, a) * (u - qpos[MI(act_qposadr, a)]) - MF(act_kd, a) * qvel[d];
    }
    act[d] = tau;
    a0[d] = tau + passive[d] - bias[d];
  }
  __syncwarp();
  if (e.lane == 0) ldl_solve_lane(e, a0);
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// collision
// ---------------------------------------------------------------------------------------
struct Con {
  float dist;
  float3 pos, n;
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

__device__ void collide(const Env& e, uint32_t& status) {
  const ModelHdr& h = *e.h;
  float* con = WS(con);
  const float *gpos = WS(gpos), *gmat = WS(gmat);
  for (int p = e.lane; p < h.npair; p += 32) {
    const int g1 = MI(pair_g1, p), g2 = MI(pair_g2, p);
    const int t1 = MI(geom_type, g1), t2 = MI(geom_type, g2);
    const float3 x1 = ld3(gpos + 3 * g1), x2 = ld3(gpos + 3 * g2);
    const float *R1 = gmat + 9 * g1, *R2 = gmat + 9 * g2;
    const float *s1 = &MF(geom_size, 3 * g1), *s2 = &MF(geom_size, 3 * g2);
    const int s0 = MI(pair_slotadr, p), ns = MI(pair_nslot, p);
    Con c[4];
    int valid = ns;   // candidates produced (others stay inactive)
    for (int i = 0; i < 4; i++) { c[i].dist = 1.f; c[i].pos = x1; c[i].n = make_float3(0.f, 0.f, 1.f); }
    if (t1 == PG_GEOM_PLANE) {
      const float3 nz = mat_col(R1, 2);
      if (t2 == PG_GEOM_SPHERE) {
        c[0] = plane_sphere(x1, nz, x2, s2[0]);
      } else if (t2 == PG_GEOM_CAPSULE) {
        const float3 a = mat_col(R2, 2);
        c[0] = plane_sphere(x1, nz, x2 - a * s2[1], s2[0]);
        c[1] = plane_sphere(x1, nz, x2 + a * s2[1], s2[0]);
      } else if (t2 == PG_GEOM_BOX) {
        float d[8];
        float3 cp[8];
        for (int v = 0; v < 8; v++) {
          const float3 l = make_float3((v & 1) ? s2[0] : -s2[0], (v & 2) ? s2[1] : -s2[1], (v & 4) ? s2[2] : -s2[2]);
          cp[v] = x2 + mat_mul(R2, l);
          d[v] = dot3(nz, cp[v] - x1);
        }
        // the 4 deepest corners (ties: lower index), kept in corner order
        unsigned chosen = 0;
        for (int r = 0; r < 4; r++) {
          int bi = -1;
          for (int v = 0; v < 8; v++)
            if (!((chosen >> v) & 1u) && (bi < 0 || d[v] < d[bi])) bi = v;
          chosen |= 1u << bi;
        }
        int i = 0;
        for (int v = 0; v < 8; v++)
          if ((chosen >> v) & 1u) {
            c[i].n = nz;
            c[i].dist = d[v];
            c[i].pos = cp[v] - nz * (0.5f * d[v]);
            i++;
          }
      }
    } else if (t1 == PG_GEOM_SPHERE) {
      if (t2 == PG_GEOM_SPHERE) {
        c[0] = sphere_sphere(x1, s1[0], x2, s2[0]);
      } else if (t2 == PG_GEOM_CAPSULE) {
        const float3 a = mat_col(R2, 2);
        const float t = fminf(fmaxf(dot3(x1 - x2, a), -s2[1]), s2[1]);
        c[0] = sphere_sphere(x1, s1[0], x2 + a * t, s2[0]);
      } else {
        c[0] = sphere_box(x1, s1[0], x2, R2, make_float3(s2[0], s2[1], s2[2]));
      }
    } else if (t1 == PG_GEOM_CAPSULE) {
      const float3 a1 = mat_col(R1, 2);
      if (t2 == PG_GEOM_CAPSULE) {
        const float3 a2 = mat_col(R2, 2);
        float u, v;
        seg_seg(x1, a1, s1[1], x2, a2, s2[1], u, v);
        c[0] = sphere_sphere(x1 + a1 * u, s1[0], x2 + a2 * v, s2[0]);
      } else {
        const float3 hb = make_float3(s2[0], s2[1], s2[2]);
        c[0] = sphere_box(x1 - a1 * s1[1], s1[0], x2, R2, hb);
        c[1] = sphere_box(x1 + a1 * s1[1], s1[0], x2, R2, hb);
      }
    } else {
      valid = box_box(x1, R1, make_float3(s1[0], s1[1], s1[2]), x2, R2, make_float3(s2[0], s2[1], s2[2]), c);
    }
    for (int i = 0; i < ns; i++) {
      float* k = con + 14 * (s0 + i);
      const bool act = i < valid && c[i].dist < h.margin;
      float3 t1v, t2v;
      contact_frame(c[i].n, t1v, t2v);
      k[0] = act ? 1.f : 0.f;
      k[1] = i < valid ? c[i].dist : 1.f;
      st3(k + 2, c[i].pos);
      st3(k + 5, c[i].n);
      st3(k + 8, t1v);
      st3(k + 11, t2v);
    }
  }
  __syncwarp();
  // at most max_contacts active contacts, kept in slot order
  if (e.lane == 0) {
    int na = 0;
    for (int s = 0; s < h.nslot; s++) {
      if (con[14 * s] != 0.f) {
        if (na >= h.max_contacts) { con[14 * s] = 0.f; status |= PG_STATUS_CAPACITY; }
        else na++;
      }
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// constraint rows
// ---------------------------------------------------------------------------------------
// row ids: contact rows encode 4 * slot + edge (edge 0..3; condim 1 uses edge 0);
// limit rows encode -1 - (2 * limit_index + side) with side 0 = lower, 1 = upper.
__device__ int assign_rows(const Env& e) {
  const ModelHdr& h = *e.h;
  int* rowslot = reinterpret_cast<int*>(WS(rowslot));
  int nrow = 0;
  if (e.lane == 0) {
    const float* con = WS(con);
    for (int p = 0; p < h.npair; p++) {
      const int s0 = MI(pair_slotadr, p), ns = MI(pair_nslot, p), ne = MI(pair_condim, p) == 3 ? 4 : 1;
      for (int s = s0; s < s0 + ns; s++)
        if (con[14 * s] != 0.f)
          for (int k = 0; k < ne; k++) rowslot[nrow++] = 4 * s + k;
    }
    const float* qpos = WS(qpos);
    for (int li = 0; li < h.nlimited; li++) {
      const int j = MI(limit_jnt, li);
      const float q = qpos[MI(jnt_qposadr, j)];
      if (q - MF(jnt_range, 2 * j) < h.margin) rowslot[nrow++] = -1 - 2 * li;
      else if (MF(jnt_range, 2 * j + 1) - q < h.margin) rowslot[nrow++] = -1 - (2 * li + 1);
    }
  }
  nrow = __shfl_sync(kFull, nrow, 0);
  __syncwarp();
  return nrow;
}

__device__ __forceinline__ int slot_pair(const Env& e, int s) {
  int p = 0;
  while (p + 1 < e.h->npair && MI(pair_slotadr, p + 1) <= s) p++;
  return p;
}

// J rows (dense over nv), row position r, velocity J qdot, Ahat, impedance, aref, D
__device__ void build_rows(const Env& e, int nrow) {
  const ModelHdr& h = *e.h;
  const int nv = h.nv;
  float* J = WS(J);
  const int* rowslot = reinterpret_cast<const int*>(WS(rowslot));
  const float *con = WS(con), *cdof = WS(cdof), *xpos = WS(xpos);
  for (int i = e.lane; i < nrow * nv; i += 32) J[i] = 0.f;
  __syncwarp();
  // contact rows: lane = dof, loop over the contacts (first row of each)
  for (int d = e.lane; d < nv; d += 32) {
    const float3 cw = ld3(cdof + 6 * d), cl = ld3(cdof + 6 * d + 3);
    const int db = MI(dof_body, d);
    (void)db;
    for (int r = 0; r < nrow; r++) {
      const int id = rowslot[r];
      if (id < 0 || (id & 3) != 0) continue;
      const int s = id >> 2, p = slot_pair(e, s);
      const int b1 = MI(geom_body, MI(pair_g1, p)), b2 = MI(geom_body, MI(pair_g2, p));
      const float* k = con + 14 * s;
      const float3 pos = ld3(k + 2);
      float3 jac = make_float3(0.f, 0.f, 0.f);
      const uint64_t m2 = (uint64_t)(uint32_t)MI(body_dofmask, 2 * b2) | ((uint64_t)(uint32_t)MI(body_dofmask, 2 * b2 + 1) << 32);
      const uint64_t m1 = (uint64_t)(uint32_t)MI(body_dofmask, 2 * b1) | ((uint64_t)(uint32_t)MI(body_dofmask, 2 * b1 + 1) << 32);
      if ((m2 >> d) & 1ull) jac = jac + cl + cross3(cw, pos - ld3(xpos + 3 * MI(body_root, b2)));
      if ((m1 >> d) & 1ull) jac = jac - (cl + cross3(cw, pos - ld3(xpos + 3 * MI(body_root, b1))));
      const float jn = dot3(ld3(k + 5), jac);
      if (MI(pair_condim, p) == 3) {
        const float mu = MF(pair_friction, p);
        const float jt1 = dot3(ld3(k + 8), jac), jt2 = dot3(ld3(k + 11), jac);
        J[(r + 0) * nv + d] = jn + mu * jt1;
        J[(r + 1) * nv + d] = jn - mu * jt1;
        J[(r + 2) * nv + d] = jn + mu * jt2;
        J[(r + 3) * nv + d] = jn - mu * jt2;
      } else {
        J[r * nv + d] = jn;
      }
    }
  }
  // limit rows
  for (int r = e.lane; r < nrow; r += 32) {
    const int id = rowslot[r];
    if (id >= 0) continue;
    const int code = -1 - id, li = code >> 1, side = code & 1;
    const int j = MI(limit_jnt, li);
    J[r * nv + MI(jnt_dofadr, j)] = side == 0 ? 1.f : -1.f;
  }
  __syncwarp();
}

// per-row position, velocity, exact Ahat = (J M^-1 J^T)_rr = sum_k z_k^2 / D_k with
// z = L^-T J_r^T (one lane per row), impedance, reference acceleration and D = 1 / R
__device__ void row_params(const Env& e, int nrow) {
  const ModelHdr& h = *e.h;
  const int nv = h.nv;
  const float *J = WS(J), *con = WS(con), *qvel = WS(qvel), *qpos = WS(qpos), *Lp = WS(L), *Dd = WS(D);
  const int* rowslot = reinterpret_cast<const int*>(WS(rowslot));
  float *rr = WS(rr), *rv = WS(rv), *aref = WS(aref), *rD = WS(rD), *Ahat = WS(Ahat), *imp = WS(imp), *Z = WS(Z);
  for (int r = e.lane; r < nrow; r += 32) {
    const int id = rowslot[r];
    float pos;
    if (id >= 0) {
      pos = con[14 * (id >> 2) + 1];
    } else {
      const int code = -1 - id, li = code >> 1, side = code & 1, j = MI(limit_jnt, li);
      const float q = qpos[MI(jnt_qposadr, j)];
      pos = side == 0 ? q - MF(jnt_range, 2 * j) : MF(jnt_range, 2 * j + 1) - q;
    }
    const float* Jr = J + r * nv;
    float* z = Z + r * nv;
    float vel = 0.f;
    for (int k = 0; k < nv; k++) { z[k] = Jr[k]; vel = fmaf(Jr[k], qvel[k], vel); }
    float A = 0.f;
    for (int k = nv - 1; k >= 0; k--) {
      const float zk = z[k];
      if (zk != 0.f) {
        const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
        for (int t = 1; t <= dk; t++) z[MI(Lcol, r0 + t)] -= Lp[r0 + t] * zk;
      }
      A = fmaf(zk * zk, 1.f / Dd[k], A);
    }
    // impedance d(r) from solimp = (d0, dwidth, width, mid, power)
    const float d0 = h.solimp[0], d1 = h.solimp[1], width = h.solimp[2], mid = h.solimp[3], pw = h.solimp[4];
    const float x = fminf(fabsf(pos) / width, 1.f);
    float y;
    if (x >= 1.f) y = 1.f;
    else if (x <= mid) y = powf(x, pw) / powf(mid, pw - 1.f);
    else y = 1.f - powf(1.f - x, pw) / powf(1.f - mid, pw - 1.f);
    const float dimp = d0 + y * (d1 - d0);
    rr[r] = pos;
    rv[r] = vel;
    Ahat[r] = A;
    imp[r] = dimp;
    aref[r] = -h.bref * vel - h.kref * dimp * pos;
    rD[r] = dimp / ((1.f - dimp) * A);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// Newton solve of  min_a 1/2 (a-a0)^T M (a-a0) + sum_r 1/2 D_r min(0, J_r a - aref_r)^2
// ---------------------------------------------------------------------------------------
// f(x) with x in shared memory (all lanes get the value)
__device__ float cost_of(const Env& e, const float* x, int nrow) {
  const ModelHdr& h = *e.h;
  const int nv = h.nv;
  const float *M = WS(M), *a0 = WS(a0), *J = WS(J), *aref = WS(aref), *rD = WS(rD);
  float part = 0.f;
  for (int j = e.lane; j < nv; j += 32) {
    float s = 0.f;
    for (int k = 0; k < nv; k++) s = fmaf(M[j * nv + k], x[k] - a0[k], s);
    part = fmaf(0.5f * (x[j] - a0[j]), s, part);
  }
  for (int r = e.lane; r < nrow; r += 32) {
    float jar = -aref[r];
    for (int k = 0; k < nv; k++) jar = fmaf(J[r * nv + k], x[k], jar);
    if (jar < 0.f) part = fmaf(0.5f * rD[r] * jar, jar, part);
  }
  return warp_sum(part);
}

// active set of x: bit r of word r/32, with jar stored (all lanes get the 4 words)
__device__ void active_set(const Env& e, const float* x, int nrow, unsigned act[4]) {
  const int nv = e.h->nv;
  const float *J = WS(J), *aref = WS(aref);
  float* jar = WS(jar);
#pragma unroll
  for (int w = 0; w < 4; w++) {
    const int r = 32 * w + e.lane;
    bool on = false;
    if (r < nrow) {
      float s = -aref[r];
      for (int k = 0; k < nv; k++) s = fmaf(J[r * nv + k], x[k], s);
      jar[r] = s;
      on = s < 0.f;
    }
    act[w] = __ballot_sync(kFull, on);
  }
  __syncwarp();
}

__device__ __forceinline__ bool bit(const unsigned act[4], int r) { return (act[r >> 5] >> (r & 31)) & 1u; }

// returns iterations used; sets converged
__device__ int newton(const Env& e, int nrow, bool& converged) {
  const ModelHdr& h = *e.h;
  const int nv = h.nv;
  float *a = WS(a), *g = WS(g), *p = WS(p), *Mp = WS(Mp), *H = WS(H), *jar = WS(jar), *Jp = WS(Jp);
  const float *M = WS(M), *a0 = WS(a0), *J = WS(J), *rD = WS(rD), *warm = WS(warm);
  converged = false;
  // warm start: qacc_warm if f(qacc_warm) < f(a0), else a0
  const float fw = cost_of(e, warm, nrow), f0 = cost_of(e, a0, nrow);
  const bool use_warm = fw < f0;
  for (int j = e.lane; j < nv; j += 32) a[j] = use_warm ? warm[j] : a0[j];
  __syncwarp();
  int it = 0;
  for (; it < h.cap;) {
    unsigned act[4];
    active_set(e, a, nrow, act);
    // gradient and Hessian rows (lane = row j of H)
    bool nz = false;
    for (int j = e.lane; j < nv; j += 32) {
      float gj = 0.f;
      for (int k = 0; k < nv; k++) gj = fmaf(M[j * nv + k], a[k] - a0[k], gj);
      for (int k = 0; k < nv; k++) H[j * nv + k] = M[j * nv + k];
      for (int r = 0; r < nrow; r++) {
        if (!bit(act, r)) continue;
        const float Dj = rD[r] * J[r * nv + j];
        gj = fmaf(Dj, jar[r], gj);
        if (Dj != 0.f)
          for (int k = 0; k < nv; k++) H[j * nv + k] = fmaf(Dj, J[r * nv + k], H[j * nv + k]);
      }
      g[j] = gj;
      nz = nz || gj != 0.f;
    }
    it++;
    if (!__any_sync(kFull, nz)) { converged = true; break; }
    __syncwarp();
    // Cholesky H = L L^T in place (lower triangle), row i owned by a lane
    bool ok = true;
    for (int k = 0; k < nv; k++) {
      const float dkk = H[k * nv + k];
      ok = ok && dkk > 0.f;
      const float dk = sqrtf(fmaxf(dkk, 1e-30f));
      const float inv = 1.f / dk;
      for (int i = k + 1 + e.lane; i < nv; i += 32) H[i * nv + k] *= inv;
      __syncwarp();
      for (int i = k + 1 + e.lane; i < nv; i += 32) {
        const float lik = H[i * nv + k];
        for (int j = k + 1; j <= i; j++) H[i * nv + j] = fmaf(-lik, H[j * nv + k], H[i * nv + j]);
      }
      if (e.lane == 0) H[k * nv + k] = dk;
      __syncwarp();
    }
    if (!ok) break;
    // p = -H^-1 g: forward (L y = -g) then backward (L^T p = y), column-oriented updates
    for (int j = e.lane; j < nv; j += 32) p[j] = -g[j];
    __syncwarp();
    for (int k = 0; k < nv; k++) {
      const float pk = p[k] / H[k * nv + k];
      for (int i = k + 1 + e.lane; i < nv; i += 32) p[i] = fmaf(-H[i * nv + k], pk, p[i]);
      __syncwarp();
      if (e.lane == 0) p[k] = pk;
      __syncwarp();
    }
    for (int k = nv - 1; k >= 0; k--) {
      const float pk = p[k] / H[k * nv + k];
      for (int i = e.lane; i < k; i += 32) p[i] = fmaf(-H[k * nv + i], pk, p[i]);
      __syncwarp();
      if (e.lane == 0) p[k] = pk;
      __syncwarp();
    }
    // exact line search on phi(alpha) = f(a + alpha p)
    float qp = 0.f, lp = 0.f;
    for (int j = e.lane; j < nv; j += 32) {
      float s = 0.f;
      for (int k = 0; k < nv; k++) s = fmaf(M[j * nv + k], p[k], s);
      Mp[j] = s;
      qp = fmaf(p[j], s, qp);
      lp = fmaf(s, a[j] - a0[j], lp);
    }
    const float quad0 = warp_sum(qp), lin0 = warp_sum(lp);
    for (int r = e.lane; r < nrow; r += 32) {
      float s = 0.f;
      for (int k = 0; k < nv; k++) s = fmaf(J[r * nv + k], p[k], s);
      Jp[r] = s;
    }
    __syncwarp();
    // phi' at each row's breakpoint (lane = row); bracket the root between the largest
    // breakpoint with phi' < 0 and the smallest with phi' >= 0
    float lo = 0.f, hi = INFINITY;
    for (int r = e.lane; r < ((nrow + 31) & ~31); r += 32) {
      float ar = -1.f;
      if (r < nrow && Jp[r] != 0.f) ar = -jar[r] / Jp[r];
      if (r < nrow && ar > 0.f) {
        float dphi = fmaf(ar, quad0, lin0);
        for (int q = 0; q < nrow; q++) {
          const float v = fmaf(ar, Jp[q], jar[q]);
          if (v < 0.f) dphi = fmaf(rD[q] * Jp[q], v, dphi);
        }
        if (dphi < 0.f) lo = fmaxf(lo, ar);
        else hi = fminf(hi, ar);
      }
    }
    lo = warp_max(lo);
    hi = warp_min(hi);
    const float amid = isinf(hi) ? lo + 1.f : 0.5f * (lo + hi);
    float qa = 0.f, la = 0.f;
    for (int r = e.lane; r < nrow; r += 32) {
      if (fmaf(amid, Jp[r], jar[r]) < 0.f) {
        const float dj = rD[r] * Jp[r];
        qa = fmaf(dj, Jp[r], qa);
        la = fmaf(dj, jar[r], la);
      }
    }
    const float qt = quad0 + warp_sum(qa), lt = lin0 + warp_sum(la);
    const float alpha = qt > 0.f ? -lt / qt : 0.f;
    for (int j = e.lane; j < nv; j += 32) a[j] = fmaf(alpha, p[j], a[j]);
    __syncwarp();
    unsigned act2[4];
    active_set(e, a, nrow, act2);
    if (act2[0] == act[0] && act2[1] == act[1] && act2[2] == act[2] && act2[3] == act[3]) {
      converged = true;
      break;
    }
  }
  return it;
}

// ---------------------------------------------------------------------------------------
// one substep
// ---------------------------------------------------------------------------------------
template <bool DEBUG>
__device__ void substep(const Env& e, uint32_t& status, float* dbg, uint32_t cnt[3]) {
  const ModelHdr& h = *e.h;
  const int nv = h.nv;
  fk(e);
  derived(e);
  if (DEBUG) {
    for (int i = e.lane; i < 3 * h.nbody; i += 32) { dbg[h.dbg_xpos + i] = WS(xpos)[i]; dbg[h.dbg_xcom + i] = WS(xipos)[i]; }
    for (int i = e.lane; i < 9 * h.nbody; i += 32) dbg[h.dbg_xmat + i] = WS(xmat)[i];
    if (e.lane < 3) dbg[h.dbg_xcom + e.lane] = 0.f;   // world body
  }
  crba(e);
  ldl_factor(e);
  rnea(e);
  smooth_acc(e);
  collide(e, status);
  const int nrow = assign_rows(e);
  build_rows(e, nrow);
  // kinematic buffers are dead from here on (the Newton / row-solve union reuses them)
  __syncwarp();
  row_params(e, nrow);
  float* a = WS(a);
  int iters = 0;
  bool conv = true;
  if (nrow == 0) {
    for (int j = e.lane; j < nv; j += 32) a[j] = WS(a0)[j];
    __syncwarp();
  } else {
    iters = newton(e, nrow, conv);
    if (!conv) status |= PG_STATUS_NOT_CONVERGED;
  }
  cnt[0] += (uint32_t)iters;
  cnt[1] += (uint32_t)nrow;
  cnt[2] += (uint32_t)(nrow * iters);
  // semi-implicit Euler
  float *qvel = WS(qvel), *qpos = WS(qpos), *warm = WS(warm);
  bool bad = false;
  for (int d = e.lane; d < nv; d += 32) {
    const float acc = a[d];
    qvel[d] = fmaf(h.h, acc, qvel[d]);
    warm[d] = acc;
    bad = bad || !isfinite(acc) || !isfinite(qvel[d]);
  }
  __syncwarp();
  for (int j = e.lane; j < h.njnt; j += 32) {
    const int qa = MI(jnt_qposadr, j), da = MI(jnt_dofadr, j);
    if (MI(jnt_type, j) == PG_JNT_FREE) {
      for (int k = 0; k < 3; k++) qpos[qa + k] = fmaf(h.h, qvel[da + k], qpos[qa + k]);
      const float3 w = make_float3(qvel[da + 3], qvel[da + 4], qvel[da + 5]);
      const float wn = sqrtf(dot3(w, w));
      Quat q{qpos[qa + 3], qpos[qa + 4], qpos[qa + 5], qpos[qa + 6]};
      if (wn > 0.f) {
        float sn, cs;
        sincosf(0.5f * h.h * wn, &sn, &cs);
        const float s = sn / wn;
        q = qmul(q, Quat{cs, w.x * s, w.y * s, w.z * s});
      }
      q = qnormalize(q);
      qpos[qa + 3] = q.w; qpos[qa + 4] = q.x; qpos[qa + 5] = q.y; qpos[qa + 6] = q.z;
      for (int k = 0; k < 7; k++) bad = bad || !isfinite(qpos[qa + k]);
    } else {
      qpos[qa] = fmaf(h.h, qvel[da], qpos[qa]);
      bad = bad || !isfinite(qpos[qa]);
    }
  }
  if (__any_sync(kFull, bad)) status |= PG_STATUS_NAN;
  __syncwarp();
  if (DEBUG) {
    for (int i = e.lane; i < nv * nv; i += 32) dbg[h.dbg_M + i] = WS(M)[i];
    for (int i = e.lane; i < nv; i += 32) {
      dbg[h.dbg_bias + i] = WS(bias)[i];
      dbg[h.dbg_passive + i] = WS(passive)[i];
      dbg[h.dbg_act + i] = WS(act)[i];
      dbg[h.dbg_a0 + i] = WS(a0)[i];
      dbg[h.dbg_qacc + i] = a[i];
      dbg[h.dbg_qvel + i] = qvel[i];
    }
    for (int i = e.lane; i < h.nq; i += 32) dbg[h.dbg_qpos + i] = qpos[i];
    for (int i = e.lane; i < 14 * h.nslot; i += 32) dbg[h.dbg_con + i] = WS(con)[i];
    const float *J = WS(J), *jar = WS(jar), *rD = WS(rD);
    for (int r = e.lane; r < nrow; r += 32) {
      float* o = dbg + h.dbg_rows + r * (nv + 7);
      for (int k = 0; k < nv; k++) o[k] = J[r * nv + k];
      o[nv] = WS(rr)[r];
      o[nv + 1] = WS(rv)[r];
      o[nv + 2] = WS(aref)[r];
      o[nv + 3] = rD[r];
      o[nv + 4] = WS(Ahat)[r];
      o[nv + 5] = WS(imp)[r];
      // force at the final acceleration
      float s = -WS(aref)[r];
      for (int k = 0; k < nv; k++) s = fmaf(J[r * nv + k], a[k], s);
      o[nv + 6] = s < 0.f ? -rD[r] * s : 0.f;
      (void)jar;
    }
    if (e.lane == 0) {
      dbg[h.dbg_nrow] = (float)nrow;
      dbg[h.dbg_iter] = (float)iters;
      dbg[h.dbg_status] = (float)status;
    }
  }
}

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
struct StepArgs {
  const uint32_t* blobs;
  const int* blob_off;
  const Tile* tiles;
  float* qpos;
  float* qvel;
  float* warm;
  uint32_t* status;
  uint32_t* stats;
  const float* ctrl;
  int64_t ld;
  int blob_words;   // max over models (shared-memory slot size)
  int n_substeps;
  float* dbg;
  Tile dbg_tile;
};

template <bool DEBUG>
__global__ void __launch_bounds__(256) step_kernel(StepArgs A) {
  extern __shared__ __align__(16) float smem[];
  const Tile tile = DEBUG ? A.dbg_tile : A.tiles[blockIdx.x];
  // model blob -> shared memory
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.blobs + A.blob_off[tile.model]);
    const int nw = reinterpret_cast<const ModelHdr*>(A.blobs + A.blob_off[tile.model])->words;
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < nw / 4; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const ModelHdr* hdr = reinterpret_cast<const ModelHdr*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ws = hdr->ws_floats;
  float* wsbase = smem + A.blob_words;
  const int count = tile.count;
  // stage the tile's state: [coord][env] runs of `count` consecutive envs (coalesced)
  {
    const int nq = hdr->nq, nv = hdr->nv, nu = hdr->nu;
    const int tot = count * (nq + 2 * nv + nu);
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int c = i / count, k = i - c * count;
      const int64_t env = tile.env0 + k;
      float* w = wsbase + k * ws;
      if (c < nq) w[hdr->w_qpos + c] = A.qpos[c * A.ld + env];
      else if (c < nq + nv) w[hdr->w_qvel + (c - nq)] = A.qvel[(c - nq) * A.ld + env];
      else if (c < nq + 2 * nv) w[hdr->w_warm + (c - nq - nv)] = A.warm[(c - nq - nv) * A.ld + env];
      else w[hdr->w_ctrl + (c - nq - 2 * nv)] = A.ctrl[(c - nq - 2 * nv) * A.ld + env];
    }
  }
  __syncthreads();
  if (warp < count) {
    Env e{hdr, reinterpret_cast<const int*>(smem), smem, wsbase + warp * ws, lane};
    uint32_t status = 0;
    // a non-finite warm start is replaced by zeros (flagged)
    {
      bool bad = false;
      for (int d = lane; d < hdr->nv; d += 32) bad = bad || !isfinite(e.w[hdr->w_warm + d]);
      if (__any_sync(kFull, bad)) {
        status |= PG_STATUS_WARM_RESET;
        for (int d = lane; d < hdr->nv; d += 32) e.w[hdr->w_warm + d] = 0.f;
      }
      __syncwarp();
    }
    const int nsub = DEBUG ? 1 : A.n_substeps;
    uint32_t cnt[3] = {0u, 0u, 0u};
    for (int s = 0; s < nsub; s++) substep<DEBUG>(e, status, A.dbg, cnt);
    if (lane == 0 && status) atomicOr(A.status + tile.env0 + warp, status);
    if (lane == 0 && A.stats)
      for (int c = 0; c < 3; c++) A.stats[c * A.ld + tile.env0 + warp] += cnt[c];
  }
  __syncthreads();
  {
    const int nq = hdr->nq, nv = hdr->nv;
    const int tot = count * (nq + 2 * nv);
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int c = i / count, k = i - c * count;
      const int64_t env = tile.env0 + k;
      const float* w = wsbase + k * ws;
      if (c < nq) A.qpos[c * A.ld + env] = w[hdr->w_qpos + c];
      else if (c < nq + nv) A.qvel[(c - nq) * A.ld + env] = w[hdr->w_qvel + (c - nq)];
      else A.warm[(c - nq - nv) * A.ld + env] = w[hdr->w_warm + (c - nq - nv)];
    }
  }
}

__global__ void reset_kernel(const int* env_model, const uint32_t* blobs, const int* blob_off, float* qpos, float* qvel,
                             float* warm, uint32_t* status, int64_t ld, int64_t n, const uint8_t* mask, const float* qpos0,
                             const float* qvel0, int nq_max, int nv_max) {
  const int64_t env = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (env >= n) return;
  if (mask && !mask[env]) return;
  for (int c = 0; c < nq_max; c++) qpos[c * ld + env] = qpos0[c * ld + env];
  for (int c = 0; c < nv_max; c++) {
    qvel[c * ld + env] = qvel0[c * ld + env];
    warm[c * ld + env] = 0.f;
  }
  status[env] = 0u;
  (void)env_model; (void)blobs; (void)blob_off;
}

}  // namespace

cudaError_t configure_step_kernels(size_t smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(step_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

static StepArgs make_args(const pg_batch* b, const pg_state* s, const float* ctrl) {
  StepArgs A;
  A.blobs = b->d_blobs;
  A.blob_off = b->d_blob_off;
  A.tiles = b->d_tiles;
  A.qpos = s->qpos;
  A.qvel = s->qvel;
  A.warm = s->qacc_warm;
  A.status = s->status;
  A.stats = s->stats;
  A.ctrl = ctrl;
  A.ld = s->ld;
  A.blob_words = b->max_blob_words;
  A.n_substeps = 1;
  A.dbg = nullptr;
  A.dbg_tile = Tile{0, 0, 0, 0};
  return A;
}

cudaError_t launch_step(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st) {
  if (b->ntiles == 0) return cudaSuccess;
  StepArgs A = make_args(b, s, ctrl);
  A.n_substeps = n_substeps;
  step_kernel<false><<<b->ntiles, 32 * b->warps, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_debug(const pg_batch* b, const pg_state* s, const float* ctrl, int64_t env, float* out, cudaStream_t st) {
  StepArgs A = make_args(b, s, ctrl);
  int model = 0;
  for (size_t k = 0; k < b->models.size(); k++)
    if (env >= b->env_off[k] && env < b->env_off[k] + b->counts[k]) model = (int)k;
  A.dbg = out;
  A.dbg_tile = Tile{model, (int)env, 1, 0};
  step_kernel<true><<<1, 32 * b->warps, b->smem_bytes, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_reset(const pg_batch* b, const pg_state* s, const uint8_t* mask, const float* qpos0, const float* qvel0,
                         cudaStream_t st) {
  if (s->n == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)((s->n + threads - 1) / threads);
  reset_kernel<<<blocks, threads, 0, st>>>(nullptr, b->d_blobs, b->d_blob_off, s->qpos, s->qvel, s->qacc_warm, s->status,
                                           s->ld, s->n, mask, qpos0, qvel0, b->nq_max, b->nv_max);
  return cudaGetLastError();
}

}  // namespace pg
