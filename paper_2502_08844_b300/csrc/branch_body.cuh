// The branch-parallel physics step: one thread per (environment, branch).
//
// A model qualifies when its kinematic tree splits into a trunk and G >= 2 branches: a branch is
// a chain of hinge/slide bodies that hangs from a trunk body or from the world (a quadruped's
// legs under its torso, a humanoid's legs and arms under its pelvis and waist, the fingers of a
// fixed hand beside a free object); the trunk is every other body (free bodies included).  Every
// contact pair touches at most one branch.  Ordering the dofs branch by branch and the trunk
// last, the mass matrix M and the Newton Hessian H = M + J_A^T D_A J_A (Sec. 3's soft-contact
// step, the solver being MJX's prior art) are block arrowheads: a dense block per branch (the
// branch is a chain, so its ancestor pattern is full), the branch-trunk coupling and the trunk
// block.  The lanes of a group (GP consecutive lanes of a warp, GP the power of two >= G) each
// own one branch: its bodies, dofs, contact pairs and limit rows.  Every lane also computes the
// trunk, identically.  Where the trunk needs the branches (composite inertias, body forces, the
// Schur complement S = H_TT - sum_l H_TB,l H_BB,l^-1 H_BT,l of the block factorisation, the
// line search's sums) the lanes add their parts with an xor butterfly of warp shuffles, which
// leaves the same bits on every lane of the group.
//
// The model is compiled in (run-time compilation per model, see branch.cpp): namespace pgb
// holds its sizes as constexpr values and its tables as __constant__ arrays, indexed here only
// at compile-time positions, so every table read folds to an immediate; a value that differs
// between branches is chosen by the lane's branch index with selects (lsel).
//
// Per substep, in the order of the step (the same method as step_device.cuh, whose primitives
// this file reuses): kinematics, bias forces (RNEA), composite-rigid-body M, the smooth
// acceleration a0 = M^-1 (tau - c), collision over the lane's pairs, the contact and limit rows
// (Jacobian, exact Ahat = J M^-1 J^T from the block factor, impedance, aref, D), the Newton solve
// with the exact breakpoint line search and its active-set termination, semi-implicit Euler.
#pragma once
#include "step_device.cuh"

namespace pgb {
using namespace pg;

constexpr int NTRI = NT * (NT + 1) / 2;   // packed lower triangle of the trunk block
constexpr int NRL = 4 * NCL + LS;         // rows of a lane: 4 per contact, then its limits

// ---- lane-group reductions (group-uniform results, bitwise equal on every lane) ----
__device__ __forceinline__ unsigned group_mask() {
  const unsigned lane = threadIdx.x & 31u;
  return GP == 32 ? 0xffffffffu : (((1u << GP) - 1u) << (lane & ~(unsigned)(GP - 1)));
}
__device__ __forceinline__ float gsum(float v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}
__device__ __forceinline__ float gmin(float v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1) v = fminf(v, __shfl_xor_sync(gm, v, o));
  return v;
}
__device__ __forceinline__ int gor(int v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1) v |= __shfl_xor_sync(gm, v, o);
  return v;
}
__device__ __forceinline__ int gand(int v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1) v &= __shfl_xor_sync(gm, v, o);
  return v;
}
__device__ __forceinline__ int gsumi(int v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}
template <int N>
__device__ __forceinline__ void gsum_arr(float (&v)[N], unsigned gm) {
#pragma unroll
  for (int o = 1; o < GP; o <<= 1)
#pragma unroll
    for (int i = 0; i < N; i++) v[i] += __shfl_xor_sync(gm, v[i], o);
}

// the lane's value of a per-branch table entry: f(g) for g = the lane's branch
template <class F>
__device__ __forceinline__ auto lsel(int br, F f) -> decltype(f(0)) {
  auto v = f(0);
#pragma unroll
  for (int g = 1; g < GP; g++)
    if (br == g) v = f(g);
  return v;
}

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ float3 c3(const float* p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float dot6(const float* a, float3 w, float3 v) {
  return a[0] * w.x + a[1] * w.y + a[2] * w.z + a[3] * v.x + a[4] * v.y + a[5] * v.z;
}
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }   // i >= j

// spatial inertia about the tree origin o (Ixx Iyy Izz Ixy Ixz Iyz, m c, m) of a body with
// frame (x, q), mass m, centre ipos and body-frame inertia In
__device__ __forceinline__ void spatial_inertia(float3 x, Quat q, float3 o, float m, float3 ip, const float In[6],
                                                float ci[10]) {
  float R[9];
  qmat(q, R);
  const float3 com = x + mat_mul(R, ip);
  const float Ib[9] = {In[0], In[3], In[4], In[3], In[1], In[5], In[4], In[5], In[2]};
  float T[9];
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int k = 0; k < 3; k++) T[3 * r + k] = R[3 * r] * Ib[k] + R[3 * r + 1] * Ib[3 + k] + R[3 * r + 2] * Ib[6 + k];
  const float3 cc = com - o;
  const float c2 = dot3(cc, cc);
  ci[0] = T[0] * R[0] + T[1] * R[1] + T[2] * R[2] + m * (c2 - cc.x * cc.x);
  ci[1] = T[3] * R[3] + T[4] * R[4] + T[5] * R[5] + m * (c2 - cc.y * cc.y);
  ci[2] = T[6] * R[6] + T[7] * R[7] + T[8] * R[8] + m * (c2 - cc.z * cc.z);
  ci[3] = T[0] * R[3] + T[1] * R[4] + T[2] * R[5] - m * cc.x * cc.y;
  ci[4] = T[0] * R[6] + T[1] * R[7] + T[2] * R[8] - m * cc.x * cc.z;
  ci[5] = T[3] * R[6] + T[4] * R[7] + T[5] * R[8] - m * cc.y * cc.z;
  ci[6] = m * cc.x;
  ci[7] = m * cc.y;
  ci[8] = m * cc.z;
  ci[9] = m;
}

// spatial inertia times a motion vector (w; v): (I w + h x v; m v - h x w)
__device__ __forceinline__ void imul(const float ci[10], float3 w, float3 v, float3& fa, float3& fl) {
  const float3 hc = make_float3(ci[6], ci[7], ci[8]);
  fa = make_float3(ci[0] * w.x + ci[3] * w.y + ci[4] * w.z, ci[3] * w.x + ci[1] * w.y + ci[5] * w.z,
                   ci[4] * w.x + ci[5] * w.y + ci[2] * w.z) +
       cross3(hc, v);
  fl = v * ci[9] - cross3(hc, w);
}

// impedance d(r) of the soft constraint (solimp = d0, dwidth, width, mid, power)
__device__ __forceinline__ float imp(float pos) {
  const float x = fminf(fabsf(pos) * (1.f / SOLIMP_WIDTH), 1.f);
  float y;
  if (x >= 1.f) y = 1.f;
  else if (x <= SOLIMP_MID) y = (SOLIMP_POWER == 2.f ? x * x : powf(x, SOLIMP_POWER)) * IMP_MID_INV;
  else y = 1.f - (SOLIMP_POWER == 2.f ? (1.f - x) * (1.f - x) : powf(1.f - x, SOLIMP_POWER)) * IMP_TAIL_INV;
  return SOLIMP_D0 + y * (SOLIMP_DW - SOLIMP_D0);
}

// ---- small dense factorisations (lower triangles of full arrays) ----
// (Square roots and divisions in this file take the hardware's reciprocal square root and
// approximate division, a few ulp from the correctly rounded result, instead of the IEEE
// sequences whose slow paths would be unrolled at every site: the kernel is bound by fetching
// its own instructions.)
// Cholesky in place: L L^T = A; dinv[i] = 1 / L_ii; false when a pivot is not positive
template <int N>
__device__ __forceinline__ bool chol(float (&A)[N][N], float (&dinv)[N]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < N; j++) {
    float s = A[j][j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= A[j][k] * A[j][k];
    ok = ok && s > 0.f;
    const float sp = fmaxf(s, 1e-30f), inv = rsqrtf(sp);
    A[j][j] = sp * inv;
    dinv[j] = inv;
#pragma unroll
    for (int i = j + 1; i < N; i++) {
      float t = A[i][j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i][k] * A[j][k];
      A[i][j] = t * inv;
    }
  }
  return ok;
}
// x <- L^-1 x
template <int N>
__device__ __forceinline__ void fwd(const float (&L)[N][N], const float (&dinv)[N], float (&x)[N]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    float s = x[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= L[i][k] * x[k];
    x[i] = s * dinv[i];
  }
}
// x <- L^-T x
template <int N>
__device__ __forceinline__ void bwd(const float (&L)[N][N], const float (&dinv)[N], float (&x)[N]) {
#pragma unroll
  for (int i = N - 1; i >= 0; i--) {
    float s = x[i];
#pragma unroll
    for (int k = i + 1; k < N; k++) s -= L[k][i] * x[k];
    x[i] = s * dinv[i];
  }
}

// The block-arrowhead factor of a symmetric matrix A (M or H): the lane's branch block A_BB (its
// Cholesky factor LB, dB), Y = LB^-1 A_BT and the trunk Schur complement's factor LS, dS.
struct Factor {
  float LB[NB][NB], dB[NB];
  float Y[NB][NT];
  float LS[NT][NT], dS[NT];
};

// Factor A (branch block AB, coupling ABT, trunk block AT0 + the lanes' parts ATl) and solve
// A x = r (r_B = rB, r_T = rT0 + the lanes' parts rTl); xB, xT out.  One group reduction of
// NTRI + NT floats.  Returns false (group-uniform) when a pivot is not positive.
__device__ __forceinline__ bool block_solve(Factor& F, const float (&AB)[NB][NB], const float (&ABT)[NB][NT],
                                            const float (&AT0)[NT][NT], const float (&ATl)[NTRI],
                                            const float (&rB)[NB], const float (&rT0)[NT], const float (&rTl)[NT],
                                            float (&xB)[NB], float (&xT)[NT], unsigned gm) {
#pragma unroll
  for (int i = 0; i < NB; i++)
#pragma unroll
    for (int k = 0; k <= i; k++) F.LB[i][k] = AB[i][k];
  const bool okB = chol(F.LB, F.dB);
  float y[NB];
#pragma unroll
  for (int i = 0; i < NB; i++) y[i] = rB[i];
  fwd(F.LB, F.dB, y);
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float col[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) col[i] = ABT[i][t];
    fwd(F.LB, F.dB, col);
#pragma unroll
    for (int i = 0; i < NB; i++) F.Y[i][t] = col[i];
  }
  // the lane's parts: ATl - Y^T Y and rTl - Y^T y, summed over the group
  float red[NTRI + NT];
#pragma unroll
  for (int t = 0; t < NT; t++) {
#pragma unroll
    for (int s = 0; s <= t; s++) {
      float v = ATl[tri(t, s)];
#pragma unroll
      for (int i = 0; i < NB; i++) v -= F.Y[i][t] * F.Y[i][s];
      red[tri(t, s)] = v;
    }
    float v = rTl[t];
#pragma unroll
    for (int i = 0; i < NB; i++) v -= F.Y[i][t] * y[i];
    red[NTRI + t] = v;
  }
  gsum_arr(red, gm);
  const int ok = gand(okB ? 1 : 0, gm);
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int s = 0; s <= t; s++) F.LS[t][s] = AT0[t][s] + red[tri(t, s)];
  const bool okS = chol(F.LS, F.dS);
#pragma unroll
  for (int t = 0; t < NT; t++) xT[t] = rT0[t] + red[NTRI + t];
  fwd(F.LS, F.dS, xT);
  bwd(F.LS, F.dS, xT);
  // x_B = LB^-T (y - Y x_T)
#pragma unroll
  for (int i = 0; i < NB; i++) {
    float v = y[i];
#pragma unroll
    for (int t = 0; t < NT; t++) v -= F.Y[i][t] * xT[t];
    xB[i] = v;
  }
  bwd(F.LB, F.dB, xB);
  return ok && okS;
}

// the Gram entries u_a^T A^-1 u_b of K row vectors (branch parts uB, trunk parts uT) with the
// factor of A: z = LB^-1 u_B, w = u_T - Y^T z, s = LS^-1 w, u_a^T A^-1 u_b = z_a.z_b + s_a.s_b
template <int K>
__device__ __forceinline__ void gram(const Factor& F, const float (&uB)[K][NB], const float (&uT)[K][NT],
                                     float (&A)[K][K]) {
  float z[K][NB], s[K][NT];
#pragma unroll
  for (int a = 0; a < K; a++) {
#pragma unroll
    for (int i = 0; i < NB; i++) z[a][i] = uB[a][i];
    fwd(F.LB, F.dB, z[a]);
#pragma unroll
    for (int t = 0; t < NT; t++) {
      float v = uT[a][t];
#pragma unroll
      for (int i = 0; i < NB; i++) v -= F.Y[i][t] * z[a][i];
      s[a][t] = v;
    }
    fwd(F.LS, F.dS, s[a]);
  }
#pragma unroll
  for (int a = 0; a < K; a++)
#pragma unroll
    for (int b = 0; b <= a; b++) {
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < NB; i++) v = fmaf(z[a][i], z[b][i], v);
#pragma unroll
      for (int t = 0; t < NT; t++) v = fmaf(s[a][t], s[b][t], v);
      A[a][b] = v;
      A[b][a] = v;
    }
}

// ---- per-lane state of one environment ----
struct Lane {
  int br;        // the lane's branch
  unsigned gm;   // its group's shuffle mask
  int64_t env, ld;
  const float* ctrl;
  const float* hf;   // the heightfield's elevations (device), or NULL
  const float* dr;   // per-environment parameters [nrand][ld] (the DR variant), or NULL
  __device__ __forceinline__ float dr_row(int k) const { return __ldg(dr + k * ld + env); }
  __device__ __forceinline__ float ctrl_row(int a) const { return __ldg(ctrl + a * ld + env); }
  // state: trunk (identical on the group's lanes) and branch
  float qT[NQT], vT[NT], wT[NT];
  float qB[NB], vB[NB], wB[NB];
  // mass matrix blocks and smooth acceleration
  float MB[NB][NB], MBT[NB][NT], MT[NT][NT];
  float a0B[NB], a0T[NT];
  // contacts (n, t1, t2 Jacobian rows) and row parameters
  float JB[NCL][3][NB], JT[NCL][3][NT];
  float mu[NCL];
  float D[NRL], aref[NRL], lsgn[LS > 0 ? LS : 1];
};

// a per-branch table entry at the lane's branch
#define LV(tab, ...) lsel(L.br, [&](int g_) { return tab[g_] __VA_ARGS__; })
#define LV0(tab) lsel(L.br, [&](int g_) { return tab[g_]; })

__device__ __forceinline__ Quat q4(const float* p) { return Quat{p[0], p[1], p[2], p[3]}; }

// frames, motion subspaces (cdof: angular; linear about the tree origin) and spatial inertias
struct Kin {
  float3 xT[BT];
  Quat qT[BT];
  float3 oT[BT];
  float cdT[NT][6];
  float ciT[BT][10];
  float3 xB[BB > 0 ? BB : 1];
  Quat qB[BB > 0 ? BB : 1];
  float3 oB;
  float cdB[NB][6];
  float ciB[BB > 0 ? BB : 1][10];
};

__device__ __forceinline__ void set6(float* d, float3 a, float3 b) {
  d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = b.x; d[4] = b.y; d[5] = b.z;
}

// one joint (hinge or slide) of a body whose frame is (x, q) so far: its cdof about o, then the
// frame after the joint
__device__ __forceinline__ void joint_1dof(int type, float3 lp, float3 la, float qv, float3 o, float3& x, Quat& q,
                                           float* cd) {
  const float3 anchor = x + qrot(q, lp), axis = qrot(q, la);
  if (type == PG_JNT_HINGE) {
    set6(cd, axis, cross3(axis, o - anchor));
    float sn, cs;
    sincosf(0.5f * qv, &sn, &cs);
    q = qmul(q, Quat{cs, la.x * sn, la.y * sn, la.z * sn});
    x = anchor - qrot(q, lp);
  } else {
    set6(cd, make_float3(0.f, 0.f, 0.f), axis);
    x = x + axis * qv;
  }
}

// a body's mass, centre of mass and inertia scale with the environment's parameters (DR): the mass
// scale (mass and inertia), the payload on body 1, the centre-of-mass offset
template <bool DR>
__device__ __forceinline__ void body_params(const Lane& L, int g, float& m, float3& ip, float& iscale) {
  iscale = 1.f;
  if (!DR) return;
  iscale = 1.f + L.dr_row(DR_MASS + g);
  m *= iscale;
  if (g == 1) m += L.dr_row(1);
  ip = ip + make_float3(L.dr_row(DR_COM + 3 * g), L.dr_row(DR_COM + 3 * g + 1), L.dr_row(DR_COM + 3 * g + 2));
}

template <bool DR = false>
__device__ __forceinline__ void kinematics(const Lane& L, Kin& K) {
  // trunk bodies in level order
#pragma unroll
  for (int k = 0; k < BT; k++) {
    float3 x = make_float3(0.f, 0.f, 0.f);
    Quat q{1.f, 0.f, 0.f, 0.f};
    const int par = kTBpar[k];
#pragma unroll
    for (int p = 0; p < BT; p++)
      if (p == par) { x = K.xT[p]; q = K.qT[p]; }
    x = x + qrot(q, c3(kTBpos[k]));
    q = qmul(q, q4(kTBquat[k]));
    const int oq = kTBorg[k];
    const float3 o = oq >= 0 ? make_float3(L.qT[oq], L.qT[oq + 1], L.qT[oq + 2]) : c3(kTBorgp[k]);
#pragma unroll
    for (int j = 0; j < NJT; j++) {
      const int type = kTJtype[k][j];
      if (type < 0) continue;
      const int qa = kTJq[k][j], d0 = kTJd[k][j];
      if (type == PG_JNT_FREE) {
        x = make_float3(L.qT[qa], L.qT[qa + 1], L.qT[qa + 2]);
        q = qnormalize(Quat{L.qT[qa + 3], L.qT[qa + 4], L.qT[qa + 5], L.qT[qa + 6]});
        float R[9];
        qmat(q, R);
#pragma unroll
        for (int i = 0; i < 3; i++) {
          set6(K.cdT[d0 + i], make_float3(0.f, 0.f, 0.f),
               make_float3(i == 0 ? 1.f : 0.f, i == 1 ? 1.f : 0.f, i == 2 ? 1.f : 0.f));
          const float3 ax = mat_col(R, i);
          set6(K.cdT[d0 + 3 + i], ax, cross3(ax, o - x));
        }
      } else {
        joint_1dof(type, c3(kTJpos[k][j]), c3(kTJaxis[k][j]), L.qT[qa], o, x, q, K.cdT[d0]);
      }
    }
    q = qnormalize(q);
    K.xT[k] = x;
    K.qT[k] = q;
    K.oT[k] = o;
    if (DR) {
      float m = kTBmass[k], sc;
      float3 ip = c3(kTBipos[k]);
      body_params<DR>(L, kTBg[k], m, ip, sc);
      float In[6];
#pragma unroll
      for (int i = 0; i < 6; i++) In[i] = sc * kTBinert[k][i];
      spatial_inertia(x, q, o, m, ip, In, K.ciT[k]);
    } else if (kTBmass[k] > 0.f) {
      spatial_inertia(x, q, o, kTBmass[k], c3(kTBipos[k]), kTBinert[k], K.ciT[k]);
    } else {
#pragma unroll
      for (int i = 0; i < 10; i++) K.ciT[k][i] = 0.f;
    }
  }
  // the lane's branch, from its attachment (a trunk body or the world)
  {
    const int oq = LV0(kLorgT);
    K.oB = oq >= 0 ? make_float3(L.qT[oq], L.qT[oq + 1], L.qT[oq + 2])
                   : make_float3(LV(kLorg, [0]), LV(kLorg, [1]), LV(kLorg, [2]));
  }
  const int att = LV0(kLatt);
#pragma unroll
  for (int b = 0; b < BB; b++) {
    float3 x = make_float3(0.f, 0.f, 0.f);
    Quat q{1.f, 0.f, 0.f, 0.f};
    if (b == 0) {
#pragma unroll
      for (int p = 0; p < BT; p++)
        if (p == att) { x = K.xT[p]; q = K.qT[p]; }
    } else {
      x = K.xB[b - 1];
      q = K.qB[b - 1];
    }
    x = x + qrot(q, make_float3(LV(kLBpos, [b][0]), LV(kLBpos, [b][1]), LV(kLBpos, [b][2])));
    q = qmul(q, Quat{LV(kLBquat, [b][0]), LV(kLBquat, [b][1]), LV(kLBquat, [b][2]), LV(kLBquat, [b][3])});
#pragma unroll
    for (int j = 0; j < bnj(b); j++) {
      const int d = bdof0(b) + j;
      const int type = LV(kLJtype, [d]);
      if (type == PG_JNT_HINGE || type == PG_JNT_SLIDE) {
        joint_1dof(type, make_float3(LV(kLJpos, [d][0]), LV(kLJpos, [d][1]), LV(kLJpos, [d][2])),
                   make_float3(LV(kLJaxis, [d][0]), LV(kLJaxis, [d][1]), LV(kLJaxis, [d][2])), L.qB[d], K.oB, x, q,
                   K.cdB[d]);
      } else {
#pragma unroll
        for (int i = 0; i < 6; i++) K.cdB[d][i] = 0.f;
      }
    }
    q = qnormalize(q);
    K.xB[b] = x;
    K.qB[b] = q;
    float m = LV(kLBmass, [b]), sc;
    float3 ip = make_float3(LV(kLBipos, [b][0]), LV(kLBipos, [b][1]), LV(kLBipos, [b][2]));
    body_params<DR>(L, LV(kLBg, [b]), m, ip, sc);
    const float In[6] = {sc * LV(kLBinert, [b][0]), sc * LV(kLBinert, [b][1]), sc * LV(kLBinert, [b][2]),
                         sc * LV(kLBinert, [b][3]), sc * LV(kLBinert, [b][4]), sc * LV(kLBinert, [b][5])};
    spatial_inertia(x, q, K.oB, m, ip, In, K.ciB[b]);
  }
}

// ---- bias forces c(q, qdot) (RNEA) ----

// the velocity and bias acceleration across one 1-dof joint
__device__ __forceinline__ void rnea_joint(const float* cd, float qd, float3& w, float3& v, float3& aw, float3& av) {
  const float3 dw = make_float3(cd[0], cd[1], cd[2]) * qd, dv = make_float3(cd[3], cd[4], cd[5]) * qd;
  aw = aw + cross3(w, dw);
  av = av + cross3(w, dv) + cross3(v, dw);
  w = w + dw;
  v = v + dv;
}

__device__ __forceinline__ void body_force(const float ci[10], float3 w, float3 v, float3 aw, float3 av, float f[6]) {
  float3 fa, fl, ia, il;
  imul(ci, aw, av, fa, fl);
  imul(ci, w, v, ia, il);
  set6(f, fa + cross3(w, ia) + cross3(v, il), fl + cross3(w, il));
}

// bias forces of every dof: cB (branch), cT (trunk)
__device__ __forceinline__ void rnea(const Lane& L, const Kin& K, float (&cB)[NB], float (&cT)[NT]) {
  const float3 g0 = make_float3(-GRAV_X, -GRAV_Y, -GRAV_Z);
  float3 wT[BT], vT[BT], awT[BT], avT[BT];
  float fT[BT][6];
#pragma unroll
  for (int k = 0; k < BT; k++) {
    float3 w = make_float3(0.f, 0.f, 0.f), v = w, aw = w, av = g0;
    const int par = kTBpar[k];
#pragma unroll
    for (int p = 0; p < BT; p++)
      if (p == par) { w = wT[p]; v = vT[p]; aw = awT[p]; av = avT[p]; }
#pragma unroll
    for (int j = 0; j < NJT; j++) {
      const int type = kTJtype[k][j];
      if (type < 0) continue;
      const int d0 = kTJd[k][j];
      if (type == PG_JNT_FREE) {
        v = v + make_float3(L.vT[d0], L.vT[d0 + 1], L.vT[d0 + 2]);
        float3 dw = make_float3(0.f, 0.f, 0.f), dv = dw;
#pragma unroll
        for (int i = 3; i < 6; i++) {
          dw = dw + c3(&K.cdT[d0 + i][0]) * L.vT[d0 + i];
          dv = dv + c3(&K.cdT[d0 + i][3]) * L.vT[d0 + i];
        }
        aw = aw + cross3(w, dw);
        av = av + cross3(w, dv) + cross3(v, dw);
        w = w + dw;
        v = v + dv;
      } else {
        rnea_joint(K.cdT[d0], L.vT[d0], w, v, aw, av);
      }
    }
    wT[k] = w; vT[k] = v; awT[k] = aw; avT[k] = av;
    body_force(K.ciT[k], w, v, aw, av, fT[k]);
  }
  // the branch
  float fB[BB > 0 ? BB : 1][6];
  {
    const int att = LV0(kLatt);
    float3 w = make_float3(0.f, 0.f, 0.f), v = w, aw = w, av = g0;
#pragma unroll
    for (int p = 0; p < BT; p++)
      if (p == att) { w = wT[p]; v = vT[p]; aw = awT[p]; av = avT[p]; }
#pragma unroll
    for (int b = 0; b < BB; b++) {
#pragma unroll
      for (int j = 0; j < bnj(b); j++) {
        const int d = bdof0(b) + j;
        rnea_joint(K.cdB[d], L.vB[d], w, v, aw, av);
      }
      body_force(K.ciB[b], w, v, aw, av, fB[b]);
    }
#pragma unroll
    for (int b = BB - 1; b >= 1; b--)
#pragma unroll
      for (int i = 0; i < 6; i++) fB[b - 1][i] += fB[b][i];
    // the branch's force on its attachment, summed over the group
    float red[BT * 6];
#pragma unroll
    for (int k = 0; k < BT; k++)
#pragma unroll
      for (int i = 0; i < 6; i++) red[6 * k + i] = (BB > 0 && k == att) ? fB[0][i] : 0.f;
    gsum_arr(red, L.gm);
#pragma unroll
    for (int k = 0; k < BT; k++)
#pragma unroll
      for (int i = 0; i < 6; i++) fT[k][i] += red[6 * k + i];
  }
#pragma unroll
  for (int k = BT - 1; k >= 1; k--) {
    const int par = kTBpar[k];
#pragma unroll
    for (int p = 0; p < BT; p++)
      if (p == par)
#pragma unroll
        for (int i = 0; i < 6; i++) fT[p][i] += fT[k][i];
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    const int k = kTDbody[t];
    cT[t] = dot6(K.cdT[t], c3(&fT[k][0]), c3(&fT[k][3]));
  }
#pragma unroll
  for (int b = 0; b < BB; b++)
#pragma unroll
    for (int j = 0; j < bnj(b); j++) {
      const int d = bdof0(b) + j;
      cB[d] = dot6(K.cdB[d], c3(&fB[b][0]), c3(&fB[b][3]));
    }
}

// ---- composite-rigid-body mass matrix (in place on the inertias) ----
template <bool DR = false>
__device__ __forceinline__ void crba(Lane& L, Kin& K) {
#pragma unroll
  for (int b = BB - 1; b >= 1; b--)
#pragma unroll
    for (int i = 0; i < 10; i++) K.ciB[b - 1][i] += K.ciB[b][i];
  {
    const int att = LV0(kLatt);
    float red[BT * 10];
#pragma unroll
    for (int k = 0; k < BT; k++)
#pragma unroll
      for (int i = 0; i < 10; i++) red[10 * k + i] = (BB > 0 && k == att) ? K.ciB[0][i] : 0.f;
    gsum_arr(red, L.gm);
#pragma unroll
    for (int k = 0; k < BT; k++)
#pragma unroll
      for (int i = 0; i < 10; i++) K.ciT[k][i] += red[10 * k + i];
  }
#pragma unroll
  for (int k = BT - 1; k >= 1; k--) {
    const int par = kTBpar[k];
#pragma unroll
    for (int p = 0; p < BT; p++)
      if (p == par)
#pragma unroll
        for (int i = 0; i < 10; i++) K.ciT[p][i] += K.ciT[k][i];
  }
  // branch rows: M_ji = cdof_i . (Ic(body j) cdof_j) for the branch's earlier dofs i and the
  // trunk dofs on the attachment's chain
  const int anc = LV0(kLanc);
#pragma unroll
  for (int b = 0; b < BB; b++)
#pragma unroll
    for (int jj = 0; jj < bnj(b); jj++) {
      const int j = bdof0(b) + jj;
      float3 fa, fl;
      imul(K.ciB[b], c3(&K.cdB[j][0]), c3(&K.cdB[j][3]), fa, fl);
#pragma unroll
      for (int i = 0; i <= j; i++) L.MB[j][i] = dot6(K.cdB[i], fa, fl);
      L.MB[j][j] += LV(kLDarm, [j]);
      if (DR && LV(kLDg, [j]) >= 0) L.MB[j][j] += L.dr_row(DR_ARM + LV(kLDg, [j]));
#pragma unroll
      for (int t = 0; t < NT; t++) L.MBT[j][t] = ((anc >> t) & 1) ? dot6(K.cdT[t], fa, fl) : 0.f;
    }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float3 fa, fl;
    imul(K.ciT[kTDbody[t]], c3(&K.cdT[t][0]), c3(&K.cdT[t][3]), fa, fl);
#pragma unroll
    for (int s = 0; s <= t; s++) L.MT[t][s] = ((kTDanc[t] >> s) & 1) ? dot6(K.cdT[s], fa, fl) : 0.f;
    L.MT[t][t] += kTDarm[t];
    if (DR) L.MT[t][t] += L.dr_row(DR_ARM + kTDg[t]);
  }
}

// actuator force of a dof with actuator a at position q and velocity qd (PD or motor)
__device__ __forceinline__ float act_force(int atype, float gear, float kp, float kd, int clim, float lo, float hi,
                                           int flim, float flo, float fhi, float u, float q, float qd) {
  if (clim) u = fminf(fmaxf(u, lo), hi);
  float tau = atype == PG_ACT_MOTOR ? gear * u : kp * (u - q) - kd * qd;
  if (flim) tau = fminf(fmaxf(tau, flo), fhi);
  return tau;
}

// ---- the lane's contacts: collision of its pairs, their Jacobian rows ----
__device__ __forceinline__ void frame_of(int side, const Kin& K, float3& x, Quat& q) {
  x = make_float3(0.f, 0.f, 0.f);
  q = Quat{1.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < BT; k++)
    if (side == k) { x = K.xT[k]; q = K.qT[k]; }
#pragma unroll
  for (int b = 0; b < BB; b++)
    if (side == BT + b) { x = K.xB[b]; q = K.qB[b]; }
}
__device__ __forceinline__ float3 origin_of(int side, const Kin& K) {
  float3 o = K.oB;
#pragma unroll
  for (int k = 0; k < BT; k++)
    if (side == k) o = K.oT[k];
  return o;
}

// collision of pair slot s; k[] its points (dist = 1 where absent); returns the point count
__device__ __forceinline__ int collide_slot(const Lane& L, const Kin& K, int s, Con k[4]) {
  const int t1 = LV(kPt1, [s]), t2 = LV(kPt2, [s]);
  float3 x1, x2, bx;
  Quat bq;
  float R1[9], R2[9];
  frame_of(LV(kPs1, [s]), K, bx, bq);
  x1 = bx + qrot(bq, make_float3(LV(kPgp1, [s][0]), LV(kPgp1, [s][1]), LV(kPgp1, [s][2])));
  qmat(qnormalize(qmul(bq, Quat{LV(kPgq1, [s][0]), LV(kPgq1, [s][1]), LV(kPgq1, [s][2]), LV(kPgq1, [s][3])})), R1);
  frame_of(LV(kPs2, [s]), K, bx, bq);
  x2 = bx + qrot(bq, make_float3(LV(kPgp2, [s][0]), LV(kPgp2, [s][1]), LV(kPgp2, [s][2])));
  qmat(qnormalize(qmul(bq, Quat{LV(kPgq2, [s][0]), LV(kPgq2, [s][1]), LV(kPgq2, [s][2]), LV(kPgq2, [s][3])})), R2);
  const float s1[3] = {LV(kPsz1, [s][0]), LV(kPsz1, [s][1]), LV(kPsz1, [s][2])};
  const float s2[3] = {LV(kPsz2, [s][0]), LV(kPsz2, [s][1]), LV(kPsz2, [s][2])};
#pragma unroll
  for (int i = 0; i < 4; i++) { k[i].dist = 1.f; k[i].pos = x1; k[i].n = make_float3(0.f, 0.f, 1.f); }
  if (t1 < 0) return 0;
  if (t1 == PG_GEOM_HFIELD) {   // the terrain: a sphere, a capsule's two end spheres, or a box as a solid
    const HGrid g{L.hf, HF_NROW, HF_NCOL, s1[0], s1[1], s1[2], 2.f * s1[0] / (float)(HF_NCOL - 1),
                  2.f * s1[1] / (float)(HF_NROW - 1)};
    if (t2 == PG_GEOM_SPHERE) {
      k[0] = hfield_sphere(g, x1, R1, x2, s2[0]);
      return 1;
    }
    if (t2 == PG_GEOM_CAPSULE) {
      const float3 a = mat_col(R2, 2);
      k[0] = hfield_sphere(g, x1, R1, x2 - a * s2[1], s2[0]);
      k[1] = hfield_sphere(g, x1, R1, x2 + a * s2[1], s2[0]);
      return 2;
    }
    const Solid sd{8, 6, make_float3(s2[0], s2[1], s2[2]), nullptr, nullptr};
    return hfield_solid(g, x1, R1, x2, R2, sd, k);
  }
  if (t1 == PG_GEOM_PLANE) {
    const float3 nz = mat_col(R1, 2);
    if (t2 == PG_GEOM_SPHERE) {
      k[0] = plane_sphere(x1, nz, x2, s2[0]);
      return 1;
    }
    if (t2 == PG_GEOM_CAPSULE) {
      const float3 a = mat_col(R2, 2);
      k[0] = plane_sphere(x1, nz, x2 - a * s2[1], s2[0]);
      k[1] = plane_sphere(x1, nz, x2 + a * s2[1], s2[0]);
      return 2;
    }
    // box: the 4 deepest corners (ties: lower index), kept in corner order
    float dd[8];
    float3 cp[8];
#pragma unroll
    for (int v = 0; v < 8; v++) {
      const float3 l = make_float3((v & 1) ? s2[0] : -s2[0], (v & 2) ? s2[1] : -s2[1], (v & 4) ? s2[2] : -s2[2]);
      cp[v] = x2 + mat_mul(R2, l);
      dd[v] = dot3(nz, cp[v] - x1);
    }
    unsigned chosen = 0;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      int bi = -1;
      float bd = 0.f;
#pragma unroll
      for (int v = 0; v < 8; v++)
        if (!((chosen >> v) & 1u) && (bi < 0 || dd[v] < bd)) { bi = v; bd = dd[v]; }
      chosen |= 1u << bi;
    }
    int i = 0;
#pragma unroll
    for (int v = 0; v < 8; v++)
      if ((chosen >> v) & 1u) {
        // i < 4 always (exactly four bits are set)
#pragma unroll
        for (int m = 0; m < 4; m++)
          if (m == i) {
            k[m].n = nz;
            k[m].dist = dd[v];
            k[m].pos = cp[v] - nz * (0.5f * dd[v]);
          }
        i++;
      }
    return 4;
  }
  if (t1 == PG_GEOM_SPHERE) {
    if (t2 == PG_GEOM_SPHERE) k[0] = sphere_sphere(x1, s1[0], x2, s2[0]);
    else if (t2 == PG_GEOM_CAPSULE) {
      const float3 a = mat_col(R2, 2);
      const float t = fminf(fmaxf(dot3(x1 - x2, a), -s2[1]), s2[1]);
      k[0] = sphere_sphere(x1, s1[0], x2 + a * t, s2[0]);
    } else {
      k[0] = sphere_box(x1, s1[0], x2, R2, make_float3(s2[0], s2[1], s2[2]));
    }
    return 1;
  }
  if (t1 == PG_GEOM_CAPSULE) {
    const float3 a1 = mat_col(R1, 2);
    if (t2 == PG_GEOM_CAPSULE) {
      const float3 a2 = mat_col(R2, 2);
      float u, v;
      seg_seg(x1, a1, s1[1], x2, a2, s2[1], u, v);
      k[0] = sphere_sphere(x1 + a1 * u, s1[0], x2 + a2 * v, s2[0]);
      return 1;
    }
    const float3 hb = make_float3(s2[0], s2[1], s2[2]);
    k[0] = sphere_box(x1 - a1 * s1[1], s1[0], x2, R2, hb);
    k[1] = sphere_box(x1 + a1 * s1[1], s1[0], x2, R2, hb);
    return 2;
  }
  return box_box(x1, R1, make_float3(s1[0], s1[1], s1[2]), x2, R2, make_float3(s2[0], s2[1], s2[2]), k);
}

// Jacobian rows (n, t1, t2) of a contact at point p of pair slot s:
// sum over the dofs of geom2's chain minus geom1's (shared ancestors cancel), column d of the
// point velocity being cdof_lin + cdof_ang x (p - o) about its tree's origin o
__device__ __forceinline__ void contact_rows(Lane& L, const Kin& K, int s, int c, float3 p, float3 n) {
  float3 t1, t2;
  contact_frame(n, t1, t2);
  const float3 o1 = origin_of(LV(kPs1, [s]), K), o2 = origin_of(LV(kPs2, [s]), K);
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int cb = LV(kPjb, [s][i]);
    float3 jac = make_float3(0.f, 0.f, 0.f);
    if (cb != 0) {
      const float3 cw = c3(&K.cdB[i][0]), cl = c3(&K.cdB[i][3]);
      jac = (cl + cross3(cw, p - K.oB)) * (float)cb;
    }
    L.JB[c][0][i] = dot3(n, jac);
    L.JB[c][1][i] = dot3(t1, jac);
    L.JB[c][2][i] = dot3(t2, jac);
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    const int ct = LV(kPjt, [s][t]);
    float3 jac = make_float3(0.f, 0.f, 0.f);
    if (ct != 0) {
      const float3 cw = c3(&K.cdT[t][0]), cl = c3(&K.cdT[t][3]);
      jac = (cl + cross3(cw, p - (ct > 0 ? o2 : o1))) * (float)ct;
    }
    L.JT[c][0][t] = dot3(n, jac);
    L.JT[c][1][t] = dot3(t1, jac);
    L.JT[c][2][t] = dot3(t2, jac);
  }
}

// J . x over one contact's three frame rows
__device__ __forceinline__ void jdot3(const Lane& L, int c, const float (&xB)[NB], const float (&xT)[NT], float& dn,
                                      float& d1, float& d2) {
  dn = d1 = d2 = 0.f;
#pragma unroll
  for (int i = 0; i < NB; i++) {
    dn = fmaf(L.JB[c][0][i], xB[i], dn);
    d1 = fmaf(L.JB[c][1][i], xB[i], d1);
    d2 = fmaf(L.JB[c][2][i], xB[i], d2);
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    dn = fmaf(L.JT[c][0][t], xT[t], dn);
    d1 = fmaf(L.JT[c][1][t], xT[t], d1);
    d2 = fmaf(L.JT[c][2][t], xT[t], d2);
  }
}

// a pyramid edge row e of a contact: n + mu t1, n - mu t1, n + mu t2, n - mu t2
__device__ __forceinline__ float edge(float mu, int e, float dn, float d1, float d2) {
  const float dt = e < 2 ? d1 : d2;
  return (e & 1) ? dn - mu * dt : dn + mu * dt;
}

// a limit slot's dof value: the branch dof or trunk dof it constrains
__device__ __forceinline__ float limit_val(const Lane& L, int kind, int d, const float (&xB)[NB], const float (&xT)[NT]) {
  float v = 0.f;
  if (kind == 1) {
#pragma unroll
    for (int i = 0; i < NB; i++)
      if (i == d) v = xB[i];
  } else if (kind == 2) {
#pragma unroll
    for (int t = 0; t < NT; t++)
      if (t == d) v = xT[t];
  }
  return v;
}

// a limit slot's joint position: the branch dof's (local index d) or the trunk joint's (trunk
// qpos index qi)
__device__ __forceinline__ float limit_q(const Lane& L, int kind, int d, int qi) {
  float v = 0.f;
  if (kind == 1) {
#pragma unroll
    for (int i = 0; i < NB; i++)
      if (i == d) v = L.qB[i];
  } else if (kind == 2) {
#pragma unroll
    for (int i = 0; i < NQT; i++)
      if (i == qi) v = L.qT[i];
  }
  return v;
}

// J_r . x for every row of the lane
__device__ __forceinline__ void rows_dot(const Lane& L, const float (&xB)[NB], const float (&xT)[NT], float (&out)[NRL]) {
#pragma unroll
  for (int c = 0; c < NCL; c++) {
    float dn, d1, d2;
    jdot3(L, c, xB, xT, dn, d1, d2);
#pragma unroll
    for (int e = 0; e < 4; e++) out[4 * c + e] = edge(L.mu[c], e, dn, d1, d2);
  }
#pragma unroll
  for (int l = 0; l < LS; l++)
    out[4 * NCL + l] = L.lsgn[l] * limit_val(L, LV(kLLk, [l]), LV(kLLd, [l]), xB, xT);
}

// the lane's part of f(x) = 1/2 (x - a0)^T M (x - a0) + sum_r 1/2 D_r min(0, J_r x - aref_r)^2
// (its branch terms of the quadratic and its rows), and the trunk term qT = 1/2 tT^T MT tT
__device__ __forceinline__ float cost_part(const Lane& L, const float (&xB)[NB], const float (&xT)[NT], float& qT) {
  float tB[NB], tT[NT];
#pragma unroll
  for (int i = 0; i < NB; i++) tB[i] = xB[i] - L.a0B[i];
#pragma unroll
  for (int t = 0; t < NT; t++) tT[t] = xT[t] - L.a0T[t];
  float f = 0.f;
#pragma unroll
  for (int i = 0; i < NB; i++) {
    float mi = 0.f;   // (M_BB tB + 2 M_BT tT)_i
#pragma unroll
    for (int k = 0; k < NB; k++) mi = fmaf(k <= i ? L.MB[i][k] : L.MB[k][i], tB[k], mi);
#pragma unroll
    for (int t = 0; t < NT; t++) mi = fmaf(2.f * L.MBT[i][t], tT[t], mi);
    f = fmaf(0.5f * tB[i], mi, f);
  }
  qT = 0.f;
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float mt = 0.f;
#pragma unroll
    for (int s = 0; s < NT; s++) mt = fmaf(s <= t ? L.MT[t][s] : L.MT[s][t], tT[s], mt);
    qT = fmaf(0.5f * tT[t], mt, qT);
  }
  float jx[NRL];
  rows_dot(L, xB, xT, jx);
#pragma unroll
  for (int r = 0; r < NRL; r++) {
    const float j = jx[r] - L.aref[r];
    if (j < 0.f) f = fmaf(0.5f * L.D[r] * j, j, f);
  }
  return f;
}

// residuals jar = J a - aref and the active set (existing rows with jar < 0)
__device__ __forceinline__ unsigned residuals(const Lane& L, const float (&aB)[NB], const float (&aT)[NT],
                                             float (&jar)[NRL]) {
  rows_dot(L, aB, aT, jar);
  unsigned act = 0u;
#pragma unroll
  for (int r = 0; r < NRL; r++) {
    jar[r] -= L.aref[r];
    if (jar[r] < 0.f && L.D[r] > 0.f) act |= 1u << r;
  }
  return act;
}

// Newton direction p = -H^-1 g at a with active set act.  `zero`: g is exactly zero.
__device__ __forceinline__ bool newton_direction(const Lane& L, const float (&aB)[NB], const float (&aT)[NT],
                                                 const float (&jar)[NRL], unsigned act, float (&pB)[NB],
                                                 float (&pT)[NT], bool& zero) {
  float tB[NB], tT[NT];
#pragma unroll
  for (int i = 0; i < NB; i++) tB[i] = aB[i] - L.a0B[i];
#pragma unroll
  for (int t = 0; t < NT; t++) tT[t] = aT[t] - L.a0T[t];
  // g_B, the lane's part of g_T, H blocks (H_TT's lane part in HTl)
  float gB[NB], gTl[NT], HB[NB][NB], HBT[NB][NT], HTl[NTRI];
#pragma unroll
  for (int i = 0; i < NB; i++) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < NB; k++) v = fmaf(k <= i ? L.MB[i][k] : L.MB[k][i], tB[k], v);
#pragma unroll
    for (int t = 0; t < NT; t++) v = fmaf(L.MBT[i][t], tT[t], v);
    gB[i] = v;
#pragma unroll
    for (int k = 0; k <= i; k++) HB[i][k] = L.MB[i][k];
#pragma unroll
    for (int t = 0; t < NT; t++) HBT[i][t] = L.MBT[i][t];
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < NB; i++) v = fmaf(L.MBT[i][t], tB[i], v);
    gTl[t] = v;
  }
#pragma unroll
  for (int i = 0; i < NTRI; i++) HTl[i] = 0.f;
#pragma unroll
  for (int c = 0; c < NCL; c++) {
    const float mu = L.mu[c];
    float Sn = 0.f, c1 = 0.f, c2 = 0.f, s1 = 0.f, s2 = 0.f, gn = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int r = 4 * c + e;
      const float D = ((act >> r) & 1u) ? L.D[r] : 0.f, DJ = D * jar[r];
      const float sg = (e & 1) ? -mu : mu;
      Sn += D;
      gn += DJ;
      if (e < 2) { c1 += sg * D; s1 += mu * mu * D; g1 += sg * DJ; }
      else { c2 += sg * D; s2 += mu * mu * D; g2 += sg * DJ; }
    }
    if (Sn == 0.f) continue;
    // gradient and the rank-3 update J^T B J in the (n, t1, t2) basis, B = [Sn c1 c2; c1 s1 0; c2 0 s2]
    float hB[NB][3], hT[NT][3];
#pragma unroll
    for (int i = 0; i < NB; i++) {
      const float na = L.JB[c][0][i], ta = L.JB[c][1][i], ua = L.JB[c][2][i];
      gB[i] += gn * na + g1 * ta + g2 * ua;
      hB[i][0] = Sn * na + c1 * ta + c2 * ua;
      hB[i][1] = c1 * na + s1 * ta;
      hB[i][2] = c2 * na + s2 * ua;
    }
#pragma unroll
    for (int t = 0; t < NT; t++) {
      const float na = L.JT[c][0][t], ta = L.JT[c][1][t], ua = L.JT[c][2][t];
      gTl[t] += gn * na + g1 * ta + g2 * ua;
      hT[t][0] = Sn * na + c1 * ta + c2 * ua;
      hT[t][1] = c1 * na + s1 * ta;
      hT[t][2] = c2 * na + s2 * ua;
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
#pragma unroll
      for (int k = 0; k <= i; k++)
        HB[i][k] += hB[i][0] * L.JB[c][0][k] + hB[i][1] * L.JB[c][1][k] + hB[i][2] * L.JB[c][2][k];
#pragma unroll
      for (int t = 0; t < NT; t++)
        HBT[i][t] += hB[i][0] * L.JT[c][0][t] + hB[i][1] * L.JT[c][1][t] + hB[i][2] * L.JT[c][2][t];
    }
#pragma unroll
    for (int t = 0; t < NT; t++)
#pragma unroll
      for (int s = 0; s <= t; s++)
        HTl[tri(t, s)] += hT[t][0] * L.JT[c][0][s] + hT[t][1] * L.JT[c][1][s] + hT[t][2] * L.JT[c][2][s];
  }
#pragma unroll
  for (int l = 0; l < LS; l++) {
    const int r = 4 * NCL + l, kind = LV(kLLk, [l]), d = LV(kLLd, [l]);
    const float D = ((act >> r) & 1u) ? L.D[r] : 0.f, gv = L.lsgn[l] * D * jar[r];
    if (kind == 1) {
#pragma unroll
      for (int i = 0; i < NB; i++)
        if (i == d) { gB[i] += gv; HB[i][i] += D; }
    } else if (kind == 2) {
#pragma unroll
      for (int t = 0; t < NT; t++)
        if (t == d) { gTl[t] += gv; HTl[tri(t, t)] += D; }
    }
  }
  // g_T = MT tT + the lanes' parts, with the Schur reduction of the factorisation: one butterfly
  float gTr[NT];
#pragma unroll
  for (int t = 0; t < NT; t++) gTr[t] = gTl[t];
  gsum_arr(gTr, L.gm);
  float gT[NT];
  int nz = 0;
#pragma unroll
  for (int i = 0; i < NB; i++) nz |= gB[i] != 0.f;
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float v = gTr[t];
#pragma unroll
    for (int s = 0; s < NT; s++) v = fmaf(s <= t ? L.MT[t][s] : L.MT[s][t], tT[s], v);
    gT[t] = v;
    nz |= v != 0.f;
  }
  zero = gor(nz, L.gm) == 0;
  if (zero) return false;
  Factor F;
  float zT[NT];
#pragma unroll
  for (int t = 0; t < NT; t++) zT[t] = 0.f;
  const bool ok = block_solve(F, HB, HBT, L.MT, HTl, gB, gT, zT, pB, pT, L.gm);
#pragma unroll
  for (int i = 0; i < NB; i++) pB[i] = -pB[i];
#pragma unroll
  for (int t = 0; t < NT; t++) pT[t] = -pT[t];
  return ok;
}

// Exact minimiser of phi(alpha) = f(a + alpha p) (convex, piecewise quadratic): the breakpoints
// alpha_r = -jar_r / Jp_r of every row of the environment walked in increasing order, the rows
// crossing at a breakpoint toggled together, until the root of phi' on the current piece comes
// before the next breakpoint.
__device__ __forceinline__ float line_search(const Lane& L, const float (&aB)[NB], const float (&aT)[NT],
                                             const float (&jar)[NRL], const float (&pB)[NB], const float (&pT)[NT]) {
  float tB[NB], tT[NT];
#pragma unroll
  for (int i = 0; i < NB; i++) tB[i] = aB[i] - L.a0B[i];
#pragma unroll
  for (int t = 0; t < NT; t++) tT[t] = aT[t] - L.a0T[t];
  // p^T M p and t^T M p: the lane's branch terms, then the trunk terms
  float qt = 0.f, lt = 0.f;
#pragma unroll
  for (int i = 0; i < NB; i++) {
    float mp = 0.f, mpt = 0.f;   // (M_BB pB + M_BT pT)_i, (M_BT tT)_i
#pragma unroll
    for (int k = 0; k < NB; k++) mp = fmaf(k <= i ? L.MB[i][k] : L.MB[k][i], pB[k], mp);
#pragma unroll
    for (int t = 0; t < NT; t++) {
      mp = fmaf(L.MBT[i][t], pT[t], mp);
      mpt = fmaf(L.MBT[i][t], tT[t], mpt);
    }
    qt = fmaf(pB[i], mp, qt);
    lt = fmaf(tB[i], mp, lt);
    lt = fmaf(pB[i], mpt, lt);
  }
  float qtT = 0.f, ltT = 0.f;
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float mp = 0.f, mpb = 0.f;   // (M_TT pT)_t, (M_TB pB)_t
#pragma unroll
    for (int s = 0; s < NT; s++) mp = fmaf(s <= t ? L.MT[t][s] : L.MT[s][t], pT[s], mp);
#pragma unroll
    for (int i = 0; i < NB; i++) mpb = fmaf(L.MBT[i][t], pB[i], mpb);
    qtT = fmaf(pT[t], mp, qtT);
    qt = fmaf(pT[t], mpb, qt);
    ltT = fmaf(tT[t], mp, ltT);
  }
  float jp[NRL], bp[NRL];
  rows_dot(L, pB, pT, jp);
  unsigned on = 0u;
#pragma unroll
  for (int r = 0; r < NRL; r++) {
    const float D = L.D[r], j = jp[r], jr = jar[r];
    if (D > 0.f && (jr < 0.f || (jr == 0.f && j < 0.f))) {
      on |= 1u << r;
      qt = fmaf(D * j, j, qt);
      lt = fmaf(D * j, jr, lt);
    }
    bp[r] = D > 0.f && j != 0.f ? __fdividef(-jr, j) : -inf_f();
  }
  qt = gsum(qt, L.gm) + qtT;
  lt = gsum(lt, L.gm) + ltT;
  float alpha = 0.f;
  for (int step = 0; step <= GP * NRL; step++) {
    const float root = qt > 0.f ? __fdividef(-lt, qt) : alpha;
    float next = inf_f();
#pragma unroll
    for (int r = 0; r < NRL; r++)
      if (bp[r] > alpha && bp[r] < next) next = bp[r];
    next = gmin(next, L.gm);
    if (root <= next) return root;
    alpha = next;
    float dq = 0.f, dl = 0.f;
#pragma unroll
    for (int r = 0; r < NRL; r++) {
      if (bp[r] != next) continue;
      const float sg = ((on >> r) & 1u) ? -1.f : 1.f, D = L.D[r];
      on ^= 1u << r;
      dq = fmaf(sg * D * jp[r], jp[r], dq);
      dl = fmaf(sg * D * jp[r], jar[r], dl);
    }
    qt += gsum(dq, L.gm);
    lt += gsum(dl, L.gm);
  }
  return qt > 0.f ? __fdividef(-lt, qt) : alpha;
}

// one substep of the lane's environment; OUT: also write its contact forces and count (the last
// substep of a pg_step_ex with outputs)
// actuator a's force: act_force, with the environment's parameters in the DR variant (the
// control clipped first, then a PD target's calibration offset and its gain scales)
template <bool DR>
__device__ __forceinline__ float act_force_env(const Lane& L, int a, int atype, float gear, float kp, float kd, int clim,
                                               float lo, float hi, int flim, float flo, float fhi, float u, float q,
                                               float qd) {
  if (!DR) return act_force(atype, gear, kp, kd, clim, lo, hi, flim, flo, fhi, u, q, qd);
  if (clim) u = fminf(fmaxf(u, lo), hi);
  if (atype != PG_ACT_MOTOR) {
    u += L.dr_row(DR_CAL + a);
    kp *= 1.f + L.dr_row(DR_KP + a);
    kd *= 1.f + L.dr_row(DR_KD + a);
  }
  return act_force(atype, gear, kp, kd, 0, lo, hi, flim, flo, fhi, u, q, qd);
}

template <bool DR = false>
__device__ __forceinline__ void substep(Lane& L, uint32_t& status, uint32_t cnt[3], bool out, const BranchArgs& A) {
  Kin K;
  kinematics<DR>(L, K);
  float cB[NB], cT[NT];
  rnea(L, K, cB, cT);
  crba<DR>(L, K);
  // smooth forces tau = passive - bias + actuation, then a0 = M^-1 tau
  float tauB[NB], tauT[NT];
#pragma unroll
  for (int i = 0; i < NB; i++) {
    float tau = -LV(kLDdamp, [i]) * L.vB[i] - cB[i];
    const int a = LV(kLDact, [i]);
    if (a >= 0) {
      const float u = L.ctrl_row(a);
      tau += act_force_env<DR>(L, a, LV(kLDatype, [i]), LV(kLDgear, [i]), LV(kLDkp, [i]), LV(kLDkd, [i]),
                               LV(kLDclim, [i]), LV(kLDcr, [i][0]), LV(kLDcr, [i][1]), LV(kLDflim, [i]),
                               LV(kLDfr, [i][0]), LV(kLDfr, [i][1]), u, L.qB[i], L.vB[i]);
    }
    tauB[i] = tau;
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    float tau = -kTDdamp[t] * L.vT[t] - cT[t];
    const int a = kTDact[t];
    if (a >= 0)
      tau += act_force_env<DR>(L, a, kTDatype[t], kTDgear[t], kTDkp[t], kTDkd[t], kTDclim[t], kTDcr[t][0],
                               kTDcr[t][1], kTDflim[t], kTDfr[t][0], kTDfr[t][1], L.ctrl_row(a), L.qT[kTDqa[t]],
                               L.vT[t]);
    tauT[t] = tau;
  }
  Factor FM;
  {
    float zl[NTRI], zT[NT];
#pragma unroll
    for (int i = 0; i < NTRI; i++) zl[i] = 0.f;
#pragma unroll
    for (int t = 0; t < NT; t++) zT[t] = 0.f;
    block_solve(FM, L.MB, L.MBT, L.MT, zl, tauB, tauT, zT, L.a0B, L.a0T, L.gm);
  }
  // contacts: collision, Jacobian rows, row parameters (one impedance per contact, exact Ahat
  // of every pyramid edge from the (n, t1, t2) Gram matrix of J M^-1 J^T)
  float dist[NCL];
#pragma unroll
  for (int s = 0; s < PS; s++) {
    Con k[4];
    const int np = collide_slot(L, K, s, k);
#pragma unroll
    for (int i = 0; i < pnp(s); i++) {
      const int c = pc0(s) + i;
      const bool valid = i < np && k[i].dist < MARGIN;
      dist[c] = valid ? k[i].dist : 1.f;
      L.mu[c] = valid && LV(kPcond, [s]) == 3 ? LV(kPmu, [s]) * (DR ? L.dr_row(0) : 1.f) : 0.f;
      contact_rows(L, K, s, c, k[i].pos, k[i].n);   // (a contact that is not active gets D = 0)
    }
  }
#pragma unroll
  for (int c = 0; c < NCL; c++) {
    const bool valid = dist[c] < MARGIN;
    const bool pyr = LV(kPcond, [pslot(c)]) == 3;
    float A[3][3];
    gram(FM, L.JB[c], L.JT[c], A);
    float dn, d1, d2;
    jdot3(L, c, L.vB, L.vT, dn, d1, d2);
    const float mu = L.mu[c], d = valid ? imp(dist[c]) : 0.f;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int r = 4 * c + e;
      const bool ex = valid && (pyr || e == 0);
      float Ah = A[0][0];
      if (pyr) {
        const int kk = e < 2 ? 1 : 2;
        const float sg = (e & 1) ? -1.f : 1.f;
        Ah = A[0][0] + 2.f * sg * mu * A[0][kk] + mu * mu * A[kk][kk];
      }
      const float v = pyr ? edge(mu, e, dn, d1, d2) : (e == 0 ? dn : 0.f);
      L.aref[r] = ex ? -BREF * v - KREF * d * dist[c] : 0.f;
      L.D[r] = ex ? __fdividef(d, (1.f - d) * Ah) : 0.f;
    }
  }
#pragma unroll
  for (int l = 0; l < LS; l++) {
    const int r = 4 * NCL + l, kind = LV(kLLk, [l]), dd = LV(kLLd, [l]);
    const float q = limit_q(L, kind, dd, LV(kLLq, [l]));
    const float lo = LV(kLLlo, [l]), hi = LV(kLLhi, [l]);
    float sgn = 0.f;
    if (kind != 0) {
      if (q - lo < MARGIN) sgn = 1.f;
      else if (hi - q < MARGIN) sgn = -1.f;
    }
    L.lsgn[l] = sgn;
    float uB[1][NB], uT[1][NT];
#pragma unroll
    for (int i = 0; i < NB; i++) uB[0][i] = (kind == 1 && i == dd) ? 1.f : 0.f;
#pragma unroll
    for (int t = 0; t < NT; t++) uT[0][t] = (kind == 2 && t == dd) ? 1.f : 0.f;
    float A[1][1];
    gram(FM, uB, uT, A);
    const float pos = sgn < 0.f ? hi - q : q - lo;
    const float vel = sgn * limit_val(L, kind, dd, L.vB, L.vT);
    const float d = sgn != 0.f ? imp(pos) : 0.f;
    L.aref[r] = sgn != 0.f ? -BREF * vel - KREF * d * pos : 0.f;
    L.D[r] = sgn != 0.f ? __fdividef(d, (1.f - d) * A[0][0]) : 0.f;
  }
  int nrow = 0;
#pragma unroll
  for (int r = 0; r < NRL; r++) nrow += L.D[r] > 0.f ? 1 : 0;
  nrow = gsumi(nrow, L.gm);
  float aB[NB], aT[NT];
  float jar[NRL];   // J a - aref at the solution (when rows exist)
  int iters = 0;
  bool conv = true;
#pragma unroll
  for (int i = 0; i < NB; i++) aB[i] = L.a0B[i];
#pragma unroll
  for (int t = 0; t < NT; t++) aT[t] = L.a0T[t];
  if (nrow > 0) {
    // warm start: qacc_warm when f(warm) < f(a0)
    float qw, q0;
    const float fw_l = cost_part(L, L.wB, L.wT, qw), f0_l = cost_part(L, L.a0B, L.a0T, q0);
    const float fw = gsum(fw_l, L.gm) + qw, f0 = gsum(f0_l, L.gm) + q0;
    if (fw < f0) {
#pragma unroll
      for (int i = 0; i < NB; i++) aB[i] = L.wB[i];
#pragma unroll
      for (int t = 0; t < NT; t++) aT[t] = L.wT[t];
    }
    unsigned act = residuals(L, aB, aT, jar);
    conv = false;
    while (iters < CAP) {
      float pB[NB], pT[NT];
      bool zero = false;
      const bool ok = newton_direction(L, aB, aT, jar, act, pB, pT, zero);
      iters++;
      if (zero) { conv = true; break; }
      if (!ok) break;
      const float alpha = line_search(L, aB, aT, jar, pB, pT);
#pragma unroll
      for (int i = 0; i < NB; i++) aB[i] = fmaf(alpha, pB[i], aB[i]);
#pragma unroll
      for (int t = 0; t < NT; t++) aT[t] = fmaf(alpha, pT[t], aT[t]);
      const unsigned act2 = residuals(L, aB, aT, jar);
      const int same = gand(act2 == act ? 1 : 0, L.gm);
      act = act2;
      if (same) { conv = true; break; }
    }
    if (!conv) status |= PG_STATUS_NOT_CONVERGED;
  }
  cnt[0] += (uint32_t)iters;
  cnt[1] += (uint32_t)nrow;
  cnt[2] += (uint32_t)(nrow * iters);
  if (out) {   // the contact forces in each contact's frame, per candidate slot of the lane's pairs
    int ncon = 0;
#pragma unroll
    for (int s = 0; s < PS; s++) {
      const int slot0 = LV(kPslot, [s]), nsl = LV(kPnslot, [s]);
#pragma unroll
      for (int i = 0; i < pnp(s); i++) {
        const int c = pc0(s) + i;
        float fe[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int r = 4 * c + e;
          fe[e] = nrow > 0 && L.D[r] > 0.f && jar[r] < 0.f ? -L.D[r] * jar[r] : 0.f;
        }
        ncon += dist[c] < MARGIN ? 1 : 0;
        if (A.out_force && i < nsl) {
          float* o = A.out_force + (int64_t)(slot0 + i) * 3 * L.ld + L.env;
          o[0] = fe[0] + fe[1] + fe[2] + fe[3];
          o[L.ld] = L.mu[c] * (fe[0] - fe[1]);
          o[2 * L.ld] = L.mu[c] * (fe[2] - fe[3]);
        }
      }
    }
    ncon = gsumi(ncon, L.gm);
    if (L.br == 0) {
      if (A.out_ncon) A.out_ncon[L.env] = ncon;
      if (A.out_force)   // the rows of a batch's larger models
        for (int sl = NSLOT; sl < A.out_nslot; sl++)
          for (int q = 0; q < 3; q++) A.out_force[((int64_t)sl * 3 + q) * L.ld + L.env] = 0.f;
    }
  }
  // semi-implicit Euler
  bool bad = false;
#pragma unroll
  for (int i = 0; i < NB; i++) {
    L.vB[i] = fmaf(HSTEP, aB[i], L.vB[i]);
    L.wB[i] = aB[i];
    L.qB[i] = fmaf(HSTEP, L.vB[i], L.qB[i]);
    bad = bad || !isfinite(aB[i]) || !isfinite(L.vB[i]) || !isfinite(L.qB[i]);
  }
#pragma unroll
  for (int t = 0; t < NT; t++) {
    L.vT[t] = fmaf(HSTEP, aT[t], L.vT[t]);
    L.wT[t] = aT[t];
    bad = bad || !isfinite(aT[t]) || !isfinite(L.vT[t]);
  }
#pragma unroll
  for (int k = 0; k < BT; k++)
#pragma unroll
    for (int j = 0; j < NJT; j++) {
      const int type = kTJtype[k][j];
      if (type < 0) continue;
      const int qa = kTJq[k][j], da = kTJd[k][j];
      if (type == PG_JNT_FREE) {
#pragma unroll
        for (int i = 0; i < 3; i++) L.qT[qa + i] = fmaf(HSTEP, L.vT[da + i], L.qT[qa + i]);
        const float3 w = make_float3(L.vT[da + 3], L.vT[da + 4], L.vT[da + 5]);
        const float w2 = dot3(w, w);
        Quat q{L.qT[qa + 3], L.qT[qa + 4], L.qT[qa + 5], L.qT[qa + 6]};
        if (w2 > 0.f) {   // rotation by h |w| about w: |h w / 2| stays far below pi
          const float inv = rsqrtf(w2);
          float sn, cs;
          sincosf(0.5f * HSTEP * (w2 * inv), &sn, &cs);
          const float s = sn * inv;
          q = qmul(q, Quat{cs, w.x * s, w.y * s, w.z * s});
        }
        q = qnormalize(q);
        L.qT[qa + 3] = q.w; L.qT[qa + 4] = q.x; L.qT[qa + 5] = q.y; L.qT[qa + 6] = q.z;
#pragma unroll
        for (int i = 0; i < 7; i++) bad = bad || !isfinite(L.qT[qa + i]);
      } else {
        L.qT[qa] = fmaf(HSTEP, L.vT[da], L.qT[qa]);
        bad = bad || !isfinite(L.qT[qa]);
      }
    }
  if (gor(bad ? 1 : 0, L.gm)) status |= PG_STATUS_NAN;
}

// The kernel: GP lanes per environment, blockDim.x / GP environments per block.  SYNC: the
// block's warps start every substep together (a barrier per substep), so that they run its long
// straight-line phases close together and share their instruction fetches; a group past the
// last environment then steps the last environment alongside (it writes nothing).
// SYNC: the block's warps meet at a barrier before every substep.  TAPE: also record the adjoint's
// substep tape (A.tape); a separate instantiation, so the plain step's code is untouched by it.
// DR: per-environment parameters (A.dr, pg_step_dr's layout), another instantiation.
template <bool SYNC, bool TAPE = false, bool DR = false>
__device__ __forceinline__ void branch_step(const BranchArgs& A) {
  const int tid = threadIdx.x;
  Lane L;
  L.br = tid & (GP - 1);
  L.gm = group_mask();
  const int64_t local = (int64_t)blockIdx.x * (blockDim.x / GP) + tid / GP;
  const bool active = local < A.n;
  if (!SYNC && !active) return;   // the whole group leaves together
  L.env = A.env0 + (active ? local : A.n - 1);
  L.ld = A.ld;
  L.ctrl = A.ctrl;
  L.hf = A.hfield;
  L.dr = DR ? A.dr : nullptr;
  const int64_t ld = A.ld, env = L.env;
#pragma unroll
  for (int i = 0; i < NQT; i++) L.qT[i] = A.qpos[kTQg[i] * ld + env];
  bool warm_bad = false;
#pragma unroll
  for (int t = 0; t < NT; t++) {
    L.vT[t] = A.qvel[kTDg[t] * ld + env];
    L.wT[t] = A.warm[kTDg[t] * ld + env];
    warm_bad = warm_bad || !isfinite(L.wT[t]);
  }
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int gd = LV(kLDg, [i]), gq = LV(kLDq, [i]);
    L.qB[i] = gd >= 0 ? A.qpos[gq * ld + env] : 0.f;
    L.vB[i] = gd >= 0 ? A.qvel[gd * ld + env] : 0.f;
    L.wB[i] = gd >= 0 ? A.warm[gd * ld + env] : 0.f;
    warm_bad = warm_bad || !isfinite(L.wB[i]);
  }
  uint32_t status = 0;
  if (gor(warm_bad ? 1 : 0, L.gm)) {   // a non-finite warm start is replaced by zeros (flagged)
    status |= PG_STATUS_WARM_RESET;
#pragma unroll
    for (int t = 0; t < NT; t++) L.wT[t] = 0.f;
#pragma unroll
    for (int i = 0; i < NB; i++) L.wB[i] = 0.f;
  }
  uint32_t cnt[3] = {0u, 0u, 0u};
  const int nsub = A.n_substeps > 0 ? A.n_substeps : NSUB;
  const bool want = A.out_force || A.out_ncon;
  for (int s = 0; s < nsub; s++) {
    if (SYNC) __syncthreads();
    float* tp = TAPE && active ? A.tape + (int64_t)s * A.tape_rows * ld + env : nullptr;
    if (TAPE && tp) {   // the state the substep starts from (each lane its branch's dofs, lane 0 the trunk's)
      if (L.br == 0) {
#pragma unroll
        for (int i = 0; i < NQT; i++) tp[kTQg[i] * ld] = L.qT[i];
#pragma unroll
        for (int t = 0; t < NT; t++) {
          tp[(A.tape_nq + kTDg[t]) * ld] = L.vT[t];
          tp[(A.tape_nq + A.tape_nv + kTDg[t]) * ld] = L.wT[t];
        }
      }
#pragma unroll
      for (int i = 0; i < NB; i++) {
        const int gd = LV(kLDg, [i]), gq = LV(kLDq, [i]);
        if (gd >= 0) {
          tp[gq * ld] = L.qB[i];
          tp[(A.tape_nq + gd) * ld] = L.vB[i];
          tp[(A.tape_nq + A.tape_nv + gd) * ld] = L.wB[i];
        }
      }
    }
    substep<DR>(L, status, cnt, want && s == nsub - 1 && active, A);
    if (TAPE && tp) {   // the solver's acceleration (the next warm start)
      if (L.br == 0)
#pragma unroll
        for (int t = 0; t < NT; t++) tp[(A.tape_nq + 2 * A.tape_nv + kTDg[t]) * ld] = L.wT[t];
#pragma unroll
      for (int i = 0; i < NB; i++) {
        const int gd = LV(kLDg, [i]);
        if (gd >= 0) tp[(A.tape_nq + 2 * A.tape_nv + gd) * ld] = L.wB[i];
      }
    }
  }
  if (!active) return;
  if (L.br == 0) {
#pragma unroll
    for (int i = 0; i < NQT; i++) A.qpos[kTQg[i] * ld + env] = L.qT[i];
#pragma unroll
    for (int t = 0; t < NT; t++) {
      A.qvel[kTDg[t] * ld + env] = L.vT[t];
      A.warm[kTDg[t] * ld + env] = L.wT[t];
    }
    if (status) A.status[env] |= status;
    if (A.stats)
#pragma unroll
      for (int k = 0; k < 3; k++) A.stats[k * ld + env] += cnt[k];
  }
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int gd = LV(kLDg, [i]), gq = LV(kLDq, [i]);
    if (gd >= 0) {
      A.qpos[gq * ld + env] = L.qB[i];
      A.qvel[gd * ld + env] = L.vB[i];
      A.warm[gd * ld + env] = L.wB[i];
    }
  }
}

}  // namespace pgb
