// Hand-written adjoint (reverse-mode sweep) of the physics step, one thread per environment: its
// device code and kernel body, shared by the library's compiled kernel (adjoint.cu) and the
// model-specialised one compiled at run time (specialize.cpp; PG_SPEC takes the model from the
// constant SpecModel<SPEC_M>).  The including unit sets PG_WITH_ELLIPTIC 0.
//
// A control step's substeps are replayed from a tape that the forward kernel wrote (the state
// at each substep's start and the solver's acceleration), last substep first.  Each substep
// recomputes the forward quantities from its start state (kinematics, RNEA, CRBA, LDL^T,
// collision, constraint rows) with the forward device code, takes the solver's acceleration
// from the tape, and then sweeps back:
//
//  * semi-implicit Euler (free-joint quaternion exponential and normalisation included);
//  * the contact solve, differentiated implicitly at its optimum with the active set A fixed.
//    The optimality condition M a + J_A^T D_A (J_A a - aref_A) = tau gives, with lambda = H^-1 abar
//    and H = M + J_A^T D_A J_A: taubar = lambda, Mbar = -lambda a^T, arefbar_A = D_A J_A lambda,
//    Dbar_i = -(J_i lambda)(J_i a - aref_i), Jbar_i = -D_i ((J_i a - aref_i) lambda + (J_i lambda) a);
//  * the row parameters (aref = -b v - k d(r) r, D = d / ((1 - d) Ahat), Ahat = (J M^-1 J^T)_rr);
//  * actuation and passive forces (controls, kp, damping);
//  * CRBA and RNEA, down to adjoints of the motion subspaces cdof and of the spatial inertias;
//  * plane contacts, down to the adjoint of the contact feature point on its body.
//
// Position dependence is then collected as spatial "virtual work".  Every pose-dependent
// quantity is attached to a frame, and its adjoint becomes a wrench (torque and force about the
// tree's reference point o, world axes) on that frame:
//
//  * a body-fixed point y with adjoint ybar gives ((y - o) x ybar, ybar);
//  * a motion vector (w; v) attached to a frame, with adjoint (wbar; vbar), gives
//    (w x wbar + v x vbar, w x vbar);
//  * a spatial inertia gives the torque and force derived in the "own spatial inertias" step below.
//
// Wrenches accumulate inward along the tree. A dof's position adjoint is its cdof dotted with the
// wrench of everything the dof moves. The reference point o is held fixed throughout. Every
// physical output (M, c, J, Ahat) is independent of the choice of o, so this gives the exact
// derivative.
//
// Scope (checked by the model compiler, `adj_ok`):
//  * any joints;
//  * pyramidal or condim-1 contacts between a world-fixed plane and spheres, capsules or boxes;
//  * joint limits and joint friction loss;
//  * motor and PD actuators.
//
// The gradient treats the solver's final iterate as the optimum. It is exact when the solver has
// converged, which the converged-solver tests check.
#pragma once
#include "step_device.cuh"

namespace pg {
namespace {


#define B(name, i) (c.w[(c.h.b_##name + (i)) * c.S])

__device__ __forceinline__ float3 B3(const Ctx& c, int off) { return W3(c, off); }
__device__ __forceinline__ void add3(const Ctx& c, int off, float3 v) {
  c.w[off * c.S] += v.x; c.w[(off + 1) * c.S] += v.y; c.w[(off + 2) * c.S] += v.z;
}
__device__ __forceinline__ Quat qconj(Quat q) { return Quat{q.w, -q.x, -q.y, -q.z}; }

// dL/dI of L = s x^T I y for the spatial inertia I (Ixx Iyy Izz Ixy Ixz Iyz, h, m) with
// I (w; v) = (Irot w + h x v; m v - h x w), added into the 10 adjoint entries at `gi`
__device__ __forceinline__ void inertia_bilinear_grad(const Ctx& c, int gi, float3 xw, float3 xv, float3 yw, float3 yv,
                                                      float s) {
  float* g = c.w + gi * c.S;
  const int S = c.S;
  g[0] += s * xw.x * yw.x;
  g[S] += s * xw.y * yw.y;
  g[2 * S] += s * xw.z * yw.z;
  g[3 * S] += s * (xw.x * yw.y + xw.y * yw.x);
  g[4 * S] += s * (xw.x * yw.z + xw.z * yw.x);
  g[5 * S] += s * (xw.y * yw.z + xw.z * yw.y);
  const float3 hb = cross3(yv, xw) - cross3(yw, xv);
  g[6 * S] += s * hb.x;
  g[7 * S] += s * hb.y;
  g[8 * S] += s * hb.z;
  g[9 * S] += s * dot3(xv, yv);
}

// wrench of the adjoint (gw; gv) of a motion vector (cw; cv) attached to a frame
__device__ __forceinline__ void motion_wrench(float3 cw, float3 cv, float3 gw, float3 gv, float3& t, float3& f) {
  t = t + cross3(cw, gw) + cross3(cv, gv);
  f = f + cross3(cw, gv);
}

__device__ __forceinline__ float3 cdof_w(const Ctx& c, int d) { return W3(c, c.h.w_cdof + 6 * d); }
__device__ __forceinline__ float3 cdof_v(const Ctx& c, int d) { return W3(c, c.h.w_cdof + 6 * d + 3); }

// d impedance / d pos (solimp = d0, dwidth, width, mid, power)
__device__ __forceinline__ float impedance_slope(const ModelHdr& h, float pos) {
  const float d0 = h.solimp[0], d1 = h.solimp[1], width = h.solimp[2], mid = h.solimp[3], pw = h.solimp[4];
  const float x = fminf(fabsf(pos) / width, 1.f);
  if (x >= 1.f) return 0.f;
  float dy;
  if (x <= mid) dy = pw * powf(x, pw - 1.f) / powf(mid, pw - 1.f);
  else dy = pw * powf(1.f - x, pw - 1.f) / powf(1.f - mid, pw - 1.f);
  const float sg = pos > 0.f ? 1.f : (pos < 0.f ? -1.f : 0.f);
  return (d1 - d0) * dy * sg / width;
}

// Hessian H = M + J_A^T D_A J_A of the active set `act` on M's packed pattern (every contact's
// dofs lie on one chain), factorised in place at HL
__device__ void hessian_factor(const Ctx& c, const unsigned act[4], int HL) {
  const ModelHdr& h = c.h;
  const int NC = h.ncol_max, MC = h.max_contacts;
  float* H = c.w + HL * c.S;
  for (int k = 0; k < h.nL; k++) H[k * c.S] = W(M, k);
  for (int k = 0; k < MC; k++) {
    const float mu = W(gmu, k);
    float Sn = 0.f, c1 = 0.f, c2 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int e = 0; e < 4; e++) {
      const int r = 4 * k + e;
      const float D = bit(act, r) ? W(rD, r) : 0.f;
      const float sg = (e & 1) ? -mu : mu;
      Sn += D;
      if (e < 2) { c1 += sg * D; s1 += mu * mu * D; }
      else { c2 += sg * D; s2 += mu * mu * D; }
    }
    if (Sn == 0.f) continue;
    const float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    const float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    for (int a = 0; a < NC; a++) {
      const int da = __float_as_int(gc[a * c.S]);
      const float na = J[a * c.S], ta = J[(NC + a) * c.S], ua = J[(2 * NC + a) * c.S];
      const float hn = Sn * na + c1 * ta + c2 * ua, ht = c1 * na + s1 * ta, hu = c2 * na + s2 * ua;
      const int ra = MI(dof_rowadr, da), depa = MI(dof_depth, da);
      for (int b = a; b < NC; b++) {
        const int db = __float_as_int(gc[b * c.S]);
        H[(ra + depa - MI(dof_depth, db)) * c.S] += hn * J[b * c.S] + ht * J[(NC + b) * c.S] + hu * J[(2 * NC + b) * c.S];
      }
    }
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int r = 4 * MC + li, d = MI(jnt_dofadr, MI(limit_jnt, li));
    if (bit(act, r)) H[MI(dof_rowadr, d) * c.S] += W(rD, r);
  }
  // friction-loss rows inside their band (outside it a row's force is the constant bound)
  for (int k = 0; k < h.nfric; k++) {
    const int r = fric_row0(h) + k, d = MI(fric_dof, k);
    if (bit(act, r)) H[MI(dof_rowadr, d) * c.S] += W(rD, r);
  }
  ldl_factor(c, HL);
}

// packed Mbar -= s (x y^T + y x^T)/2-style symmetric update: for the packed entry (j, i) the
// adjoint of a full-matrix gradient G is G_ji + G_ij (i != j) or G_jj; here G = -s x y^T
__device__ void mbar_outer(const Ctx& c, int X, int Y, float s) {
  const ModelHdr& h = c.h;
  if (s == 0.f) return;
  const float* x = c.w + X * c.S;
  const float* y = c.w + Y * c.S;
  for (int j = 0; j < h.nv; j++) {
    const int r0 = MI(dof_rowadr, j), dj = MI(dof_depth, j);
    const float xj = x[j * c.S], yj = y[j * c.S];
    B(M, r0) -= s * xj * yj;
    for (int t = 1; t <= dj; t++) {
      const int i = MI(Lcol, r0 + t);
      B(M, r0 + t) -= s * (xj * y[i * c.S] + x[i * c.S] * yj);
    }
  }
}

// the five outer products of one contact's Ahat adjoint in one pass over the packed entries:
// Mbar -= Ann wn wn^T + An1 wn w1^T + An2 wn w2^T + A11 w1 w1^T + A22 w2 w2^T (w at offset Wo)
__device__ void mbar_ahat(const Ctx& c, int Wo, float Ann, float An1, float An2, float A11, float A22) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, S = c.S;
  const float* wn = c.w + Wo * S;
  const float* w1 = c.w + (Wo + nv) * S;
  const float* w2 = c.w + (Wo + 2 * nv) * S;
  for (int j = 0; j < nv; j++) {
    const int r0 = MI(dof_rowadr, j), dj = MI(dof_depth, j);
    const float nj = wn[j * S], aj = w1[j * S], bj = w2[j * S];
    // g_j = (G + G^T) row j applied to the ancestors i below
    const float pn = 2.f * Ann * nj + An1 * aj + An2 * bj, p1 = An1 * nj + 2.f * A11 * aj, p2 = An2 * nj + 2.f * A22 * bj;
    B(M, r0) -= Ann * nj * nj + An1 * nj * aj + An2 * nj * bj + A11 * aj * aj + A22 * bj * bj;
    for (int t = 1; t <= dj; t++) {
      const int i = MI(Lcol, r0 + t);
      B(M, r0 + t) -= pn * wn[i * S] + p1 * w1[i * S] + p2 * w2[i * S];
    }
  }
}

// x_s <- A^-1 x_s for three nv-vectors at X, X + nv, X + 2 nv with the packed factor of A, in one
// pass (three independent update chains; indices and factor entries loaded once)
__device__ void ldl_solve3(const Ctx& c, int A, int X) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, S = c.S;
  const float* a = c.w + A * S;
  float* x0 = c.w + X * S;
  float* x1 = c.w + (X + nv) * S;
  float* x2 = c.w + (X + 2 * nv) * S;
  PG_SPEC_UNROLL
  for (int k = nv - 1; k >= 0; k--) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    const float y0 = x0[k * S], y1 = x1[k * S], y2 = x2[k * S];
    for (int t = 1; t <= dk; t++) {
      const int i = MI(Lcol, r0 + t);
      const float l = a[(r0 + t) * S];
      const float z0 = x0[i * S], z1 = x1[i * S], z2 = x2[i * S];
      x0[i * S] = z0 - l * y0;
      x1[i * S] = z1 - l * y1;
      x2[i * S] = z2 - l * y2;
    }
  }
  PG_SPEC_UNROLL
  for (int k = 0; k < nv; k++) {
    const float d = a[MI(dof_rowadr, k) * S];
    x0[k * S] /= d;
    x1[k * S] /= d;
    x2[k * S] /= d;
  }
  PG_SPEC_UNROLL
  for (int k = 0; k < nv; k++) {
    const int r0 = MI(dof_rowadr, k), dk = MI(dof_depth, k);
    float s0 = x0[k * S], s1 = x1[k * S], s2 = x2[k * S];
    for (int t = 1; t <= dk; t++) {
      const int i = MI(Lcol, r0 + t);
      const float l = a[(r0 + t) * S];
      s0 -= l * x0[i * S];
      s1 -= l * x1[i * S];
      s2 -= l * x2[i * S];
    }
    x0[k * S] = s0;
    x1[k * S] = s1;
    x2[k * S] = s2;
  }
}

// ---------------------------------------------------------------------------------------
// reverse of semi-implicit Euler: b_q, b_v hold the adjoint of the post-substep state on entry;
// on exit b_q holds the pre-state position adjoint (this step's share), b_v the adjoint of the
// new velocity, and b_a = h * b_v the adjoint of the acceleration
// ---------------------------------------------------------------------------------------
__device__ void integrate_vjp(const Ctx& c) {
  const ModelHdr& h = c.h;
  const float dt = h.h;
  for (int j = 0; j < h.njnt; j++) {
    const int qa = MI(jnt_qposadr, j), da = MI(jnt_dofadr, j);
    if (MI(jnt_type, j) == PG_JNT_FREE) {
      for (int k = 0; k < 3; k++) B(v, da + k) += dt * B(q, qa + k);
      float3 w;
      w.x = fmaf(dt, W(a, da + 3), W(qvel, da + 3));
      w.y = fmaf(dt, W(a, da + 4), W(qvel, da + 4));
      w.z = fmaf(dt, W(a, da + 5), W(qvel, da + 5));
      const float wn = sqrtf(dot3(w, w));
      const Quat q{W(qpos, qa + 3), W(qpos, qa + 4), W(qpos, qa + 5), W(qpos, qa + 6)};
      float sn = 0.f, cs = 1.f;
      Quat e{1.f, 0.f, 0.f, 0.f};
      if (wn > 0.f) {
        sincosf(0.5f * dt * wn, &sn, &cs);
        const float s = sn / wn;
        e = Quat{cs, w.x * s, w.y * s, w.z * s};
      }
      const Quat r = qmul(q, e);
      const float rn = sqrtf(r.w * r.w + r.x * r.x + r.y * r.y + r.z * r.z);
      const Quat qn{r.w / rn, r.x / rn, r.y / rn, r.z / rn};
      const Quat qb{B(q, qa + 3), B(q, qa + 4), B(q, qa + 5), B(q, qa + 6)};
      const float pr = qn.w * qb.w + qn.x * qb.x + qn.y * qb.y + qn.z * qb.z;
      const Quat rb{(qb.w - qn.w * pr) / rn, (qb.x - qn.x * pr) / rn, (qb.y - qn.y * pr) / rn, (qb.z - qn.z * pr) / rn};
      const Quat qbar = qmul(rb, qconj(e));
      const Quat eb = qmul(qconj(q), rb);
      B(q, qa + 3) = qbar.w; B(q, qa + 4) = qbar.x; B(q, qa + 5) = qbar.y; B(q, qa + 6) = qbar.z;
      const float3 ev = make_float3(eb.x, eb.y, eb.z);
      float3 wb;
      if (wn > 0.f) {
        const float3 u = w * (1.f / wn);
        const float ue = dot3(u, ev);
        wb = u * (-sn * 0.5f * dt * eb.w + cs * 0.5f * dt * ue) + (ev - u * ue) * (sn / wn);
      } else {
        wb = ev * (0.5f * dt);
      }
      add3(c, c.h.b_v + da + 3, wb);
    } else {
      B(v, da) += dt * B(q, qa);
    }
  }
  for (int d = 0; d < h.nv; d++) B(a, d) = dt * B(v, d);
}

// ---------------------------------------------------------------------------------------
// one substep backward.  On entry the workspace holds the substep's recomputed forward state
// (through row_params, a from the tape, residuals and active set `act`) and b_q / b_v the adjoint
// of the post-substep state; on exit b_q / b_v hold the adjoint of the pre-substep state.
// Parameter and control adjoints are added into gpar / gu (global, [k * ld + env]).
// ---------------------------------------------------------------------------------------
__device__ void substep_vjp(const Ctx& c, int nc, const unsigned act[4], float* gpar, float* gu, int64_t ld) {
  const ModelHdr& h = c.h;
  const int nv = h.nv, NC = h.ncol_max, MC = h.max_contacts, nb = h.nbody;
  const int64_t env = c.env;

  // ---- integration, then lambda = H^-1 abar (in b_a) ----
  integrate_vjp(c);
  hessian_factor(c, act, h.w_HL);
  ldl_solve(c, h.w_HL, h.b_a);

  // accumulators of the following phases (each buffer's space is shared outside its phases)
  for (int k = 0; k < h.nL; k++) B(M, k) = 0.f;
  for (int k = 0; k < 6 * nv; k++) B(cdof, k) = 0.f;
  for (int k = 0; k < 10 * nb; k++) B(I, k) = 0.f;
  for (int k = 0; k < 6 * nb; k++) B(wr, k) = 0.f;

  // ---- forces: taubar = lambda ----
  for (int d = 0; d < nv; d++) {
    const float lam = B(a, d);
    B(bias, d) = -lam;
    B(v, d) -= MF(dof_damping, d) * lam;
    gpar[(nb + d) * ld + env] -= W(qvel, d) * lam;
  }
  for (int k = 0; k < h.nu; k++) {
    const int d = MI(act_dof, k);
    const float lam = B(a, d);
    const float u0 = c.ctrl[k * c.ld + env];
    float u = u0;
    bool pass = true;
    if (MI(act_ctrllimited, k)) {
      u = fminf(fmaxf(u0, MF(act_range, 2 * k)), MF(act_range, 2 * k + 1));
      pass = u0 > MF(act_range, 2 * k) && u0 < MF(act_range, 2 * k + 1);
    }
    if (MI(act_forcelimited, k)) {   // a force clipped at its limit is constant: no derivative
      const float f = MI(act_type, k) == PG_ACT_MOTOR
                          ? MF(act_gear, k) * u
                          : MF(act_kp, k) * (u - W(qpos, MI(act_qposadr, k))) - MF(act_kd, k) * W(qvel, d);
      if (f < MF(act_forcerange, 2 * k) || f > MF(act_forcerange, 2 * k + 1)) continue;
    }
    if (MI(act_type, k) == PG_ACT_MOTOR) {
      if (pass) gu[k * ld + env] += MF(act_gear, k) * lam;
    } else {
      const int qa = MI(act_qposadr, k);
      if (pass) gu[k * ld + env] += MF(act_kp, k) * lam;
      B(q, qa) -= MF(act_kp, k) * lam;
      B(v, d) -= MF(act_kd, k) * lam;
      gpar[(nb + nv + k) * ld + env] += (u - W(qpos, qa)) * lam;
    }
  }
  // Mbar = -lambda a^T (packed)
  mbar_outer(c, h.b_a, h.w_a, 1.f);

  // ---- constraint rows ----
  rows_dot(c, h.b_a, h.w_Jp);   // J lambda per row
  for (int k = 0; k < nc; k++) {
    const float mu = W(gmu, k);
    const bool pyr = W(gcond, k) == 3.f;
    const float dist = W(con, kConFloats * k + 1);
    float al[4], be[4], ga[4], Ab[4];
    float distb = 0.f;
    bool any = false;
    for (int e = 0; e < 4; e++) {
      const int r = 4 * k + e;
      al[e] = be[e] = ga[e] = Ab[e] = 0.f;
      if (!bit(act, r)) continue;
      any = true;
      const float D = W(rD, r), jl = W(Jp, r), jar = W(jar, r), d = W(imp, r), A = W(Ahat, r);
      const float arefb = D * jl, Db = -jl * jar;
      al[e] = -D * jar;
      be[e] = -D * jl;
      ga[e] = -h.bref * arefb;
      float db = -h.kref * dist * arefb + Db / ((1.f - d) * (1.f - d) * A);
      Ab[e] = -Db * D / A;
      distb += -h.kref * d * arefb + db * impedance_slope(h, dist);
    }
    if (!any) continue;
    // Ahat of the edges from A_nn, A_n1, A_n2, A_11, A_22
    float Ann, An1 = 0.f, An2 = 0.f, A11 = 0.f, A22 = 0.f;
    float Sa, a1 = 0.f, a2 = 0.f, Sb, b1 = 0.f, b2 = 0.f, Sg, g1 = 0.f, g2 = 0.f;
    if (pyr) {
      Ann = Ab[0] + Ab[1] + Ab[2] + Ab[3];
      An1 = 2.f * mu * (Ab[0] - Ab[1]);
      An2 = 2.f * mu * (Ab[2] - Ab[3]);
      A11 = mu * mu * (Ab[0] + Ab[1]);
      A22 = mu * mu * (Ab[2] + Ab[3]);
      Sa = al[0] + al[1] + al[2] + al[3]; a1 = mu * (al[0] - al[1]); a2 = mu * (al[2] - al[3]);
      Sb = be[0] + be[1] + be[2] + be[3]; b1 = mu * (be[0] - be[1]); b2 = mu * (be[2] - be[3]);
      Sg = ga[0] + ga[1] + ga[2] + ga[3]; g1 = mu * (ga[0] - ga[1]); g2 = mu * (ga[2] - ga[3]);
    } else {
      Ann = Ab[0]; Sa = al[0]; Sb = be[0]; Sg = ga[0];
    }
    const float* J = c.w + (h.w_J + 3 * NC * k) * c.S;
    const float* gc = c.w + (h.w_gcol + NC * k) * c.S;
    const int p = con_pair(c, k);
    const int ncol = MI(pair_ncol, p), ca = MI(pair_coladr, p);
    // w_x = M^-1 J_x^T for x = n, t1, t2
    for (int s = 0; s < 3; s++) {
      const int wo = h.b_w + s * nv;
      for (int i = 0; i < nv; i++) c.w[(wo + i) * c.S] = 0.f;
      for (int a = 0; a < ncol; a++) c.w[(wo + __float_as_int(gc[a * c.S])) * c.S] += J[(s * NC + a) * c.S];
    }
    ldl_solve3(c, h.w_L, h.b_w);
    // Mbar from Ahat = J M^-1 J^T
    mbar_ahat(c, h.b_w, Ann, An1, An2, A11, A22);
    // row velocities v_r = J_r qvel
    // Jacobian adjoint per column -> cdof adjoint and contact-point adjoint
    const int co = h.w_con + kConFloats * k;
    const float3 pos = W3(c, co + 2), n = W3(c, co + 5);
    float3 t1, t2;
    contact_frame(n, t1, t2);
    const int g1i = MI(pair_g1, p), g2i = MI(pair_g2, p);
    const int gb1 = MI(geom_body, g1i), gb2 = MI(geom_body, g2i);
    const float3 o1 = tree_origin(c, gb1), o2 = tree_origin(c, gb2);
    // on a heightfield the contact frame turns with the state (at the terrain's edges and
    // vertices): the adjoints of n, t1 and t2 through the Jacobian rows J_x[a] = x . P_a
    const bool turns = MI(geom_type, g1i) == PG_GEOM_HFIELD;
    float3 posb = make_float3(0.f, 0.f, 0.f);
    float3 nb = make_float3(0.f, 0.f, 0.f), t1b = nb, t2b = nb;
    for (int a = 0; a < ncol; a++) {
      const int d = MI(col_dof, ca + a), sg = MI(col_sign, ca + a);
      const float lam = B(a, d), acc = W(a, d), vel = W(qvel, d);
      const float wn = B(w, d), w1 = B(w, nv + d), w2 = B(w, 2 * nv + d);
      const float Jn = J[a * c.S], Jt = J[(NC + a) * c.S], Ju = J[(2 * NC + a) * c.S];
      // v_r adjoint into qvel: sum_e gamma_e J_e
      B(v, d) += Sg * Jn + g1 * Jt + g2 * Ju;
      const float jn = Sa * lam + Sb * acc + Sg * vel + 2.f * Ann * wn + An1 * w1 + An2 * w2;
      const float j1 = a1 * lam + b1 * acc + g1 * vel + An1 * wn + 2.f * A11 * w1;
      const float j2 = a2 * lam + b2 * acc + g2 * vel + An2 * wn + 2.f * A22 * w2;
      const float3 jb = (n * jn + t1 * j1 + t2 * j2) * (float)sg;
      const float3 cw = cdof_w(c, d);
      const float3 r = pos - (sg > 0 ? o2 : o1);
      add3(c, h.b_cdof + 6 * d + 3, jb);
      add3(c, h.b_cdof + 6 * d, cross3(r, jb));
      posb = posb + cross3(jb, cw);
      if (turns) {
        const float3 P = (cdof_v(c, d) + cross3(cw, r)) * (float)sg;
        nb = nb + P * jn;
        t1b = t1b + P * j1;
        t2b = t2b + P * j2;
      }
    }
    // contact point and depth -> the feature point y on geom2's body (geom1 is a world plane):
    // dist = n.(y - p0) - r_s, pos = y - n (r_s + dist / 2)
    float3 yb = posb - n * (0.5f * dot3(n, posb)) + n * distb;
    float3 bx;
    Quat bq;
    body_frame(c, gb2, bx, bq);
    const float3 x2 = bx + qrot(bq, T3(&MF(geom_pos, 3 * g2i)));
    float R2[9];
    qmat(qnormalize(qmul(bq, Quat{MF(geom_quat, 4 * g2i), MF(geom_quat, 4 * g2i + 1), MF(geom_quat, 4 * g2i + 2),
                                  MF(geom_quat, 4 * g2i + 3)})), R2);
    const float* s2 = &MF(geom_size, 3 * g2i);
    const int feat = (int)W(con, kConFloats * k + 8);
    const int t2y = MI(geom_type, g2i);
    float3 y = x2;
    if (t2y == PG_GEOM_CAPSULE) y = x2 + mat_col(R2, 2) * (feat ? s2[1] : -s2[1]);
    else if (t2y == PG_GEOM_BOX)
      y = x2 + mat_mul(R2, make_float3((feat & 1) ? s2[0] : -s2[0], (feat & 2) ? s2[1] : -s2[1], (feat & 4) ? s2[2] : -s2[2]));
    if (t2y == PG_GEOM_CYLINDER) {
      // rim point y = cap centre + r E, E = c1 e + c2 (a x e) with e = -perp / |perp|,
      // perp = n - (n.a) a: E turns with the axis a, so beyond the rigid motion of a body-fixed
      // point y gains r (dE - dtheta x E); its adjoint is the couple r (a x abar - E x ybar)
      const float3 a = mat_col(R2, 2);
      const float s = dot3(n, a);
      const float3 perp = n - a * s;
      const float pl = sqrtf(dot3(perp, perp));
      const bool fixed = pl < 1e-4f;   // e is the cylinder's own x axis: y is a body-fixed point
      const float3 e = fixed ? mat_col(R2, 0) : perp * (-1.f / pl);
      const float3 bv = cross3(a, e);
      const float c1 = feat >= 2 ? -0.5f : 1.f, c2 = feat == 2 ? 0.8660254f : (feat == 3 ? -0.8660254f : 0.f);
      const float3 E = e * c1 + bv * c2;
      const float hs = (s >= 0.f ? -s2[1] : s2[1]) * (feat == 1 ? -1.f : 1.f);
      y = x2 + a * hs + E * s2[0];
      if (!fixed) {
        const float3 eb = yb * c1 + cross3(yb, a) * c2;
        const float3 perpb = (eb - e * dot3(e, eb)) * (-1.f / pl);
        const float3 ab = cross3(e, yb) * c2 - n * dot3(perpb, a) - perpb * s;
        add3(c, h.b_wr + 6 * gb2, (cross3(a, ab) - cross3(E, yb)) * s2[0]);
      }
    }
    if (turns) {
      // the frame: t2 = n x t1, t1 = t / |t|, t = n x e_k (e_k fixed by n's smallest component)
      nb = nb + cross3(t1, t2b);
      t1b = t1b + cross3(t2b, n);
      {
        const float a0 = fabsf(n.x), a1 = fabsf(n.y), a2 = fabsf(n.z);
        int kk = 0;
        if (a1 < a0) kk = 1;
        if (a2 < (kk == 0 ? a0 : a1)) kk = 2;
        const float3 ek = make_float3(kk == 0 ? 1.f : 0.f, kk == 1 ? 1.f : 0.f, kk == 2 ? 1.f : 0.f);
        const float3 t = cross3(n, ek);
        const float3 tb = (t1b - t1 * dot3(t1, t1b)) * rsqrtf(dot3(t, t));
        nb = nb + cross3(ek, tb);
      }
      // pos = y - n (r + dist / 2)
      const float rs = s2[0];
      nb = nb - posb * (rs + 0.5f * dist);
      // n = (y - q) / |y - q| with q the closest terrain point: at a face (or below the terrain)
      // n is the triangle's normal and constant; on an edge of direction u,
      // dn/dy = (I - n n^T)(I - u u^T) / |y - q|; at a vertex, (I - n n^T) / |y - q|
      float3 gx;
      Quat gq;
      body_frame(c, gb1, gx, gq);
      const float3 x1 = gx + qrot(gq, T3(&MF(geom_pos, 3 * g1i)));
      float R1[9];
      qmat(qnormalize(qmul(gq, Quat{MF(geom_quat, 4 * g1i), MF(geom_quat, 4 * g1i + 1), MF(geom_quat, 4 * g1i + 2),
                                    MF(geom_quat, 4 * g1i + 3)})), R1);
      const float* s1 = &MF(geom_size, 3 * g1i);
      const HGrid g{c.hf, h.hf_nrow, h.hf_ncol, s1[0], s1[1], s1[2], 2.f * s1[0] / (float)(h.hf_ncol - 1),
                    2.f * s1[1] / (float)(h.hf_nrow - 1)};
      HFeature f{0, make_float3(0.f, 0.f, 0.f)};
      hfield_sphere<true>(g, x1, R1, y, rs, &f);
      if (f.kind != 0) {
        float3 v = nb - n * dot3(n, nb);
        if (f.kind == 1) {
          const float3 U = mat_mul(R1, f.u);
          v = v - U * dot3(U, v);
        }
        yb = yb + v * (1.f / (dist + rs));
      }
    }
    add3(c, h.b_wr + 6 * gb2, cross3(y - o2, yb));
    add3(c, h.b_wr + 6 * gb2 + 3, yb);
  }
  for (int li = 0; li < h.nlimited; li++) {
    const int r = 4 * MC + li;
    if (!bit(act, r)) continue;
    const int j = MI(limit_jnt, li), d = MI(jnt_dofadr, j), qa = MI(jnt_qposadr, j);
    const float sgn = W(lsgn, li);
    const float D = W(rD, r), jl = W(Jp, r), jar = W(jar, r), dd = W(imp, r), A = W(Ahat, r), pos = W(rr, r);
    const float arefb = D * jl, Db = -jl * jar;
    B(v, d) += sgn * (-h.bref * arefb);
    const float db = -h.kref * pos * arefb + Db / ((1.f - dd) * (1.f - dd) * A);
    B(q, qa) += sgn * (-h.kref * dd * arefb + db * impedance_slope(h, pos));
    // Ahat = (M^-1)_dd
    const int wo = h.b_w;
    for (int i = 0; i < nv; i++) c.w[(wo + i) * c.S] = 0.f;
    c.w[(wo + d) * c.S] = 1.f;
    ldl_solve(c, h.w_L, wo);
    mbar_outer(c, wo, wo, -Db * D / A);
  }
  // friction-loss rows inside their band: as a limit row at zero position (aref = -b v, constant
  // impedance); outside the band the row's force is the constant bound and passes nothing back
  for (int k = 0; k < h.nfric; k++) {
    const int r = fric_row0(h) + k;
    if (!bit(act, r)) continue;
    const int d = MI(fric_dof, k);
    const float D = W(rD, r), jl = W(Jp, r), jar = W(jar, r), A = W(Ahat, r);
    const float arefb = D * jl, Db = -jl * jar;
    B(v, d) += -h.bref * arefb;
    const int wo = h.b_w;
    for (int i = 0; i < nv; i++) c.w[(wo + i) * c.S] = 0.f;
    c.w[(wo + d) * c.S] = 1.f;
    ldl_solve(c, h.w_L, wo);
    mbar_outer(c, wo, wo, -Db * D / A);
  }

  // ---- CRBA backward: Mbar -> cdof and composite inertia adjoints ----
  // M_ji = cdof_i . (Ic_b cdof_j) for the packed entries (j, i) of row j (b = body of j).  Ic_b
  // and the bilinear gradient are linear, so with u = sum_i Mbar_ji cdof_i (i over row j):
  //   cdof_i bar += Mbar_ji Ic_b cdof_j;  cdof_j bar += Ic_b u;  Ic_b bar += d(u^T Ic_b cdof_j)/dIc_b
  // (the diagonal entry is counted on both sides, as its derivative needs).
  for (int j = 0; j < nv; j++) {
    const int b = MI(dof_body, j), ci = h.w_cinert + 10 * b;
    const float3 cwj = cdof_w(c, j), cvj = cdof_v(c, j);
    float3 fa, fl;
    inert_mul(c, ci, cwj, cvj, fa, fl);
    const int r0 = MI(dof_rowadr, j), n = MI(dof_depth, j) + 1;
    float3 uw = make_float3(0.f, 0.f, 0.f), uv = uw;
    for (int t = 0; t < n; t++) {
      const float mb = B(M, r0 + t);
      const int i = MI(Lcol, r0 + t);
      uw = uw + cdof_w(c, i) * mb;
      uv = uv + cdof_v(c, i) * mb;
      add3(c, h.b_cdof + 6 * i, fa * mb);
      add3(c, h.b_cdof + 6 * i + 3, fl * mb);
    }
    float3 ga, gl;
    inert_mul(c, ci, uw, uv, ga, gl);
    add3(c, h.b_cdof + 6 * j, ga);
    add3(c, h.b_cdof + 6 * j + 3, gl);
    inertia_bilinear_grad(c, h.b_I + 10 * b, uw, uv, cwj, cvj, 1.f);
  }
  // composite -> own: Ibar_own(b) = sum over b and its ancestors of Ibar_composite
  for (int b = 1; b < nb; b++) {
    const int p = MI(body_parent, b);
    if (p == 0) continue;
    for (int k = 0; k < 10; k++) B(I, 10 * b + k) += B(I, 10 * p + k);
  }

  // ---- RNEA backward ----
  for (int k = 0; k < 6 * nb; k++) { B(vel, k) = 0.f; B(acc, k) = 0.f; }
  for (int d = 0; d < nv; d++) {
    const int f = h.w_cfrc + 6 * MI(dof_body, d);
    const float bb = B(bias, d);
    add3(c, h.b_cdof + 6 * d, W3(c, f) * bb);
    add3(c, h.b_cdof + 6 * d + 3, W3(c, f + 3) * bb);
  }
  for (int b = 1; b < nb; b++) {   // own-force adjoint: the bias adjoints of b's dofs and ancestors'
    const int p = MI(body_parent, b);
    float3 Fa = make_float3(0.f, 0.f, 0.f), Fl = Fa;
    if (p != 0) { Fa = B3(c, h.b_frc + 6 * p); Fl = B3(c, h.b_frc + 6 * p + 3); }
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    for (int j = j0; j < j0 + nj; j++) {
      const int d0 = MI(jnt_dofadr, j), ndof = MI(jnt_type, j) == PG_JNT_FREE ? 6 : 1;
      for (int d = d0; d < d0 + ndof; d++) {
        Fa = Fa + cdof_w(c, d) * B(bias, d);
        Fl = Fl + cdof_v(c, d) * B(bias, d);
      }
    }
    S3(c, h.b_frc + 6 * b, Fa);
    S3(c, h.b_frc + 6 * b + 3, Fl);
  }
  for (int b = nb - 1; b >= 1; b--) {
    const int p = MI(body_parent, b), ci = h.w_ci0 + 10 * b;
    float3 w = W3(c, h.w_cvel + 6 * b), v = W3(c, h.w_cvel + 6 * b + 3);
    const float3 aw = W3(c, h.w_cacc + 6 * b), av = W3(c, h.w_cacc + 6 * b + 3);
    const float3 Fa = B3(c, h.b_frc + 6 * b), Fl = B3(c, h.b_frc + 6 * b + 3);
    float3 ia, il;
    inert_mul(c, ci, w, v, ia, il);
    float3 wb = cross3(ia, Fa) + cross3(il, Fl);
    float3 vb = cross3(il, Fa);
    const float3 iab = cross3(Fa, w), ilb = cross3(Fa, v) + cross3(Fl, w);
    float3 awb, avb;
    inert_mul(c, ci, Fa, Fl, awb, avb);
    inertia_bilinear_grad(c, h.b_I + 10 * b, Fa, Fl, aw, av, 1.f);
    inertia_bilinear_grad(c, h.b_I + 10 * b, iab, ilb, w, v, 1.f);
    float3 gw, gv;
    inert_mul(c, ci, iab, ilb, gw, gv);
    wb = wb + gw + B3(c, h.b_vel + 6 * b);
    vb = vb + gv + B3(c, h.b_vel + 6 * b + 3);
    awb = awb + B3(c, h.b_acc + 6 * b);
    avb = avb + B3(c, h.b_acc + 6 * b + 3);
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    for (int j = j0 + nj - 1; j >= j0; j--) {
      const int d0 = MI(jnt_dofadr, j);
      const bool fr = MI(jnt_type, j) == PG_JNT_FREE;
      const int dr = fr ? d0 + 3 : d0, ndr = fr ? 3 : 1;
      float3 dw = make_float3(0.f, 0.f, 0.f), dv = dw;
      for (int d = dr; d < dr + ndr; d++) {
        dw = dw + cdof_w(c, d) * W(qvel, d);
        dv = dv + cdof_v(c, d) * W(qvel, d);
      }
      const float3 w0 = w - dw, v0 = v - dv;
      const float3 dwb = wb + cross3(awb, w0) + cross3(avb, v0);
      const float3 dvb = vb + cross3(avb, w0);
      wb = wb + cross3(dw, awb) + cross3(dv, avb);
      vb = vb + cross3(dw, avb);
      for (int d = dr; d < dr + ndr; d++) {
        const float qd = W(qvel, d);
        add3(c, h.b_cdof + 6 * d, dwb * qd);
        add3(c, h.b_cdof + 6 * d + 3, dvb * qd);
        B(v, d) += dot3(cdof_w(c, d), dwb) + dot3(cdof_v(c, d), dvb);
      }
      w = w0;
      v = v0;
      if (fr) {   // the translation was added to v before the rotations
        for (int k = 0; k < 3; k++) B(v, d0 + k) += k == 0 ? vb.x : (k == 1 ? vb.y : vb.z);
        v = v - make_float3(W(qvel, d0), W(qvel, d0 + 1), W(qvel, d0 + 2));
      }
    }
    if (p != 0) {
      add3(c, h.b_vel + 6 * p, wb);
      add3(c, h.b_vel + 6 * p + 3, vb);
      add3(c, h.b_acc + 6 * p, awb);
      add3(c, h.b_acc + 6 * p + 3, avb);
    }
  }

  // ---- own spatial inertias -> wrenches and mass adjoints ----
  for (int b = 1; b < nb; b++) {
    const int gi = h.b_I + 10 * b;
    const float G00 = B(I, 10 * b), G11 = B(I, 10 * b + 1), G22 = B(I, 10 * b + 2);
    const float G01 = 0.5f * B(I, 10 * b + 3), G02 = 0.5f * B(I, 10 * b + 4), G12 = 0.5f * B(I, 10 * b + 5);
    const float3 hb = W3(c, gi + 6);
    const float mbar_direct = B(I, 10 * b + 9);
    float3 x;
    Quat q;
    body_frame(c, b, x, q);
    float R[9];
    qmat(q, R);
    const float3 com = x + mat_mul(R, T3(&MF(body_ipos, 3 * b)));
    const float3 r = com - tree_origin(c, b);
    const float m = MF(body_mass, b);
    const float* In = &MF(body_inertia, 6 * b);
    const float Ib[9] = {In[0], In[3], In[4], In[3], In[1], In[5], In[4], In[5], In[2]};
    float T[9], A[9];
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) T[3 * i + k] = R[3 * i] * Ib[k] + R[3 * i + 1] * Ib[3 + k] + R[3 * i + 2] * Ib[6 + k];
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) A[3 * i + k] = T[3 * i] * R[3 * k] + T[3 * i + 1] * R[3 * k + 1] + T[3 * i + 2] * R[3 * k + 2];
    const float G[9] = {G00, G01, G02, G01, G11, G12, G02, G12, G22};
    float X[9];   // A G - G A (skew)
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) {
        float s = 0.f;
        for (int l = 0; l < 3; l++) s += A[3 * i + l] * G[3 * l + k] - G[3 * i + l] * A[3 * l + k];
        X[3 * i + k] = s;
      }
    float3 t = make_float3(2.f * X[5], 2.f * X[6], 2.f * X[1]);
    const float trG = G00 + G11 + G22;
    const float3 Gr = make_float3(G00 * r.x + G01 * r.y + G02 * r.z, G01 * r.x + G11 * r.y + G12 * r.z,
                                  G02 * r.x + G12 * r.y + G22 * r.z);
    const float3 rb = (r * (2.f * trG) - Gr * 2.f + hb) * m;
    t = t + cross3(r, rb);
    add3(c, h.b_wr + 6 * b, t);
    add3(c, h.b_wr + 6 * b + 3, rb);
    float GA = 0.f;
    for (int k = 0; k < 9; k++) GA += G[k] * A[k];
    const float gm = (m > 0.f ? GA / m : 0.f) + trG * dot3(r, r) - dot3(r, Gr) + dot3(hb, r) + mbar_direct;
    gpar[b * ld + env] += gm;
  }

  // ---- inward sweep: wrenches -> position adjoints ----
  for (int b = nb - 1; b >= 1; b--) {
    const int p = MI(body_parent, b);
    float3 t = B3(c, h.b_wr + 6 * b), f = B3(c, h.b_wr + 6 * b + 3);
    const int j0 = MI(body_jntadr, b), nj = MI(body_jntnum, b);
    for (int j = j0 + nj - 1; j >= j0; j--) {
      const int d0 = MI(jnt_dofadr, j), qa = MI(jnt_qposadr, j);
      if (MI(jnt_type, j) == PG_JNT_FREE) {
        for (int k = 3; k < 6; k++)
          motion_wrench(cdof_w(c, d0 + k), cdof_v(c, d0 + k), B3(c, h.b_cdof + 6 * (d0 + k)), B3(c, h.b_cdof + 6 * (d0 + k) + 3), t, f);
        B(q, qa) += f.x; B(q, qa + 1) += f.y; B(q, qa + 2) += f.z;
        const float3 phi = make_float3(dot3(cdof_w(c, d0 + 3), t) + dot3(cdof_v(c, d0 + 3), f),
                                       dot3(cdof_w(c, d0 + 4), t) + dot3(cdof_v(c, d0 + 4), f),
                                       dot3(cdof_w(c, d0 + 5), t) + dot3(cdof_v(c, d0 + 5), f));
        const Quat q{W(qpos, qa + 3), W(qpos, qa + 4), W(qpos, qa + 5), W(qpos, qa + 6)};
        const float qn = sqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
        const Quat qh{q.w / qn, q.x / qn, q.y / qn, q.z / qn};
        const Quat g = qmul(qh, Quat{0.f, phi.x, phi.y, phi.z});
        const float s = 2.f / qn;
        B(q, qa + 3) += s * g.w; B(q, qa + 4) += s * g.x; B(q, qa + 5) += s * g.y; B(q, qa + 6) += s * g.z;
      } else {
        const float3 cw = cdof_w(c, d0), cv = cdof_v(c, d0);
        B(q, qa) += dot3(cw, t) + dot3(cv, f);
        motion_wrench(cw, cv, B3(c, h.b_cdof + 6 * d0), B3(c, h.b_cdof + 6 * d0 + 3), t, f);
      }
    }
    if (p != 0) {
      add3(c, h.b_wr + 6 * p, t);
      add3(c, h.b_wr + 6 * p + 3, f);
    }
  }
}

// ---------------------------------------------------------------------------------------
// the kernel: one control step backward for every environment
// ---------------------------------------------------------------------------------------
struct VjpArgs {
  const float* tape;     // [S][tape_rows][ld] of this control step: qpos | qvel | warm | qacc
  const float* ctrl;     // [nu_max][ld]
  const float* gq;       // [nq_max][ld] loss cotangent of the post-step qpos, or NULL
  const float* gv;       // [nv_max][ld] loss cotangent of the post-step qvel, or NULL
  float* adj_q;          // [nq_max][ld] in: adjoint of the post-step state, out: of the pre-step state
  float* adj_v;          // [nv_max][ld]
  float* g_ctrl;         // [nu_max][ld] out
  float* g_params;       // [np_max][ld] accumulated: body masses | dof damping | actuator kp
  float* ws;             // global-memory workspaces (soa == 0): element i of env e at ws[i * ld + e]
  int64_t ld;
  int soa;               // > 0: workspaces in shared memory, blocks of soa environments, element i
                         // of the block's environment l at [i * soa + l]
  int64_t n;
  int tape_rows, nq_max, nv_max;
  int n_substeps;
  int nmodels;
  int64_t env_end[kMaxModels];
  int model_off[kMaxModels];
  const float* hfield[kMaxModels];   // each model's heightfield elevations (device), or NULL
  uint32_t blob[kMaxParamWords];     // the models' adjoint blobs (adjoint header + tables)
};
static_assert(sizeof(VjpArgs) <= 32764, "the reverse sweep's argument block must fit the kernel parameter space");

// SMEM: the workspace is in shared memory (blocks of A.soa environments, or of the specialised
// model's constant width); otherwise in global memory at A.ws with stride ld.
template <int SPEC_M = 0, bool SMEM = true>
__device__ __forceinline__ void vjp_body(const VjpArgs& A) {
  extern __shared__ __align__(16) float vjp_ws[];
  const int64_t env = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (env >= A.n) return;
#ifdef PG_SPEC
  const uint32_t* blob = SpecModel<SPEC_M>::blob_adj();   // the run-time compiled build: one model
  const int m = 0;
#else
  int m = 0;
  while (m < A.nmodels - 1 && env >= A.env_end[m]) m++;
  const uint32_t* blob = A.blob + A.model_off[m];
#endif
  const ModelHdr& h = *reinterpret_cast<const ModelHdr*>(blob);
  const int64_t ld = A.ld;
#ifdef PG_SPEC
  constexpr int kSoa = SMEM ? SpecModel<SPEC_M>::vjp_soa : 0;
#else
  const int kSoa = SMEM ? A.soa : 0;
#endif
  float* w = SMEM ? vjp_ws + threadIdx.x : A.ws + env;
  Ctx c{h, SMEM ? kSoa : (int)ld, reinterpret_cast<const int*>(blob), reinterpret_cast<const float*>(blob), w, A.ctrl, ld, env,
        A.hfield[m], nullptr};
  for (int k = 0; k < h.nq; k++) B(q, k) = A.adj_q[k * ld + env] + (A.gq ? A.gq[k * ld + env] : 0.f);
  for (int k = 0; k < h.nv; k++) B(v, k) = A.adj_v[k * ld + env] + (A.gv ? A.gv[k * ld + env] : 0.f);
  for (int k = 0; k < h.nu; k++) A.g_ctrl[k * ld + env] = 0.f;
  const int nsub = A.n_substeps > 0 ? A.n_substeps : h.substeps;
  const int64_t ent = (int64_t)A.tape_rows * ld;
  for (int s = nsub - 1; s >= 0; s--) {
    const float* tp = A.tape + s * ent + env;
    for (int k = 0; k < h.nq; k++) W(qpos, k) = tp[k * ld];
    for (int k = 0; k < h.nv; k++) W(qvel, k) = tp[(A.nq_max + k) * ld];   // (the warm start is not needed)
    kinematics(c);
    for (int k = 0; k < 10 * h.nbody; k++) W(ci0, k) = W(cinert, k);
    rnea(c);
    crba(c);
    // M's factor and reciprocal pivots (the sweep needs no forces and no a0)
    for (int k = 0; k < h.nL; k++) W(L, k) = W(M, k);
    ldl_factor(c, h.w_L);
    for (int k = 0; k < h.nv; k++) W(Dinv, k) = 1.f / W(L, MI(dof_rowadr, k));
    uint32_t status = 0;
    const int nc = collide<false>(c, status, nullptr);
    build_rows(c, nc);
    row_params(c, nc);
    for (int k = 0; k < h.nv; k++) W(a, k) = tp[(A.nq_max + 2 * A.nv_max + k) * ld];
    unsigned act[4];
    residuals(c, act);
    substep_vjp(c, nc, act, A.g_params, A.g_ctrl, ld);
  }
  for (int k = 0; k < h.nq; k++) A.adj_q[k * ld + env] = B(q, k);
  for (int k = 0; k < h.nv; k++) A.adj_v[k * ld + env] = B(v, k);
}

}  // namespace
}  // namespace pg
