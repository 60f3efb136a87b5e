// Device functions of the locomotion task around the step (pg_env_step, pg_env_reset): the
// joint targets from the policy's action, the observation, the reward table, termination,
// truncation and automatic reset (App. B, "Observation and Action" and "Reward and
// Termination").  One thread per environment, as the step kernel; the state lives in the
// step's workspace (the final substep's qpos / qvel) and in the caller's [rows][ld] arrays.
//
// Readings where the paper leaves a choice:
//   * base linear velocity = the free joint's world velocity rotated into the base frame;
//     angular velocity = the free joint's (already base-frame) rate;
//   * the orientation term's phi_body,xy = the xy part of gravity's direction in the base frame;
//   * observed joint positions are q - q_default over the actuated joints;
//   * tau of the torque and energy terms = the PD torque at the step's final state, and the
//     energy term sums |qdot_j tau_j|;
//   * a foot's air time grows by the control step before the touchdown test and restarts at
//     zero while it touches the ground;
//   * the stand-still term is |cmd_xy| as the table prints it;
//   * turning over = the base's z axis below the horizon (R_zz < 0), or a non-finite state.
#pragma once
#include "step_device.cuh"

namespace pg {
namespace {

// q_des = q_default + scale a (absolute) or q_des_prev + scale a (relative), clipped to a
// limited actuator's control range; written to the task state's q_des rows, which are the
// step's PD targets
__device__ void env_targets(const Ctx& c, const EnvArgs& E) {
  const EnvTask& T = E.task;
  const int64_t ld = c.ld, env = c.env;
  for (int a = 0; a < T.nu; a++) {
    float* qd = E.state + a * ld + env;
    const float base = T.mode == PG_ACTION_ABSOLUTE ? T.q_default[a] : *qd;
    float u = fmaf(T.scale, E.actions[a * ld + env], base);
    if (MI(act_ctrllimited, a)) u = fminf(fmaxf(u, MF(act_range, 2 * a)), MF(act_range, 2 * a + 1));
    *qd = u;
  }
}

// rotation of the floating base from its free joint's quaternion (qp: its qpos, stride ld)
__device__ __forceinline__ void base_rotation(const float* qp, int64_t ld, float R[9]) {
  qmat(qnormalize(Quat{qp[3 * ld], qp[4 * ld], qp[5 * ld], qp[6 * ld]}), R);
}

// observation of environment env from the [coord][ld] state arrays: gravity direction, base
// linear and angular velocity (base frame), joint positions from q_default, joint velocities,
// previous action (a_prev rows, or zero when NULL), command
__device__ void env_observe(const Ctx& c, const EnvTask& T, const float* qpos, const float* qvel, const float* a_prev,
                            const float* cmd, float* obs) {
  const int64_t ld = c.ld, env = c.env;
  float R[9];
  base_rotation(qpos + T.base_qpos * ld + env, ld, R);
  const float* bv = qvel + T.base_dof * ld + env;
  const float3 v = mat_tmul(R, make_float3(bv[0], bv[ld], bv[2 * ld]));
  float* o = obs + env;
  o[0] = -R[6]; o[ld] = -R[7]; o[2 * ld] = -R[8];
  o[3 * ld] = v.x; o[4 * ld] = v.y; o[5 * ld] = v.z;
  o[6 * ld] = bv[3 * ld]; o[7 * ld] = bv[4 * ld]; o[8 * ld] = bv[5 * ld];
  const int nu = T.nu;
  for (int a = 0; a < nu; a++) {
    o[(9 + a) * ld] = qpos[MI(act_qposadr, a) * ld + env] - T.q_default[a];
    o[(9 + nu + a) * ld] = qvel[MI(act_dof, a) * ld + env];
    o[(9 + 2 * nu + a) * ld] = a_prev ? a_prev[a * ld + env] : 0.f;
  }
  for (int k = 0; k < 3; k++) o[(9 + 3 * nu + k) * ld] = cmd[k * ld + env];
}

// a new episode for environment env: state <- (qpos0, qvel0), zero warm start and status, the
// task state's defaults
__device__ void env_restart(const Ctx& c, const EnvArgs& E, float* qpos, float* qvel, float* warm, uint32_t* status) {
  const ModelHdr& h = c.h;
  const EnvTask& T = E.task;
  const int64_t ld = c.ld, env = c.env;
  for (int k = 0; k < h.nq; k++) qpos[k * ld + env] = E.qpos0[k * ld + env];
  for (int k = 0; k < h.nv; k++) {
    qvel[k * ld + env] = E.qvel0[k * ld + env];
    warm[k * ld + env] = 0.f;
  }
  status[env] = 0u;
  float* st = E.state + env;
  for (int a = 0; a < T.nu; a++) {
    st[a * ld] = T.q_default[a];
    st[(T.nu + a) * ld] = 0.f;
  }
  for (int k = 2 * T.nu; k < 2 * T.nu + 2 * T.nfeet + 1; k++) st[k * ld] = 0.f;
}

// After the physics substeps (the workspace holds the final qpos / qvel, already stored to the
// state arrays): the reward terms on the final state, the reward, termination and truncation,
// the task state's update or the episode's restart, and the observation of the state the next
// action acts on.  dt is the control step (substeps x timestep).
__device__ void env_finish(const Ctx& c, const EnvArgs& E, float dt, float* qpos, float* qvel, float* warm,
                           uint32_t* status) {
  const ModelHdr& h = c.h;
  const EnvTask& T = E.task;
  const int64_t ld = c.ld, env = c.env;
  const int nu = T.nu, nf = T.nfeet;
  float* st = E.state + env;
  kinematics<false>(c);   // body frames and motion subspaces of the final state
  bool finite = true;
  for (int k = 0; k < h.nq; k++) finite = finite && isfinite(W(qpos, k));
  for (int k = 0; k < h.nv; k++) finite = finite && isfinite(W(qvel, k));
  const int bq = T.base_qpos, bd = T.base_dof;
  float R[9];
  qmat(qnormalize(Quat{W(qpos, bq + 3), W(qpos, bq + 4), W(qpos, bq + 5), W(qpos, bq + 6)}), R);
  const float3 g = make_float3(-R[6], -R[7], -R[8]);
  const float3 v = mat_tmul(R, make_float3(W(qvel, bd), W(qvel, bd + 1), W(qvel, bd + 2)));
  const float3 w = make_float3(W(qvel, bd + 3), W(qvel, bd + 4), W(qvel, bd + 5));
  const float cx = E.cmd[env], cy = E.cmd[ld + env], cw = E.cmd[2 * ld + env];
  const bool term = !finite || R[8] < 0.f;
  const float step_n = st[(2 * nu + 2 * nf) * ld] + 1.f;
  const bool trunc = !term && step_n >= (float)T.episode_length;
  const bool done = term || trunc;

  float r[PG_NTERMS];
  const float ex = cx - v.x, ey = cy - v.y, ez = cw - w.z;
  r[PG_R_LIN_VEL] = expf(-(ex * ex + ey * ey) / T.sig_v);
  r[PG_R_ANG_VEL] = expf(-(ez * ez) / T.sig_w);
  // feet: height, contact and horizontal velocity of each foot sphere
  float air_r = 0.f, clear = 0.f, slip = 0.f;
  for (int f = 0; f < nf; f++) {
    const int b = T.foot_body[f];
    float3 xb;
    Quat qb;
    body_frame(c, b, xb, qb);
    const float3 p = xb + qrot(qb, make_float3(T.foot_pos[3 * f], T.foot_pos[3 * f + 1], T.foot_pos[3 * f + 2]));
    const float height = p.z - T.foot_r[f];
    const bool on = height < T.contact_height;
    const float3 o = tree_origin(c, b);
    float3 vf = make_float3(0.f, 0.f, 0.f);
    const int dl = T.foot_lastdof[f];
    if (dl >= 0) {
      const int r0 = MI(dof_rowadr, dl), n = MI(dof_depth, dl) + 1;
      for (int t = 0; t < n; t++) {
        const int d = MI(Lcol, r0 + t);
        const float3 cwd = W3(c, h.w_cdof + 6 * d), cld = W3(c, h.w_cdof + 6 * d + 3);
        vf = vf + (cld + cross3(cwd, p - o)) * W(qvel, d);
      }
    }
    const float vxy2 = vf.x * vf.x + vf.y * vf.y;
    const float air = st[(2 * nu + f) * ld] + dt;
    const bool was_on = st[(2 * nu + nf + f) * ld] >= 0.5f;
    if (on && !was_on) air_r += fminf(fmaxf(air - T.air_min, 0.f), T.air_max - T.air_min);
    const float dz = height - T.clearance;
    clear += dz * dz * sqrtf(sqrtf(vxy2));
    if (on) slip += vxy2;
    if (!done) {
      st[(2 * nu + f) * ld] = on ? 0.f : air;
      st[(2 * nu + nf + f) * ld] = on ? 1.f : 0.f;
    }
  }
  r[PG_R_AIR_TIME] = air_r;
  r[PG_R_CLEARANCE] = clear;
  r[PG_R_SLIP] = slip;
  r[PG_R_ORIENTATION] = g.x * g.x + g.y * g.y;
  // actuated joints: PD torque at the final state against this step's targets
  float torque = 0.f, energy = 0.f, jpos = 0.f, rate = 0.f;
  for (int a = 0; a < nu; a++) {
    const float q = W(qpos, MI(act_qposadr, a)), qd = W(qvel, MI(act_dof, a));
    const float tau = actuator_force(c, a, st[a * ld]);
    torque += tau * tau;
    energy += fabsf(qd * tau);
    const float dq = q - T.q_default[a];
    jpos += dq * dq;
    const float da = E.actions[a * ld + env] - st[(nu + a) * ld];
    rate += da * da;
  }
  r[PG_R_TORQUE] = torque;
  r[PG_R_JOINT_POS] = jpos;
  r[PG_R_ACTION_RATE] = rate;
  r[PG_R_ENERGY] = energy;
  r[PG_R_POSE] = expf(-jpos);
  r[PG_R_TERMINATION] = term ? 1.f : 0.f;
  r[PG_R_STAND_STILL] = sqrtf(cx * cx + cy * cy);
  r[PG_R_LIN_Z] = v.z * v.z;
  r[PG_R_ANG_XY] = w.x * w.x + w.y * w.y;
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < PG_NTERMS; i++) sum = fmaf(T.weight[i], r[i], sum);
  E.reward[env] = fmaxf(sum, 0.f);
  E.done[env] = done ? 1.f : 0.f;
  E.truncated[env] = trunc ? 1.f : 0.f;
  if (E.terms)
#pragma unroll
    for (int i = 0; i < PG_NTERMS; i++) E.terms[i * ld + env] = r[i];
  if (done) {
    env_restart(c, E, qpos, qvel, warm, status);
  } else {
    for (int a = 0; a < nu; a++) st[(nu + a) * ld] = E.actions[a * ld + env];
    st[(2 * nu + 2 * nf) * ld] = step_n;
  }
  env_observe(c, T, qpos, qvel, E.state + nu * ld, E.cmd, E.obs);
}

}  // namespace
}  // namespace pg
