"""FP64 oracle of the locomotion task around the step (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg import this
module.  It follows the paper's locomotion appendix (App. B):
  * "Observation and Action": the observation list (gravity in the body frame, base linear and
    angular velocity, joint positions and velocities, previous action, command), the absolute
    and relative joint-target mappings and the PD law (eq. pd_mapping);
  * "Reward and Termination": the reward table, the weighted sum clipped at zero, and
    termination when the robot turns over;
  * automatic reset of finished episodes, which the training loop needs between episodes.
The physics step is the oracle's own (`OracleModel.rollout`), the base frame comes from the
oracle's forward kinematics (`body_frames`) and foot velocities from its point Jacobian.

Readings where the paper leaves a choice (each also listed in the design notes):
  * v_xy, v_z and w are in the base frame; the linear velocity is the free joint's (base-origin)
    velocity rotated into the base frame, the angular velocity is the free joint's own.
  * "phi_body,xy" of the orientation term is the xy part of the gravity direction in the base
    frame.
  * "joint positions" in the observation are q - q_default of the actuated joints.
  * tau in the torque and energy terms is the PD torque at the step's final state (clipped by
    the actuator's torque limits), and
    "|qdot . tau|" is the sum of |qdot_j tau_j|.
  * T_air grows by the control step before the touchdown test; it restarts at zero while the
    foot touches the ground.
  * The stand-still term is |cmd_xy| as printed.
  * Turning over means the base's z axis points below the horizon (R_zz < 0); a non-finite
    state also terminates.
  * The observation after the step describes the state the next action acts on: after a reset,
    the new episode's first state with a zero previous action.

Arrays are per environment (plain vectors); the task is a `workloads.Task`.
"""
from __future__ import annotations

import numpy as np

from paper_2502_08844_b300 import workloads as W

NT = len(W.TERMS)
T = {k: i for i, k in enumerate(W.TERMS)}


def _addresses(m):
    """qpos and dof address of every joint (free 7 / 6, hinge and slide 1 / 1)."""
    qa, da, q, d = [], [], 0, 0
    for t in m.jnt_type:
        qa.append(q); da.append(d)
        q += 7 if t == W.FREE else 1
        d += 6 if t == W.FREE else 1
    return np.array(qa), np.array(da)


class OracleTask:
    """The task's tables in FP64 (the float32 inputs the CUDA library receives, widened)."""

    def __init__(self, om, task: W.Task):
        m = om.src
        self.om, self.m, self.task = om, m, task
        qa, da = _addresses(m)
        self.act_q = qa[m.act_jnt]
        self.act_d = da[m.act_jnt]
        self.kp = m.act_kp.astype(np.float64)
        self.kd = m.act_kd.astype(np.float64)
        self.limited = m.act_ctrllimited.astype(bool)
        self.lo = m.act_ctrlrange[:, 0].astype(np.float64)
        self.hi = m.act_ctrlrange[:, 1].astype(np.float64)
        if m.act_forcelimited is not None:   # torque limits clip the PD torque
            self.flo = m.act_forcerange[:, 0].astype(np.float64)
            self.fhi = m.act_forcerange[:, 1].astype(np.float64)
        self.q_default = task.q_default.astype(np.float64)
        self.scale = float(np.float32(task.action_scale))
        self.foot_geom = task.foot_geom.astype(int)
        self.foot_body = m.geom_body[self.foot_geom].astype(int)
        self.foot_r = m.geom_size[self.foot_geom, 0].astype(np.float64)
        self.weight = task.weight.astype(np.float64)
        self.nu, self.nf = m.nu, task.nfeet
        self.nobs = 12 + 3 * m.nu
        self.state_rows = 2 * m.nu + 2 * task.nfeet + 1
        f = lambda x: float(np.float32(x))
        self.contact_height, self.clearance = f(task.contact_height), f(task.clearance_height)
        self.sig_v, self.sig_w = f(task.sigma_lin_vel), f(task.sigma_ang_vel)
        self.air_min, self.air_max = f(task.air_time_min), f(task.air_time_max)
        # per-environment calibration offsets of the PD actuators (randomisation): the actuators act
        # as if their targets were q_des + calibration (set it on a task built on the substituted
        # model of oracle.randomize)
        self.calibration = np.zeros(m.nu)

    # ---- task state layout: q_des [nu] | previous action [nu] | air time [nf] | contact [nf] | step
    def split(self, st):
        nu, nf = self.nu, self.nf
        return (st[:nu].copy(), st[nu:2 * nu].copy(), st[2 * nu:2 * nu + nf].copy(),
                st[2 * nu + nf:2 * nu + 2 * nf].copy(), float(st[2 * nu + 2 * nf]))

    def join(self, q_des, a_prev, air, contact, step):
        return np.concatenate([q_des, a_prev, air, contact, [step]])

    def initial_task_state(self):
        return self.join(self.q_default.copy(), np.zeros(self.nu), np.zeros(self.nf), np.zeros(self.nf), 0.0)

    # ---- App. B "Observation and Action" -------------------------------------------------
    def targets(self, a, q_des_prev):
        """q_des = q_default + k_a a (absolute) or q_des_prev + k_a a (relative), clipped to the
        actuator's control range where it is limited (the PD target of eq. pd_mapping)."""
        base = self.q_default if self.task.action_mode == W.ABSOLUTE else q_des_prev
        q = base + self.scale * np.asarray(a, np.float64)
        return np.where(self.limited, np.clip(q, self.lo, self.hi), q)

    def base_frame(self, qpos):
        """Rotation of body 1 (the floating base) from the oracle's forward kinematics."""
        R, _, _ = self.om.body_frames(qpos)
        return R[1]

    def observation(self, qpos, qvel, a_prev, cmd):
        """(a) gravity direction in the base frame, (b) base linear and angular velocity,
        (c) joint positions (from q_default) and velocities, (d) previous action, (e) command."""
        R = self.base_frame(qpos)
        g = R.T @ np.array([0.0, 0.0, -1.0])
        v = R.T @ np.asarray(qvel[0:3], np.float64)
        w = np.asarray(qvel[3:6], np.float64)
        q = np.asarray(qpos, np.float64)[self.act_q] - self.q_default
        qd = np.asarray(qvel, np.float64)[self.act_d]
        return np.concatenate([g, v, w, q, qd, np.asarray(a_prev, np.float64), np.asarray(cmd, np.float64)])

    # ---- feet ------------------------------------------------------------------------------
    def feet(self, qpos, qvel):
        """World centre, height of the lowest point above z = 0, and velocity of each foot
        sphere (point Jacobian of the centre on its body times qvel)."""
        _, P = self.om.geom_frames(qpos)
        pos = P[self.foot_geom]
        height = pos[:, 2] - self.foot_r
        vel = np.zeros((self.nf, 3))
        for f in range(self.nf):
            Jv, _ = self.om.point_jacobian(qpos, self.foot_body[f], pos[f])
            vel[f] = Jv @ np.asarray(qvel, np.float64)
        return pos, height, vel

    # ---- App. B "Reward and Termination" -----------------------------------------------------
    def terminated(self, qpos, qvel):
        if not (np.all(np.isfinite(qpos)) and np.all(np.isfinite(qvel))):
            return True
        return bool(self.base_frame(qpos)[2, 2] < 0.0)

    def terms(self, qpos, qvel, q_des, a, a_prev, cmd, air, contact, dt, terminated):
        """The reward table's terms without coefficients, and the feet's new air time and
        contact flags."""
        R = self.base_frame(qpos)
        g = R.T @ np.array([0.0, 0.0, -1.0])
        v = R.T @ np.asarray(qvel[0:3], np.float64)
        w = np.asarray(qvel[3:6], np.float64)
        cmd = np.asarray(cmd, np.float64)
        m_lim = None if self.m.act_forcelimited is None else self.m.act_forcelimited.astype(bool)
        q = np.asarray(qpos, np.float64)[self.act_q]
        qd = np.asarray(qvel, np.float64)[self.act_d]
        tau = self.kp * (q_des + self.calibration - q) - self.kd * qd
        if m_lim is not None:
            tau = np.where(m_lim, np.clip(tau, self.flo, self.fhi), tau)
        _, height, vel = self.feet(qpos, qvel)
        on = height < self.contact_height
        air_now = air + dt
        touchdown = on & (contact < 0.5)
        vxy2 = vel[:, 0] ** 2 + vel[:, 1] ** 2
        r = np.zeros(NT)
        r[T["lin_vel"]] = np.exp(-((cmd[0] - v[0]) ** 2 + (cmd[1] - v[1]) ** 2) / self.sig_v)
        r[T["ang_vel"]] = np.exp(-(cmd[2] - w[2]) ** 2 / self.sig_w)
        r[T["air_time"]] = np.sum(np.clip((air_now - self.air_min) * touchdown, 0.0, self.air_max - self.air_min))
        r[T["clearance"]] = np.sum((height - self.clearance) ** 2 * np.sqrt(np.sqrt(vxy2)))
        r[T["slip"]] = np.sum(on * vxy2)
        r[T["orientation"]] = g[0] ** 2 + g[1] ** 2
        r[T["torque"]] = np.sum(tau ** 2)
        dq = q - self.q_default
        r[T["joint_pos"]] = np.sum(dq ** 2)
        r[T["action_rate"]] = np.sum((np.asarray(a, np.float64) - np.asarray(a_prev, np.float64)) ** 2)
        r[T["energy"]] = np.sum(np.abs(qd * tau))
        r[T["pose"]] = np.exp(-np.sum(dq ** 2))
        r[T["termination"]] = 1.0 if terminated else 0.0
        r[T["stand_still"]] = np.hypot(cmd[0], cmd[1])
        r[T["lin_z"]] = v[2] ** 2
        r[T["ang_xy"]] = w[0] ** 2 + w[1] ** 2
        return r, np.where(on, 0.0, air_now), on.astype(np.float64)

    def reward(self, r):
        """Weighted sum of the terms, clipped to stay non-negative."""
        return max(float(self.weight @ r), 0.0)

    # ---- one environment step ---------------------------------------------------------------
    def reset(self, qpos0, qvel0, cmd):
        """A new episode: the initial state, the task state's defaults and its observation."""
        st = self.initial_task_state()
        q = np.asarray(qpos0, np.float64).copy(); v = np.asarray(qvel0, np.float64).copy()
        return q, v, np.zeros(self.m.nv), st, self.observation(q, v, np.zeros(self.nu), cmd)

    def step(self, qpos, qvel, warm, task_state, a, cmd, qpos0, qvel0, n_substeps, solver_cap=None):
        """One environment step of one environment: targets, physics, reward, termination,
        truncation, reset, observation.  Returns a dict."""
        q_des_prev, a_prev, air, contact, step = self.split(np.asarray(task_state, np.float64))
        q_des = self.targets(a, q_des_prev)
        qn, vn, wn, status = self.om.rollout(np.asarray(qpos, np.float64)[None], np.asarray(qvel, np.float64)[None],
                                             (q_des + self.calibration)[None, None], n_substeps,
                                             qacc_warm=np.asarray(warm, np.float64)[None], solver_cap=solver_cap)
        qn, vn, wn = qn[0], vn[0], wn[0]
        dt = n_substeps * float(np.float32(self.m.timestep))
        term = self.terminated(qn, vn)
        r, air_n, contact_n = self.terms(qn, vn, q_des, a, a_prev, cmd, air, contact, dt, term)
        rew = self.reward(r)
        step_n = step + 1.0
        trunc = (not term) and step_n >= self.task.episode_length
        done = term or trunc
        out = dict(q_des=q_des, qpos_final=qn, qvel_final=vn, terms=r, reward=rew, done=float(done),
                   truncated=float(trunc), terminated=term)
        if done:
            q, v, wz, st, obs = self.reset(qpos0, qvel0, cmd)
        else:
            q, v, wz = qn, vn, wn
            st = self.join(q_des, np.asarray(a, np.float64), air_n, contact_n, step_n)
            obs = self.observation(q, v, a, cmd)
        out.update(qpos=q, qvel=v, warm=wz, task_state=st, obs=obs)
        return out
