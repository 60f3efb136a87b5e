// C ABI of the locomotion task around the step (declared in include/pg.h): task compilation
// from a model and a description, and the argument checks and launches of pg_env_reset and
// pg_env_step (the kernels are the step kernel's ENV variant and env_reset_kernel in step.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {
namespace {

// the model's host tables (the blob's words: int32 tables and float32 tables)
int ti(const pg_model* m, int off, int i) { return (int)m->blob[(size_t)off + i]; }
float tf(const pg_model* m, int off, int i) {
  float f;
  std::memcpy(&f, &m->blob[(size_t)off + i], 4);
  return f;
}

// last dof of the chain that moves body b: its own last dof, else its nearest ancestor's; -1
// when no joint moves it
int last_dof(const pg_model* m, int b) {
  const ModelHdr& h = m->hdr;
  while (b > 0) {
    const int nj = ti(m, h.o_body_jntnum, b);
    if (nj > 0) {
      const int j = ti(m, h.o_body_jntadr, b) + nj - 1;
      return ti(m, h.o_jnt_dofadr, j) + (ti(m, h.o_jnt_type, j) == PG_JNT_FREE ? 5 : 0);
    }
    b = ti(m, h.o_body_parent, b);
  }
  return -1;
}

int check_env_call(const pg_batch* b, const pg_task* t, const pg_state* s, const float* task_state) {
  if (!b || !t || !s) return set_error(PG_EINVAL, "NULL batch, task or state");
  if (b->models.size() != 1 || b->models[0] != t->model)
    return set_error(PG_EUNSUPPORTED, "an environment step needs a batch of the task's model only");
  if (s->n != b->n) return set_error(PG_EINVAL, "state.n differs from the batch's environment count");
  if (s->ld < s->n) return set_error(PG_EINVAL, "state.ld must be >= state.n");
  if (b->n > 0 && (!s->qpos || !s->qvel || !s->qacc_warm || !s->status || !task_state))
    return set_error(PG_EINVAL, "NULL state array");
  return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" {

int pg_task_compile(const pg_model* m, const pg_task_desc* d, pg_task** out) {
  if (!out) return set_error(PG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!m || !d) return set_error(PG_EINVAL, "NULL model or description");
  const ModelHdr& h = m->hdr;
  if (d->action_mode != PG_ACTION_ABSOLUTE && d->action_mode != PG_ACTION_RELATIVE)
    return set_error(PG_EINVAL, "action_mode must be PG_ACTION_ABSOLUTE or PG_ACTION_RELATIVE");
  if (!std::isfinite(d->action_scale)) return set_error(PG_EINVAL, "action_scale must be finite");
  if (d->nfeet < 0 || d->nfeet > PG_MAX_FEET) return set_error(PG_EINVAL, "nfeet must be 0 .. PG_MAX_FEET");
  if (d->nfeet > 0 && !d->foot_geom) return set_error(PG_EINVAL, "NULL foot_geom");
  if (h.nu > 0 && !d->q_default) return set_error(PG_EINVAL, "NULL q_default");
  if (!(d->sigma_lin_vel > 0.f) || !(d->sigma_ang_vel > 0.f)) return set_error(PG_EINVAL, "sigmas must be > 0");
  if (!(d->air_time_max >= d->air_time_min)) return set_error(PG_EINVAL, "air_time_max must be >= air_time_min");
  if (d->episode_length < 1) return set_error(PG_EINVAL, "episode_length must be >= 1");
  for (int i = 0; i < PG_NTERMS; i++)
    if (!std::isfinite(d->weight[i])) return set_error(PG_EINVAL, "reward weights must be finite");
  // the model: a free joint on body 1 (the base), PD position actuators on hinge / slide joints
  if (h.nbody < 2 || ti(m, h.o_body_jntnum, 1) < 1 || ti(m, h.o_jnt_type, ti(m, h.o_body_jntadr, 1)) != PG_JNT_FREE)
    return set_error(PG_EUNSUPPORTED, "a locomotion task needs a free joint on body 1");
  for (int a = 0; a < h.nu; a++)
    if (ti(m, h.o_act_type, a) != PG_ACT_POSITION)
      return set_error(PG_EUNSUPPORTED, "a locomotion task needs PD position actuators");
  pg_task* t = new (std::nothrow) pg_task();
  if (!t) return set_error(PG_ENOMEM, "host allocation failed");
  EnvTask& T = t->task;
  std::memset(&T, 0, sizeof(T));
  const int j0 = ti(m, h.o_body_jntadr, 1);
  T.mode = d->action_mode;
  T.nu = h.nu;
  T.nfeet = d->nfeet;
  T.episode_length = d->episode_length;
  T.base_qpos = ti(m, h.o_jnt_qposadr, j0);
  T.base_dof = ti(m, h.o_jnt_dofadr, j0);
  T.scale = d->action_scale;
  T.contact_height = d->contact_height;
  T.clearance = d->clearance_height;
  T.sig_v = d->sigma_lin_vel;
  T.sig_w = d->sigma_ang_vel;
  T.air_min = d->air_time_min;
  T.air_max = d->air_time_max;
  for (int i = 0; i < PG_NTERMS; i++) T.weight[i] = d->weight[i];
  for (int a = 0; a < h.nu; a++) {
    if (!std::isfinite(d->q_default[a])) {
      delete t;
      return set_error(PG_EINVAL, "q_default must be finite");
    }
    T.q_default[a] = d->q_default[a];
  }
  for (int f = 0; f < d->nfeet; f++) {
    const int g = d->foot_geom[f];
    if (g < 0 || g >= h.ngeom || ti(m, h.o_geom_type, g) != PG_GEOM_SPHERE) {
      delete t;
      return set_error(PG_EINVAL, "every foot must be a sphere geom of the model");
    }
    const int b = ti(m, h.o_geom_body, g);
    T.foot_body[f] = b;
    T.foot_lastdof[f] = last_dof(m, b);
    for (int k = 0; k < 3; k++) T.foot_pos[3 * f + k] = tf(m, h.o_geom_pos, 3 * g + k);
    T.foot_r[f] = tf(m, h.o_geom_size, 3 * g);
  }
  t->model = m;
  t->nobs = 12 + 3 * h.nu;
  t->state_rows = 2 * h.nu + 2 * d->nfeet + 1;
  *out = t;
  return PG_OK;
}

int pg_task_info(const pg_task* t, pg_task_sizes* out) {
  if (!t || !out) return set_error(PG_EINVAL, "NULL argument");
  out->nobs = t->nobs;
  out->nterms = PG_NTERMS;
  out->state_rows = t->state_rows;
  return PG_OK;
}

void pg_task_free(pg_task* t) { delete t; }

int pg_env_reset(const pg_batch* b, const pg_task* t, pg_state* s, float* task_state, const float* qpos0,
                 const float* qvel0, const float* cmd, float* obs, void* stream) {
  int rc = check_env_call(b, t, s, task_state);
  if (rc) return rc;
  if (b->n == 0) return PG_OK;
  if (!qpos0 || !qvel0 || !cmd || !obs) return set_error(PG_EINVAL, "NULL qpos0, qvel0, cmd or obs");
  EnvArgs E;
  std::memset(&E, 0, sizeof(E));
  E.state = task_state; E.cmd = cmd; E.qpos0 = qpos0; E.qvel0 = qvel0; E.obs = obs; E.task = t->task;
  cudaError_t e = launch_env_reset(b, s, E, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("environment reset launch: ") + cudaGetErrorString(e));
  return PG_OK;
}

int pg_env_step(const pg_batch* b, const pg_task* t, pg_state* s, float* task_state, const float* actions,
                const float* cmd, const float* qpos0, const float* qvel0, int n_substeps, float* obs, float* reward,
                float* done, float* truncated, float* terms, const float* params, void* stream) {
  int rc = check_env_call(b, t, s, task_state);
  if (rc) return rc;
  if (n_substeps < 0) return set_error(PG_EINVAL, "n_substeps must be >= 0 (0: the model's own)");
  if (b->n == 0) return PG_OK;
  if ((t->task.nu > 0 && !actions) || !cmd || !qpos0 || !qvel0 || !obs || !reward || !done || !truncated)
    return set_error(PG_EINVAL, "NULL argument");
  EnvArgs E;
  E.state = task_state; E.actions = actions; E.cmd = cmd; E.qpos0 = qpos0; E.qvel0 = qvel0;
  E.obs = obs; E.reward = reward; E.done = done; E.truncated = truncated; E.terms = terms;
  E.task = t->task;
  cudaError_t e = launch_env_step(b, s, E, n_substeps, (cudaStream_t)stream, params);
  if (e != cudaSuccess) return set_error(PG_ECUDA, std::string("environment step launch: ") + cudaGetErrorString(e));
  return PG_OK;
}

}  // extern "C"
