// The branch-parallel step kernel's model plan (branch_body.cuh): the split of a compiled model
// into a trunk and branches, and the per-model constants the kernel is compiled with.
//
// Branches are found from the leaves: a branch is the longest chain that ends at a leaf body,
// climbs through bodies with exactly one child and no free joint, and stops below the world, a
// free body or a body with several children.  Every other body is trunk.  A model qualifies for
// the kernel when it has 2 to 8 branches, every contact pair touches at most one branch, at
// most one actuator drives each dof, the friction cone is pyramidal, its pairs are primitives up
// to boxes (geom1 may be a heightfield), and it has no joint friction loss and no more candidate
// contact points than max_contacts (so no contact is ever dropped); the sizes must also fit the
// kernel's register budget.  Otherwise
// pg_batch_specialize keeps the thread-per-environment kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_host.h"
#include "pg_internal.h"

namespace pg {

namespace {

struct Src {
  std::string s;
  void line(const std::string& x) { s += x + "\n"; }
  static std::string f(double v) {
    char b[48];
    snprintf(b, sizeof(b), "%.9gf", v);
    std::string r(b);
    if (r.find_first_of(".eEn") == std::string::npos) r.insert(r.size() - 1, ".0");
    return r;
  }
  void ci(const std::string& name, int v) { line("constexpr int " + name + " = " + std::to_string(v) + ";"); }
  void cf(const std::string& name, double v) { line("constexpr float " + name + " = " + f(v) + ";"); }
  // __constant__ tables, flattened row-major with the given extents
  void ti(const std::string& name, const std::string& dims, const std::vector<int>& v) {
    std::string x = "__constant__ const int " + name + dims + " = {";
    for (size_t i = 0; i < v.size(); i++) x += (i ? "," : "") + std::to_string(v[i]);
    line(x + "};");
  }
  void tf(const std::string& name, const std::string& dims, const std::vector<float>& v) {
    std::string x = "__constant__ const float " + name + dims + " = {";
    for (size_t i = 0; i < v.size(); i++) x += (i ? "," : "") + f(v[i]);
    line(x + "};");
  }
  // a __device__ constexpr function of one index returning vals[i]
  void fn(const std::string& name, const std::vector<int>& vals) {
    std::string x = "__device__ constexpr int " + name + "(int i) { return ";
    for (size_t i = 0; i < vals.size(); i++) x += "i == " + std::to_string(i) + " ? " + std::to_string(vals[i]) + " : ";
    line(x + "0; }");
  }
};

std::string dims(std::initializer_list<int> d) {
  std::string s;
  for (int x : d) s += "[" + std::to_string(std::max(x, 1)) + "]";
  return s;
}

}  // namespace

// Returns PG_OK and the generated constants (the head of the run-time compiled source), or
// PG_EUNSUPPORTED with the reason the model does not qualify.
int branch_plan(const pg_model* m, std::string& src, std::string& why, int& lanes_per_env, int& threads,
                int& branches) {
  const ModelHdr& h = m->hdr;
  const int* I = reinterpret_cast<const int*>(m->blob.data());
  const float* F = reinterpret_cast<const float*>(m->blob.data());
#define TI(name, i) (I[h.o_##name + (i)])
#define TF(name, i) (F[h.o_##name + (i)])
  auto no = [&](const std::string& r) {
    why = r;
    return PG_EUNSUPPORTED;
  };
  if (h.cone != PG_CONE_PYRAMIDAL) return no("the elliptic cone");
  if (h.nfric > 0) return no("joint friction loss");
  if (h.nslot > h.max_contacts) return no("more candidate contact points than max_contacts");
  const int nb = h.nbody;
  std::vector<int> parent(nb), nchild(nb, 0), free_body(nb, 0);
  for (int b = 0; b < nb; b++) parent[b] = TI(body_parent, b);
  for (int b = 1; b < nb; b++) nchild[parent[b]]++;
  std::vector<int> jnt_body(h.njnt, 0);
  for (int b = 1; b < nb; b++)
    for (int j = TI(body_jntadr, b); j < TI(body_jntadr, b) + TI(body_jntnum, b); j++) {
      jnt_body[j] = b;
      if (TI(jnt_type, j) == PG_JNT_FREE) free_body[b] = 1;
    }
  // ---- branches (chains to the leaves) and trunk ----
  std::vector<std::vector<int>> chains;
  std::vector<int> lane_of(nb, -1), slot_of(nb, -1);
  for (int b = 1; b < nb; b++) {
    if (nchild[b] != 0 || free_body[b]) continue;
    std::vector<int> c{b};
    int p = parent[b];
    while (p != 0 && nchild[p] == 1 && !free_body[p]) { c.push_back(p); p = parent[p]; }
    std::reverse(c.begin(), c.end());
    chains.push_back(c);
  }
  const int G = (int)chains.size();
  if (G < 2) return no("fewer than 2 branches");
  if (G > 8) return no("more than 8 branches");
  int GP = 1;
  while (GP < G) GP *= 2;
  int BB = 0;
  for (int l = 0; l < G; l++) {
    BB = std::max(BB, (int)chains[l].size());
    for (int s = 0; s < (int)chains[l].size(); s++) { lane_of[chains[l][s]] = l; slot_of[chains[l][s]] = s; }
  }
  std::vector<int> bnj(BB, 0);
  for (int l = 0; l < G; l++)
    for (int s = 0; s < (int)chains[l].size(); s++) bnj[s] = std::max(bnj[s], TI(body_jntnum, chains[l][s]));
  std::vector<int> bdof0(BB, 0);
  int NB = 0;
  for (int s = 0; s < BB; s++) { bdof0[s] = NB; NB += bnj[s]; }
  std::vector<int> trunk;   // trunk bodies in level order
  std::vector<int> tslot(nb, -1);
  for (int b = 1; b < nb; b++)
    if (lane_of[b] < 0) { tslot[b] = (int)trunk.size(); trunk.push_back(b); }
  const int BT = (int)trunk.size();
  if (BT < 1) return no("no trunk body");
  if (BT > 4) return no("more than 4 trunk bodies");
  // trunk-local qpos and dof indices (global order)
  std::vector<int> tq_of(h.nq, -1), td_of(h.nv, -1), tq_g, td_g;
  int NJT = 0;
  for (int k = 0; k < BT; k++) {
    const int b = trunk[k];
    NJT = std::max(NJT, TI(body_jntnum, b));
    for (int j = TI(body_jntadr, b); j < TI(body_jntadr, b) + TI(body_jntnum, b); j++) {
      const int free = TI(jnt_type, j) == PG_JNT_FREE;
      for (int i = 0; i < (free ? 7 : 1); i++) { tq_of[TI(jnt_qposadr, j) + i] = (int)tq_g.size(); tq_g.push_back(TI(jnt_qposadr, j) + i); }
      for (int i = 0; i < (free ? 6 : 1); i++) { td_of[TI(jnt_dofadr, j) + i] = (int)td_g.size(); td_g.push_back(TI(jnt_dofadr, j) + i); }
    }
  }
  const int NT = (int)td_g.size(), NQT = (int)tq_g.size();
  if (NT < 1) return no("a trunk without dofs");
  if (NT > 12) return no("more than 12 trunk dofs");
  if (NB > 9) return no("more than 9 dofs in a branch");
  // ancestors-or-self of every body as global dof bit masks
  std::vector<uint64_t> anc(nb, 0);
  for (int b = 1; b < nb; b++) {
    anc[b] = anc[parent[b]];
    for (int j = TI(body_jntadr, b); j < TI(body_jntadr, b) + TI(body_jntnum, b); j++)
      for (int i = 0; i < (TI(jnt_type, j) == PG_JNT_FREE ? 6 : 1); i++) anc[b] |= 1ull << (TI(jnt_dofadr, j) + i);
  }
  auto trunk_mask = [&](uint64_t g) {
    int mk = 0;
    for (int t = 0; t < NT; t++)
      if ((g >> td_g[t]) & 1ull) mk |= 1 << t;
    return mk;
  };
  // the tree origin of a body: its root's free joint position (trunk-local qpos), else the root's
  // fixed position
  auto origin = [&](int b, int& oq, float o[3]) {
    const int r = TI(body_root, b), fa = TI(root_freeadr, r);
    oq = fa >= 0 ? tq_of[fa] : -1;
    for (int k = 0; k < 3; k++) o[k] = fa >= 0 ? 0.f : TF(body_pos, 3 * r + k);
  };
  // actuator of each dof (at most one)
  std::vector<int> dof_act(h.nv, -1);
  for (int a = 0; a < h.nu; a++) {
    if (dof_act[TI(act_dof, a)] >= 0) return no("two actuators on one dof");
    dof_act[TI(act_dof, a)] = a;
  }
  Src S;
  // ---- trunk tables ----
  std::vector<int> tbpar(BT), tborg(BT), tjtype(BT * NJT, -1), tjq(BT * NJT, 0), tjd(BT * NJT, 0), tbg(BT, 0),
      lbg(GP * BB, 0);
  std::vector<float> tbpos(3 * BT), tbquat(4 * BT), tbmass(BT), tbipos(3 * BT), tbinert(6 * BT), tborgp(3 * BT),
      tjpos(3 * BT * NJT, 0.f), tjaxis(3 * BT * NJT, 0.f);
  for (int k = 0; k < BT; k++) {
    const int b = trunk[k];
    tbpar[k] = parent[b] == 0 ? -1 : tslot[parent[b]];
    if (parent[b] != 0 && tslot[parent[b]] < 0) return no("a trunk body below a branch");
    for (int i = 0; i < 3; i++) { tbpos[3 * k + i] = TF(body_pos, 3 * b + i); tbipos[3 * k + i] = TF(body_ipos, 3 * b + i); }
    for (int i = 0; i < 4; i++) tbquat[4 * k + i] = TF(body_quat, 4 * b + i);
    for (int i = 0; i < 6; i++) tbinert[6 * k + i] = TF(body_inertia, 6 * b + i);
    tbmass[k] = TF(body_mass, b);
    tbg[k] = b;
    origin(b, tborg[k], &tborgp[3 * k]);
    for (int jj = 0; jj < TI(body_jntnum, b); jj++) {
      const int j = TI(body_jntadr, b) + jj, e = k * NJT + jj;
      tjtype[e] = TI(jnt_type, j);
      tjq[e] = tq_of[TI(jnt_qposadr, j)];
      tjd[e] = td_of[TI(jnt_dofadr, j)];
      for (int i = 0; i < 3; i++) { tjpos[3 * e + i] = TF(jnt_pos, 3 * j + i); tjaxis[3 * e + i] = TF(jnt_axis, 3 * j + i); }
    }
  }
  std::vector<int> tdbody(NT), tdanc(NT), tdact(NT, -1), tdatype(NT, 0), tdqa(NT, 0), tdclim(NT, 0), tdflim(NT, 0);
  std::vector<float> tddamp(NT), tdarm(NT), tdgear(NT, 0.f), tdkp(NT, 0.f), tdkd(NT, 0.f), tdcr(2 * NT, 0.f), tdfr(2 * NT, 0.f);
  for (int t = 0; t < NT; t++) {
    const int d = td_g[t], b = TI(dof_body, d);
    tdbody[t] = tslot[b];
    uint64_t a = 0;   // ancestors-or-self of dof d: its body's ancestors up to d itself
    for (int x = 0; x <= d; x++)
      if (((anc[b] >> x) & 1ull) && (TI(dof_body, x) != b || x <= d)) a |= 1ull << x;
    tdanc[t] = trunk_mask(a);
    tddamp[t] = TF(dof_damping, d);
    tdarm[t] = TF(dof_armature, d);
    const int ac = dof_act[d];
    if (ac >= 0) {
      tdact[t] = ac; tdatype[t] = TI(act_type, ac); tdqa[t] = tq_of[TI(act_qposadr, ac)];
      tdgear[t] = TF(act_gear, ac); tdkp[t] = TF(act_kp, ac); tdkd[t] = TF(act_kd, ac);
      tdclim[t] = TI(act_ctrllimited, ac); tdflim[t] = TI(act_forcelimited, ac);
      for (int i = 0; i < 2; i++) { tdcr[2 * t + i] = TF(act_range, 2 * ac + i); tdfr[2 * t + i] = TF(act_forcerange, 2 * ac + i); }
    }
  }
  // ---- branch tables (padding: zero mass, no joints, unit armature) ----
  std::vector<int> latt(GP, -1), lanc(GP, 0), lorgT(GP, -1);
  std::vector<float> lorg(3 * GP, 0.f);
  std::vector<float> lbpos(GP * BB * 3, 0.f), lbquat(GP * BB * 4, 0.f), lbmass(GP * BB, 0.f), lbipos(GP * BB * 3, 0.f),
      lbinert(GP * BB * 6, 0.f);
  for (int i = 0; i < GP * BB; i++) lbquat[4 * i] = 1.f;
  std::vector<int> ljtype(GP * NB, -1), ldg(GP * NB, -1), ldq(GP * NB, -1), ldact(GP * NB, -1), ldatype(GP * NB, 0),
      ldclim(GP * NB, 0), ldflim(GP * NB, 0);
  std::vector<float> ljpos(GP * NB * 3, 0.f), ljaxis(GP * NB * 3, 0.f), lddamp(GP * NB, 0.f), ldarm(GP * NB, 1.f),
      ldgear(GP * NB, 0.f), ldkp(GP * NB, 0.f), ldkd(GP * NB, 0.f), ldcr(GP * NB * 2, 0.f), ldfr(GP * NB * 2, 0.f);
  std::vector<int> bdof_local(h.nv, -1);   // global dof -> local dof index in its branch
  for (int l = 0; l < G; l++) {
    const std::vector<int>& c = chains[l];
    const int top = c[0];
    latt[l] = parent[top] == 0 ? -1 : tslot[parent[top]];
    lanc[l] = trunk_mask(anc[parent[top]]);
    origin(top, lorgT[l], &lorg[3 * l]);
    for (int s = 0; s < (int)c.size(); s++) {
      const int b = c[s], e = l * BB + s;
      for (int i = 0; i < 3; i++) { lbpos[3 * e + i] = TF(body_pos, 3 * b + i); lbipos[3 * e + i] = TF(body_ipos, 3 * b + i); }
      for (int i = 0; i < 4; i++) lbquat[4 * e + i] = TF(body_quat, 4 * b + i);
      for (int i = 0; i < 6; i++) lbinert[6 * e + i] = TF(body_inertia, 6 * b + i);
      lbmass[e] = TF(body_mass, b);
      lbg[e] = b;
      for (int jj = 0; jj < TI(body_jntnum, b); jj++) {
        const int j = TI(body_jntadr, b) + jj, d = bdof0[s] + jj, e2 = l * NB + d, gd = TI(jnt_dofadr, j);
        ljtype[e2] = TI(jnt_type, j);
        for (int i = 0; i < 3; i++) { ljpos[3 * e2 + i] = TF(jnt_pos, 3 * j + i); ljaxis[3 * e2 + i] = TF(jnt_axis, 3 * j + i); }
        ldg[e2] = gd; ldq[e2] = TI(jnt_qposadr, j);
        bdof_local[gd] = d;
        lddamp[e2] = TF(dof_damping, gd); ldarm[e2] = TF(dof_armature, gd);
        const int ac = dof_act[gd];
        if (ac >= 0) {
          ldact[e2] = ac; ldatype[e2] = TI(act_type, ac); ldgear[e2] = TF(act_gear, ac); ldkp[e2] = TF(act_kp, ac);
          ldkd[e2] = TF(act_kd, ac); ldclim[e2] = TI(act_ctrllimited, ac); ldflim[e2] = TI(act_forcelimited, ac);
          for (int i = 0; i < 2; i++) { ldcr[2 * e2 + i] = TF(act_range, 2 * ac + i); ldfr[2 * e2 + i] = TF(act_forcerange, 2 * ac + i); }
        }
      }
    }
  }
  // ---- contact pairs, per lane in pair order ----
  auto side = [&](int b) { return b == 0 ? -1 : (lane_of[b] >= 0 ? BT + slot_of[b] : tslot[b]); };
  std::vector<std::vector<int>> lpairs(GP);
  for (int p = 0; p < h.npair; p++) {
    const int g1 = TI(pair_g1, p), g2 = TI(pair_g2, p);
    const int t1 = TI(geom_type, g1), t2 = TI(geom_type, g2);
    if ((t1 > PG_GEOM_BOX && t1 != PG_GEOM_HFIELD) || t2 > PG_GEOM_BOX)
      return no("a pair type outside the branch kernel");
    const int b1 = TI(geom_body, g1), b2 = TI(geom_body, g2);
    const int l1 = lane_of[b1], l2 = lane_of[b2];
    if (l1 >= 0 && l2 >= 0) return no("a contact pair between branch bodies");
    int l = l1 >= 0 ? l1 : l2;
    if (l < 0) {   // trunk or world on both sides: the lane with the fewest pairs so far
      l = 0;
      for (int x = 1; x < G; x++)
        if (lpairs[x].size() < lpairs[l].size()) l = x;
    }
    lpairs[l].push_back(p);
  }
  int PS = 0;
  for (int l = 0; l < G; l++) PS = std::max(PS, (int)lpairs[l].size());
  std::vector<int> pnp(std::max(PS, 1), 0), pc0(std::max(PS, 1), 0);
  for (int l = 0; l < G; l++)
    for (int s = 0; s < (int)lpairs[l].size(); s++) pnp[s] = std::max(pnp[s], TI(pair_nslot, lpairs[l][s]));
  int NCL = 0;
  for (int s = 0; s < PS; s++) { pc0[s] = NCL; NCL += pnp[s]; }
  std::vector<int> pt1(GP * PS, -1), pt2(GP * PS, -1), ps1(GP * PS, -1), ps2(GP * PS, -1), pcond(GP * PS, 0),
      pjb(GP * PS * NB, 0), pjt(GP * PS * NT, 0), pslotadr(GP * PS, 0), pnslot(GP * PS, 0);
  std::vector<float> pgp1(GP * PS * 3, 0.f), pgq1(GP * PS * 4, 0.f), psz1(GP * PS * 3, 0.f), pgp2(GP * PS * 3, 0.f),
      pgq2(GP * PS * 4, 0.f), psz2(GP * PS * 3, 0.f), pmu(GP * PS, 0.f);
  for (int i = 0; i < GP * PS; i++) { pgq1[4 * i] = 1.f; pgq2[4 * i] = 1.f; }
  for (int l = 0; l < G; l++)
    for (int s = 0; s < (int)lpairs[l].size(); s++) {
      const int p = lpairs[l][s], e = l * PS + s;
      const int g1 = TI(pair_g1, p), g2 = TI(pair_g2, p);
      pt1[e] = TI(geom_type, g1); pt2[e] = TI(geom_type, g2);
      ps1[e] = side(TI(geom_body, g1)); ps2[e] = side(TI(geom_body, g2));
      pcond[e] = TI(pair_condim, p); pmu[e] = TF(pair_friction, p);
      pslotadr[e] = TI(pair_slotadr, p); pnslot[e] = TI(pair_nslot, p);
      for (int i = 0; i < 3; i++) {
        pgp1[3 * e + i] = TF(geom_pos, 3 * g1 + i); psz1[3 * e + i] = TF(geom_size, 3 * g1 + i);
        pgp2[3 * e + i] = TF(geom_pos, 3 * g2 + i); psz2[3 * e + i] = TF(geom_size, 3 * g2 + i);
      }
      for (int i = 0; i < 4; i++) { pgq1[4 * e + i] = TF(geom_quat, 4 * g1 + i); pgq2[4 * e + i] = TF(geom_quat, 4 * g2 + i); }
      for (int a = 0; a < TI(pair_ncol, p); a++) {
        const int d = TI(col_dof, TI(pair_coladr, p) + a), sg = TI(col_sign, TI(pair_coladr, p) + a);
        if (td_of[d] >= 0) pjt[e * NT + td_of[d]] = sg;
        else if (bdof_local[d] >= 0 && lane_of[TI(dof_body, d)] == l) pjb[e * NB + bdof_local[d]] = sg;
        else return no("a contact column outside its lane");
      }
    }
  // ---- limit rows: branch joints on their lane, trunk joints on the lane with the fewest ----
  std::vector<std::vector<int>> llim(GP);
  for (int i = 0; i < h.nlimited; i++) {
    const int j = TI(limit_jnt, i), b = jnt_body[j];
    int l = lane_of[b];
    if (l < 0) {
      l = 0;
      for (int x = 1; x < G; x++)
        if (llim[x].size() < llim[l].size()) l = x;
    }
    llim[l].push_back(j);
  }
  int LS = 0;
  for (int l = 0; l < G; l++) LS = std::max(LS, (int)llim[l].size());
  std::vector<int> llk(GP * std::max(LS, 1), 0), lld(GP * std::max(LS, 1), 0), llq(GP * std::max(LS, 1), 0);
  std::vector<float> lllo(GP * std::max(LS, 1), 0.f), llhi(GP * std::max(LS, 1), 0.f);
  for (int l = 0; l < G; l++)
    for (int s = 0; s < (int)llim[l].size(); s++) {
      const int j = llim[l][s], e = l * LS + s, gd = TI(jnt_dofadr, j), gq = TI(jnt_qposadr, j);
      if (td_of[gd] >= 0) { llk[e] = 2; lld[e] = td_of[gd]; llq[e] = tq_of[gq]; }
      else { llk[e] = 1; lld[e] = bdof_local[gd]; llq[e] = bdof_local[gd]; }
      lllo[e] = TF(jnt_range, 2 * j); llhi[e] = TF(jnt_range, 2 * j + 1);
    }
  if (4 * NCL + LS > 32) return no("more than 32 constraint rows per branch");
  if (NCL > 8) return no("more than 8 contact points per branch");
  // ---- the source head ----
  const int envs_per_block = 32 / GP;
  lanes_per_env = GP;
  threads = 32;
  branches = G;
  S.line("// generated: branch-parallel step kernel constants for one model");
  S.line("#define PG_WITH_ELLIPTIC 0");
  S.line("#include \"pg_internal.h\"");
  S.line("namespace pgb {");
  S.ci("GP", GP); S.ci("G", G); S.ci("NT", NT); S.ci("NQT", NQT); S.ci("BT", BT); S.ci("NJT", std::max(NJT, 1));
  S.ci("NB", std::max(NB, 1)); S.ci("BB", BB); S.ci("PS", PS); S.ci("NCL", NCL); S.ci("LS", LS);
  S.ci("NTH", threads); S.ci("EPB", envs_per_block); S.ci("CAP", h.cap); S.ci("NSUB", h.substeps);
  S.ci("HF_NROW", std::max(h.hf_nrow, 2)); S.ci("HF_NCOL", std::max(h.hf_ncol, 2));
  // rows of pg_step_dr's per-environment parameters
  S.ci("DR_COM", h.dr_com); S.ci("DR_ARM", h.dr_arm); S.ci("DR_CAL", h.dr_cal); S.ci("DR_KP", h.dr_kp);
  S.ci("DR_KD", h.dr_kd); S.ci("DR_MASS", h.dr_mass);
  S.cf("HSTEP", h.h); S.cf("GRAV_X", h.grav[0]); S.cf("GRAV_Y", h.grav[1]); S.cf("GRAV_Z", h.grav[2]);
  S.cf("KREF", h.kref); S.cf("BREF", h.bref); S.cf("MARGIN", h.margin);
  S.cf("SOLIMP_D0", h.solimp[0]); S.cf("SOLIMP_DW", h.solimp[1]); S.cf("SOLIMP_WIDTH", h.solimp[2]);
  S.cf("SOLIMP_MID", h.solimp[3]); S.cf("SOLIMP_POWER", h.solimp[4]);
  S.cf("IMP_MID_INV", h.imp_mid_inv); S.cf("IMP_TAIL_INV", h.imp_tail_inv);
  S.fn("bnj", bnj); S.fn("bdof0", bdof0); S.fn("pnp", pnp); S.fn("pc0", pc0);
  std::vector<int> pslot(std::max(NCL, 1), 0);
  for (int s = 0; s < PS; s++)
    for (int i = 0; i < pnp[s]; i++) pslot[pc0[s] + i] = s;
  S.fn("pslot", pslot);
  S.ti("kTBpar", dims({BT}), tbpar); S.ti("kTBorg", dims({BT}), tborg);
  S.tf("kTBpos", dims({BT, 3}), tbpos); S.tf("kTBquat", dims({BT, 4}), tbquat); S.tf("kTBmass", dims({BT}), tbmass);
  S.tf("kTBipos", dims({BT, 3}), tbipos); S.tf("kTBinert", dims({BT, 6}), tbinert); S.tf("kTBorgp", dims({BT, 3}), tborgp);
  S.ti("kTBg", dims({BT}), tbg); S.ti("kLBg", dims({GP, BB}), lbg);
  const int njt = std::max(NJT, 1);
  if (NJT == 0) { tjtype.assign(BT, -1); tjq.assign(BT, 0); tjd.assign(BT, 0); tjpos.assign(3 * BT, 0.f); tjaxis.assign(3 * BT, 0.f); }
  S.ti("kTJtype", dims({BT, njt}), tjtype); S.ti("kTJq", dims({BT, njt}), tjq); S.ti("kTJd", dims({BT, njt}), tjd);
  S.tf("kTJpos", dims({BT, njt, 3}), tjpos); S.tf("kTJaxis", dims({BT, njt, 3}), tjaxis);
  S.ti("kTDbody", dims({NT}), tdbody); S.ti("kTDanc", dims({NT}), tdanc); S.ti("kTDact", dims({NT}), tdact);
  S.ti("kTDatype", dims({NT}), tdatype); S.ti("kTDqa", dims({NT}), tdqa); S.ti("kTDclim", dims({NT}), tdclim);
  S.ti("kTDflim", dims({NT}), tdflim); S.ti("kTDg", dims({NT}), td_g); S.ti("kTQg", dims({NQT}), tq_g);
  S.tf("kTDdamp", dims({NT}), tddamp); S.tf("kTDarm", dims({NT}), tdarm); S.tf("kTDgear", dims({NT}), tdgear);
  S.tf("kTDkp", dims({NT}), tdkp); S.tf("kTDkd", dims({NT}), tdkd); S.tf("kTDcr", dims({NT, 2}), tdcr);
  S.tf("kTDfr", dims({NT, 2}), tdfr);
  S.ti("kLatt", dims({GP}), latt); S.ti("kLanc", dims({GP}), lanc); S.ti("kLorgT", dims({GP}), lorgT);
  S.tf("kLorg", dims({GP, 3}), lorg);
  S.tf("kLBpos", dims({GP, BB, 3}), lbpos); S.tf("kLBquat", dims({GP, BB, 4}), lbquat); S.tf("kLBmass", dims({GP, BB}), lbmass);
  S.tf("kLBipos", dims({GP, BB, 3}), lbipos); S.tf("kLBinert", dims({GP, BB, 6}), lbinert);
  const int nbb = std::max(NB, 1);
  S.ti("kLJtype", dims({GP, nbb}), ljtype); S.tf("kLJpos", dims({GP, nbb, 3}), ljpos); S.tf("kLJaxis", dims({GP, nbb, 3}), ljaxis);
  S.ti("kLDg", dims({GP, nbb}), ldg); S.ti("kLDq", dims({GP, nbb}), ldq); S.ti("kLDact", dims({GP, nbb}), ldact);
  S.ti("kLDatype", dims({GP, nbb}), ldatype); S.ti("kLDclim", dims({GP, nbb}), ldclim); S.ti("kLDflim", dims({GP, nbb}), ldflim);
  S.tf("kLDdamp", dims({GP, nbb}), lddamp); S.tf("kLDarm", dims({GP, nbb}), ldarm); S.tf("kLDgear", dims({GP, nbb}), ldgear);
  S.tf("kLDkp", dims({GP, nbb}), ldkp); S.tf("kLDkd", dims({GP, nbb}), ldkd); S.tf("kLDcr", dims({GP, nbb, 2}), ldcr);
  S.tf("kLDfr", dims({GP, nbb, 2}), ldfr);
  const int ps = std::max(PS, 1);
  if (PS == 0) {
    pt1.assign(GP, -1); pt2.assign(GP, -1); ps1.assign(GP, -1); ps2.assign(GP, -1); pcond.assign(GP, 0);
    pjb.assign(GP * nbb, 0); pjt.assign(GP * NT, 0); pgp1.assign(3 * GP, 0.f); pgq1.assign(4 * GP, 0.f);
    psz1.assign(3 * GP, 0.f); pgp2.assign(3 * GP, 0.f); pgq2.assign(4 * GP, 0.f); psz2.assign(3 * GP, 0.f);
    pmu.assign(GP, 0.f);
    pslotadr.assign(GP, 0); pnslot.assign(GP, 0);
  }
  S.ti("kPt1", dims({GP, ps}), pt1); S.ti("kPt2", dims({GP, ps}), pt2); S.ti("kPs1", dims({GP, ps}), ps1);
  S.ti("kPs2", dims({GP, ps}), ps2); S.ti("kPcond", dims({GP, ps}), pcond);
  S.ti("kPslot", dims({GP, ps}), pslotadr); S.ti("kPnslot", dims({GP, ps}), pnslot);
  S.ci("NSLOT", h.nslot);
  S.ti("kPjb", dims({GP, ps, nbb}), pjb); S.ti("kPjt", dims({GP, ps, NT}), pjt);
  S.tf("kPgp1", dims({GP, ps, 3}), pgp1); S.tf("kPgq1", dims({GP, ps, 4}), pgq1); S.tf("kPsz1", dims({GP, ps, 3}), psz1);
  S.tf("kPgp2", dims({GP, ps, 3}), pgp2); S.tf("kPgq2", dims({GP, ps, 4}), pgq2); S.tf("kPsz2", dims({GP, ps, 3}), psz2);
  S.tf("kPmu", dims({GP, ps}), pmu);
  S.ti("kLLk", dims({GP, std::max(LS, 1)}), llk); S.ti("kLLd", dims({GP, std::max(LS, 1)}), lld);
  S.ti("kLLq", dims({GP, std::max(LS, 1)}), llq);
  S.tf("kLLlo", dims({GP, std::max(LS, 1)}), lllo); S.tf("kLLhi", dims({GP, std::max(LS, 1)}), llhi);
  S.line("}  // namespace pgb");
  S.line("#include \"branch_body.cuh\"");
  S.line("extern \"C\" __global__ void __launch_bounds__(32) pg_step_branch(const __grid_constant__ pg::BranchArgs A) "
         "{ pgb::branch_step<false>(A); }");
  S.line("extern \"C\" __global__ void __launch_bounds__(256) pg_step_branch_sync(const __grid_constant__ pg::BranchArgs A) "
         "{ pgb::branch_step<true>(A); }");
  S.line("extern \"C\" __global__ void __launch_bounds__(256) pg_step_branch_dr(const __grid_constant__ pg::BranchArgs A) "
         "{ pgb::branch_step<true, false, true>(A); }");
  if (m->hdr.adj_ok)   // the adjoint's tape replay (only for models inside its scope)
    S.line("extern \"C\" __global__ void __launch_bounds__(256) pg_step_branch_tape(const __grid_constant__ pg::BranchArgs A) "
           "{ pgb::branch_step<true, true>(A); }");
  src = S.s;
  return PG_OK;
#undef TI
#undef TF
}

// environments [env0, env0 + count) of a state.  k: blocks of one warp (32 / lanes environments
// each).  k_sync (when not NULL): blocks of W warps whose warps start every substep together; W is
// envs_per_block / (32 / lanes) when envs_per_block > 0 (1 to 8), else the warps per SM the launch
// needs for one wave (at most 8).
cudaError_t launch_branch_range(cudaKernel_t k, cudaKernel_t k_sync, int lanes, int64_t env0, int64_t count,
                                const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                                const pg_step_out* out, int nslot, float* tape, int tape_rows, int tape_nq,
                                int tape_nv, int envs_per_block, const float* hfield, const float* dr) {
  if (count <= 0) return cudaSuccess;
  BranchArgs A;
  A.hfield = hfield;
  A.dr = dr;
  A.out_force = out ? out->contact_force : nullptr;
  A.out_ncon = out ? out->ncon : nullptr;
  A.out_nslot = nslot;
  A.tape = tape;
  A.tape_rows = tape_rows;
  A.tape_nq = tape_nq;
  A.tape_nv = tape_nv;
  A.qpos = s->qpos;
  A.qvel = s->qvel;
  A.warm = s->qacc_warm;
  A.status = s->status;
  A.stats = s->stats;
  A.ctrl = ctrl;
  A.ld = s->ld;
  A.env0 = env0;
  A.n = count;
  A.n_substeps = n_substeps;
  const int epw = 32 / lanes;   // environments per warp
  void* params[] = {&A};
  if (k_sync) {
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms < 1) sms = 1;
    }
    const int64_t warps = (count + epw - 1) / epw;
    const int w = envs_per_block > 0 ? std::min(8, std::max(1, envs_per_block / epw))
                                     : (int)std::min<int64_t>(8, std::max<int64_t>(1, (warps + sms - 1) / sms));
    const int64_t per_block = (int64_t)w * epw;
    return cudaLaunchKernel((const void*)k_sync, dim3((unsigned)((count + per_block - 1) / per_block)), dim3(32 * w),
                            params, 0, st);
  }
  return cudaLaunchKernel((const void*)k, dim3((unsigned)((count + epw - 1) / epw)), dim3(32), params, 0, st);
}

cudaError_t launch_branch(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, cudaStream_t st,
                          const pg_step_out* out) {
  return launch_branch_range(b->branch_kernel, b->branch_kernel_sync, b->branch_lanes, 0, s->n, s, ctrl, n_substeps,
                             st, out, b->nslot_max, nullptr, 0, 0, 0, b->envs_per_cta_req, b->hfield_ptr[0]);
}

cudaError_t launch_branch_dr(const pg_batch* b, const pg_state* s, const float* ctrl, const float* dr, int n_substeps,
                             cudaStream_t st) {
  return launch_branch_range(nullptr, b->branch_kernel_dr, b->branch_lanes, 0, s->n, s, ctrl, n_substeps, st, nullptr,
                             b->nslot_max, nullptr, 0, 0, 0, b->envs_per_cta_req, b->hfield_ptr[0], dr);
}

cudaError_t launch_branch_tape(const pg_batch* b, const pg_state* s, const float* ctrl, int n_substeps, float* tape,
                               int tape_rows, cudaStream_t st) {
  return launch_branch_range(nullptr, b->branch_kernel_tape, b->branch_lanes, 0, s->n, s, ctrl, n_substeps, st,
                             nullptr, b->nslot_max, tape, tape_rows, b->nq_max, b->nv_max, b->envs_per_cta_req,
                             b->hfield_ptr[0]);
}

}  // namespace pg
