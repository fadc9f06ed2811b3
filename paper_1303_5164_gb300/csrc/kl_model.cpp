// Host implementation of the performance model (Section 4.4), pruning
// (Section 4.3) and the greedy co-schedule planner (Algorithm 1).
//
// Model, in the paper's terms:
//   * One warp scheduler = one virtual SM: warps, blocks and bandwidth of the
//     SM divided by the scheduler count (Section 4.4, multiple schedulers).
//   * Warps are ready or idle; with the uncoalesced extension idle splits into
//     idle-coalesced / idle-uncoalesced, each with its own latency.
//   * A Markov step is one round: each ready warp issues one instruction; the
//     round lasts (ready warps) cycles, or 1 cycle when none is ready.
//   * Ready -> idle with probability R_m (split by the uncoalesced fraction);
//     idle -> ready with probability min(1, round / L).
//   * L of a class = L0 + b0 + a0 * (sectors per instruction of the class) *
//     (idle warps of the state) / (DRAM sectors per cycle of the virtual SM):
//     the linear contention model, read as the bandwidth shared among the
//     outstanding requests.
//   * Joint state = tuple of per-kernel states; transition = product of the
//     per-kernel transitions (kernels are independent).
//   * Steady state by GTH elimination; IPC_k = E[ready_k] / E[round length]
//     (Eqs. modelIPC, ipc_k1, ipc_k2); CP (Eq. cp); dT (Eq. executiontime).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernelet.h"

namespace kl {
namespace model {

constexpr double kCpTie = 1e-12;
constexpr double kDtTie = 1e-9;

// Next-state distribution of one kernel, indexed like its local state list.
struct LocalStates {
  int w = 0;
  bool three = false;
  // local state k -> (idle coalesced, idle uncoalesced)
  std::vector<int> ic, iu;
  std::vector<int> index;  // (ic * (w+1) + iu) -> local id, -1 if invalid
  void init(int w_, bool three_) {
    w = w_;
    three = three_;
    ic.clear();
    iu.clear();
    index.assign((w + 1) * (w + 1), -1);
    for (int c = 0; c <= w; ++c)
      for (int u = 0; u <= (three ? w - c : 0); ++u) {
        index[c * (w + 1) + u] = (int)ic.size();
        ic.push_back(c);
        iu.push_back(u);
      }
  }
  int size() const { return (int)ic.size(); }
  int id(int c, int u) const { return index[c * (w + 1) + u]; }
};

static void binomial(int n, double p, std::vector<double>& out) {
  out.assign(n + 1, 0.0);
  if (p <= 0.0) {
    out[0] = 1.0;
    return;
  }
  if (p >= 1.0) {
    out[n] = 1.0;
    return;
  }
  // C(n,x) p^x (1-p)^(n-x) via the recurrence on x
  double q = 1.0 - p, v = std::pow(q, n);
  out[0] = v;
  for (int x = 0; x < n; ++x) {
    v = v * (double)(n - x) / (double)(x + 1) * p / q;
    out[x + 1] = v;
  }
}

static double choose(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

struct KernelIn {
  const kl_profile* p;
  int w;
  bool three;
};

// Distribution of the next local state of kernel k from local state s, given
// the round length d and the idle warps I of the joint state.
static void local_row(const KernelIn& k, const LocalStates& ls, int s, double d, int I, const kl_model_params& g,
                      std::vector<double>& row) {
  const double Bv = g.dram_bytes_per_s / g.sector_bytes / (g.f_sm_hz * g.n_sm * g.n_sched);
  row.assign(ls.size(), 0.0);
  const int c = ls.ic[s], u = ls.iu[s], r = k.w - c - u;
  const double Lc = k.p->L0 + g.b0 + g.a0 * k.p->m_c * I / Bv;
  std::vector<double> wc, wu;
  binomial(c, std::min(1.0, d / Lc), wc);
  if (!k.three) {
    std::vector<double> st;
    binomial(r, k.p->R_m, st);
    for (int x = 0; x <= c; ++x)
      for (int y = 0; y <= r; ++y) row[ls.id(c - x + y, 0)] += wc[x] * st[y];
    return;
  }
  const double Lu = k.p->L0 + g.b0 + g.a0 * k.p->m_u * I / Bv;
  binomial(u, std::min(1.0, d / Lu), wu);
  const double pc = k.p->R_m * (1.0 - k.p->f_u), pu = k.p->R_m * k.p->f_u, ps = 1.0 - k.p->R_m;
  for (int yc = 0; yc <= r; ++yc)
    for (int yu = 0; yu + yc <= r; ++yu) {
      const double pm = choose(r, yc) * choose(r - yc, yu) * std::pow(pc, yc) * std::pow(pu, yu) *
                        std::pow(ps, r - yc - yu);
      if (pm == 0.0) continue;
      for (int xc = 0; xc <= c; ++xc) {
        if (wc[xc] == 0.0) continue;
        for (int xu = 0; xu <= u; ++xu) {
          if (wu[xu] == 0.0) continue;
          row[ls.id(c - xc + yc, u - xu + yu)] += pm * wc[xc] * wu[xu];
        }
      }
    }
}

// GTH (Grassmann-Taqqu-Heyman) stationary vector of a row-stochastic n x n
// matrix (destroyed). Returns false if a state cannot reach a lower one.
static bool gth(std::vector<double>& P, int n, std::vector<double>& pi) {
  for (int k = n - 1; k >= 1; --k) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += P[(size_t)k * n + j];
    if (!(s > 0.0)) return false;
    for (int i = 0; i < k; ++i) P[(size_t)i * n + k] /= s;
    for (int i = 0; i < k; ++i) {
      const double f = P[(size_t)i * n + k];
      if (f == 0.0) continue;
      double* Pi = &P[(size_t)i * n];
      const double* Pk = &P[(size_t)k * n];
      for (int j = 0; j < k; ++j) Pi[j] += f * Pk[j];
    }
  }
  pi.assign(n, 0.0);
  pi[0] = 1.0;
  double tot = 1.0;
  for (int k = 1; k < n; ++k) {
    double v = 0.0;
    for (int i = 0; i < k; ++i) v += pi[i] * P[(size_t)i * n + k];
    pi[k] = v;
    tot += v;
  }
  for (double& v : pi) v /= tot;
  return true;
}

// Per-kernel IPC on one virtual SM. Returns 0 or a negative kl_status.
int ipc(const kl_model_params& g, const kl_profile* const* profiles, const int* warps, int nk, int states,
        double* out) {
  if (nk < 1 || nk > 4) return KL_EINVAL;
  std::vector<KernelIn> ks(nk);
  std::vector<LocalStates> ls(nk);
  size_t n = 1;
  for (int k = 0; k < nk; ++k) {
    if (warps[k] < 0 || warps[k] > 64) return KL_EINVAL;
    const kl_profile* p = profiles[k];
    if (!(p->R_m >= 0.0 && p->R_m <= 1.0) || !(p->f_u >= 0.0 && p->f_u <= 1.0) || !(p->L0 >= 0.0))
      return KL_EINVAL;
    ks[k] = KernelIn{p, warps[k], states == 3 && p->f_u > 0.0};
    ls[k].init(warps[k], ks[k].three);
    n *= (size_t)ls[k].size();
    if (n > 4096) return KL_EINVAL;
  }
  // joint state id = mixed radix over the kernels' local ids (kernel 0 fastest)
  std::vector<int> radix(nk);
  for (int k = 0; k < nk; ++k) radix[k] = ls[k].size();
  std::vector<double> P(n * n, 0.0), ready(n * nk), dur(n);
  std::vector<std::vector<double>> rows(nk);
  std::vector<int> loc(nk);
  for (size_t s = 0; s < n; ++s) {
    size_t t = s;
    int I = 0, R = 0;
    for (int k = 0; k < nk; ++k) {
      loc[k] = (int)(t % radix[k]);
      t /= radix[k];
      const int idle = ls[k].ic[loc[k]] + ls[k].iu[loc[k]];
      I += idle;
      R += ks[k].w - idle;
      ready[s * nk + k] = ks[k].w - idle;
    }
    const double d = R > 0 ? (double)R : 1.0;
    dur[s] = d;
    for (int k = 0; k < nk; ++k) local_row(ks[k], ls[k], loc[k], d, I, g, rows[k]);
    // product of the per-kernel rows over every combination of next states
    std::vector<int> nx(nk, 0);
    for (;;) {
      double pr = 1.0;
      size_t id = 0, mul = 1;
      for (int k = 0; k < nk; ++k) {
        pr *= rows[k][nx[k]];
        id += (size_t)nx[k] * mul;
        mul *= radix[k];
      }
      if (pr != 0.0) P[s * n + id] += pr;
      int k = 0;
      while (k < nk && ++nx[k] == radix[k]) nx[k++] = 0;
      if (k == nk) break;
    }
  }
  std::vector<double> pi;
  if (!gth(P, (int)n, pi)) return KL_EINVAL;
  double den = 0.0;
  for (size_t s = 0; s < n; ++s) den += pi[s] * dur[s];
  for (int k = 0; k < nk; ++k) {
    double num = 0.0;
    for (size_t s = 0; s < n; ++s) num += pi[s] * ready[s * nk + k];
    out[k] = num / den;
  }
  return KL_OK;
}

int warps_on_vsm(uint32_t blocks, uint32_t warps_per_block, uint32_t n_sched) {
  if (blocks == 0) return 0;
  int w = (int)std::floor((double)blocks * warps_per_block / n_sched + 0.5);
  return std::max(1, w);
}

double cp(double ca, double ia, double cb, double ib) { return 1.0 - 1.0 / (ca / ia + cb / ib); }

// Split order: min dT (Eq. executiontime) for the balanced policy, max CP
// for max-CP; values equal within rounding (dT 1e-9 relative, CP 1e-12) tie,
// and ties go to the larger CP, then the more even split, then more K1 slots.
bool split_better(uint32_t policy, uint32_t a, uint32_t b, double cp_e, double dT_e, uint32_t ba, uint32_t bb,
                  double cp_b, double dT_b) {
  if (policy != KL_RATIO_MAX_CP) {
    const double scale = std::max(dT_e, dT_b);
    if (std::fabs(dT_e - dT_b) > kDtTie * scale) return dT_e < dT_b;
  }
  if (std::fabs(cp_e - cp_b) > kCpTie) return cp_e > cp_b;
  const uint32_t ue = a > b ? a - b : b - a, ub = ba > bb ? ba - bb : bb - ba;
  if (ue != ub) return ue < ub;
  return a > ba;
}

// Pair evaluation over every split; arrays sized slots-1, index a-1.
int pair(const kl_model_params& g, const kl_profile& pa, const kl_profile& pb, uint32_t slots, int states,
         uint32_t policy, uint32_t fixed_a, double* cA, double* cB, double* cpv, double* dT, double* solo,
         uint32_t* best_a) {
  if (slots < 2) return KL_EINVAL;
  const kl_profile* pp[2] = {&pa, &pb};
  double ia, ib;
  int w = warps_on_vsm(slots, pa.warps_per_block, g.n_sched);
  int rc = ipc(g, pp, &w, 1, states, &ia);
  if (rc) return rc;
  w = warps_on_vsm(slots, pb.warps_per_block, g.n_sched);
  rc = ipc(g, pp + 1, &w, 1, states, &ib);
  if (rc) return rc;
  ia *= g.n_sched;
  ib *= g.n_sched;
  solo[0] = ia;
  solo[1] = ib;
  uint32_t best = 0;
  for (uint32_t a = 1; a < slots; ++a) {
    const uint32_t b = slots - a;
    int ww[2] = {warps_on_vsm(a, pa.warps_per_block, g.n_sched), warps_on_vsm(b, pb.warps_per_block, g.n_sched)};
    double o[2];
    rc = ipc(g, pp, ww, 2, states, o);
    if (rc) return rc;
    const int i = (int)a - 1;
    cA[i] = o[0] * g.n_sched;
    cB[i] = o[1] * g.n_sched;
    cpv[i] = cp(cA[i], ia, cB[i], ib);
    dT[i] = std::fabs(pa.I_block * (double)(a * g.n_sm) / cA[i] - pb.I_block * (double)(b * g.n_sm) / cB[i]);
    if (best == 0 || split_better(policy, a, slots - a, cpv[i], dT[i], best, slots - best, cpv[best - 1],
                                  dT[best - 1]))
      best = a;
  }
  if (policy == KL_RATIO_FIXED) best = std::min(std::max(fixed_a, 1u), slots - 1);
  *best_a = best;
  return KL_OK;
}

// A phase of n kernels sharing each SM, kernel k on slots[k] of its slots
// (Section 2.2: a co-schedule runs n >= 1 slices at once; the heterogeneous
// chain of Section 4.4 extends to more than two kernels): the concurrent IPC
// per SM of each, its solo IPC at `total` slots (full occupancy), and CP by
// Eq. cp with n terms. A kernel with no slot has IPC 0 and adds nothing.
int phase(const kl_model_params& g, const kl_profile* const* pp, const uint32_t* slots, int n, uint32_t total,
          int states, double* cipc, double* solo, double* cpv) {
  if (n < 1 || n > 4 || total < 1) return KL_EINVAL;
  int w[4];
  uint32_t used = 0;
  for (int k = 0; k < n; ++k) {
    w[k] = warps_on_vsm(slots[k], pp[k]->warps_per_block, g.n_sched);
    used += slots[k];
  }
  if (used > total) return KL_EINVAL;
  double o[4];
  int rc = ipc(g, pp, w, n, states, o);
  if (rc) return rc;
  double sum = 0.0;
  for (int k = 0; k < n; ++k) {
    int ws = warps_on_vsm(total, pp[k]->warps_per_block, g.n_sched);
    double v;
    rc = ipc(g, pp + k, &ws, 1, states, &v);
    if (rc) return rc;
    solo[k] = v * g.n_sched;
    cipc[k] = o[k] * g.n_sched;
    if (solo[k] > 0.0) sum += cipc[k] / solo[k];
  }
  *cpv = sum > 0.0 ? 1.0 - 1.0 / sum : 0.0;
  return KL_OK;
}

bool pruned(double pur_a, double mur_a, double pur_b, double mur_b, double ap, double am) {
  if (ap < 0.0 || am < 0.0) return false;
  return std::fabs(pur_a - pur_b) < ap && std::fabs(mur_a - mur_b) < am;
}

}  // namespace model
}  // namespace kl

using namespace kl;

extern "C" int kl_model_ipc(const kl_model_params* gp, const kl_profile* profiles, const uint32_t* warps,
                            uint32_t n, uint32_t model_states, double* ipc_out) {
  if (!gp || !profiles || !warps || !ipc_out || n < 1 || n > 4) return KL_EINVAL;
  if (model_states != 2 && model_states != 3) return KL_EINVAL;
  const kl_profile* pp[4];
  int w[4];
  for (uint32_t k = 0; k < n; ++k) {
    pp[k] = &profiles[k];
    w[k] = (int)warps[k];
  }
  double v[4];
  int rc = model::ipc(*gp, pp, w, (int)n, (int)model_states, v);
  if (rc) return rc;
  for (uint32_t k = 0; k < n; ++k) ipc_out[k] = v[k] * gp->n_sched;
  return KL_OK;
}

extern "C" int kl_model_pair(const kl_model_params* gp, const kl_profile* pa, const kl_profile* pb,
                             uint32_t slots, uint32_t model_states, uint32_t policy, uint32_t fixed_a,
                             double* cipc_a, double* cipc_b, double* cp, double* dT, double* solo_ipc,
                             uint32_t* best_a) {
  if (!gp || !pa || !pb || !cipc_a || !cipc_b || !cp || !dT || !solo_ipc || !best_a) return KL_EINVAL;
  if (slots < 2 || slots > KL_MAX_SLOTS || (model_states != 2 && model_states != 3) || policy > 2)
    return KL_EINVAL;
  return model::pair(*gp, *pa, *pb, slots, (int)model_states, policy, fixed_a, cipc_a, cipc_b, cp, dT, solo_ipc,
                     best_a);
}

extern "C" int kl_model_phase(const kl_model_params* gp, const kl_profile* profiles, const uint32_t* slots,
                              uint32_t n, uint32_t total_slots, uint32_t model_states, double* cipc_out,
                              double* solo_out, double* cp_out) {
  if (!gp || !profiles || !slots || !cipc_out || !solo_out || !cp_out || n < 1 || n > 4) return KL_EINVAL;
  if (total_slots < 1 || total_slots > KL_MAX_SLOTS || (model_states != 2 && model_states != 3)) return KL_EINVAL;
  const kl_profile* pp[4];
  for (uint32_t k = 0; k < n; ++k) pp[k] = &profiles[k];
  return model::phase(*gp, pp, slots, (int)n, total_slots, (int)model_states, cipc_out, solo_out, cp_out);
}

extern "C" int kl_count_pruned(const double* pur, const double* mur, uint32_t n, double ap, double am,
                               uint32_t* out) {
  if (!pur || !mur || !out) return KL_EINVAL;
  uint32_t c = 0;
  for (uint32_t i = 0; i < n; ++i)
    for (uint32_t j = i + 1; j < n; ++j) c += model::pruned(pur[i], mur[i], pur[j], mur[j], ap, am);
  *out = c;
  return KL_OK;
}

// Greedy plan (Algorithm 1) simulated with model rates: a kernel with
// per-SM IPC c advances c * n_sm / I_block blocks per cycle.
extern "C" int kl_plan(const kl_model_params* gp, const kl_profile* tp, uint32_t n_types, const uint32_t* types,
                       const uint64_t* blocks, uint32_t n, uint32_t slots, uint32_t model_states, uint32_t policy,
                       double alpha_p, double alpha_m, kl_phase* phases, double* phase_cycles, uint32_t cap,
                       uint32_t* n_phases, double* makespan) {
  if (!gp || !tp || !types || !blocks || !n_phases || !makespan || slots < 2 || slots > KL_MAX_SLOTS)
    return KL_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (types[i] >= n_types || !tp[types[i]].valid) return KL_EINVAL;
  // per type pair: balanced split and rates (cached)
  const uint32_t T = n_types;
  std::vector<double> cpt(T * T, 0.0), ca(T * T, 0.0), cb(T * T, 0.0), solo(T, 0.0);
  std::vector<uint32_t> sa(T * T, 0);
  std::vector<char> have(T * T, 0), have_solo(T, 0);
  std::vector<double> a1(slots), b1(slots), c1(slots), d1(slots);
  auto eval = [&](uint32_t ta, uint32_t tb) -> int {
    const uint32_t k = ta * T + tb;
    if (have[k]) return 0;
    double so[2];
    uint32_t best;
    int rc = model::pair(*gp, tp[ta], tp[tb], slots, (int)model_states, policy, slots / 2, a1.data(), b1.data(),
                         c1.data(), d1.data(), so, &best);
    if (rc) return rc;
    have[k] = 1;
    sa[k] = best;
    cpt[k] = c1[best - 1];
    ca[k] = a1[best - 1];
    cb[k] = b1[best - 1];
    solo[ta] = so[0];
    solo[tb] = so[1];
    have_solo[ta] = have_solo[tb] = 1;
    return 0;
  };
  auto solo_ipc = [&](uint32_t t) -> double {
    if (!have_solo[t]) {
      int w = model::warps_on_vsm(slots, tp[t].warps_per_block, gp->n_sched);
      const kl_profile* pp = &tp[t];
      double v = 0.0;
      if (model::ipc(*gp, &pp, &w, 1, (int)model_states, &v) == 0) solo[t] = v * gp->n_sched;
      have_solo[t] = 1;
    }
    return solo[t];
  };
  std::vector<double> rem(n);
  std::vector<uint32_t> R;
  for (uint32_t i = 0; i < n; ++i) {
    rem[i] = (double)blocks[i];
    if (blocks[i] > 0) R.push_back(i);
  }
  uint32_t np = 0;
  double total = 0.0;
  while (!R.empty()) {
    kl_phase ph{};
    double dur;
    if (R.size() == 1) {
      const uint32_t a = R[0];
      const double rate = solo_ipc(types[a]) * gp->n_sm / tp[types[a]].I_block;
      dur = rem[a] / rate;
      rem[a] = 0.0;
      R.clear();
      ph.A = (int32_t)a;
      ph.B = -1;
      ph.slots_a = slots;
    } else {
      // FindCoSchedule: candidate pairs, prune (fall back to all), argmax CP
      int32_t bi = -1, bj = -1;
      double best = 0.0;
      for (int pass = 0; pass < 2 && bi < 0; ++pass)
        for (size_t x = 0; x < R.size(); ++x)
          for (size_t y = x + 1; y < R.size(); ++y) {
            const uint32_t i = std::min(R[x], R[y]), j = std::max(R[x], R[y]);
            const kl_profile &pi_ = tp[types[i]], &pj = tp[types[j]];
            if (pass == 0 && model::pruned(pi_.PUR, pi_.MUR, pj.PUR, pj.MUR, alpha_p, alpha_m)) continue;
            int rc = eval(types[i], types[j]);
            if (rc) return rc;
            const double c = cpt[types[i] * T + types[j]];
            // pairs are visited in ascending (i, j); a CP tie keeps the earlier one
            if (bi < 0 || c > best + model::kCpTie) {
              best = c;
              bi = (int32_t)i;
              bj = (int32_t)j;
            }
          }
      const uint32_t k = types[bi] * T + types[bj];
      const double rA = ca[k] * gp->n_sm / tp[types[bi]].I_block;
      const double rB = cb[k] * gp->n_sm / tp[types[bj]].I_block;
      const double tA = rem[bi] / rA, tB = rem[bj] / rB;
      dur = std::min(tA, tB);
      rem[bi] -= dur * rA;
      rem[bj] -= dur * rB;
      if (tA <= tB) {
        rem[bi] = 0.0;
        R.erase(std::find(R.begin(), R.end(), (uint32_t)bi));
      }
      if (tB <= tA) {
        rem[bj] = 0.0;
        R.erase(std::find(R.begin(), R.end(), (uint32_t)bj));
      }
      ph.A = bi;
      ph.B = bj;
      ph.slots_a = sa[k];
      ph.slots_b = slots - sa[k];
      ph.cp = best;
    }
    if (phases && np < cap) {
      phases[np] = ph;
      if (phase_cycles) phase_cycles[np] = dur;
    }
    ++np;
    total += dur;
  }
  *n_phases = np;
  *makespan = total;
  return KL_OK;
}
