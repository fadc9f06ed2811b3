// Host runtime behind the C ABI: the pending set R, admission, the CP table
// the device planner reads, launch of the persistent co-scheduler (or of the
// plain-launch baselines), completion tracking and statistics.
//
// Algorithm 1 split between host and device: the host adds arriving kernels
// to R (kl_submit) and evaluates the performance model once per set of kernel
// types (the paper re-uses a kernel's earlier slice size when it was submitted
// before; here the CP / balanced-split table per type pair is cached the same
// way); FindCoSchedule and the "repeat the co-schedule until a kernel runs out"
// loop run on the device (kl_cosched.cu).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kernelet.h"
#include "kl_internal.h"
#include "tenants.cuh"

namespace kl {
int cosched_occupancy(int* ctas_per_sm, int build);
int cosched_launch(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t n_sm, uint32_t slots, uint32_t smem_bytes,
                   int build, cudaStream_t stream, uint32_t extra_ctas = 0);
int native_launch_tenant(uint32_t type, const void* args, cudaStream_t s);
int stage_copy(const CopySeg* segs, uint32_t n, cudaStream_t s);
int class_launch(int type, TenantDev* T, RunDev* R, uint32_t grid, cudaStream_t stream);
namespace model {
int pair(const kl_model_params& g, const kl_profile& pa, const kl_profile& pb, uint32_t slots, int states,
         uint32_t policy, uint32_t fixed_a, double* cA, double* cB, double* cpv, double* dT, double* solo,
         uint32_t* best_a);
int phase(const kl_model_params& g, const kl_profile* const* pp, const uint32_t* slots, int n, uint32_t total,
          int states, double* cipc, double* solo, double* cpv);
bool pruned(double pur_a, double mur_a, double pur_b, double mur_b, double ap, double am);
}  // namespace model
}  // namespace kl

using namespace kl;

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t args_size_of(uint32_t type) {
  switch (type) {
    case KL_T_GATHER: return sizeof(kl_args_gather);
    case KL_T_BLACKSCHOLES: return sizeof(kl_args_blackscholes);
    case KL_T_GEMM_F32: return sizeof(kl_args_gemm_f32);
    case KL_T_SPMV_CSR: return sizeof(kl_args_spmv_csr);
    case KL_T_PCHASE: return sizeof(kl_args_pchase);
    case KL_T_TRIAD: return sizeof(kl_args_triad);
    case KL_T_HIST256: return sizeof(kl_args_hist256);
    case KL_T_ESCAPE: return sizeof(kl_args_escape);
    case KL_T_BITONIC: return sizeof(kl_args_bitonic);
    case KL_T_MATADD: return sizeof(kl_args_matadd);
    case KL_T_GEMM_BF16: return sizeof(kl_args_gemm_bf16);
    case KL_T_TEA: return sizeof(kl_args_tea);
    case KL_T_SAD: return sizeof(kl_args_sad);
    case KL_T_STENCIL: return sizeof(kl_args_stencil);
    case KL_T_MRIQ: return sizeof(kl_args_mriq);
    case KL_T_TESTMIX: return sizeof(kl_args_testmix);
    case KL_T_BS255: return sizeof(kl_args_blackscholes);
    case KL_T_HIST1024: return sizeof(kl_args_hist256);
    case KL_T_GEMM_F32_BIG: return sizeof(kl_args_gemm_f32);
    default: return 0;
  }
}

bool a16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Argument checks a plain launch of the tenant would need to be safe.
int validate_args(uint32_t type, const void* a) {
  switch (type) {
    // the resource-heavy variants take their base type's arguments
    case KL_T_BS255: return validate_args(KL_T_BLACKSCHOLES, a);
    case KL_T_HIST1024: return validate_args(KL_T_HIST256, a);
    case KL_T_GEMM_F32_BIG: return validate_args(KL_T_GEMM_F32, a);
    case KL_T_TESTMIX: {
      const kl_args_testmix* t = (const kl_args_testmix*)a;
      if (!t->in || !t->out || t->n_in == 0 || (t->n_in & (t->n_in - 1)) || t->nthreads == 0) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_GATHER: {
      const kl_args_gather* g = (const kl_args_gather*)a;
      if (!g->a || !g->idx || !g->out || g->n == 0 || !a16(g->idx) || !a16(g->out)) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_BLACKSCHOLES: {
      const kl_args_blackscholes* b = (const kl_args_blackscholes*)a;
      if (!b->S || !b->K || !b->r || !b->v || !b->T || !b->call || !b->put || b->n == 0) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_GEMM_F32: {
      const kl_args_gemm_f32* g = (const kl_args_gemm_f32*)a;
      if (!g->A || !g->B || !g->C || g->M == 0 || g->N == 0 || g->K == 0) return KL_EINVAL;
      if (g->N % 4 || g->K % 4 || !a16(g->A) || !a16(g->B) || !a16(g->C)) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_SPMV_CSR: {
      const kl_args_spmv_csr* s = (const kl_args_spmv_csr*)a;
      if (!s->rowptr || !s->col || !s->val || !s->x || !s->y || s->nrows == 0 || s->ncols == 0) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_PCHASE: {
      const kl_args_pchase* p = (const kl_args_pchase*)a;
      if (!p->next || !p->start || !p->end || p->N == 0 || p->nchasers == 0) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_TRIAD: {
      const kl_args_triad* t = (const kl_args_triad*)a;
      if (!t->a || !t->b || !t->c || t->n == 0 || !a16(t->a) || !a16(t->b) || !a16(t->c)) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_HIST256: {
      const kl_args_hist256* h = (const kl_args_hist256*)a;
      if (!h->data || !h->hist || h->n == 0 || !a16(h->data)) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_ESCAPE: {
      const kl_args_escape* e = (const kl_args_escape*)a;
      if (!e->count || e->width == 0 || e->height == 0) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_BITONIC: {
      const kl_args_bitonic* b = (const kl_args_bitonic*)a;
      if (!b->in || !b->out || b->log2n < 1 || b->log2n > 30) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_MATADD: {
      const kl_args_matadd* m = (const kl_args_matadd*)a;
      if (!m->a || !m->b || !m->c || m->n == 0 || m->n % 16) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_GEMM_BF16: {
      const kl_args_gemm_bf16* g = (const kl_args_gemm_bf16*)a;
      if (!g->A || !g->Bt || !g->C || !g->tmaps || g->M == 0 || g->N == 0 || g->K == 0) return KL_EINVAL;
      if (g->K % 8 || g->N % 4 || !a16(g->A) || !a16(g->Bt) || !a16(g->C) || ((uintptr_t)g->tmaps & 63u))
        return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_TEA: {
      const kl_args_tea* t = (const kl_args_tea*)a;
      if (!t->in || !t->out || t->n == 0 || !a16(t->in) || !a16(t->out)) return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_SAD: {
      const kl_args_sad* d = (const kl_args_sad*)a;
      if (!d->cur || !d->ref || !d->sad || d->width < 4 || d->height < 4 || d->width % 4 || d->height % 4 ||
          d->range < 1 || d->range > 16)
        return KL_EINVAL;
      return KL_OK;
    }
    case KL_T_STENCIL: {
      const kl_args_stencil* t = (const kl_args_stencil*)a;
      if (!t->in || !t->out || t->nx == 0 || t->ny == 0 || t->nz == 0) return KL_EINVAL;
      if ((uint64_t)t->nx * t->ny * t->nz >= (1ull << 32)) return KL_EINVAL;  // 32-bit point index
      return KL_OK;
    }
    case KL_T_MRIQ: {
      const kl_args_mriq* m = (const kl_args_mriq*)a;
      if (!m->kx || !m->ky || !m->kz || !m->phiR || !m->phiI || !m->phiMag || !m->x || !m->y || !m->z || !m->Qr ||
          !m->Qi || m->numK == 0 || m->numX == 0)
        return KL_EINVAL;
      return KL_OK;
    }
    default: return KL_EINVAL;
  }
}

// Built-in model inputs used until measured profiles are loaded: rough
// instruction mixes by construction of each tenant body (flagged as such by
// kl_profile.valid = 2).
kl_profile builtin_profile(uint32_t type) {
  kl_profile p{};
  p.m_c = 4.0;
  p.m_u = 32.0;
  p.warps_per_block = 8;
  p.valid = 2;
  switch (type) {
    case KL_T_GATHER: p.R_m = 0.30; p.f_u = 0.8; p.L0 = 900; p.I_block = 8 * 40; p.PUR = 0.05; p.MUR = 0.50; break;
    case KL_T_BLACKSCHOLES: p.R_m = 0.03; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 300; p.PUR = 0.60; p.MUR = 0.30; break;
    case KL_T_GEMM_F32: p.R_m = 0.01; p.f_u = 0.0; p.L0 = 700; p.I_block = 8 * 40000; p.PUR = 0.80; p.MUR = 0.05; break;
    case KL_T_SPMV_CSR: p.R_m = 0.25; p.f_u = 0.5; p.L0 = 900; p.I_block = 8 * 120; p.PUR = 0.15; p.MUR = 0.60; break;
    case KL_T_PCHASE: p.R_m = 0.30; p.f_u = 1.0; p.L0 = 1000; p.I_block = 8 * 1000; p.PUR = 0.01; p.MUR = 0.10; break;
    case KL_T_TRIAD: p.R_m = 0.20; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 60; p.PUR = 0.05; p.MUR = 0.90; break;
    case KL_T_HIST256: p.R_m = 0.05; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 600; p.PUR = 0.40; p.MUR = 0.40; break;
    case KL_T_ESCAPE: p.R_m = 0.001; p.f_u = 0.0; p.L0 = 700; p.I_block = 8 * 1500; p.PUR = 0.70; p.MUR = 0.01; break;
    case KL_T_BITONIC: p.R_m = 0.10; p.f_u = 0.0; p.L0 = 500; p.I_block = 8 * 400; p.PUR = 0.30; p.MUR = 0.30; break;
    case KL_T_MATADD: p.R_m = 0.25; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 12; p.PUR = 0.05; p.MUR = 0.70; break;
    case KL_T_GEMM_BF16: p.R_m = 0.02; p.f_u = 0.0; p.L0 = 700; p.I_block = 8 * 200; p.PUR = 0.10; p.MUR = 0.10; break;
    case KL_T_TEA: p.R_m = 0.002; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 1600; p.PUR = 0.90; p.MUR = 0.05; break;
    case KL_T_SAD: p.R_m = 0.25; p.f_u = 0.3; p.L0 = 500; p.I_block = 8 * 150; p.PUR = 0.40; p.MUR = 0.10; break;
    case KL_T_STENCIL: p.R_m = 0.2; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 60; p.PUR = 0.20; p.MUR = 0.60; break;
    case KL_T_MRIQ: p.R_m = 0.001; p.f_u = 0.0; p.L0 = 500; p.I_block = 8 * 20000; p.PUR = 0.85; p.MUR = 0.01; break;
    case KL_T_TESTMIX: p.R_m = 0.10; p.f_u = 0.0; p.L0 = 900; p.I_block = 8 * 400; p.PUR = 0.40; p.MUR = 0.40; break;
    case KL_T_BS255: p = builtin_profile(KL_T_BLACKSCHOLES); p.warps_per_block = 4; p.I_block *= 8; break;
    case KL_T_HIST1024: p = builtin_profile(KL_T_HIST256); p.warps_per_block = 32; p.I_block *= 16; break;
    case KL_T_GEMM_F32_BIG: p = builtin_profile(KL_T_GEMM_F32); p.I_block *= 16; break;
    default: p.valid = 0; break;
  }
  return p;
}

struct Pending {
  TenantDev td;
  uint64_t footprint;
  uint64_t t_submit;
  kl_handle handle;
  bool caller_slice;     // the descriptor set slice_blocks (never resized)
  uint32_t slice_alone;  // the least its slice shrinks to (the type's alone-tuned slice)
};

struct Record {
  kl_tenant_stats st{};
  kl_handle handle = 0;
};

enum RunKind { kNone = 0, kCosched = 1, kBaseline = 2, kServe = 3, kServeBase = 4 };

// One kernel of a serving run, by sequence number.
struct ServeRec {
  uint64_t t_submit;
  uint64_t footprint;
  uint64_t t_done_host;
  uint32_t state;    // KL_RUNNING until reaped
  uint32_t total;    // thread blocks
  ServeDone done;    // device record (co-scheduled serving)
};

uint32_t pow2_at_least(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return (uint32_t)p;
}

}  // namespace

struct kl_runtime {
  std::mutex mu;
  kl_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  uint32_t n_sm = 0, slots = 0, occupancy = 0;
  uint32_t slots_light = 0;   // CTAs per SM of the light build (0: not used)
  uint32_t flight_slots = 0;  // CTAs per SM of the in-flight / last run
  uint32_t cap = 0, cap_phases = 0;
  uint32_t ring_slots = 0, phase_slots = 0;  // powers of two >= cap, cap_phases
  TenantDev* d_tenants = nullptr;
  RunDev* d_run = nullptr;
  PhaseDev* d_phases = nullptr;
  TenantDev* h_tenants = nullptr;
  RunDev* h_run = nullptr;
  PhaseDev* h_phases = nullptr;
  TenantDev* hd_tenants = nullptr;  // device addresses of the three pinned buffers above
  RunDev* hd_run = nullptr;
  PhaseDev* hd_phases = nullptr;
  std::vector<Pending> pending;
  uint64_t pending_footprint = 0;
  uint64_t run_id = 1;       // id of the run the pending set will become
  // in-flight / last run
  int kind = kNone;
  bool in_flight = false;
  uint64_t flight_id = 0;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;   // around the persistent launch
  std::vector<Pending> flight;      // tenants of the in-flight run
  std::vector<cudaEvent_t> tenant_ev;  // baseline per-tenant completion events
  std::map<uint64_t, std::vector<Record>> history;  // retired runs (last few)
  kl_run_stats last{};
  std::vector<kl_phase> last_phases;
  // model
  kl_model_params mp{};
  kl_profile prof[KL_T_COUNT];
  bool table_valid = false;
  bool table_override = false;  // kl_set_cp_table: measured CPs instead of the model
  uint32_t table_slots = 0;     // slots per SM the cached table was computed for
  int table_chain = -1;         // chain-lane type of the cached table (KL_CFG_PHASE_MODEL)
  double cp[KL_T_COUNT][KL_T_COUNT];
  uint32_t slots_a[KL_T_COUNT][KL_T_COUNT];
  uint32_t allowed[KL_T_COUNT][KL_T_COUNT];
  uint32_t table_types = 0;  // bit mask of types in the cached table
  // baselines
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_join;
  cudaEvent_t ev_fork = nullptr;
  // serving (kind kServe: persistent kernel fed through mapped memory;
  // kServeBase: one plain launch per arrival on stream seq % s_nstreams)
  bool serve_on = false;            // between kl_serve_start and kl_serve_stop
  int serve_mode = 0;
  uint32_t s_ring = 0, s_phase_slots = 0;
  TenantDev* sd_ring = nullptr;     // device tenant ring
  PhaseDev* sd_phases = nullptr;    // device phase ring
  PhaseDev* sh_phases = nullptr;    // pinned copy of the phase ring after the run
  TenantDev* sm_ring = nullptr;     // mapped: descriptors the host publishes
  uint32_t* sm_ctl = nullptr;       // mapped: [0] tail, [32] stop request
  ServeDone* sm_done = nullptr;     // mapped: completion records
  unsigned long long* sm_cq = nullptr;  // mapped: completion queue
  TenantDev* sdm_ring = nullptr;    // device addresses of the mapped buffers
  uint32_t* sdm_ctl = nullptr;
  ServeDone* sdm_done = nullptr;
  unsigned long long* sdm_cq = nullptr;
  uint32_t s_tail = 0, s_head = 0, s_inflight = 0, s_nstreams = 0;
  uint32_t s_published = 0;         // kernels [0, s_published) are visible to the device / launched
  std::vector<TenantDev> s_staged;  // kServeBase: staged descriptors not yet launched, in order
  uint64_t s_footprint = 0;
  std::vector<ServeRec> s_recs;
  std::vector<std::deque<std::pair<uint32_t, cudaEvent_t>>> s_stream_q;  // kServeBase
  std::vector<cudaEvent_t> s_free_ev;
  std::deque<kl_handle> completed;  // serving: handles completed, not yet returned by kl_reap
  bool s_joined = false;            // kServeBase: side streams joined and ev_done recorded
};

namespace {

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? KL_OK : KL_ECUDA; }

kl_handle make_handle(uint64_t run, uint32_t idx) { return (run << 32) | (uint64_t)(idx + 1u); }
void split_handle(kl_handle h, uint64_t* run, uint32_t* idx) {
  *run = h >> 32;
  *idx = (uint32_t)(h & 0xffffffffu) - 1u;
}

// CP table for every pair of types in `mask` (Section 4.4 model + Section 4.3
// pruning). Cached until profiles, parameters or the type set change.
// chain: with KL_CFG_PHASE_MODEL, the multi-stage type the chain lane will run
// beside every pair (-1: none); the table then holds each pair's CP as the
// three-kernel phase the device runs (pair on S - chain_slots slots, that
// type on the chain lane), at the split of the pair that maximises it.
int ensure_table(kl_runtime* rt, uint32_t mask, uint32_t S, int chain = -1) {
  if (rt->table_override) return KL_OK;
  mask &= (1u << KL_T_MAIN_COUNT) - 1u;  // the planner pairs the co-scheduler's types only
  const uint32_t cs = std::max(1u, std::min(rt->cfg.chain_slots, S > 1 ? S - 1 : 1u));
  if (chain >= 0 && S < cs + 2) chain = -1;  // no room for a pair beside the lane
  const bool same = rt->table_valid && rt->table_slots == S && rt->table_chain == chain;
  if (same && (rt->table_types & mask) == mask) return KL_OK;
  const uint32_t want = mask | (same ? rt->table_types : 0u);
  std::vector<double> a(S), b(S), c(S), d(S);
  for (uint32_t i = 0; i < KL_T_COUNT; ++i)
    for (uint32_t j = 0; j < KL_T_COUNT; ++j) {
      rt->cp[i][j] = 0.0;
      rt->slots_a[i][j] = S / 2 ? S / 2 : 1;
      rt->allowed[i][j] = 1;
    }
  if (S >= 2) {
    for (uint32_t i = 0; i < KL_T_COUNT; ++i) {
      if (!(want & (1u << i))) continue;
      for (uint32_t j = 0; j < KL_T_COUNT; ++j) {
        if (!(want & (1u << j))) continue;
        double solo[2];
        uint32_t best = 1;
        int rc = model::pair(rt->mp, rt->prof[i], rt->prof[j], S, (int)rt->cfg.model_states, rt->cfg.ratio_policy,
                             rt->cfg.fixed_slots_a, a.data(), b.data(), c.data(), d.data(), solo, &best);
        if (rc) return rc;
        rt->cp[i][j] = c[best - 1];
        rt->slots_a[i][j] = best;
        if (chain >= 0) {
          const kl_profile* pp[3] = {&rt->prof[i], &rt->prof[j], &rt->prof[chain]};
          double bestcp = -1e300;
          for (uint32_t sa = 1; sa + cs < S; ++sa) {
            const uint32_t sl[3] = {sa, S - cs - sa, cs};
            double ci[3], so[3], cpv = 0.0;
            rc = model::phase(rt->mp, pp, sl, 3, S, (int)rt->cfg.model_states, ci, so, &cpv);
            if (rc) return rc;
            if (cpv > bestcp + 1e-12) {
              bestcp = cpv;
              rt->cp[i][j] = cpv;
              rt->slots_a[i][j] = sa;
            }
          }
        }
        rt->allowed[i][j] = model::pruned(rt->prof[i].PUR, rt->prof[i].MUR, rt->prof[j].PUR, rt->prof[j].MUR,
                                          rt->cfg.alpha_p, rt->cfg.alpha_m)
                                ? 0u
                                : 1u;
      }
    }
  }
  rt->table_types = want;
  rt->table_slots = S;
  rt->table_chain = chain;
  rt->table_valid = true;
  return KL_OK;
}

void record_history(kl_runtime* rt, uint64_t id, std::vector<Record>&& recs) {
  rt->history[id] = std::move(recs);
  while (rt->history.size() > 8) rt->history.erase(rt->history.begin());
}

// Serving: a kernel of the serving run has completed (lock held).
void serve_finish(kl_runtime* rt, uint32_t seq, uint32_t state) {
  ServeRec& r = rt->s_recs[seq];
  r.state = state;
  r.t_done_host = now_ns();
  rt->s_inflight--;
  rt->s_footprint -= r.footprint;
  rt->completed.push_back(make_handle(rt->flight_id, seq));
  while (rt->completed.size() > (1u << 20)) rt->completed.pop_front();
}

// Serving: collect the completions published since the last call (lock held).
// Co-scheduled: completion queue entries in mapped memory, tagged with their
// position so a stale entry is never mistaken for a new one. Plain launches:
// per stream, the oldest outstanding event (kernels of a stream finish in order).
int serve_reap(kl_runtime* rt) {
  if (rt->kind == kServe) {
    const uint32_t mask = rt->s_ring - 1u;
    for (;;) {
      const unsigned long long e = __atomic_load_n(&rt->sm_cq[rt->s_head & mask], __ATOMIC_ACQUIRE);
      if ((uint32_t)(e >> 32) != rt->s_head + 1u) break;
      const uint32_t seq = (uint32_t)e;
      rt->s_head++;
      if (seq >= rt->s_recs.size() || rt->s_recs[seq].state != KL_RUNNING) continue;
      rt->s_recs[seq].done = rt->sm_done[seq & mask];
      serve_finish(rt, seq, KL_DONE);
    }
  } else if (rt->kind == kServeBase) {
    for (auto& q : rt->s_stream_q) {
      while (!q.empty()) {
        cudaError_t e = cudaEventQuery(q.front().second);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return KL_ECUDA;
        serve_finish(rt, q.front().first, KL_DONE);
        rt->s_free_ev.push_back(q.front().second);
        q.pop_front();
      }
    }
  }
  return KL_OK;
}

// Retire a serving run whose stream work has completed (lock held).
int retire_serve(kl_runtime* rt) {
  int run_err = KL_OK;
  serve_reap(rt);
  uint64_t t_launch = 0;
  if (rt->kind == kServe) {
    const RunDev& R = *rt->h_run;
    run_err = R.error;
    t_launch = R.t_launch;
    const uint64_t np = (uint64_t)R.phase_seq + 1;
    const uint64_t first = np > rt->s_phase_slots ? np - rt->s_phase_slots : 0;
    rt->last_phases.clear();
    for (uint64_t k = first; k < np; ++k) {
      const PhaseDev& p = rt->sh_phases[k & (rt->s_phase_slots - 1)];
      kl_phase q{};
      q.A = p.A;
      q.B = p.B;
      q.slots_a = p.slots_a;
      q.slots_b = p.slots_b;
      q.cp = p.cp;
      q.t_ns = p.t;
      q.trigger = p.trigger;
      q.n_pending = p.n_pending;
      q.pending_mask = p.pending;
      q.done_a = p.done_a;
      q.done_b = p.done_b;
      q.prev_done_a = p.prev_done_a;
      q.prev_done_b = p.prev_done_b;
      rt->last_phases.push_back(q);
    }
    rt->last = kl_run_stats{};
    rt->last.n_phases = (uint32_t)std::min<uint64_t>(np, 0xffffffffu);
    rt->last.t_launch_ns = R.t_launch;
    rt->last.t_end_ns = R.t_end;
    rt->last.slot_wait_ns = R.wait_ns;
    rt->last.stage_wait_ns = R.stage_wait_ns;
    rt->last.plan_ns = R.plan_ns;
  } else {
    rt->last = kl_run_stats{};
    rt->last_phases.clear();
  }
  const uint32_t n = (uint32_t)rt->s_recs.size();
  std::vector<Record> recs(n);
  for (uint32_t i = 0; i < n; ++i) {
    ServeRec& s = rt->s_recs[i];
    Record& r = recs[i];
    r.handle = make_handle(rt->flight_id, i);
    r.st.t_submit_ns = s.t_submit;
    r.st.t_done_host_ns = s.t_done_host;
    r.st.t_launch_ns = t_launch;
    if (s.state == KL_DONE) {
      r.st.state = KL_DONE;
      r.st.t_start_ns = s.done.t_start;
      r.st.t_end_ns = s.done.t_end;
      r.st.slices = s.done.slices;
      r.st.blocks = s.done.blocks;
      if (rt->kind == kServeBase) r.st.blocks = s.total;
    } else {
      // admitted but never completed: the run ended on an error (or before the
      // device took the kernel in)
      r.st.state = KL_ERROR;
      r.st.error = run_err ? run_err : KL_ESTATE;
    }
  }
  rt->last.n_tenants = n;
  rt->last.error = run_err;
  rt->last.slots_per_sm = rt->flight_slots;
  rt->last.grid_ctas = rt->flight_slots * rt->n_sm;
  float ms = 0.f;
  rt->last.kernel_ns = cudaEventElapsedTime(&ms, rt->ev_k0, rt->ev_k1) == cudaSuccess ? (uint64_t)((double)ms * 1e6) : 0;
  rt->last.run_ns = cudaEventElapsedTime(&ms, rt->ev_start, rt->ev_done) == cudaSuccess ? (uint64_t)((double)ms * 1e6) : 0;
  record_history(rt, rt->flight_id, std::move(recs));
  rt->s_recs.clear();
  rt->s_recs.shrink_to_fit();
  rt->in_flight = false;
  rt->kind = kNone;
  return run_err;
}

// Move a finished run into the history. Caller holds the lock and has seen
// ev_done complete.
int retire(kl_runtime* rt) {
  if (!rt->in_flight) return KL_OK;
  if (rt->kind == kServe || rt->kind == kServeBase) return retire_serve(rt);
  const uint32_t n = (uint32_t)rt->flight.size();
  std::vector<Record> recs(n);
  int run_err = KL_OK;
  if (rt->kind == kCosched) {
    const RunDev& R = *rt->h_run;
    run_err = R.error;
    uint32_t np = std::min(R.phase_seq + 1, rt->cap_phases);
    rt->last_phases.clear();
    for (uint32_t k = 0; k < np; ++k) {
      const PhaseDev& p = rt->h_phases[k];
      kl_phase q{};
      q.A = p.A;
      q.B = p.B;
      q.slots_a = p.slots_a;
      q.slots_b = p.slots_b;
      q.cp = p.cp;
      q.t_ns = p.t;
      q.trigger = p.trigger;
      q.n_pending = p.n_pending;
      q.pending_mask = p.pending;
      q.done_a = p.done_a;
      q.done_b = p.done_b;
      q.prev_done_a = p.prev_done_a;
      q.prev_done_b = p.prev_done_b;
      rt->last_phases.push_back(q);
    }
    for (uint32_t i = 0; i < n; ++i) {
      const TenantDev& t = rt->h_tenants[i];
      Record& r = recs[i];
      r.handle = rt->flight[i].handle;
      r.st.t_submit_ns = rt->flight[i].t_submit;
      r.st.t_start_ns = t.t_start;
      r.st.t_end_ns = t.t_end;
      r.st.t_launch_ns = R.t_launch;
      r.st.slices = t.slices;
      r.st.blocks = t.done;
      if (t.done == t.total && t.status == KL_DONE) {
        r.st.state = KL_DONE;
      } else {
        r.st.state = KL_ERROR;
        r.st.error = run_err ? run_err : KL_ESTATE;
      }
    }
    rt->last.n_tenants = n;
    rt->last.n_phases = np;
    rt->last.error = run_err;
    rt->last.slots_per_sm = rt->flight_slots;
    rt->last.grid_ctas = rt->flight_slots * rt->n_sm;
    rt->last.t_launch_ns = R.t_launch;
    rt->last.t_end_ns = R.t_end;
    rt->last.slot_wait_ns = R.wait_ns;
    rt->last.stage_wait_ns = R.stage_wait_ns;
    rt->last.plan_ns = R.plan_ns;
    for (int c = 1; c < 4; ++c) rt->last.class_ctas[c] = R.cls_ctas[c];
    float ms = 0.f;
    rt->last.kernel_ns =
        cudaEventElapsedTime(&ms, rt->ev_k0, rt->ev_k1) == cudaSuccess ? (uint64_t)((double)ms * 1e6) : 0;
    rt->last.run_ns =
        cudaEventElapsedTime(&ms, rt->ev_start, rt->ev_done) == cudaSuccess ? (uint64_t)((double)ms * 1e6) : 0;
  } else {
    // baseline: per-tenant completion from events relative to the fork
    for (uint32_t i = 0; i < n; ++i) {
      Record& r = recs[i];
      r.handle = rt->flight[i].handle;
      r.st.state = KL_DONE;
      r.st.t_submit_ns = rt->flight[i].t_submit;
      float ms = 0.f;
      if (i < rt->tenant_ev.size() && cudaEventElapsedTime(&ms, rt->ev_start, rt->tenant_ev[i]) == cudaSuccess)
        r.st.t_end_ns = (uint64_t)((double)ms * 1e6);
      r.st.blocks = (uint32_t)tn::total_blocks(rt->flight[i].td.type, rt->flight[i].td.args);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, rt->ev_start, rt->ev_done);
    rt->last = kl_run_stats{};
    rt->last.n_tenants = n;
    rt->last.t_launch_ns = 0;
    rt->last.t_end_ns = (uint64_t)((double)ms * 1e6);
    rt->last.kernel_ns = rt->last.t_end_ns;
    rt->last.run_ns = rt->last.t_end_ns;
    rt->last_phases.clear();
  }
  record_history(rt, rt->flight_id, std::move(recs));
  rt->flight.clear();
  rt->in_flight = false;
  rt->kind = kNone;
  return run_err;
}

// Non-blocking check of the in-flight run.
int progress(kl_runtime* rt) {
  if (!rt->in_flight) return KL_OK;
  if (rt->kind == kServe || rt->kind == kServeBase) {
    if (serve_reap(rt) != KL_OK) return KL_ECUDA;
    if (rt->kind == kServeBase && !rt->s_joined) return KL_EAGAIN;
  }
  cudaError_t e = cudaEventQuery(rt->ev_done);
  if (e == cudaErrorNotReady) return KL_EAGAIN;
  if (e != cudaSuccess) return KL_ECUDA;
  retire(rt);
  return KL_OK;
}

int wait_flight(kl_runtime* rt, std::unique_lock<std::mutex>& lk, uint64_t timeout_ns) {
  const uint64_t t0 = now_ns();
  for (;;) {
    int rc = progress(rt);
    if (rc != KL_EAGAIN) return rc;
    if (now_ns() - t0 >= timeout_ns) return KL_ETIMEDOUT;
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::microseconds(20));
    lk.lock();
  }
}

// Plain-launch server: join the side streams into the runtime stream and
// record the run's end event (lock held).
int serve_join(kl_runtime* rt) {
  int rc = KL_OK;
  for (uint32_t k = 0; k < rt->s_nstreams && !rc; ++k) {
    rc = cuda_ok(cudaEventRecord(rt->side_join[k], rt->side[k]));
    if (!rc) rc = cuda_ok(cudaStreamWaitEvent(rt->stream, rt->side_join[k], 0));
  }
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k1, rt->stream));
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_done, rt->stream));
  rt->s_joined = true;
  return rc;
}

// A slice never exceeds the kernel, and the queue counter (which can overshoot
// by one slice per CTA when a kernel runs out) stays below 2^32.
uint32_t clamp_slice(const kl_runtime* rt, uint32_t slice, uint32_t total) {
  const uint64_t ctas = (uint64_t)rt->n_sm * std::max(rt->slots, rt->slots_light);
  uint64_t sl = std::min<uint64_t>(slice, total);
  while (sl > 1 && (uint64_t)total + sl * (ctas + 1) >= (1ull << 32)) sl >>= 1;
  return (uint32_t)std::max<uint64_t>(sl, 1);
}

// Serving, plain launches: launch a descriptor on stream seq % nstreams and
// queue its completion event (lock held).
int serve_base_launch(kl_runtime* rt, const TenantDev& td) {
  const uint32_t seq = td.index;
  const uint32_t k = seq % rt->s_nstreams;
  cudaEvent_t e = nullptr;
  if (!rt->s_free_ev.empty()) {
    e = rt->s_free_ev.back();
    rt->s_free_ev.pop_back();
  } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    return KL_ECUDA;
  }
  if (native_launch_tenant(td.type, td.args, rt->side[k]) != 0 || cudaEventRecord(e, rt->side[k]) != cudaSuccess) {
    rt->s_free_ev.push_back(e);
    return KL_ECUDA;
  }
  rt->s_stream_q[k].emplace_back(seq, e);
  return KL_OK;
}

// Serving: make every admitted kernel up to s_tail visible (lock held).
// Co-scheduled: one release store of the new tail into the mapped control
// word; the device's dispatcher copies the descriptors in and re-plans.
// Plain launches: launch the staged descriptors in order.
int serve_flush(kl_runtime* rt) {
  if (rt->s_published == rt->s_tail) return KL_OK;
  if (rt->kind == kServe) {
    __atomic_store_n(&rt->sm_ctl[0], rt->s_tail, __ATOMIC_RELEASE);
  } else {
    for (const TenantDev& td : rt->s_staged) {
      int rc = serve_base_launch(rt, td);
      if (rc) return rc;
    }
    rt->s_staged.clear();
  }
  for (uint32_t q = rt->s_published; q < rt->s_tail; ++q) rt->s_recs[q].state = KL_RUNNING;
  rt->s_published = rt->s_tail;
  return KL_OK;
}

// Serving: admit one kernel to the running server (lock held). Co-scheduled:
// write the descriptor into the mapped ring; plain launches: keep it in order.
// With `publish` the kernel (and every one staged before it) becomes visible
// at once (serve_flush); without, it waits for the next publish, and a
// serving run that stops first never runs it.
int serve_publish(kl_runtime* rt, TenantDev td, uint64_t footprint, kl_handle* out, bool publish = true) {
  int p = progress(rt);
  if (p == KL_ECUDA) return KL_ECUDA;
  if (!rt->in_flight || (rt->kind != kServe && rt->kind != kServeBase)) return KL_ESTATE;  // the run has ended
  if (rt->kind == kServeBase && rt->s_joined) return KL_ESTATE;
  if (rt->kind == kServe && __atomic_load_n(&rt->sm_ctl[32], __ATOMIC_RELAXED)) return KL_ESTATE;  // stopping
  if (rt->kind == kServe && tn::resource_class(td.type) != tn::kClassMain) return KL_EINVAL;
  if (rt->kind == kServe && !tn::in_plain_build(td.type) && !(rt->cfg.flags & KL_CFG_SERVE_TC)) return KL_EINVAL;
  if (rt->s_inflight >= rt->cap) return KL_EAGAIN;
  if (rt->cfg.mem_cap_bytes && rt->s_footprint + footprint > rt->cfg.mem_cap_bytes) return KL_EAGAIN;
  const uint32_t seq = rt->s_tail;
  if (seq >= 0xfffffff0u) return KL_EOVERFLOW;
  td.index = seq;
  td.slice = clamp_slice(rt, td.slice, td.total);
  if (rt->kind == kServe)
    memcpy(&rt->sm_ring[seq & (rt->s_ring - 1u)], &td, sizeof(td));
  else
    rt->s_staged.push_back(td);
  ServeRec r{};
  r.t_submit = now_ns();
  r.footprint = footprint;
  r.state = KL_PENDING;  // until published
  r.total = td.total;
  rt->s_recs.push_back(r);
  rt->s_tail = seq + 1u;
  rt->s_inflight++;
  rt->s_footprint += footprint;
  *out = make_handle(rt->flight_id, seq);
  return publish ? serve_flush(rt) : KL_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" int kl_abi_version(void) { return KL_ABI_VERSION; }

extern "C" const char* kl_strerror(int code) {
  switch (code) {
    case KL_OK: return "ok";
    case KL_EINVAL: return "invalid argument";
    case KL_ENOMEM: return "out of memory";
    case KL_EAGAIN: return "try again (queue full, over the memory cap, or a run in flight)";
    case KL_ETIMEDOUT: return "host wait timed out";
    case KL_ECUDA: return "CUDA runtime error";
    case KL_EDEVICE_TIMEOUT: return "device-side wait exceeded its limit";
    case KL_ESTATE: return "invalid state";
    case KL_ENOTFOUND: return "unknown handle";
    case KL_EOVERFLOW: return "device table overflow";
    default: return "unknown status";
  }
}

extern "C" int kl_config_default(kl_config* c) {
  if (!c) return KL_EINVAL;
  memset(c, 0, sizeof(*c));
  c->device = 0;
  c->slots_per_sm = 0;
  c->max_tenants = 4096;
  c->model_states = 3;
  c->ratio_policy = KL_RATIO_BALANCED;
  c->fixed_slots_a = 2;
  c->device_wait_limit_ns = 2000000000ull;
  c->mem_cap_bytes = 0;
  c->alpha_p = -1.0;
  c->alpha_m = -1.0;
  c->flags = KL_CFG_BACKFILL | KL_CFG_FILL_TYPES | KL_CFG_CHAIN_LANE | KL_CFG_WIDE_FILL | KL_CFG_LIGHT_BUILD |
             KL_CFG_DEEP_FILL | KL_CFG_PHASE_MODEL;
  c->chain_slots = 2;
  return KL_OK;
}

extern "C" int kl_tenant_shape_of(uint32_t type, const void* args, uint32_t args_size, kl_tenant_shape* out) {
  if (!out || !args || type >= KL_T_COUNT || args_size != args_size_of(type)) return KL_EINVAL;
  int rc = validate_args(type, args);
  if (rc) return rc;
  unsigned char blob[KL_MAX_ARGS_BYTES] = {0};
  memcpy(blob, args, args_size);
  memset(out, 0, sizeof(*out));
  out->grid[0] = tn::stage_blocks(type, blob, 0);
  out->grid[1] = out->grid[2] = 1;
  out->block[0] = tn::block_threads(type);
  out->block[1] = out->block[2] = 1;
  out->nstages = tn::nstages(type, blob);
  out->smem_bytes = tn::smem_bytes(type);
  out->total_blocks = tn::total_blocks(type, blob);
  return KL_OK;
}

extern "C" int kl_gemm_bf16_tensor_maps(const kl_args_gemm_bf16* a, void* out_host) {
  if (!a || !out_host) return KL_EINVAL;
  if (!a->A || !a->Bt || a->M == 0 || a->N == 0 || a->K == 0 || a->K % 8 || !a16(a->A) || !a16(a->Bt))
    return KL_EINVAL;
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn)
        return KL_ECUDA;
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
  }
  CUtensorMap maps[2];
  const void* base[2] = {a->A, a->Bt};
  const uint32_t rows[2] = {a->M, a->N};
  const uint32_t box_rows[2] = {(uint32_t)tn::kBfBM, (uint32_t)tn::kBfBN};
  for (int i = 0; i < 2; ++i) {
    const cuuint64_t dims[2] = {a->K, rows[i]};           // innermost first: K, then rows
    const cuuint64_t strides[1] = {(cuuint64_t)a->K * 2};  // bytes between rows
    const cuuint32_t box[2] = {(cuuint32_t)tn::kBfBK, box_rows[i]};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base[i]), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return KL_ECUDA;
  }
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  memcpy(out_host, maps, sizeof(maps));
  return KL_OK;
}

extern "C" int kl_create(const kl_config* cfg_in, void* cuda_stream, kl_runtime** out) {
  if (!out) return KL_EINVAL;
  *out = nullptr;
  kl_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    kl_config_default(&cfg);
  if (cfg.model_states != 2 && cfg.model_states != 3) return KL_EINVAL;
  if (cfg.max_tenants == 0 || cfg.max_tenants > (1u << 20)) return KL_EINVAL;
  if (cfg.slots_per_sm > KL_MAX_SLOTS || cfg.ratio_policy > 2) return KL_EINVAL;
  if (cfg.device_wait_limit_ns == 0) cfg.device_wait_limit_ns = 2000000000ull;
  if (cudaSetDevice(cfg.device) != cudaSuccess) return KL_ECUDA;
  kl_runtime* rt = new (std::nothrow) kl_runtime();
  if (!rt) return KL_ENOMEM;
  rt->cfg = cfg;
  rt->device = cfg.device;
  rt->stream = (cudaStream_t)cuda_stream;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, cfg.device) != cudaSuccess) goto fail_cuda;
  rt->n_sm = (uint32_t)std::min(v, kMaxSM);
  {
    int occ = 0;
    // the tensor-core build reaches the same residency: its CTAs give up the
    // TMEM allocation permit right after allocating (see acquire_tmem)
    int occ_tc = 0;     // also raises the tensor-core build's dynamic shared memory limit
    int occ_light = 0;  // and the light build's
    if (cosched_occupancy(&occ, tn::kBuildPlain) != 0 || occ < 1 ||
        cosched_occupancy(&occ_tc, tn::kBuildFull) != 0 || cosched_occupancy(&occ_light, tn::kBuildLight) != 0)
      goto fail_cuda;
    rt->occupancy = (uint32_t)occ;
    uint32_t s = cfg.slots_per_sm ? cfg.slots_per_sm : (uint32_t)occ;
    s = std::min<uint32_t>(std::min<uint32_t>(s, (uint32_t)occ), KL_MAX_SLOTS);
    rt->slots = s;
    // a fixed slot count pins every run to it; otherwise runs of light types
    // use the light build when it holds more CTAs per SM
    const uint32_t sl = std::min<uint32_t>((uint32_t)std::max(occ_light, 0), KL_MAX_SLOTS);
    rt->slots_light = (cfg.slots_per_sm == 0 && sl > s) ? sl : 0u;
  }
  // the device indexes tenants and phases modulo a power of two (a ring in
  // serving mode); a batch run never wraps: n <= cap tenants, <= 4 cap + 16 phases
  rt->cap = cfg.max_tenants;
  rt->cap_phases = 4 * rt->cap + 16;
  rt->ring_slots = pow2_at_least(rt->cap);
  rt->phase_slots = pow2_at_least(rt->cap_phases);
  if (cudaMalloc(&rt->d_tenants, sizeof(TenantDev) * rt->ring_slots) != cudaSuccess) goto fail_mem;
  if (cudaMalloc(&rt->d_run, sizeof(RunDev)) != cudaSuccess) goto fail_mem;
  if (cudaMalloc(&rt->d_phases, sizeof(PhaseDev) * rt->phase_slots) != cudaSuccess) goto fail_mem;
  if (cudaMallocHost(&rt->h_tenants, sizeof(TenantDev) * rt->ring_slots) != cudaSuccess) goto fail_mem;
  if (cudaMallocHost(&rt->h_run, sizeof(RunDev)) != cudaSuccess) goto fail_mem;
  if (cudaMallocHost(&rt->h_phases, sizeof(PhaseDev) * rt->phase_slots) != cudaSuccess) goto fail_mem;
  // device addresses of the pinned image (the SM-side staging copies use them)
  if (cudaHostGetDevicePointer((void**)&rt->hd_tenants, rt->h_tenants, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&rt->hd_run, rt->h_run, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&rt->hd_phases, rt->h_phases, 0) != cudaSuccess)
    goto fail_cuda;
  if (cudaEventCreate(&rt->ev_start) != cudaSuccess || cudaEventCreate(&rt->ev_done) != cudaSuccess ||
      cudaEventCreate(&rt->ev_k0) != cudaSuccess || cudaEventCreate(&rt->ev_k1) != cudaSuccess ||
      cudaEventCreateWithFlags(&rt->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    goto fail_cuda;
  // model defaults: device properties, built-in profiles
  {
    rt->mp.n_sm = rt->n_sm;
    rt->mp.n_sched = 4;
    int khz = 0;
    rt->mp.f_sm_hz = (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, cfg.device) == cudaSuccess && khz > 0)
                         ? khz * 1e3
                         : 1.9e9;
    rt->mp.dram_bytes_per_s = 6.75e12;
    rt->mp.sector_bytes = 32.0;
    rt->mp.a0 = 1.0;
    rt->mp.b0 = 0.0;
    for (uint32_t t = 0; t < KL_T_COUNT; ++t) rt->prof[t] = builtin_profile(t);
  }
  *out = rt;
  return KL_OK;
fail_mem:
  kl_destroy(rt);
  return KL_ENOMEM;
fail_cuda:
  kl_destroy(rt);
  return KL_ECUDA;
}

extern "C" int kl_destroy(kl_runtime* rt) {
  if (!rt) return KL_EINVAL;
  int rc = KL_OK;
  {
    std::unique_lock<std::mutex> lk(rt->mu);
    if (rt->in_flight && rt->kind == kServe) __atomic_store_n(&rt->sm_ctl[32], 1u, __ATOMIC_RELEASE);
    if (rt->in_flight && rt->kind == kServeBase && !rt->s_joined) serve_join(rt);
    if (rt->in_flight) {
      int w = wait_flight(rt, lk, rt->cfg.device_wait_limit_ns * 4 + 1000000000ull);
      if (w == KL_ETIMEDOUT) rc = KL_ESTATE;
    }
  }
  if (rc == KL_ESTATE) return rc;  // leave resources: the GPU may still use them
  cudaFree(rt->d_tenants);
  cudaFree(rt->d_run);
  cudaFree(rt->d_phases);
  cudaFreeHost(rt->h_tenants);
  cudaFreeHost(rt->h_run);
  cudaFreeHost(rt->h_phases);
  cudaFree(rt->sd_ring);
  cudaFree(rt->sd_phases);
  cudaFreeHost(rt->sh_phases);
  cudaFreeHost(rt->sm_ring);
  cudaFreeHost(rt->sm_ctl);
  cudaFreeHost(rt->sm_done);
  cudaFreeHost(rt->sm_cq);
  for (cudaEvent_t e : rt->s_free_ev) cudaEventDestroy(e);
  for (auto& q : rt->s_stream_q)
    for (auto& x : q) cudaEventDestroy(x.second);
  if (rt->ev_start) cudaEventDestroy(rt->ev_start);
  if (rt->ev_done) cudaEventDestroy(rt->ev_done);
  if (rt->ev_k0) cudaEventDestroy(rt->ev_k0);
  if (rt->ev_k1) cudaEventDestroy(rt->ev_k1);
  if (rt->ev_fork) cudaEventDestroy(rt->ev_fork);
  for (cudaEvent_t e : rt->tenant_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : rt->side_join) cudaEventDestroy(e);
  for (cudaStream_t s : rt->side) cudaStreamDestroy(s);
  delete rt;
  return KL_OK;
}

static int submit_impl(kl_runtime* rt, const kl_kernel_desc* d, kl_handle* out, bool publish) {
  if (!rt || !d || !out) return KL_EINVAL;
  *out = 0;
  if (d->type >= KL_T_COUNT || !d->args || d->args_size != args_size_of(d->type)) return KL_EINVAL;
  if (d->block[0] != tn::block_threads(d->type) || d->block[1] != 1 || d->block[2] != 1) return KL_EINVAL;
  kl_tenant_shape sh;
  int rc = kl_tenant_shape_of(d->type, d->args, d->args_size, &sh);
  if (rc) return rc;
  if (d->grid[0] != sh.grid[0] || d->grid[1] != 1 || d->grid[2] != 1) return KL_EINVAL;
  if (d->smem_bytes != 0 && d->smem_bytes < sh.smem_bytes) return KL_EINVAL;
  if (sh.total_blocks == 0 || sh.total_blocks >= (1ull << 31)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  TenantDev td;
  memset(&td, 0, sizeof(td));
  td.type = d->type;
  td.slice = d->slice_blocks                   ? d->slice_blocks
             : rt->prof[d->type].slice_blocks ? rt->prof[d->type].slice_blocks
                                              : default_slice(d->type);
  td.total = (uint32_t)sh.total_blocks;
  td.nstages = sh.nstages;
  td.blocks0 = sh.grid[0];
  memcpy(td.args, d->args, d->args_size);
  if (rt->serve_on) return serve_publish(rt, td, d->footprint_bytes, out, publish);
  if (rt->pending.size() >= rt->cap) return KL_EAGAIN;
  if (rt->cfg.mem_cap_bytes && rt->pending_footprint + d->footprint_bytes > rt->cfg.mem_cap_bytes) return KL_EAGAIN;
  Pending p;
  p.td = td;
  p.td.index = (uint32_t)rt->pending.size();
  p.footprint = d->footprint_bytes;
  p.t_submit = now_ns();
  p.handle = make_handle(rt->run_id, p.td.index);
  p.caller_slice = d->slice_blocks != 0;
  p.slice_alone = std::max(1u, rt->prof[d->type].slice_blocks_alone);
  rt->pending.push_back(p);
  rt->pending_footprint += d->footprint_bytes;
  *out = p.handle;
  return KL_OK;
}

extern "C" int kl_submit(kl_runtime* rt, const kl_kernel_desc* d, kl_handle* out) {
  return submit_impl(rt, d, out, true);
}

extern "C" int kl_submit_staged(kl_runtime* rt, const kl_kernel_desc* d, kl_handle* out) {
  return submit_impl(rt, d, out, false);
}

extern "C" int kl_submit_batch(kl_runtime* rt, const kl_kernel_desc* descs, uint32_t n, kl_handle* out,
                               uint32_t* n_done) {
  if (n_done) *n_done = 0;
  if (!rt || (n && (!descs || !out))) return KL_EINVAL;
  int rc = KL_OK;
  uint32_t k = 0;
  for (; k < n; ++k) {
    rc = submit_impl(rt, &descs[k], &out[k], false);
    if (rc) break;
  }
  if (n_done) *n_done = k;
  // one publish for the whole burst (serving: one tail store, one re-plan)
  const int pr = kl_publish(rt);
  return rc ? rc : pr;
}

extern "C" int kl_publish(kl_runtime* rt) {
  if (!rt) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  if (!rt->serve_on || !rt->in_flight || (rt->kind != kServe && rt->kind != kServeBase)) return KL_OK;
  return serve_flush(rt);
}

// Plan and start the pending set; caller holds rt->mu.
static int launch_locked(kl_runtime* rt) {
  if (rt->in_flight && progress(rt) == KL_EAGAIN) return KL_EAGAIN;
  const uint32_t n = (uint32_t)rt->pending.size();
  if (n == 0) return KL_OK;
  if (cudaSetDevice(rt->device) != cudaSuccess) return KL_ECUDA;
  uint32_t mask = 0, smem = tn::kMinCtaSmem, cls_mask = 0;
  for (const Pending& p : rt->pending) {
    const int c = tn::resource_class(p.td.type);
    if (c != tn::kClassMain) {
      cls_mask |= 1u << c;  // run by its resource-class kernel beside the co-scheduler
      continue;
    }
    mask |= 1u << p.td.type;
    smem = std::max(smem, tn::smem_bytes(p.td.type));  // dynamic shared memory of this run's CTAs
  }
  const bool has_main = mask != 0u;
  // the smallest build that holds every type of the run (tn::run_block)
  int build = tn::kBuildPlain;
  bool all_light = true;
  for (uint32_t t = 0; t < KL_T_MAIN_COUNT; ++t)
    if ((mask >> t) & 1u) {
      if (!tn::in_plain_build(t)) build = tn::kBuildFull;
      all_light = all_light && tn::in_light_build(t);
    }
  if (all_light && !cls_mask && (rt->cfg.flags & KL_CFG_LIGHT_BUILD) && rt->slots_light && !rt->table_override)
    build = tn::kBuildLight;
  uint32_t S = build == tn::kBuildLight ? rt->slots_light : rt->slots;
  const uint32_t S_build = S;
  // a resource-class CTA takes up to half an SM's registers: the co-scheduler
  // keeps two slots per SM beside it
  if (cls_mask && has_main) S = std::min<uint32_t>(S, 2u);
  // KL_CFG_PHASE_MODEL: the multi-stage type with the most blocks pending is
  // what the chain lane runs beside the pairs
  int chain = -1;
  if ((rt->cfg.flags & KL_CFG_PHASE_MODEL) && (rt->cfg.flags & KL_CFG_CHAIN_LANE)) {
    uint64_t most = 0;
    uint64_t per_type[KL_T_COUNT] = {0};
    for (const Pending& p : rt->pending)
      if (p.td.nstages > 1 && tn::resource_class(p.td.type) == tn::kClassMain) per_type[p.td.type] += p.td.total;
    for (uint32_t t = 0; t < KL_T_MAIN_COUNT; ++t)
      if (per_type[t] > most) {
        most = per_type[t];
        chain = (int)t;
      }
  }
  int rc = has_main && S >= 1 ? ensure_table(rt, mask, S, chain) : KL_OK;
  if (rc) return rc;
  // device image: run state, tenants, the "plan first" phase
  RunDev& R = *rt->h_run;
  memset(&R, 0, sizeof(R));
  R.n_tenants = n;
  R.slots = S;
  R.max_phases = std::min(rt->cap_phases, 4 * n + 16);
  R.n_types = KL_T_COUNT;
  R.wait_limit_ns = rt->cfg.device_wait_limit_ns;
  R.flags = rt->cfg.flags;
  R.serve = 0;
  R.plan_seed = rt->cfg.plan_seed;
  R.chain_slots = std::max(1u, std::min(rt->cfg.chain_slots, S - 1));
  R.ring_mask = rt->ring_slots - 1;
  R.phase_mask = rt->phase_slots - 1;
  memcpy(R.cp, rt->cp, sizeof(R.cp));
  memcpy(R.slots_a, rt->slots_a, sizeof(R.slots_a));
  memcpy(R.allowed, rt->allowed, sizeof(R.allowed));
  R.n_sm = rt->n_sm;
  R.quota_exit = (cls_mask && has_main) ? 1u : 0u;
  // resource classes present in the run, each run by its class kernel with
  // two CTAs per SM (they take the room the co-scheduler's two slots leave)
  int cls_list[tn::kNumClasses];
  uint32_t ncls = 0;
  for (int c = 1; c < tn::kNumClasses; ++c)
    if ((cls_mask >> c) & 1u) cls_list[ncls++] = c;
  // Slices are tuned with several kernels of a type sharing the GPU; a run of
  // few or small kernels could then hand out too few slices to balance its
  // CTAs. Slices the run can hand out at once (a multi-stage kernel counts two
  // stages: the others keep the slots busy at its barriers), summed over the
  // co-scheduler's kernels: below four per CTA, the slices the caller did not
  // set shrink by the missing factor, but never below the type's alone-tuned
  // slice (the paper's rule for a kernel without company).
  uint32_t shrink = 1;
  if (has_main) {
    uint64_t avail = 0;
    for (const Pending& p : rt->pending) {
      if (tn::resource_class(p.td.type) != tn::kClassMain) continue;
      const uint64_t per_stage = std::max<uint64_t>(1u, p.td.total / std::max(1u, p.td.nstages));
      avail += (per_stage + p.td.slice - 1) / p.td.slice * std::min(2u, std::max(1u, p.td.nstages));
    }
    const uint64_t want = 4ull * rt->n_sm * S;
    if (avail < want) shrink = (uint32_t)((want + avail - 1) / avail);
  }
  for (uint32_t i = 0; i < n; ++i) {
    TenantDev td = rt->pending[i].td;
    if (shrink > 1 && !rt->pending[i].caller_slice)
      td.slice = std::max(std::min(td.slice, rt->pending[i].slice_alone), td.slice / shrink);
    td.slice = clamp_slice(rt, td.slice, td.total);
    rt->h_tenants[i] = td;
  }
  PhaseDev first{};
  first.A = -2;
  first.B = -1;
  for (int f = 0; f < kFill; ++f) first.fill[f] = -1;
  first.chain[0] = first.chain[1] = -1;
  rt->h_phases[0] = first;
  cudaStream_t s = rt->stream;
  // the run's image goes in and its results come out through the SMs (the
  // pinned host image is device-accessible), not the copy engines: a caller's
  // bulk transfers queued on those engines must not delay the launch
  const CopySeg in[3] = {{rt->d_tenants, rt->hd_tenants, sizeof(TenantDev) * n},
                         {rt->d_run, rt->hd_run, sizeof(RunDev)},
                         {rt->d_phases, rt->hd_phases, sizeof(PhaseDev)}};
  const CopySeg out[3] = {{rt->hd_tenants, rt->d_tenants, sizeof(TenantDev) * n},
                          {rt->hd_run, rt->d_run, sizeof(RunDev)},
                          {rt->hd_phases, rt->d_phases, sizeof(PhaseDev) * R.max_phases}};
  // resource-class kernels run on side streams forked from the runtime stream
  // after the image is in, and joined back before the image comes out
  while (rt->side.size() < ncls) {
    cudaStream_t q;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) return KL_ECUDA;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return KL_ECUDA;
    rt->side.push_back(q);
    rt->side_join.push_back(e);
  }
  static const int cls_type[tn::kNumClasses] = {-1, KL_T_BS255, KL_T_HIST1024, KL_T_GEMM_F32_BIG};
  rc = cuda_ok(cudaEventRecord(rt->ev_start, s));
  if (!rc && stage_copy(in, 3, s) != 0) rc = KL_ECUDA;
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k0, s));
  if (!rc && ncls) rc = cuda_ok(cudaEventRecord(rt->ev_fork, s));
  // the co-scheduler first: its CTAs take their two slots on every SM before
  // the class CTAs fill the rest
  if (!rc && has_main &&
      cosched_launch(rt->d_tenants, rt->d_run, rt->d_phases, rt->n_sm, S, smem, build, s, R.quota_exit ? rt->n_sm : 0u) != 0)
    rc = KL_ECUDA;
  for (uint32_t q = 0; q < ncls && !rc; ++q) {
    rc = cuda_ok(cudaStreamWaitEvent(rt->side[q], rt->ev_fork, 0));
    if (!rc && class_launch(cls_type[cls_list[q]], rt->d_tenants, rt->d_run, 2u * rt->n_sm, rt->side[q]) != 0)
      rc = KL_ECUDA;
    if (!rc && q > 0) rc = cuda_ok(cudaEventRecord(rt->side_join[q], rt->side[q]));
  }
  // The room the class kernels held goes back to the co-scheduler when they
  // are all done: behind them on the first side stream, the quota that made
  // extra co-scheduler CTAs leave is lifted and a second grid of the
  // co-scheduler joins the same run (its CTAs take the freed slots and pull
  // from the same plan; if the run has ended they leave at once).
  if (!rc && ncls) {
    for (uint32_t q = 1; q < ncls && !rc; ++q) rc = cuda_ok(cudaStreamWaitEvent(rt->side[0], rt->side_join[q], 0));
    if (!rc && has_main && S_build > S) {
      rc = cuda_ok(cudaMemsetAsync(&rt->d_run->quota_exit, 0, sizeof(uint32_t), rt->side[0]));
      if (!rc && cosched_launch(rt->d_tenants, rt->d_run, rt->d_phases, rt->n_sm, S_build - S, smem, build,
                                rt->side[0], 0u) != 0)
        rc = KL_ECUDA;
    }
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->side_join[0], rt->side[0]));
  }
  for (uint32_t q = 0; q < ncls && !rc; ++q) rc = cuda_ok(cudaStreamWaitEvent(s, rt->side_join[q], 0));
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k1, s));
  if (!rc && stage_copy(out, 3, s) != 0) rc = KL_ECUDA;
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_done, s));
  if (rc) return rc;
  rt->flight.swap(rt->pending);
  rt->pending.clear();
  rt->pending_footprint = 0;
  rt->in_flight = true;
  rt->kind = kCosched;
  rt->flight_id = rt->run_id++;
  rt->flight_slots = S;
  return KL_OK;
}

extern "C" int kl_launch(kl_runtime* rt) {
  if (!rt) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  if (rt->serve_on) return KL_ESTATE;
  return launch_locked(rt);
}

extern "C" int kl_launch_baseline(kl_runtime* rt, int mode, uint32_t nstreams) {
  if (!rt || (mode != KL_BASE_SERIAL && mode != KL_BASE_MULTISTREAM)) return KL_EINVAL;
  if (mode == KL_BASE_MULTISTREAM && (nstreams == 0 || nstreams > 256)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  if (rt->serve_on) return KL_ESTATE;
  if (rt->in_flight && progress(rt) == KL_EAGAIN) return KL_EAGAIN;
  const uint32_t n = (uint32_t)rt->pending.size();
  if (n == 0) return KL_OK;
  if (cudaSetDevice(rt->device) != cudaSuccess) return KL_ECUDA;
  while (rt->tenant_ev.size() < n) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return KL_ECUDA;
    rt->tenant_ev.push_back(e);
  }
  if (mode == KL_BASE_MULTISTREAM) {
    while (rt->side.size() < nstreams) {
      cudaStream_t s;
      cudaEvent_t e;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return KL_ECUDA;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return KL_ECUDA;
      rt->side.push_back(s);
      rt->side_join.push_back(e);
    }
  }
  cudaStream_t s = rt->stream;
  int rc = cuda_ok(cudaEventRecord(rt->ev_start, s));
  if (mode == KL_BASE_SERIAL) {
    for (uint32_t i = 0; i < n && !rc; ++i) {
      if (native_launch_tenant(rt->pending[i].td.type, rt->pending[i].td.args, s) != 0) rc = KL_ECUDA;
      if (!rc) rc = cuda_ok(cudaEventRecord(rt->tenant_ev[i], s));
    }
  } else {
    rc = rc ? rc : cuda_ok(cudaEventRecord(rt->ev_fork, s));
    for (uint32_t k = 0; k < nstreams && !rc; ++k) rc = cuda_ok(cudaStreamWaitEvent(rt->side[k], rt->ev_fork, 0));
    for (uint32_t i = 0; i < n && !rc; ++i) {
      cudaStream_t si = rt->side[i % nstreams];
      if (native_launch_tenant(rt->pending[i].td.type, rt->pending[i].td.args, si) != 0) rc = KL_ECUDA;
      if (!rc) rc = cuda_ok(cudaEventRecord(rt->tenant_ev[i], si));
    }
    for (uint32_t k = 0; k < nstreams && !rc; ++k) {
      rc = cuda_ok(cudaEventRecord(rt->side_join[k], rt->side[k]));
      if (!rc) rc = cuda_ok(cudaStreamWaitEvent(s, rt->side_join[k], 0));
    }
  }
  if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_done, s));
  if (rc) return rc;
  rt->flight.swap(rt->pending);
  rt->pending.clear();
  rt->pending_footprint = 0;
  rt->in_flight = true;
  rt->kind = kBaseline;
  rt->flight_id = rt->run_id++;
  rt->flight_slots = rt->slots;
  return KL_OK;
}

// Serving buffers, allocated at the first co-scheduled kl_serve_start: the
// device tenant and phase rings, and the mapped host ring, control words,
// completion records and completion queue.
static int serve_alloc(kl_runtime* rt) {
  if (rt->sd_ring) return KL_OK;
  const uint32_t ring = pow2_at_least(std::max<uint64_t>(65536, 4ull * rt->cap));
  const uint32_t nph = 65536;
  void* p = nullptr;
  if (cudaMalloc(&rt->sd_ring, sizeof(TenantDev) * ring) != cudaSuccess) return KL_ENOMEM;
  if (cudaMalloc(&rt->sd_phases, sizeof(PhaseDev) * nph) != cudaSuccess) return KL_ENOMEM;
  if (cudaMallocHost(&rt->sh_phases, sizeof(PhaseDev) * nph) != cudaSuccess) return KL_ENOMEM;
  if (cudaHostAlloc(&p, sizeof(TenantDev) * ring, cudaHostAllocMapped) != cudaSuccess) return KL_ENOMEM;
  rt->sm_ring = (TenantDev*)p;
  if (cudaHostAlloc(&p, 256, cudaHostAllocMapped) != cudaSuccess) return KL_ENOMEM;
  rt->sm_ctl = (uint32_t*)p;
  if (cudaHostAlloc(&p, sizeof(ServeDone) * ring, cudaHostAllocMapped) != cudaSuccess) return KL_ENOMEM;
  rt->sm_done = (ServeDone*)p;
  if (cudaHostAlloc(&p, sizeof(unsigned long long) * ring, cudaHostAllocMapped) != cudaSuccess) return KL_ENOMEM;
  rt->sm_cq = (unsigned long long*)p;
  if (cudaHostGetDevicePointer((void**)&rt->sdm_ring, rt->sm_ring, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&rt->sdm_ctl, rt->sm_ctl, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&rt->sdm_done, rt->sm_done, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&rt->sdm_cq, rt->sm_cq, 0) != cudaSuccess)
    return KL_ECUDA;
  rt->s_ring = ring;
  rt->s_phase_slots = nph;
  return KL_OK;
}

extern "C" int kl_serve_start(kl_runtime* rt, int mode, uint32_t nstreams, uint64_t idle_limit_ns) {
  if (!rt) return KL_EINVAL;
  if (mode != KL_SERVE_COSCHED && mode != KL_BASE_SERIAL && mode != KL_BASE_MULTISTREAM) return KL_EINVAL;
  if (mode == KL_BASE_MULTISTREAM && (nstreams == 0 || nstreams > 256)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  if (rt->serve_on) return KL_ESTATE;
  if (rt->in_flight && progress(rt) == KL_EAGAIN) return KL_EAGAIN;
  if (cudaSetDevice(rt->device) != cudaSuccess) return KL_ECUDA;
  int rc = KL_OK;
  cudaStream_t s = rt->stream;
  if (mode == KL_SERVE_COSCHED) {
    rc = serve_alloc(rt);
    if (rc) return rc;
    rc = ensure_table(rt, (1u << KL_T_COUNT) - 1u, rt->slots);  // arrivals may be of any type
    if (rc) return rc;
    memset(rt->sm_ctl, 0, 256);
    memset(rt->sm_cq, 0, sizeof(unsigned long long) * rt->s_ring);
    RunDev& R = *rt->h_run;
    memset(&R, 0, sizeof(R));
    R.slots = rt->slots;
    R.n_sm = rt->n_sm;
    R.max_phases = rt->s_phase_slots;
    R.n_types = KL_T_COUNT;
    R.wait_limit_ns = rt->cfg.device_wait_limit_ns;
    R.flags = rt->cfg.flags;
    R.serve = 1;
    R.plan_seed = rt->cfg.plan_seed;
    R.chain_slots = std::max(1u, std::min(rt->cfg.chain_slots, rt->slots - 1));
    R.age_limit_ns = rt->cfg.age_limit_ns ? rt->cfg.age_limit_ns : 5000000ull;
    R.ring_mask = rt->s_ring - 1u;
    R.phase_mask = rt->s_phase_slots - 1u;
    R.idle_limit_ns = idle_limit_ns ? idle_limit_ns : 60000000000ull;
    R.host_ring = rt->sdm_ring;
    R.host_ctl = rt->sdm_ctl;
    R.host_done = rt->sdm_done;
    R.host_cq = rt->sdm_cq;
    memcpy(R.cp, rt->cp, sizeof(R.cp));
    memcpy(R.slots_a, rt->slots_a, sizeof(R.slots_a));
    memcpy(R.allowed, rt->allowed, sizeof(R.allowed));
    PhaseDev first{};
    first.A = kPhasePlan;
    first.B = -1;
    for (int f = 0; f < kFill; ++f) first.fill[f] = -1;
    first.chain[0] = first.chain[1] = -1;
    rt->sh_phases[0] = first;
    rc = cuda_ok(cudaEventRecord(rt->ev_start, s));
    if (!rc) rc = cuda_ok(cudaMemcpyAsync(rt->d_run, rt->h_run, sizeof(RunDev), cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_ok(cudaMemcpyAsync(rt->sd_phases, rt->sh_phases, sizeof(PhaseDev), cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k0, s));
    // dynamic shared memory of the largest type a serving run can receive
    const bool tc = (rt->cfg.flags & KL_CFG_SERVE_TC) != 0;
    uint32_t smem = tn::kMinCtaSmem;
    // the types the launched build holds (resource-class variants never run in it)
    for (uint32_t t = 0; t < KL_T_COUNT; ++t)
      if (tn::in_plain_build(t) || (tc && tn::in_build(tn::kBuildFull, t))) smem = std::max(smem, tn::smem_bytes(t));
    if (!rc && cosched_launch(rt->sd_ring, rt->d_run, rt->sd_phases, rt->n_sm, rt->slots, smem,
                              tc ? tn::kBuildFull : tn::kBuildPlain, s) != 0)
      rc = KL_ECUDA;
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k1, s));
    if (!rc) rc = cuda_ok(cudaMemcpyAsync(rt->h_run, rt->d_run, sizeof(RunDev), cudaMemcpyDeviceToHost, s));
    if (!rc)
      rc = cuda_ok(cudaMemcpyAsync(rt->sh_phases, rt->sd_phases, sizeof(PhaseDev) * rt->s_phase_slots,
                                   cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_done, s));
    if (rc) return rc;
    rt->kind = kServe;
  } else {
    const uint32_t ns = mode == KL_BASE_SERIAL ? 1u : nstreams;
    while (rt->side.size() < ns) {
      cudaStream_t q;
      cudaEvent_t e;
      if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) return KL_ECUDA;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return KL_ECUDA;
      rt->side.push_back(q);
      rt->side_join.push_back(e);
    }
    rc = cuda_ok(cudaEventRecord(rt->ev_start, s));
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_k0, s));
    if (!rc) rc = cuda_ok(cudaEventRecord(rt->ev_fork, s));
    for (uint32_t k = 0; k < ns && !rc; ++k) rc = cuda_ok(cudaStreamWaitEvent(rt->side[k], rt->ev_fork, 0));
    if (rc) return rc;
    rt->s_nstreams = ns;
    rt->s_stream_q.assign(ns, {});
    rt->s_joined = false;
    rt->kind = kServeBase;
  }
  rt->serve_on = true;
  rt->serve_mode = mode;
  rt->in_flight = true;
  rt->flight_id = rt->run_id++;  // kernels still pending keep their handles: they arrive first
  rt->flight_slots = rt->slots;
  rt->s_tail = rt->s_head = rt->s_inflight = rt->s_published = 0;
  rt->s_staged.clear();
  rt->s_footprint = 0;
  rt->s_recs.clear();
  rt->completed.clear();
  std::vector<Pending> early;
  early.swap(rt->pending);
  rt->pending_footprint = 0;
  kl_handle h = 0;
  for (const Pending& p : early) {
    rc = serve_publish(rt, p.td, p.footprint, &h);
    if (rc) return rc;
    rt->s_recs.back().t_submit = p.t_submit;
  }
  return KL_OK;
}

extern "C" int kl_serve_stop(kl_runtime* rt, uint64_t timeout_ns) {
  if (!rt) return KL_EINVAL;
  std::unique_lock<std::mutex> lk(rt->mu);
  if (!rt->serve_on) return KL_ESTATE;
  int rc = KL_OK;
  if (rt->in_flight && rt->kind == kServe) __atomic_store_n(&rt->sm_ctl[32], 1u, __ATOMIC_RELEASE);
  if (rt->in_flight && rt->kind == kServeBase && !rt->s_joined) rc = serve_join(rt);
  if (rc) return rc;
  if (rt->in_flight) {
    rc = wait_flight(rt, lk, timeout_ns);
    if (rc == KL_ETIMEDOUT || rc == KL_ECUDA) return rc;
  }
  rt->serve_on = false;
  return rt->last.error;
}

extern "C" int kl_reap(kl_runtime* rt, kl_handle* out, uint32_t cap, uint32_t* n) {
  if (!rt || !n || (cap && !out)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  *n = 0;
  int p = progress(rt);
  if (p == KL_ECUDA) return p;
  while (*n < cap && !rt->completed.empty()) {
    out[(*n)++] = rt->completed.front();
    rt->completed.pop_front();
  }
  return KL_OK;
}

static int lookup(kl_runtime* rt, kl_handle h, kl_tenant_stats* st) {
  uint64_t run;
  uint32_t idx;
  split_handle(h, &run, &idx);
  if (h == 0) return KL_ENOTFOUND;
  if (run == rt->run_id) {
    if (idx >= rt->pending.size() || rt->pending[idx].handle != h) return KL_ENOTFOUND;
    memset(st, 0, sizeof(*st));
    st->state = KL_PENDING;
    st->t_submit_ns = rt->pending[idx].t_submit;
    return KL_OK;
  }
  if (rt->in_flight && run == rt->flight_id && (rt->kind == kServe || rt->kind == kServeBase)) {
    if (idx >= rt->s_recs.size()) return KL_ENOTFOUND;
    const ServeRec& r = rt->s_recs[idx];
    memset(st, 0, sizeof(*st));
    st->state = (int32_t)r.state;
    st->t_submit_ns = r.t_submit;
    st->t_done_host_ns = r.t_done_host;
    if (r.state == KL_DONE) {
      st->t_start_ns = r.done.t_start;
      st->t_end_ns = r.done.t_end;
      st->slices = r.done.slices;
      st->blocks = rt->kind == kServe ? r.done.blocks : r.total;
    }
    return KL_OK;
  }
  if (rt->in_flight && run == rt->flight_id) {
    if (idx >= rt->flight.size()) return KL_ENOTFOUND;
    memset(st, 0, sizeof(*st));
    st->state = KL_RUNNING;
    st->t_submit_ns = rt->flight[idx].t_submit;
    return KL_OK;
  }
  auto it = rt->history.find(run);
  if (it == rt->history.end() || idx >= it->second.size()) return KL_ENOTFOUND;
  *st = it->second[idx].st;
  return KL_OK;
}

extern "C" int kl_poll(kl_runtime* rt, kl_handle h, int* state) {
  if (!rt || !state) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  int p = progress(rt);
  if (p != KL_OK && p != KL_EAGAIN) return p;
  kl_tenant_stats st;
  int rc = lookup(rt, h, &st);
  if (rc) return rc;
  *state = st.state;
  return KL_OK;
}

extern "C" int kl_wait(kl_runtime* rt, kl_handle h, uint64_t timeout_ns) {
  if (!rt) return KL_EINVAL;
  std::unique_lock<std::mutex> lk(rt->mu);
  kl_tenant_stats st;
  int rc = lookup(rt, h, &st);
  if (rc) return rc;
  if (st.state == KL_PENDING) return KL_ESTATE;  // not launched: waiting would never end
  const uint64_t t0 = now_ns();
  for (uint32_t spins = 0; st.state == KL_RUNNING; ++spins) {
    int p = progress(rt);
    if (p == KL_ECUDA) return p;
    rc = lookup(rt, h, &st);
    if (rc) return rc;
    if (st.state != KL_RUNNING) break;
    if (now_ns() - t0 >= timeout_ns) return KL_ETIMEDOUT;
    lk.unlock();
    if (spins < 64)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    lk.lock();
  }
  return st.state == KL_DONE ? KL_OK : (st.error ? st.error : KL_ESTATE);
}

extern "C" int kl_drain(kl_runtime* rt, uint64_t timeout_ns) {
  if (!rt) return KL_EINVAL;
  std::unique_lock<std::mutex> lk(rt->mu);
  if (rt->serve_on) return KL_ESTATE;
  int rc;
  if (rt->in_flight) {
    rc = wait_flight(rt, lk, timeout_ns);
    if (rc == KL_ETIMEDOUT || rc == KL_ECUDA) return rc;
  }
  if (!rt->pending.empty()) {
    rc = launch_locked(rt);
    if (rc) return rc;
  }
  if (rt->in_flight) {
    rc = wait_flight(rt, lk, timeout_ns);
    if (rc == KL_ETIMEDOUT || rc == KL_ECUDA) return rc;
  }
  return rt->last.error;
}

extern "C" int kl_wait_run(kl_runtime* rt, uint64_t timeout_ns) {
  if (!rt) return KL_EINVAL;
  std::unique_lock<std::mutex> lk(rt->mu);
  if (rt->serve_on) return KL_ESTATE;
  if (rt->in_flight) {
    const int rc = wait_flight(rt, lk, timeout_ns);
    if (rc == KL_ETIMEDOUT || rc == KL_ECUDA) return rc;
  }
  return rt->last.error;
}

extern "C" int kl_get_stats(kl_runtime* rt, kl_handle h, kl_tenant_stats* out) {
  if (!rt || !out) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  progress(rt);
  return lookup(rt, h, out);
}

extern "C" int kl_get_run_stats(kl_runtime* rt, kl_run_stats* out) {
  if (!rt || !out) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  progress(rt);
  *out = rt->last;
  if (out->slots_per_sm == 0) {  // no run retired yet: the plain build's
    out->slots_per_sm = rt->slots;
    out->grid_ctas = rt->slots * rt->n_sm;
  }
  return KL_OK;
}

extern "C" int kl_get_phases(kl_runtime* rt, kl_phase* out, uint32_t cap, uint32_t* n) {
  if (!rt || !n || (cap && !out)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  progress(rt);
  *n = (uint32_t)rt->last_phases.size();
  for (uint32_t i = 0; i < cap && i < *n; ++i) out[i] = rt->last_phases[i];
  return KL_OK;
}

extern "C" int kl_set_profiles(kl_runtime* rt, const kl_profile* p, uint32_t n) {
  if (!rt || !p || n > KL_T_COUNT) return KL_EINVAL;
  for (uint32_t t = 0; t < n; ++t)
    if (p[t].valid && (!(p[t].R_m >= 0.0 && p[t].R_m <= 1.0) || !(p[t].f_u >= 0.0 && p[t].f_u <= 1.0) ||
                       !(p[t].L0 >= 0.0) || !(p[t].I_block > 0.0) || p[t].warps_per_block == 0))
      return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  for (uint32_t t = 0; t < n; ++t)
    if (p[t].valid) rt->prof[t] = p[t];
  rt->table_valid = false;
  return KL_OK;
}

extern "C" int kl_set_model_params(kl_runtime* rt, const kl_model_params* mp) {
  if (!rt || !mp || mp->n_sm == 0 || mp->n_sched == 0 || !(mp->f_sm_hz > 0) || !(mp->dram_bytes_per_s > 0) ||
      !(mp->sector_bytes > 0))
    return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  rt->mp = *mp;
  rt->table_valid = false;
  return KL_OK;
}

extern "C" int kl_get_model_params(kl_runtime* rt, kl_model_params* out) {
  if (!rt || !out) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  *out = rt->mp;
  return KL_OK;
}

extern "C" int kl_set_cp_table(kl_runtime* rt, const double* cp, const uint32_t* slots_a) {
  if (!rt || (!cp) != (!slots_a)) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  if (!cp) {
    rt->table_override = false;
    rt->table_valid = false;
    return KL_OK;
  }
  for (uint32_t k = 0; k < KL_T_COUNT * KL_T_COUNT; ++k)
    if (slots_a[k] < 1 || slots_a[k] + 1 > rt->slots || !std::isfinite(cp[k])) return KL_EINVAL;
  for (uint32_t i = 0; i < KL_T_COUNT; ++i)
    for (uint32_t j = 0; j < KL_T_COUNT; ++j) {
      rt->cp[i][j] = cp[i * KL_T_COUNT + j];
      rt->slots_a[i][j] = slots_a[i * KL_T_COUNT + j];
      rt->allowed[i][j] = 1;
    }
  rt->table_override = true;
  rt->table_valid = true;
  rt->table_types = (1u << KL_T_COUNT) - 1u;
  return KL_OK;
}

extern "C" int kl_get_cp_table(kl_runtime* rt, double* cp, uint32_t* slots_a, uint8_t* allowed) {
  if (!rt) return KL_EINVAL;
  std::lock_guard<std::mutex> lk(rt->mu);
  int rc = ensure_table(rt, (1u << KL_T_COUNT) - 1, rt->slots);
  if (rc) return rc;
  for (uint32_t i = 0; i < KL_T_COUNT; ++i)
    for (uint32_t j = 0; j < KL_T_COUNT; ++j) {
      if (cp) cp[i * KL_T_COUNT + j] = rt->cp[i][j];
      if (slots_a) slots_a[i * KL_T_COUNT + j] = rt->slots_a[i][j];
      if (allowed) allowed[i * KL_T_COUNT + j] = (uint8_t)rt->allowed[i][j];
    }
  return KL_OK;
}
