// Persistent co-scheduler kernel: the device half of Kernelet's Algorithm 1.
//
// grid = numSM x S CTAs of 256 threads; each CTA takes a per-SM slot number
// from a ticket on its %smid. The current co-schedule <K1, K2, size1, size2>
// (Algorithm 1) is a published phase: slots [0, size1) of every SM run K1 and
// slots [size1, S) run K2, so size1 * numSM blocks of K1 and size2 * numSM
// blocks of K2 are co-resident, the pair's slice ratio. A CTA pulls its next
// slice — a contiguous range of the kernel's block IDs (Section 2.2) — with
// one atomicAdd on the kernel's queue counter and runs it with rectified block
// indices (Section 4.1). When a kernel has handed out its last block, the CTA
// that sees it claims the re-plan and runs FindCoSchedule (Algorithm 1,
// procedure) over the pending set on the device: the largest CP pair among
// the unpruned candidates, CP and balanced slot split taken from the table the
// Markov model (Section 4.4) filled in on the host. Multi-stage kernels are
// chains of grids: blocks of stage s run only after stage s-1 completed.
//
// Serving mode keeps the kernel running while the host keeps submitting:
// kernels are numbered by submission and live in a ring of tenant slots; CTA 0
// is a dispatcher that copies newly published descriptors from mapped host
// memory into the device ring and re-plans on every arrival (Algorithm 1: a
// new kernel joins R and the co-schedule is recomputed on the residuals).
//
// No wait in this kernel is unbounded: every spin has a globaltimer deadline
// after which the run records KL_EDEVICE_TIMEOUT (or, when serving and idle,
// ends the run) and every CTA returns.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>

#include "kl_internal.h"
#include "tenants.cuh"

namespace kl {

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smid() {
  uint32_t s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// host-mapped words (system scope)
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// SplitMix64 finaliser (Steele, Lea and Flood 2014; Vigna's constants): the
// random plans of KL_CFG_RANDOM_PLAN are a function of (seed, phase number).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Co-resident CTAs per SM: 4 x 256 threads at up to 64 registers each (plain
// and full builds), 8 x 256 at up to 32 registers (light build).
constexpr int kCtasPerSm = 4;
constexpr int kCtasPerSmLight = 8;
constexpr int ctas_per_sm(int build) { return build == tn::kBuildLight ? kCtasPerSmLight : kCtasPerSm; }

enum : uint32_t { kActRun = 0, kActWait = 1, kActExit = 2, kActReplan = 3, kActIntake = 4 };
enum : int { kPulled = 0, kBlocked = 1, kExhausted = 2 };

struct CtaCtl {
  int32_t tenant;
  uint32_t g0, g1;
  uint32_t action;
  uint32_t seq;
  int32_t trigger;
  int32_t wait_failed;
  uint32_t from, to;   // dispatcher: kernels to copy in
  uint32_t mine;       // dispatcher: this CTA claimed the re-plan
  uint32_t own;        // the slice came from this slot's own kernel in the current phase
  uint32_t own_seq;    // ... the phase that gave the slot that kernel
  int32_t pf_tenant;   // a slice claimed ahead while the previous one ran (-1: none)
  uint32_t pf_g0, pf_g1;
  uint32_t pf_more;    // the phase was still own_seq when that slice was claimed
  uint32_t backoff;    // thread 0: current sleep between polls (ns)
  unsigned long long wait_since;  // thread 0: start of the current wait (0: not waiting)
  int32_t args_of;     // kernel whose arguments s_args holds (-1: none)
  unsigned long long acc_wait, acc_stage, acc_plan;  // this CTA's time accounting (thread 0)
};

__device__ __forceinline__ void set_error(RunDev* R, int32_t code, uint32_t info) {
  if (atomicCAS(reinterpret_cast<int*>(&R->error), 0, code) == 0) R->error_info = info;
}

__device__ __forceinline__ TenantDev& tenant(TenantDev* T, const RunDev* R, uint32_t seq) {
  return T[seq & R->ring_mask];
}
__device__ __forceinline__ PhaseDev* phase(PhaseDev* P, const RunDev* R, uint32_t seq) {
  return &P[seq & R->phase_mask];
}

// Thread 0 only: try to take the next slice of tenant t. `rank` is this CTA's
// position among the slots of its SM that serve t: while the stage has fewer
// blocks left than rank * numSM, the slot leaves them to lower ranks, so a
// kernel with few blocks spreads one per SM instead of stacking on some SMs.
// Stage containing cumulative block g, from the descriptor's block counts
// (no argument parsing on the scheduler's path).
__device__ __forceinline__ tn::Stage stage_at(const TenantDev& d, uint32_t type, uint32_t g) {
  const uint32_t total = d.total, b0 = d.blocks0;
  if (d.nstages == 1u) return tn::Stage{0u, 0u, total};
  if (type == KL_T_BITONIC) {
    const uint32_t s = g / b0;
    return tn::Stage{s, s * b0, (s + 1u) * b0};
  }
  return g < b0 ? tn::Stage{0u, 0u, b0} : tn::Stage{1u, b0, total};
}

__device__ __forceinline__ int try_pull(TenantDev* T, const RunDev* R, int32_t t, uint32_t rank, uint32_t n_sm,
                                        uint32_t& g0, uint32_t& g1) {
  TenantDev& d = tenant(T, R, (uint32_t)t);
  // serving: a phase read just before the slot was refilled names an older kernel
  if (d.index != (uint32_t)t) return kExhausted;
  const uint32_t total = d.total;
  uint32_t n = ld_relaxed(&d.next);
  if (n >= total) return kExhausted;
  tn::Stage st = stage_at(d, d.type, n);
  if (st.begin > ld_relaxed(&d.done)) return kBlocked;  // previous stage still running
  if ((uint64_t)rank * n_sm >= (uint64_t)(st.end - n)) return kBlocked;
  uint32_t a = atomicAdd(&d.next, d.slice);
  if (a >= total) return kExhausted;
  g0 = a;
  g1 = min(a + d.slice, total);
  if (a == 0) {
    d.t_start = gtimer();
    d.status = KL_RUNNING;
  }
  if (g1 == total) d.drained = 1u;
  atomicAdd(&d.slices, 1u);
  return kPulled;
}

// Per-warp partial results of the pending-set scan, in the re-planning CTA's
// dynamic shared memory (free between tenant blocks).
struct ScanPart {
  uint32_t npend;
  int32_t first;
  unsigned long long pmask;
  uint32_t nlow, nms;
  int32_t lowp[kFill + 2];
  int32_t lowms[4];
  int32_t low1[KL_T_MAIN_COUNT], low2[KL_T_MAIN_COUNT];
};
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kPlanScratch = sizeof(ScanPart) * kWarps + 16;
static_assert(kPlanScratch <= tn::kMinCtaSmem, "re-plan scratch fits the smallest dynamic shared memory");

// FindCoSchedule on the device (Algorithm 1, procedure), all threads of one
// CTA. Pending = kernels with blocks not yet handed out, among sequence
// numbers [scan_lo, end) (end = kernels submitted; in serving mode, copied
// in); each warp scans a contiguous eighth of that range and thread 0 merges
// the eight partial results in order. For every pair of pending kernels CP
// depends only on their types, so the best pair of a type pair is its two
// lowest sequence numbers; the winner is the largest CP among unpruned type
// pairs (all pairs when every one is pruned), ties to the smallest (i, j). One
// pending kernel runs alone on every slot; none ends a batch run, or idles a
// serving run until the next arrival.
__device__ __noinline__ void replan(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t seq_old, int32_t trigger, char* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ScanPart* parts = reinterpret_cast<ScanPart*>(smem);
  uint32_t* bounds = reinterpret_cast<uint32_t*>(parts + kWarps);
  if (threadIdx.x == 0) {
    bounds[0] = ld_relaxed(&R->scan_lo);
    bounds[1] = R->serve ? ld_acquire(&R->intake) : R->n_tenants;
  }
  __syncthreads();
  const uint32_t lo = bounds[0], hi = bounds[1];
  {
    int32_t low1[KL_T_MAIN_COUNT], low2[KL_T_MAIN_COUNT];
#pragma unroll
    for (int t = 0; t < KL_T_MAIN_COUNT; ++t) low1[t] = low2[t] = -1;
    uint32_t npend = 0, nlow = 0, nms = 0;
    unsigned long long pmask = 0ull;
    int32_t lowp[kFill + 2], lowms[4];
    int32_t first_pending = -1;
    const uint32_t nchunk = hi > lo ? (hi - lo + 31u) / 32u : 0u;
    const uint32_t cpw = (nchunk + kWarps - 1) / kWarps;
    const uint32_t b0 = lo + 32u * min(nchunk, (uint32_t)warp * cpw);
    const uint32_t b1 = lo + 32u * min(nchunk, (uint32_t)(warp + 1) * cpw);
    for (uint32_t base = b0; base < b1; base += 32) {
      const uint32_t i = base + lane;
      bool pend = false, multi = false;
      uint32_t ty = 0;
      if (i < hi) {
        const TenantDev& d = tenant(T, R, i);
        // static fields through L2: in serving mode the slot may have been refilled
        ty = __ldcg(&d.type);
        // kernels of the resource-heavy classes are their class kernels' business
        pend = ld_relaxed(&d.next) < __ldcg(&d.total) && tn::resource_class(ty) == tn::kClassMain;
        multi = __ldcg(&d.nstages) > 1u;
      }
      const uint32_t pb = __ballot_sync(0xffffffffu, pend);
      npend += __popc(pb);
      if (pb && first_pending < 0) first_pending = (int32_t)(base + __ffs(pb) - 1);
      if (base < 64) pmask |= (unsigned long long)pb << base;
      for (uint32_t m = pb; m && nlow < (uint32_t)kFill + 2u; m &= m - 1) lowp[nlow++] = (int32_t)(base + __ffs(m) - 1);
      const uint32_t msb = __ballot_sync(0xffffffffu, pend && multi);
      for (uint32_t m = msb; m && nms < 4; m &= m - 1) lowms[nms++] = (int32_t)(base + __ffs(m) - 1);
#pragma unroll
      for (int t = 0; t < KL_T_MAIN_COUNT; ++t) {
        uint32_t m = __ballot_sync(0xffffffffu, pend && ty == (uint32_t)t);
        if (m && low1[t] < 0) {
          low1[t] = (int32_t)(base + __ffs(m) - 1);
          m &= m - 1;
        }
        if (m && low2[t] < 0) low2[t] = (int32_t)(base + __ffs(m) - 1);
      }
    }
    if (lane == 0) {
      ScanPart& q = parts[warp];
      q.npend = npend;
      q.first = first_pending;
      q.pmask = pmask;
      q.nlow = nlow;
      q.nms = nms;
      for (uint32_t f = 0; f < nlow; ++f) q.lowp[f] = lowp[f];
      for (uint32_t f = 0; f < nms; ++f) q.lowms[f] = lowms[f];
#pragma unroll
      for (int t = 0; t < KL_T_MAIN_COUNT; ++t) {
        q.low1[t] = low1[t];
        q.low2[t] = low2[t];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  // merge in warp order (warp w scanned lower sequence numbers than warp w+1)
  int32_t low1[KL_T_MAIN_COUNT], low2[KL_T_MAIN_COUNT];
  for (int t = 0; t < KL_T_MAIN_COUNT; ++t) low1[t] = low2[t] = -1;
  uint32_t npend = 0, nlow = 0, nms = 0;
  unsigned long long pmask = 0ull;
  int32_t lowp[kFill + 2], lowms[4];
  int32_t first_pending = -1;
  for (int w = 0; w < kWarps; ++w) {
    const ScanPart& q = parts[w];
    npend += q.npend;
    pmask |= q.pmask;
    if (first_pending < 0) first_pending = q.first;
    for (uint32_t f = 0; f < q.nlow && nlow < (uint32_t)kFill + 2u; ++f) lowp[nlow++] = q.lowp[f];
    for (uint32_t f = 0; f < q.nms && nms < 4; ++f) lowms[nms++] = q.lowms[f];
    for (int t = 0; t < KL_T_MAIN_COUNT; ++t) {
      const int32_t c[2] = {q.low1[t], q.low2[t]};
      for (int k = 0; k < 2; ++k) {
        if (c[k] < 0) break;
        if (low1[t] < 0)
          low1[t] = c[k];
        else if (low2[t] < 0)
          low2[t] = c[k];
      }
    }
  }
  // kernels below the first pending one are all handed out: skip them next time
  st_release(&R->scan_lo, first_pending >= 0 ? (uint32_t)first_pending : hi);
  PhaseDev ph;
  ph.A = R->serve ? kPhaseIdle : kPhaseEnd;
  ph.B = -1;
  ph.slots_a = R->slots;
  ph.slots_b = 0;
  ph.cp = 0.0;
  ph.trigger = trigger;
  ph.n_pending = npend;
  ph.pending = pmask;
  ph.intake_seen = hi;
  ph.pad2 = 0;
  if (npend == 1) {
    for (int t = 0; t < KL_T_MAIN_COUNT; ++t)
      if (low1[t] >= 0) ph.A = low1[t];
  } else if (npend >= 2) {
    int32_t aged = -1;
    // MC comparison (KL_CFG_RANDOM_PLAN): a uniformly random pair of pending
    // kernel types (the lowest pending kernel of each) and a random split
    if ((R->flags & KL_CFG_RANDOM_PLAN) && R->slots >= 2) {
      const unsigned long long r = splitmix64(R->plan_seed ^ (0xD1B54A32D192ED03ull * (seq_old + 1ull)));
      uint32_t nc = 0;
      for (int ta = 0; ta < KL_T_MAIN_COUNT; ++ta)
        for (int tb = ta; tb < KL_T_MAIN_COUNT; ++tb)
          nc += low1[ta] >= 0 && (ta == tb ? low2[ta] >= 0 : low1[tb] >= 0);
      uint32_t pick = (uint32_t)((r & 0xFFFFFFFFull) % nc);
      for (int ta = 0; ta < KL_T_MAIN_COUNT && aged < 0; ++ta)
        for (int tb = ta; tb < KL_T_MAIN_COUNT && aged < 0; ++tb) {
          if (!(low1[ta] >= 0 && (ta == tb ? low2[ta] >= 0 : low1[tb] >= 0))) continue;
          if (pick-- != 0u) continue;
          ph.A = min(low1[ta], ta == tb ? low2[ta] : low1[tb]);
          ph.B = max(low1[ta], ta == tb ? low2[ta] : low1[tb]);
          ph.slots_a = 1u + (uint32_t)((r >> 32) % (R->slots - 1u));
          ph.slots_b = R->slots - ph.slots_a;
          ph.cp = R->cp[tenant(T, R, (uint32_t)ph.A).type][tenant(T, R, (uint32_t)ph.B).type];
          aged = ph.A;  // a pair is chosen: skip the selections below
        }
    }
    // serving: the oldest pending kernel (lowest sequence number) has waited
    // past the age limit: it goes first, with its best partner by CP
    if (aged < 0 && R->serve && first_pending >= 0 && R->age_limit_ns != ~0ull) {
      const unsigned long long ta = __ldcg(&tenant(T, R, (uint32_t)first_pending).t_arrive);
      if (ta != 0ull && gtimer() - ta > R->age_limit_ns) aged = first_pending;
    }
    if (aged >= 0 && ph.B < 0) {
      const uint32_t tya = tenant(T, R, (uint32_t)aged).type;
      double best = 0.0;
      int32_t bj = -1;
      for (int pass = 0; pass < 2 && bj < 0; ++pass)
        for (int tb = 0; tb < KL_T_MAIN_COUNT; ++tb) {
          const int32_t j = low1[tb] != aged ? low1[tb] : low2[tb];
          if (j < 0) continue;
          const uint32_t tyj = tenant(T, R, (uint32_t)j).type;
          if (pass == 0 && !R->allowed[tya][tyj]) continue;
          const double c = R->cp[tya][tyj];
          if (bj < 0 || c > best + 1e-12 || (fabs(c - best) <= 1e-12 && j < bj)) {
            best = c;
            bj = j;
          }
        }
      if (bj >= 0) {
        ph.A = aged;
        ph.B = bj;
        ph.cp = best;
        ph.slots_a = R->slots_a[tya][tenant(T, R, (uint32_t)bj).type];
        ph.slots_b = R->slots - ph.slots_a;
      }
    }
    for (int pass = 0; pass < 2 && aged < 0; ++pass) {
      double best = 0.0;
      int32_t bi = -1, bj = -1;
      for (int ta = 0; ta < KL_T_MAIN_COUNT; ++ta) {
        if (low1[ta] < 0) continue;
        for (int tb = ta; tb < KL_T_MAIN_COUNT; ++tb) {
          int32_t i, j;
          if (ta == tb) {
            if (low2[ta] < 0) continue;
            i = low1[ta];
            j = low2[ta];
          } else {
            if (low1[tb] < 0) continue;
            i = min(low1[ta], low1[tb]);
            j = max(low1[ta], low1[tb]);
          }
          const uint32_t tyi = tenant(T, R, i).type, tyj = tenant(T, R, j).type;
          if (pass == 0 && !R->allowed[tyi][tyj]) continue;
          const double c = R->cp[tyi][tyj];
          // CP equal within 1e-12 is a tie, resolved to the smaller (i, j)
          const bool tie = fabs(c - best) <= 1e-12;
          if (bi < 0 || (!tie && c > best) || (tie && (i < bi || (i == bi && j < bj)))) {
            best = c;
            bi = i;
            bj = j;
          }
        }
      }
      if (bi >= 0) {
        ph.A = bi;
        ph.B = bj;
        ph.cp = best;
        ph.slots_a = R->slots_a[tenant(T, R, bi).type][tenant(T, R, bj).type];
        ph.slots_b = R->slots - ph.slots_a;
        break;
      }
    }
  }
  // backfill candidates: the next pending kernel of A's type and of B's type
  // (more of the work the pair is doing), then the lowest pending multi-stage
  // kernel (a long chain of dependent grids: started early, its stage
  // barriers overlap other work instead of forming the tail of the run), then
  // the lowest pending sequence numbers
  for (int f = 0; f < kFill; ++f) ph.fill[f] = -1;
  // two candidates per slot of an SM (8 at 4 slots, 16 at 8): kernels with
  // fewer blocks than the GPU has slots still fill it
  const uint32_t nfill = (R->flags & KL_CFG_WIDE_FILL) ? min((uint32_t)kFill, 2u * R->slots) : 4u;
  uint32_t c = 0;
  if (ph.A >= 0 && (R->flags & KL_CFG_FILL_TYPES)) {
    const uint32_t ta = tenant(T, R, ph.A).type;
    const int32_t sa = low1[ta] != ph.A ? low1[ta] : low2[ta];
    if (sa >= 0 && sa != ph.B) ph.fill[c++] = sa;
    if (ph.B >= 0) {
      const uint32_t tb = tenant(T, R, ph.B).type;
      const int32_t sb = low1[tb] != ph.B ? low1[tb] : low2[tb];
      if (sb >= 0 && sb != ph.A && (c == 0 || sb != ph.fill[0])) ph.fill[c++] = sb;
    }
  }
  // chain lane: the two lowest multi-stage kernels outside the pair
  ph.chain[0] = ph.chain[1] = -1;
  {
    uint32_t nc = 0;
    for (uint32_t f = 0; f < nms && nc < 2; ++f)
      if (lowms[f] != ph.A && lowms[f] != ph.B) ph.chain[nc++] = lowms[f];
  }
  for (int k = 0; k < 2 && c < nfill; ++k) {
    bool dup = ph.chain[k] < 0;
    for (uint32_t q = 0; q < c; ++q) dup |= ph.chain[k] == ph.fill[q];
    if (!dup) ph.fill[c++] = ph.chain[k];
    if (!(R->flags & KL_CFG_WIDE_FILL)) break;  // the narrow list takes the lowest chain only
  }
  for (uint32_t f = 0; f < nlow && c < nfill; ++f) {
    bool dup = lowp[f] == ph.A || lowp[f] == ph.B;
    for (uint32_t q = 0; q < c; ++q) dup |= lowp[f] == ph.fill[q];
    if (!dup) ph.fill[c++] = lowp[f];
  }
  const uint32_t seq = seq_old + 1;
  if (!R->serve && seq >= R->max_phases) {
    set_error(R, KL_EOVERFLOW, seq);
    ph.A = kPhaseEnd;
    ph.B = -1;
  }
  // block counts at this instant: per-phase measured progress of each kernel
  ph.done_a = ph.A >= 0 ? ld_relaxed(&tenant(T, R, ph.A).done) : 0u;
  ph.done_b = ph.B >= 0 ? ld_relaxed(&tenant(T, R, ph.B).done) : 0u;
  {
    const int32_t pa = __ldcg(&phase(P, R, seq_old)->A), pb = __ldcg(&phase(P, R, seq_old)->B);
    ph.prev_done_a = pa >= 0 ? ld_relaxed(&tenant(T, R, pa).done) : 0u;
    ph.prev_done_b = pb >= 0 ? ld_relaxed(&tenant(T, R, pb).done) : 0u;
  }
  ph.t = gtimer();
  const uint32_t slot = R->serve ? seq : min(seq, R->max_phases - 1);
  *phase(P, R, slot) = ph;
  __threadfence();
  st_release(&R->phase_seq, slot);
}

__device__ __forceinline__ void complete_tenant(TenantDev& d, RunDev* R) {
  unsigned long long now = gtimer();
  d.t_end = now;
  __threadfence();
  st_release(&d.status, KL_DONE);
  if (R->serve) {
    // the host reaps completions from the queue while the run goes on: the
    // record first, then the queue entry that publishes it
    ServeDone& r = R->host_done[d.index & R->ring_mask];
    r.slices = d.slices;
    r.blocks = d.total;
    r.t_start = d.t_start;
    r.t_end = now;
    r.seq1 = d.index + 1u;
    __threadfence_system();
    const uint32_t pos = atomicAdd(&R->cq_pos, 1u);
    st_release_sys64(R->host_cq + (pos & R->ring_mask), ((unsigned long long)(pos + 1u) << 32) | d.index);
  }
  atomicAdd(&R->n_complete, 1u);
  atomicMax(&R->t_end, now);
}

// Serving mode, CTA 0: copy arrivals in, re-plan, end the run on request.
__device__ void dispatcher(TenantDev* T, RunDev* R, PhaseDev* P, CtaCtl& ctl, char* smem) {
  const int tid = threadIdx.x;
  unsigned long long last_arrival = gtimer();
  unsigned long long stop_since = 0;
  for (;;) {
    if (tid == 0) {
      ctl.action = kActWait;
      const unsigned long long now = gtimer();
      const uint32_t intake = ld_relaxed(&R->intake);
      const uint32_t tail = ld_acquire_sys(R->host_ctl);
      const uint32_t room = ld_relaxed(&R->scan_lo) + R->ring_mask + 1u;  // slots the device may fill
      if (ld_relaxed(reinterpret_cast<uint32_t*>(&R->error)) != 0) {
        ctl.action = kActExit;
      } else if (tail > intake && room > intake) {
        ctl.action = kActIntake;
        ctl.from = intake;
        ctl.to = min(tail, room);
        last_arrival = now;
      } else {
        const bool quiet = ld_relaxed(&R->n_complete) == intake && tail == intake;
        const bool stop = ld_acquire_sys(R->host_ctl + 32) != 0;
        if (quiet && (stop || now - last_arrival > R->idle_limit_ns)) {
          // end of the run: publish the final phase (claimed like a re-plan)
          if (stop_since == 0) stop_since = now;
          const uint32_t seq = ld_acquire(&R->phase_seq);
          if (ld_relaxed(&R->phase_claim) == seq && atomicCAS(&R->phase_claim, seq, seq + 1) == seq) {
            PhaseDev* e = phase(P, R, seq + 1);
            e->A = kPhaseEnd;
            e->B = -1;
            e->chain[0] = e->chain[1] = -1;
            e->intake_seen = intake;
            e->t = now;
            __threadfence();
            st_release(&R->phase_seq, seq + 1);
            ctl.action = kActExit;
          } else if (now - stop_since > R->wait_limit_ns) {
            set_error(R, KL_EDEVICE_TIMEOUT, 4u);
            ctl.action = kActExit;
          }
        }
      }
      if (ctl.action == kActWait) __nanosleep(256);
    }
    __syncthreads();
    const uint32_t action = ctl.action;
    if (action == kActExit) return;
    if (action == kActIntake) {
      if (tid < 32) {
        // 256-byte descriptors, 8 bytes per lane; the host zeroed the dynamic part
        for (uint32_t s = ctl.from; s < ctl.to; ++s) {
          const unsigned long long* src =
              reinterpret_cast<const unsigned long long*>(&R->host_ring[s & R->ring_mask]);
          unsigned long long* dst = reinterpret_cast<unsigned long long*>(&T[s & R->ring_mask]);
          dst[tid] = ld_volatile64(src + tid);
        }
        __syncwarp();
        if (tid == 0) {
          const unsigned long long now = gtimer();
          for (uint32_t s = ctl.from; s < ctl.to; ++s) T[s & R->ring_mask].t_arrive = now;
        }
        __threadfence();
      }
      __syncthreads();
      // re-plan on arrival (Algorithm 1); if a re-plan is already running,
      // the workers see intake > intake_seen and ask for another
      if (tid == 0) {
        st_release(&R->intake, ctl.to);
        const uint32_t seq = ld_acquire(&R->phase_seq);
        ctl.seq = seq;
        // KL_CFG_LAZY_ARRIVAL: a running pair keeps the GPU; arrivals join R
        // and are planned when a kernel of the pair runs out
        const bool pair_running = __ldcg(&phase(P, R, seq)->B) >= 0;
        ctl.mine = !((R->flags & KL_CFG_LAZY_ARRIVAL) && pair_running) && ld_relaxed(&R->phase_claim) == seq &&
                   atomicCAS(&R->phase_claim, seq, seq + 1) == seq;
      }
      __syncthreads();
      if (ctl.mine) replan(T, R, P, ctl.seq, -1, smem);
    }
    __syncthreads();
  }
}

// BUILD: tn::kBuildPlain, kBuildFull (the only one that can run the
// tensor-core BF16 GEMM tenant) or kBuildLight; the host picks the smallest
// build that holds every type of the run (see tn::run_block).
template <int BUILD>
__global__ void __launch_bounds__(kThreads, ctas_per_sm(BUILD)) cosched_kernel(TenantDev* __restrict__ T, RunDev* __restrict__ R,
                                                                      PhaseDev* __restrict__ P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaCtl ctl;
  __shared__ uint32_t s_slot;
  __shared__ uint32_t s_tmem;  // TMEM columns of this CTA (BF16 GEMM blocks)
  __shared__ __align__(16) unsigned char s_args[KL_MAX_ARGS_BYTES];  // arguments of the running slice
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint32_t sm = smid() & (kMaxSM - 1);
    const uint32_t ticket = atomicAdd(&R->sm_ticket[sm], 1u);
    // with resource classes beside it the grid carries extra CTAs and each
    // SM keeps `slots` of them; the others leave at once, freeing the room
    s_slot = (R->quota_exit && ticket >= R->slots) ? 0xffffffffu : ticket % R->slots;
    atomicCAS(&R->t_launch, 0ull, gtimer());
  }
  __syncthreads();
  if (s_slot == 0xffffffffu) return;
  const tn::BlockCtx tcx{&s_tmem, &R->error, R->wait_limit_ns};
  if constexpr (BUILD == tn::kBuildFull) tn::acquire_tmem(tcx);
  if (R->serve && blockIdx.x == 0) {
    dispatcher(T, R, P, ctl, smem);
    if constexpr (BUILD == tn::kBuildFull) tn::release_tmem(tcx);
    if (tid == 0) atomicAdd(&R->ctas_done, 1u);
    return;
  }
  // The loop keeps no scheduler state in registers across a slice: thread 0
  // re-reads it from shared memory and the run state at each decision, so the
  // tenant bodies get the registers (at the light build's 32 they spill
  // otherwise).
  if (tid == 0) {
    ctl.wait_since = 0ull;
    ctl.backoff = 32u;
    ctl.acc_wait = ctl.acc_stage = ctl.acc_plan = 0ull;
    ctl.pf_tenant = -1;
    ctl.args_of = -1;
  }

  for (;;) {
    if (tid == 0) {
      const uint32_t slot = s_slot;
      const uint32_t S = R->slots;
      const uint32_t n_sm = R->n_sm;
      const unsigned long long limit = R->wait_limit_ns;
      ctl.action = kActWait;
      ctl.tenant = -1;
      ctl.own = 0;
      bool idle = false;
      if (ld_relaxed(reinterpret_cast<uint32_t*>(&R->error)) != 0) {
        ctl.action = kActExit;
      } else if (ctl.pf_tenant >= 0) {
        // run the slice claimed ahead (its blocks are this CTA's now) and
        // claim the one after it again while it runs
        ctl.action = kActRun;
        ctl.tenant = ctl.pf_tenant;
        ctl.g0 = ctl.pf_g0;
        ctl.g1 = ctl.pf_g1;
        ctl.own = ctl.pf_more;  // a re-plan since: this slice, then the phase again
        ctl.pf_tenant = -1;
      } else {
        const uint32_t seq = ld_acquire(&R->phase_seq);
        PhaseDev* pp = phase(P, R, seq);  // published by another CTA: read through L2
        PhaseDev ph;
        ph.A = __ldcg(&pp->A);
        ph.B = __ldcg(&pp->B);
        ph.slots_a = __ldcg(&pp->slots_a);
        if (ph.A == kPhaseEnd) {
          ctl.action = kActExit;
        } else {
          bool need_replan = ph.A == kPhasePlan;
          int32_t trig = -1;
          // serving: kernels arrived after this plan was made; re-plan now
          if (R->serve && ld_relaxed(&R->intake) > __ldcg(&pp->intake_seen) &&
              !((R->flags & KL_CFG_LAZY_ARRIVAL) && __ldcg(&pp->B) >= 0) && ld_relaxed(&R->phase_claim) == seq &&
              atomicCAS(&R->phase_claim, seq, seq + 1) == seq) {
            ctl.action = kActReplan;
            ctl.seq = seq;
            ctl.trigger = -1;
          }
          idle = ph.A == kPhaseIdle;
          // chain lane: the last slot of every SM serves pending multi-stage
          // kernels first (their stage barriers then overlap the pair's work)
          if (ph.A >= 0 && ctl.action == kActWait && (R->flags & KL_CFG_CHAIN_LANE) && slot + R->chain_slots >= S) {
            for (int f = 0; f < 2; ++f) {
              const int32_t c = __ldcg(&pp->chain[f]);
              if (c < 0) break;
              uint32_t g0 = 0, g1 = 0;
              if (try_pull(T, R, c, 0u, n_sm, g0, g1) == kPulled) {
                ctl.action = kActRun;
                ctl.tenant = c;
                ctl.g0 = g0;
                ctl.g1 = g1;
                break;
              }
            }
          }
          if (ph.A >= 0 && ctl.action == kActWait) {
            const bool mine_is_b = ph.B >= 0 && slot >= ph.slots_a;
            const int32_t t1 = mine_is_b ? ph.B : ph.A;
            const int32_t t2 = mine_is_b ? ph.A : ph.B;
            const uint32_t rank1 = mine_is_b ? slot - ph.slots_a : slot;
            const uint32_t rank2 = mine_is_b ? slot : slot + (S - ph.slots_a);
            uint32_t g0 = 0, g1 = 0;
            int r = try_pull(T, R, t1, rank1, n_sm, g0, g1);
            if (r == kPulled) {
              ctl.action = kActRun;
              ctl.tenant = t1;
              ctl.g0 = g0;
              ctl.g1 = g1;
              ctl.own = 1;
              ctl.own_seq = seq;
            } else {
              if (r == kExhausted) {
                need_replan = true;
                trig = t1;
              }
              // the phase is over for this slot: re-plan first if nobody else does
              if (need_replan && ld_relaxed(&R->phase_claim) == seq &&
                  atomicCAS(&R->phase_claim, seq, seq + 1) == seq) {
                ctl.action = kActReplan;
                ctl.seq = seq;
                ctl.trigger = trig;
              } else if (t2 >= 0) {
                int r2 = try_pull(T, R, t2, rank2, n_sm, g0, g1);
                if (r2 == kPulled) {
                  ctl.action = kActRun;
                  ctl.tenant = t2;
                  ctl.g0 = g0;
                  ctl.g1 = g1;
                } else if (r2 == kExhausted) {
                  need_replan = true;
                  trig = t2;
                }
              }
            }
          }
          if (ctl.action == kActWait && need_replan && ld_relaxed(&R->phase_claim) == seq &&
              atomicCAS(&R->phase_claim, seq, seq + 1) == seq) {
            ctl.action = kActReplan;
            ctl.seq = seq;
            ctl.trigger = trig;
          }
          // backfill: the pair cannot use this slot right now (stage barrier,
          // spread rule, re-plan in flight), so take a slice of another
          // pending kernel instead of idling
          if (ctl.action == kActWait && (R->flags & KL_CFG_BACKFILL) && ph.A >= 0) {
            for (int f = 0; f < kFill; ++f) {
              const int32_t c = __ldcg(&pp->fill[f]);
              if (c < 0) break;
              uint32_t g0 = 0, g1 = 0;
              if (try_pull(T, R, c, 0u, n_sm, g0, g1) == kPulled) {
                ctl.action = kActRun;
                ctl.tenant = c;
                ctl.g0 = g0;
                ctl.g1 = g1;
                break;
              }
            }
          }
          // deep fill (batch runs): neither the pair nor the fill list has a
          // slice for this slot (kernels with fewer slices than the GPU has
          // slots), so take one from the lowest kernel in submission order
          // that still has blocks to hand out. fill_cursor moves past the
          // prefix of drained kernels; a kernel at a stage barrier is skipped
          // without moving it.
          if (ctl.action == kActWait && (R->flags & KL_CFG_DEEP_FILL) && !R->serve && ph.A >= 0) {
            const uint32_t c0 = ld_relaxed(&R->fill_cursor);
            bool prefix = true;
            for (uint32_t j = c0; j < R->n_tenants && j < c0 + 8u; ++j) {
              uint32_t g0 = 0, g1 = 0;
              const int r = tn::resource_class(__ldcg(&tenant(T, R, j).type)) != tn::kClassMain
                                ? kExhausted  // a class kernel's kernel: not for this slot
                                : try_pull(T, R, (int32_t)j, 0u, n_sm, g0, g1);
              if (r == kPulled) {
                ctl.action = kActRun;
                ctl.tenant = (int32_t)j;
                ctl.g0 = g0;
                ctl.g1 = g1;
                break;
              }
              if (r == kExhausted && prefix)
                atomicMax(&R->fill_cursor, j + 1u);
              else
                prefix = false;
            }
          }
        }
      }
      if (ctl.action == kActWait) {
        const unsigned long long now = gtimer();
        if (ctl.wait_since == 0) ctl.wait_since = now;
        // an idle serving run waits for arrivals; its dispatcher ends the run
        const unsigned long long lim = (R->serve && idle) ? R->idle_limit_ns + limit : limit;
        if (now - ctl.wait_since > lim) {
          set_error(R, KL_EDEVICE_TIMEOUT, 1u);
          ctl.action = kActExit;
        } else {
          __nanosleep(ctl.backoff);
          ctl.backoff = min(ctl.backoff * 2, 256u);
        }
      } else {
        if (ctl.wait_since != 0) ctl.acc_wait += gtimer() - ctl.wait_since;
        ctl.wait_since = 0;
        ctl.backoff = 32;
      }
    }
    __syncthreads();
    const uint32_t action = ctl.action;
    if (action == kActExit) break;
    if (action == kActReplan) {
      const unsigned long long t0 = tid == 0 ? gtimer() : 0ull;
      replan(T, R, P, ctl.seq, ctl.trigger, smem);
      if (tid == 0) ctl.acc_plan += gtimer() - t0;
    } else if (action == kActRun) {
      TenantDev& d = tenant(T, R, (uint32_t)ctl.tenant);
      const uint32_t type = d.type;
      uint32_t g = ctl.g0;
      const uint32_t g1 = ctl.g1;
      static_assert(KL_MAX_ARGS_BYTES % 16 == 0 && offsetof(TenantDev, args) % 16 == 0, "argument copy");
      if (ctl.args_of != ctl.tenant) {  // uniform: read after the barrier that published the action
        if (tid < (int)(KL_MAX_ARGS_BYTES / 16))
          reinterpret_cast<uint4*>(s_args)[tid] = __ldcg(reinterpret_cast<const uint4*>(d.args) + tid);
        __syncthreads();
        if (tid == 0) ctl.args_of = ctl.tenant;
      }
      // Claim-ahead (batch runs): a slot running its own kernel of the phase
      // claims that kernel's next slice now and reads the claim after this
      // slice, so the atomic's round trip overlaps the blocks instead of
      // preceding the next slice. Only while the kernel has many slices left
      // (the spread rule matters only near its end) and for one-stage kernels
      // (no stage barrier between the two slices). The phase number is read
      // alongside: after a re-plan the slot runs the slice it already owns and
      // then reads the new phase. A serving run reads the phase before every
      // slice instead: that is where arrivals are noticed.
      uint32_t pf_a = 0xffffffffu, pf_seq = 0;  // the only values held across the blocks
      if (tid == 0 && ctl.own && !R->serve && d.nstages == 1u) {
        const uint32_t S = R->slots, n_sm = R->n_sm;
        const uint32_t sl = d.slice;
        if ((uint64_t)g1 + 2ull * S * n_sm * sl < (uint64_t)d.total) {
          pf_a = atomicAdd(&d.next, sl);
          pf_seq = ld_relaxed(&R->phase_seq);
        }
      }
      while (g < g1) {
        const tn::Stage st = stage_at(d, type, g);
        if (st.begin > 0) {
          // the previous stage must be complete before any block of this one runs
          if (tid == 0) {
            ctl.wait_failed = 0;
            unsigned long long since = gtimer();
            uint32_t bo = 32;
            while (ld_acquire(&d.done) < st.begin) {
              if (gtimer() - since > R->wait_limit_ns) {
                set_error(R, KL_EDEVICE_TIMEOUT, 2u);
                ctl.wait_failed = 1;
                break;
              }
              __nanosleep(bo);
              bo = min(bo * 2, 256u);
            }
            ctl.acc_stage += gtimer() - since;
          }
          __syncthreads();
          if (ctl.wait_failed) break;
        }
        const uint32_t ge = min(g1, st.end);
        const tn::BlockCtx cx{&s_tmem, &R->error, R->wait_limit_ns};
        tn::run_slice<BUILD>(type, s_args, st, g, ge, smem, cx);  // ends with a CTA barrier
        if (tid == 0) {
          // a later stage reads what this one wrote: release before counting
          if (d.nstages > 1) __threadfence();
          const uint32_t cnt = ge - g;
          const uint32_t old = atomicAdd(&d.done, cnt);
          if (old + cnt == d.total) complete_tenant(d, R);
        }
        g = ge;
      }
      if (tid == 0 && pf_a != 0xffffffffu && pf_a < d.total) {
        const uint32_t total = d.total;
        ctl.pf_tenant = ctl.tenant;
        ctl.pf_g0 = pf_a;
        ctl.pf_g1 = min(pf_a + d.slice, total);
        ctl.pf_more = pf_seq == ctl.own_seq;
        if (ctl.pf_g1 == total) d.drained = 1u;
        atomicAdd(&d.slices, 1u);
      }
    }
    __syncthreads();
  }
  if constexpr (BUILD == tn::kBuildFull) tn::release_tmem(tcx);
  if (tid == 0) {
    atomicAdd(&R->wait_ns, ctl.acc_wait);
    atomicAdd(&R->stage_wait_ns, ctl.acc_stage);
    atomicAdd(&R->plan_ns, ctl.acc_plan);
    atomicAdd(&R->ctas_done, 1u);
  }
}

// ------------------------------------------------------------------ resource classes
// A resource-heavy tenant type (tn::resource_class != 0) cannot run in a
// co-scheduler slot: its blocks need more threads, registers or shared memory
// than a slot holds, and compiling it into the co-scheduler would raise every
// slot's resources to its size (the merged-kernel cost of Section 6). It runs
// in a persistent kernel of its own, launched after the co-scheduler for the
// run with two CTAs per SM. The co-scheduler keeps two slots per SM (its
// further CTAs leave at once), which leaves room for one class CTA beside them
// on every SM; the other class CTAs wait for room and take over as the
// co-scheduler's kernels, or another class's, run out. A class CTA pulls
// slices of its class's kernels in submission order from the same device
// queues and leaves when none has blocks left; it never waits on the
// co-scheduler or another class, nor they on it.
template <int TYPE>
__device__ __forceinline__ void class_block(const void* args, const tn::Stage& st, uint32_t vb, char* smem) {
  if constexpr (TYPE == KL_T_BS255)
    tn::bs255_block(*reinterpret_cast<const kl_args_blackscholes*>(args), vb);
  else if constexpr (TYPE == KL_T_HIST1024)
    tn::hist1024_block(*reinterpret_cast<const kl_args_hist256*>(args), st.s, vb, smem);
  else if constexpr (TYPE == KL_T_GEMM_F32_BIG)
    tn::gemm_big_block(*reinterpret_cast<const kl_args_gemm_f32*>(args), vb, smem);
}

template <int TYPE>
__global__ void __launch_bounds__(tn::block_threads(TYPE), 2) class_kernel(TenantDev* __restrict__ T,
                                                                          RunDev* __restrict__ R) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int s_go;
  __shared__ int32_t s_t;
  __shared__ uint32_t s_g0, s_g1, s_fail;
  __shared__ __align__(16) unsigned char s_args[KL_MAX_ARGS_BYTES];
  constexpr int C = tn::resource_class(TYPE);
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_go = 0;
    s_t = -1;
    atomicCAS(&R->t_launch, 0ull, gtimer());
  }
  __syncthreads();
  uint32_t cursor = 0;  // kernels below it have handed out every block (thread 0)
  for (;;) {
    if (tid == 0) {
      s_t = -2;  // -2: nothing left for the class; >= 0: a slice was pulled
      const unsigned long long t0 = gtimer();
      for (;;) {
        if (ld_relaxed(reinterpret_cast<uint32_t*>(&R->error)) != 0) break;
        bool blocked = false;
        for (uint32_t j = cursor; j < R->n_tenants; ++j) {
          if (__ldcg(&tenant(T, R, j).type) != (uint32_t)TYPE) {
            if (j == cursor) ++cursor;
            continue;
          }
          uint32_t g0 = 0, g1 = 0;
          const int r = try_pull(T, R, (int32_t)j, 0u, R->n_sm, g0, g1);
          if (r == kPulled) {
            s_t = (int32_t)j;
            s_g0 = g0;
            s_g1 = g1;
            break;
          }
          if (r == kExhausted && j == cursor)
            ++cursor;
          else if (r == kBlocked)
            blocked = true;
        }
        if (s_t >= 0 || !blocked) break;
        if (gtimer() - t0 > R->wait_limit_ns) {  // a stage barrier that never opens
          set_error(R, KL_EDEVICE_TIMEOUT, 5u);
          break;
        }
        __nanosleep(128);
      }
    }
    __syncthreads();
    const int32_t t = s_t;
    if (t < 0) break;
    if (tid == 0 && !s_go) {
      s_go = 1;
      atomicAdd(&R->cls_ctas[C], 1u);  // a CTA of the class that found work
    }
    TenantDev& d = tenant(T, R, (uint32_t)t);
    if (tid < (int)(KL_MAX_ARGS_BYTES / 16))
      reinterpret_cast<uint4*>(s_args)[tid] = __ldcg(reinterpret_cast<const uint4*>(d.args) + tid);
    __syncthreads();
    for (uint32_t g = s_g0; g < s_g1;) {
      const tn::Stage st = stage_at(d, (uint32_t)TYPE, g);
      if (st.begin > 0) {
        if (tid == 0) {
          s_fail = 0;
          const unsigned long long since = gtimer();
          while (ld_acquire(&d.done) < st.begin) {
            if (gtimer() - since > R->wait_limit_ns) {
              set_error(R, KL_EDEVICE_TIMEOUT, 6u);
              s_fail = 1;
              break;
            }
            __nanosleep(128);
          }
        }
        __syncthreads();
        if (s_fail) break;
      }
      const uint32_t ge = min(s_g1, st.end);
      for (uint32_t b = g; b < ge; ++b) {
        class_block<TYPE>(s_args, st, b - st.begin, smem);
        __syncthreads();
      }
      if (tid == 0) {
        if (d.nstages > 1) __threadfence();
        const uint32_t cnt = ge - g;
        const uint32_t old = atomicAdd(&d.done, cnt);
        if (old + cnt == d.total) complete_tenant(d, R);
      }
      g = ge;
    }
    __syncthreads();
  }
  if (tid == 0) atomicAdd(&R->ctas_done, 1u);
}

int class_launch(int type, TenantDev* T, RunDev* R, uint32_t grid, cudaStream_t stream) {
  const uint32_t smem = tn::smem_bytes((uint32_t)type);
  switch (type) {
    case KL_T_BS255: class_kernel<KL_T_BS255><<<grid, tn::block_threads(KL_T_BS255), smem, stream>>>(T, R); break;
    case KL_T_HIST1024:
      class_kernel<KL_T_HIST1024><<<grid, tn::block_threads(KL_T_HIST1024), smem, stream>>>(T, R);
      break;
    case KL_T_GEMM_F32_BIG: {
      static bool attr = false;
      if (!attr) {
        if (cudaFuncSetAttribute(class_kernel<KL_T_GEMM_F32_BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
          return -1;
        attr = true;
      }
      class_kernel<KL_T_GEMM_F32_BIG><<<grid, tn::block_threads(KL_T_GEMM_F32_BIG), smem, stream>>>(T, R);
      break;
    }
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Run staging through the SMs: copies between the runtime's pinned host image
// (device-accessible) and its device queue, so that a launch never waits
// behind the caller's bulk transfers queued on the copy engines.
struct CopyList {
  CopySeg seg[4];
  uint32_t n;
};

__global__ void __launch_bounds__(kThreads) stage_copy_kernel(CopyList L) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nth = (size_t)gridDim.x * blockDim.x;
  for (uint32_t k = 0; k < L.n && k < 4u; ++k) {
    const CopySeg sg = L.seg[k];
    if ((((uintptr_t)sg.dst | (uintptr_t)sg.src | sg.bytes) & 15u) == 0) {
      uint4* d = static_cast<uint4*>(sg.dst);
      const uint4* s = static_cast<const uint4*>(sg.src);
      for (size_t i = tid; i < sg.bytes / 16u; i += nth) d[i] = s[i];
    } else {
      unsigned char* d = static_cast<unsigned char*>(sg.dst);
      const unsigned char* s = static_cast<const unsigned char*>(sg.src);
      for (size_t i = tid; i < sg.bytes; i += nth) d[i] = s[i];
    }
  }
}

// dst/src pairs (device-accessible pointers) copied by one kernel on stream s
int stage_copy(const CopySeg* segs, uint32_t n, cudaStream_t s) {
  if (n == 0 || n > 4) return -1;
  CopyList L{};
  size_t total = 0;
  for (uint32_t k = 0; k < n; ++k) {
    L.seg[k] = segs[k];
    total += segs[k].bytes;
  }
  L.n = n;
  const uint32_t blocks = (uint32_t)std::min<size_t>(64, std::max<size_t>(1, total / (16u * kThreads * 4u)));
  stage_copy_kernel<<<blocks, kThreads, 0, s>>>(L);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------------ host side

template <int BUILD>
static int occupancy_of(int* ctas_per_sm) {
  const uint32_t smem = BUILD == tn::kBuildLight ? tn::kMaxLightSmem : tn::kMaxTenantSmem;
  cudaError_t e =
      cudaFuncSetAttribute(cosched_kernel<BUILD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, cosched_kernel<BUILD>, kThreads, smem);
  return e == cudaSuccess ? 0 : -1;
}

int cosched_occupancy(int* ctas_per_sm, int build) {
  switch (build) {
    case tn::kBuildPlain: return occupancy_of<tn::kBuildPlain>(ctas_per_sm);
    case tn::kBuildFull: return occupancy_of<tn::kBuildFull>(ctas_per_sm);
    case tn::kBuildLight: return occupancy_of<tn::kBuildLight>(ctas_per_sm);
    default: return -1;
  }
}

int cosched_launch(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t n_sm, uint32_t slots, uint32_t smem_bytes,
                   int build, cudaStream_t stream, uint32_t extra_ctas) {
  dim3 grid(n_sm * slots + extra_ctas), block(kThreads);
  switch (build) {
    case tn::kBuildPlain: cosched_kernel<tn::kBuildPlain><<<grid, block, smem_bytes, stream>>>(T, R, P); break;
    case tn::kBuildFull: cosched_kernel<tn::kBuildFull><<<grid, block, smem_bytes, stream>>>(T, R, P); break;
    case tn::kBuildLight:
      if (smem_bytes > tn::kMaxLightSmem) return -1;
      cosched_kernel<tn::kBuildLight><<<grid, block, smem_bytes, stream>>>(T, R, P);
      break;
    default: return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kl
