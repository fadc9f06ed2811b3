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
// No wait in this kernel is unbounded: every spin has a globaltimer deadline
// after which the run records KL_EDEVICE_TIMEOUT and every CTA returns.
#include <cuda_runtime.h>
#include <stdint.h>

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

// Co-resident CTAs per SM: 4 x 256 threads at up to 64 registers each.
constexpr int kCtasPerSm = 4;

enum : uint32_t { kActRun = 0, kActWait = 1, kActExit = 2, kActReplan = 3 };
enum : int { kPulled = 0, kBlocked = 1, kExhausted = 2 };

struct CtaCtl {
  int32_t tenant;
  uint32_t g0, g1;
  uint32_t action;
  uint32_t seq;
  int32_t trigger;
  int32_t wait_failed;
};

__device__ __forceinline__ void set_error(RunDev* R, int32_t code, uint32_t info) {
  if (atomicCAS(reinterpret_cast<int*>(&R->error), 0, code) == 0) R->error_info = info;
}

// Thread 0 only: try to take the next slice of tenant t. `rank` is this CTA's
// position among the slots of its SM that serve t: while the stage has fewer
// blocks left than rank * numSM, the slot leaves them to lower ranks, so a
// kernel with few blocks spreads one per SM instead of stacking on some SMs.
__device__ __forceinline__ int try_pull(TenantDev* T, int32_t t, uint32_t rank, uint32_t n_sm, uint32_t& g0,
                                        uint32_t& g1) {
  TenantDev& d = T[t];
  const uint32_t total = d.total;
  uint32_t n = ld_relaxed(&d.next);
  if (n >= total) return kExhausted;
  tn::Stage st = tn::stage_of(d.type, d.args, n);
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

// FindCoSchedule on the device (Algorithm 1, procedure), warp 0 of one CTA.
// Pending = kernels with blocks not yet handed out. For every pair of pending
// kernels CP depends only on their types, so the best pair of a type pair is
// its two lowest submit indices; the winner is the largest CP among unpruned
// type pairs (all pairs when every one is pruned), ties to the smallest
// (i, j). One pending kernel runs alone on every slot; none ends the run.
__device__ void replan(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t seq_old, int32_t trigger) {
  const int lane = threadIdx.x & 31;
  int32_t low1[KL_T_COUNT], low2[KL_T_COUNT];
#pragma unroll
  for (int t = 0; t < KL_T_COUNT; ++t) low1[t] = low2[t] = -1;
  uint32_t npend = 0;
  unsigned long long pmask = 0ull;
  int32_t lowp[6];
  uint32_t nlow = 0;
  int32_t lowms = -1;  // lowest pending kernel with more than one stage
  const uint32_t n = R->n_tenants;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane;
    bool pend = false;
    uint32_t ty = 0;
    if (i < n) {
      ty = T[i].type;
      pend = ld_relaxed(&T[i].next) < T[i].total;
    }
    const uint32_t pb = __ballot_sync(0xffffffffu, pend);
    npend += __popc(pb);
    if (base < 64) pmask |= (unsigned long long)pb << base;
    for (uint32_t m = pb; m && nlow < 6; m &= m - 1) lowp[nlow++] = (int32_t)(base + __ffs(m) - 1);
    const uint32_t msb = __ballot_sync(0xffffffffu, pend && T[min(i, n - 1)].nstages > 1);
    if (msb && lowms < 0) lowms = (int32_t)(base + __ffs(msb) - 1);
#pragma unroll
    for (int t = 0; t < KL_T_COUNT; ++t) {
      uint32_t m = __ballot_sync(0xffffffffu, pend && ty == (uint32_t)t);
      if (m && low1[t] < 0) {
        low1[t] = (int32_t)(base + __ffs(m) - 1);
        m &= m - 1;
      }
      if (m && low2[t] < 0) low2[t] = (int32_t)(base + __ffs(m) - 1);
    }
  }
  if (lane != 0) return;
  PhaseDev ph;
  ph.A = -1;
  ph.B = -1;
  ph.slots_a = R->slots;
  ph.slots_b = 0;
  ph.cp = 0.0;
  ph.trigger = trigger;
  ph.n_pending = npend;
  ph.pending = pmask;
  if (npend == 1) {
    for (int t = 0; t < KL_T_COUNT; ++t)
      if (low1[t] >= 0) ph.A = low1[t];
  } else if (npend >= 2) {
    for (int pass = 0; pass < 2 && ph.A < 0; ++pass) {
      double best = 0.0;
      int32_t bi = -1, bj = -1;
      for (int ta = 0; ta < KL_T_COUNT; ++ta) {
        if (low1[ta] < 0) continue;
        for (int tb = ta; tb < KL_T_COUNT; ++tb) {
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
          const uint32_t tyi = T[i].type, tyj = T[j].type;
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
        ph.slots_a = R->slots_a[T[bi].type][T[bj].type];
        ph.slots_b = R->slots - ph.slots_a;
      }
    }
  }
  // backfill candidates: the next pending kernel of A's type and of B's type
  // (more of the work the pair is doing), then the lowest pending indices
  for (int f = 0; f < 4; ++f) ph.fill[f] = -1;
  uint32_t c = 0;
  if (ph.A >= 0 && (R->flags & KL_CFG_FILL_TYPES)) {
    const uint32_t ta = T[ph.A].type;
    const int32_t sa = low1[ta] != ph.A ? low1[ta] : low2[ta];
    if (sa >= 0 && sa != ph.B) ph.fill[c++] = sa;
    if (ph.B >= 0) {
      const uint32_t tb = T[ph.B].type;
      const int32_t sb = low1[tb] != ph.B ? low1[tb] : low2[tb];
      if (sb >= 0 && sb != ph.A && (c == 0 || sb != ph.fill[0])) ph.fill[c++] = sb;
    }
  }
  // then the lowest pending multi-stage kernel (a long chain of dependent
  // grids: started early, its stage barriers overlap other work instead of
  // forming the tail of the run), then the lowest pending indices
  if (lowms >= 0 && c < 4 && lowms != ph.A && lowms != ph.B && (c == 0 || lowms != ph.fill[0]) &&
      (c < 2 || lowms != ph.fill[1]))
    ph.fill[c++] = lowms;
  for (uint32_t f = 0; f < nlow && c < 4; ++f) {
    bool dup = lowp[f] == ph.A || lowp[f] == ph.B;
    for (uint32_t q = 0; q < c; ++q) dup |= lowp[f] == ph.fill[q];
    if (!dup) ph.fill[c++] = lowp[f];
  }
  const uint32_t seq = seq_old + 1;
  if (seq >= R->max_phases) {
    set_error(R, KL_EOVERFLOW, seq);
    ph.A = -1;
    ph.B = -1;
  }
  // block counts at this instant: per-phase measured progress of each kernel
  ph.done_a = ph.A >= 0 ? ld_relaxed(&T[ph.A].done) : 0u;
  ph.done_b = ph.B >= 0 ? ld_relaxed(&T[ph.B].done) : 0u;
  {
    const int32_t pa = __ldcg(&P[seq_old].A), pb = __ldcg(&P[seq_old].B);
    ph.prev_done_a = pa >= 0 ? ld_relaxed(&T[pa].done) : 0u;
    ph.prev_done_b = pb >= 0 ? ld_relaxed(&T[pb].done) : 0u;
  }
  ph.t = gtimer();
  P[min(seq, R->max_phases - 1)] = ph;
  __threadfence();
  st_release(&R->phase_seq, min(seq, R->max_phases - 1));
}

__device__ __forceinline__ void complete_tenant(TenantDev& d, RunDev* R) {
  unsigned long long now = gtimer();
  d.t_end = now;
  __threadfence();
  st_release(&d.status, KL_DONE);
  atomicAdd(&R->n_complete, 1u);
  atomicMax(&R->t_end, now);
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) cosched_kernel(TenantDev* __restrict__ T, RunDev* __restrict__ R,
                                                             PhaseDev* __restrict__ P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaCtl ctl;
  __shared__ uint32_t s_slot;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint32_t sm = smid() & (kMaxSM - 1);
    const uint32_t ticket = atomicAdd(&R->sm_ticket[sm], 1u);
    s_slot = ticket % R->slots;
    atomicCAS(&R->t_launch, 0ull, gtimer());
  }
  __syncthreads();
  const uint32_t slot = s_slot;
  const uint32_t S = R->slots;
  const uint32_t n_sm = gridDim.x / S;
  const unsigned long long limit = R->wait_limit_ns;
  unsigned long long wait_since = 0;
  uint32_t backoff = 32;

  for (;;) {
    if (tid == 0) {
      ctl.action = kActWait;
      ctl.tenant = -1;
      if (ld_relaxed(reinterpret_cast<uint32_t*>(&R->error)) != 0) {
        ctl.action = kActExit;
      } else {
        const uint32_t seq = ld_acquire(&R->phase_seq);
        PhaseDev ph;  // published by another CTA: read through L2
        ph.A = __ldcg(&P[seq].A);
        ph.B = __ldcg(&P[seq].B);
        ph.slots_a = __ldcg(&P[seq].slots_a);
        if (ph.A == -1) {
          ctl.action = kActExit;
        } else {
          bool need_replan = (ph.A == -2);
          int32_t trig = -1;
          if (!need_replan) {
            const bool mine_is_b = ph.B >= 0 && slot >= ph.slots_a;
            const int32_t t1 = mine_is_b ? ph.B : ph.A;
            const int32_t t2 = mine_is_b ? ph.A : ph.B;
            const uint32_t rank1 = mine_is_b ? slot - ph.slots_a : slot;
            const uint32_t rank2 = mine_is_b ? slot : slot + (S - ph.slots_a);
            uint32_t g0 = 0, g1 = 0;
            int r = try_pull(T, t1, rank1, n_sm, g0, g1);
            if (r == kPulled) {
              ctl.action = kActRun;
              ctl.tenant = t1;
              ctl.g0 = g0;
              ctl.g1 = g1;
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
                int r2 = try_pull(T, t2, rank2, n_sm, g0, g1);
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
            for (int f = 0; f < 4; ++f) {
              const int32_t c = __ldcg(&P[seq].fill[f]);
              if (c < 0) break;
              uint32_t g0 = 0, g1 = 0;
              if (try_pull(T, c, 0u, n_sm, g0, g1) == kPulled) {
                ctl.action = kActRun;
                ctl.tenant = c;
                ctl.g0 = g0;
                ctl.g1 = g1;
                break;
              }
            }
          }
        }
      }
      if (ctl.action == kActWait) {
        const unsigned long long now = gtimer();
        if (wait_since == 0) wait_since = now;
        if (now - wait_since > limit) {
          set_error(R, KL_EDEVICE_TIMEOUT, 1u);
          ctl.action = kActExit;
        } else {
          __nanosleep(backoff);
          backoff = min(backoff * 2, 256u);
        }
      } else {
        wait_since = 0;
        backoff = 32;
      }
    }
    __syncthreads();
    const uint32_t action = ctl.action;
    if (action == kActExit) break;
    if (action == kActReplan) {
      if (tid < 32) replan(T, R, P, ctl.seq, ctl.trigger);
    } else if (action == kActRun) {
      const int32_t t = ctl.tenant;
      TenantDev& d = T[t];
      const uint32_t type = d.type;
      uint32_t g = ctl.g0;
      const uint32_t g1 = ctl.g1;
      while (g < g1) {
        const tn::Stage st = tn::stage_of(type, d.args, g);
        if (st.begin > 0) {
          // the previous stage must be complete before any block of this one runs
          if (tid == 0) {
            ctl.wait_failed = 0;
            unsigned long long since = gtimer();
            uint32_t bo = 32;
            while (ld_acquire(&d.done) < st.begin) {
              if (gtimer() - since > limit) {
                set_error(R, KL_EDEVICE_TIMEOUT, 2u);
                ctl.wait_failed = 1;
                break;
              }
              __nanosleep(bo);
              bo = min(bo * 2, 256u);
            }
          }
          __syncthreads();
          if (ctl.wait_failed) break;
        }
        const uint32_t ge = min(g1, st.end);
        for (uint32_t b = g; b < ge; ++b) {
          tn::run_block(type, d.args, st, b, smem);
          __syncthreads();  // shared memory is reused by the next block
        }
        if (tid == 0) {
          // a later stage reads what this one wrote: release before counting
          if (d.nstages > 1) __threadfence();
          const uint32_t cnt = ge - g;
          const uint32_t old = atomicAdd(&d.done, cnt);
          if (old + cnt == d.total) complete_tenant(d, R);
        }
        g = ge;
      }
    }
    __syncthreads();
  }
  if (tid == 0) atomicAdd(&R->ctas_done, 1u);
}

// ------------------------------------------------------------------ host side

int cosched_occupancy(int* ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(cosched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tn::kMaxTenantSmem);
  if (e != cudaSuccess) return -1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, cosched_kernel, kThreads,
                                                    tn::kMaxTenantSmem);
  return e == cudaSuccess ? 0 : -1;
}

int cosched_launch(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t n_sm, uint32_t slots,
                   cudaStream_t stream) {
  dim3 grid(n_sm * slots), block(kThreads);
  cosched_kernel<<<grid, block, tn::kMaxTenantSmem, stream>>>(T, R, P);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace kl
