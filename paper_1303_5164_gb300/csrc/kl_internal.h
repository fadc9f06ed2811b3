// Internal layouts shared by the host runtime (kl_runtime.cpp) and the device
// code (kl_cosched.cu, kl_native.cu). Not part of the public ABI.
#pragma once
#include <stdint.h>
#include "kernelet.h"

namespace kl {

constexpr int kThreads = KL_BLOCK_THREADS;
constexpr int kMaxSM = 256;
constexpr int kNoTenant = -1;
constexpr int kFill = 16;     // backfill candidates per phase, at most (see replan)

// Pull granularity per type (blocks per slice) when the descriptor leaves it to
// the runtime; chosen so one atomic covers roughly 16-64 KB of traffic or one
// long block.
inline uint32_t default_slice(uint32_t type) {
  switch (type) {
    case KL_T_GATHER: return 4;
    case KL_T_BLACKSCHOLES: return 8;
    case KL_T_GEMM_F32: return 1;
    case KL_T_SPMV_CSR: return 8;
    case KL_T_PCHASE: return 1;
    case KL_T_TRIAD: return 2;
    case KL_T_HIST256: return 2;
    case KL_T_ESCAPE: return 8;
    case KL_T_BITONIC: return 2;
    case KL_T_MATADD: return 8;
    case KL_T_GEMM_BF16: return 1;
    case KL_T_TEA: return 4;
    case KL_T_SAD: return 8;
    case KL_T_STENCIL: return 4;
    case KL_T_MRIQ: return 1;
    default: return 1;
  }
}

// One submitted kernel in device memory (128-byte aligned, 256 bytes).
// Static fields are written by the host before the launch; dynamic fields are
// zero at launch and owned by the device during the run.
struct alignas(128) TenantDev {
  // ---- static
  uint32_t type;          // kl_tenant_type
  uint32_t slice;         // blocks per slice (pull granularity)
  uint32_t total;         // thread blocks summed over stages
  uint32_t nstages;
  uint32_t index;         // submit index within the run
  uint32_t blocks0;       // blocks of stage 0 (stages after it: equal size for the bitonic sort,
                          // one more stage holding the rest otherwise)
  unsigned long long t_arrive;  // serving: globaltimer when the device took the kernel in
  alignas(16) unsigned char args[KL_MAX_ARGS_BYTES];
  // ---- dynamic (own 128-byte line, away from the arguments)
  alignas(128) uint32_t next;     // next block to hand out (cumulative over stages)
  uint32_t done;                  // blocks finished (cumulative over stages)
  uint32_t drained;               // 1 once every block has been handed out
  uint32_t status;                // kl_state
  uint32_t slices;                // slices pulled
  uint32_t pad1;
  unsigned long long t_start;     // globaltimer of the first pulled slice
  unsigned long long t_end;       // globaltimer when the last block finished
};
static_assert(sizeof(TenantDev) == 256, "TenantDev layout");

struct PhaseDev {
  int32_t A, B;             // tenant indices; B < 0 solo; A < 0 = end of run
  uint32_t slots_a, slots_b;
  double cp;
  unsigned long long t;
  int32_t trigger;
  uint32_t n_pending;          // kernels with blocks left when the phase was chosen
  unsigned long long pending;  // bit i: kernel i (i < 64) was pending
  int32_t fill[kFill];         // other pending kernels for backfill (-1 ends the list)
  uint32_t done_a, done_b;     // blocks finished by this phase's A, B when it was published
  uint32_t prev_done_a;        // ... and by the previous phase's A, B at the same moment
  uint32_t prev_done_b;
  uint32_t intake_seen;        // kernels known to the device when the phase was chosen
  uint32_t pad2;
  int32_t chain[2];            // lowest pending multi-stage kernels outside A, B (chain lane)
};
static_assert(sizeof(PhaseDev) == 144, "PhaseDev layout");

// Serving mode: per-kernel completion record in mapped host memory, written
// by the device before the kernel's entry in the completion queue.
struct ServeDone {
  uint32_t seq1;                 // sequence number + 1
  uint32_t slices;
  uint32_t blocks;
  uint32_t pad;
  unsigned long long t_start;    // globaltimer
  unsigned long long t_end;
};
static_assert(sizeof(ServeDone) == 32, "ServeDone layout");

// Phase entries with A < 0: -1 ends the run, -2 asks for the first plan,
// -3 means nothing is pending (serving mode waits for arrivals).
constexpr int32_t kPhaseEnd = -1, kPhasePlan = -2, kPhaseIdle = -3;

// Run-wide state of one co-scheduled launch.
struct alignas(128) RunDev {
  // ---- static (host-written)
  uint32_t n_tenants;
  uint32_t slots;              // CTAs per SM
  uint32_t max_phases;
  uint32_t n_types;
  uint32_t flags;              // kl_config.flags
  uint32_t serve;              // 1: serving mode (tenant ring, dispatcher CTA 0)
  uint32_t chain_slots;        // chain lane: the last chain_slots slots of every SM
  uint32_t pad_s;
  unsigned long long age_limit_ns;    // serving: pending longer than this -> paired first
  unsigned long long plan_seed;       // KL_CFG_RANDOM_PLAN: seed of the random plans
  unsigned long long wait_limit_ns;
  uint32_t ring_mask;          // tenant slots - 1 (power of two); tenant seq -> slot
  uint32_t phase_mask;         // phase slots - 1 (power of two)
  unsigned long long idle_limit_ns;   // serving: exit after this long without arrivals
  TenantDev* host_ring;        // serving: descriptors written by the host (mapped memory)
  uint32_t* host_ctl;          // serving: [0] published tail, [32] stop request (mapped)
  ServeDone* host_done;        // serving: per tenant slot, completion record (mapped)
  unsigned long long* host_cq; // serving: completion queue, entry k = (k + 1) << 32 | seq (mapped)
  double cp[KL_T_COUNT][KL_T_COUNT];          // CP of (type row as K1, type col as K2)
  uint32_t slots_a[KL_T_COUNT][KL_T_COUNT];   // slots of the K1 (row) kernel
  uint32_t allowed[KL_T_COUNT][KL_T_COUNT];   // 1 = pair survives pruning
  // ---- dynamic (zero at launch)
  alignas(128) uint32_t phase_seq;   // index of the published phase
  uint32_t phase_claim;              // == phase_seq unless a re-plan is in progress
  uint32_t n_complete;               // tenants finished
  int32_t error;                     // first kl_status error
  uint32_t error_info;
  uint32_t ctas_done;
  unsigned long long t_launch;       // globaltimer, first CTA
  unsigned long long t_end;          // globaltimer, last completion
  uint32_t intake;                   // serving: kernels copied into the device ring
  uint32_t scan_lo;                  // lowest sequence number that may still be pending
  uint32_t cq_pos;                   // serving: completion queue entries written
  unsigned long long wait_ns;        // summed over CTAs: time with nothing to pull
  unsigned long long stage_wait_ns;  // summed over CTAs: time at stage barriers inside a slice
  unsigned long long plan_ns;        // summed over CTAs: time re-planning
  alignas(128) uint32_t fill_cursor; // deep fill: kernels below this one are all drained
  alignas(128) uint32_t sm_ticket[kMaxSM];
  // ---- resource classes (static, host-written)
  uint32_t n_sm;                      // SMs of the device (the grid may carry extra CTAs)
  uint32_t quota_exit;                // 1: main CTAs past `slots` on their SM exit at once
  // ---- resource classes (dynamic, zero at launch)
  uint32_t cls_ctas[4];               // CTAs of class c that found work (index 0 unused)
};

// One device-side copy (kl_cosched.cu, stage_copy): dst and src are
// device-accessible pointers (device memory or pinned host memory).
struct CopySeg {
  void* dst;
  const void* src;
  unsigned long long bytes;
};

}  // namespace kl
