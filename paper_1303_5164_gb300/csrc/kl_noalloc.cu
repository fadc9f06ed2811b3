// kl_run_noalloc: one co-scheduled run of a small batch without allocating.
//
// Some callers cannot allocate device memory at the point where they want to
// run work: frameworks whose caching allocator has reserved the device memory
// up front (a raw cudaMalloc then fails or fragments their pool), and
// latency-critical host threads that must not call cudaMalloc / cudaFree on the
// hot path because those calls can synchronize the whole device. For them this
// entry point runs the same persistent co-scheduler kernel as kl_launch, with
// its queue, run state and phase log in a file-scope device array instead of
// memory from kl_create. The caller still owns and passes every input and
// output buffer through the kernel descriptors.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call rewrites all of it that must start at zero. Calls whose
// GPU work overlaps (several host threads, or several streams) race on it and
// must not be issued concurrently.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernelet.h"
#include "kl_internal.h"
#include "tenants.cuh"

namespace kl {
int cosched_occupancy(int* ctas_per_sm, int build);
int cosched_launch(TenantDev* T, RunDev* R, PhaseDev* P, uint32_t n_sm, uint32_t slots, uint32_t smem_bytes,
                   int build, cudaStream_t stream, uint32_t extra_ctas = 0);

namespace {

constexpr uint32_t kMaxT = KL_NOALLOC_MAX_TENANTS;
constexpr uint32_t kMaxPhases = 4 * kMaxT + 16;
constexpr uint32_t kPhaseSlots = 512;  // the device indexes phases modulo a power of two
static_assert((kMaxT & (kMaxT - 1)) == 0, "tenant slots must be a power of two");
static_assert(kPhaseSlots >= kMaxPhases, "phase slots");
constexpr size_t kRunOff = sizeof(TenantDev) * kMaxT;
constexpr size_t kPhaseOff = (kRunOff + sizeof(RunDev) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kPhaseOff + sizeof(PhaseDev) * kPhaseSlots;
constexpr int kMaxDevices = 64;
// the sizes the header documents: 64 x 256 B tenants + the 7,296 B run state
// (rounded to 7,424 B) + 512 x 144 B phases; the phase ring is a power of two,
// so 512 slots for the at most 4 x 64 + 16 = 272 phases of a run
static_assert(kScratchBytes == KL_NOALLOC_SCRATCH_BYTES, "documented size of the device array");

// Device scratch of the allocation-free path (the only storage it uses).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal. In host code the
// array's name is only a host-side stand-in, so the address is taken once per
// device with cudaGetSymbolAddress while that device is current.
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mu;

struct HostImage {
  TenantDev t[kMaxT];
  RunDev run;
  PhaseDev ph0;
};
static_assert(sizeof(HostImage) <= 23936, "documented size of the stack image");

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" int kl_run_noalloc(const kl_kernel_desc* descs, uint32_t n, const double* cp_table,
                              const uint32_t* slots_a_table, void* cuda_stream, uint64_t wait_limit_ns,
                              int32_t* states) {
  if (!descs || n == 0) return KL_EINVAL;
  if (n > kMaxT) return KL_EOVERFLOW;  // more kernels than the fixed scratch holds
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KL_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return KL_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KL_ECUDA;
      g_scratch_ptr[dev] = p;
    }
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  TenantDev* dT = reinterpret_cast<TenantDev*>(base);
  RunDev* dR = reinterpret_cast<RunDev*>(base + kRunOff);
  PhaseDev* dP = reinterpret_cast<PhaseDev*>(base + kPhaseOff);

  int occ = 0, nsm = 0;
  int occ_tc = 0;  // also raises the tensor-core build's dynamic shared memory limit
  if (cosched_occupancy(&occ, tn::kBuildPlain) != 0 || occ < 1 || cosched_occupancy(&occ_tc, tn::kBuildFull) != 0)
    return KL_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return KL_ECUDA;
  const uint32_t S = (uint32_t)(occ < KL_MAX_SLOTS ? occ : KL_MAX_SLOTS);
  const uint32_t n_sm = (uint32_t)(nsm < kMaxSM ? nsm : kMaxSM);

  // the whole image lives on the caller's stack: no heap, no device allocation
  HostImage img;
  memset(&img, 0, sizeof(img));
  for (uint32_t i = 0; i < n; ++i) {
    const kl_kernel_desc& d = descs[i];
    kl_tenant_shape sh;
    if (d.type >= KL_T_MAIN_COUNT || !d.args) return KL_EINVAL;  // the co-scheduler's types only
    int rc = kl_tenant_shape_of(d.type, d.args, d.args_size, &sh);
    if (rc) return rc;
    if (d.block[0] != KL_BLOCK_THREADS || d.block[1] != 1 || d.block[2] != 1) return KL_EINVAL;
    if (d.grid[0] != sh.grid[0] || d.grid[1] != 1 || d.grid[2] != 1) return KL_EINVAL;
    if (d.smem_bytes != 0 && d.smem_bytes < sh.smem_bytes) return KL_EINVAL;
    if (sh.total_blocks == 0 || sh.total_blocks >= (1ull << 24)) return KL_EINVAL;
    TenantDev& t = img.t[i];
    t.type = d.type;
    t.total = (uint32_t)sh.total_blocks;
    t.nstages = sh.nstages;
    t.blocks0 = sh.grid[0];
    t.index = i;
    // a slice never exceeds the kernel, and the queue counter (which can
    // overshoot by one slice per CTA when a kernel runs out) stays below 2^32
    uint64_t sl = d.slice_blocks ? d.slice_blocks : default_slice(d.type);  // as kl_submit without profiles
    if (sl > t.total) sl = t.total;
    while (sl > 1 && (uint64_t)t.total + sl * ((uint64_t)n_sm * S + 1) >= (1ull << 32)) sl >>= 1;
    t.slice = (uint32_t)sl;
    memcpy(t.args, d.args, d.args_size);
  }
  RunDev& R = img.run;
  R.n_tenants = n;
  R.slots = S;
  R.n_sm = n_sm;
  R.max_phases = 4 * n + 16;
  R.n_types = KL_T_COUNT;
  R.flags = KL_CFG_BACKFILL;
  R.chain_slots = 1;
  R.ring_mask = kMaxT - 1;
  R.phase_mask = kPhaseSlots - 1;
  R.wait_limit_ns = wait_limit_ns ? wait_limit_ns : 2000000000ull;
  for (uint32_t a = 0; a < KL_T_COUNT; ++a)
    for (uint32_t b = 0; b < KL_T_COUNT; ++b) {
      R.cp[a][b] = cp_table ? cp_table[a * KL_T_COUNT + b] : 0.0;
      uint32_t sa = slots_a_table ? slots_a_table[a * KL_T_COUNT + b] : S / 2;
      const uint32_t hi = S > 1 ? S - 1 : 1;  // both kernels of a pair keep a slot when S >= 2
      R.slots_a[a][b] = sa < 1 ? 1 : (sa > hi ? hi : sa);
      R.allowed[a][b] = 1;
    }
  img.ph0.A = -2;
  img.ph0.B = -1;
  for (int f = 0; f < kFill; ++f) img.ph0.fill[f] = -1;
  img.ph0.chain[0] = img.ph0.chain[1] = -1;

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemcpyAsync(dT, img.t, sizeof(TenantDev) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dR, &img.run, sizeof(RunDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dP, &img.ph0, sizeof(PhaseDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return KL_ECUDA;
  bool tc = false;
  for (uint32_t i = 0; i < n; ++i) tc |= !tn::in_plain_build(descs[i].type);  // a full-build type
  if (cosched_launch(dT, dR, dP, n_sm, S, tn::kMaxTenantSmem, tc ? tn::kBuildFull : tn::kBuildPlain, s) != 0)
    return KL_ECUDA;
  if (cudaMemcpyAsync(img.t, dT, sizeof(TenantDev) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&img.run, dR, sizeof(RunDev), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return KL_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KL_ECUDA;
  int result = img.run.error;
  for (uint32_t i = 0; i < n; ++i) {
    const bool ok = img.t[i].done == img.t[i].total && img.t[i].status == KL_DONE;
    if (states) states[i] = ok ? KL_DONE : KL_ERROR;
    if (!ok && result == KL_OK) result = KL_ESTATE;
  }
  return result;
}
