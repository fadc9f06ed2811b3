// Plain launches of the tenant kernels (one grid per stage, blockIdx.x as the
// block index): the comparators the co-scheduler is measured against — serial
// FIFO on one stream and concurrent multi-stream launches — and the unsliced
// reference execution for the slicing-overhead measurement (Section 5.2).
// One instantiation per type so each gets its own register allocation.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "kl_internal.h"
#include "tenants.cuh"

namespace kl {

struct ArgsBlob {
  alignas(16) unsigned char b[KL_MAX_ARGS_BYTES];
};

// Device-side errors of plain launches (a BF16 GEMM wait that ran out).
__device__ int g_native_error;

template <int TYPE>
__global__ void __launch_bounds__(kThreads) native_kernel(ArgsBlob args, uint32_t stage) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint32_t s_tmem;
  const tn::Stage st{stage, 0u, 0u};
  const tn::BlockCtx cx{&s_tmem, &g_native_error, 2000000000ull};
  if constexpr (TYPE == KL_T_GEMM_BF16) tn::acquire_tmem(cx);
  tn::run_block<tn::kBuildFull>(TYPE, args.b, st, blockIdx.x, smem, cx);
  if constexpr (TYPE == KL_T_GEMM_BF16) tn::release_tmem(cx);
}

// Plain launches of the resource-heavy variants, at their own block sizes.
template <int TYPE>
__global__ void __launch_bounds__(tn::block_threads(TYPE), 1) native_heavy_kernel(ArgsBlob args, uint32_t stage) {
  extern __shared__ __align__(16) char smem[];
  const tn::Stage st{stage, 0u, 0u};
  if constexpr (TYPE == KL_T_BS255)
    tn::bs255_block(*reinterpret_cast<const kl_args_blackscholes*>(args.b), blockIdx.x);
  else if constexpr (TYPE == KL_T_HIST1024)
    tn::hist1024_block(*reinterpret_cast<const kl_args_hist256*>(args.b), st.s, blockIdx.x, smem);
  else if constexpr (TYPE == KL_T_GEMM_F32_BIG)
    tn::gemm_big_block(*reinterpret_cast<const kl_args_gemm_f32*>(args.b), blockIdx.x, smem);
}

template <int TYPE>
static cudaError_t launch_heavy(const void* args, uint32_t stage, uint32_t blocks, cudaStream_t s) {
  ArgsBlob blob;
  memcpy(blob.b, args, KL_MAX_ARGS_BYTES);
  const uint32_t sm = tn::smem_bytes(TYPE);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(native_heavy_kernel<TYPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  native_heavy_kernel<TYPE><<<blocks, tn::block_threads(TYPE), sm, s>>>(blob, stage);
  return cudaGetLastError();
}

template <int TYPE>
static cudaError_t launch_one(const void* args, uint32_t stage, uint32_t blocks, cudaStream_t s) {
  ArgsBlob blob;
  memcpy(blob.b, args, KL_MAX_ARGS_BYTES);
  const uint32_t sm = tn::smem_bytes(TYPE);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(native_kernel<TYPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  native_kernel<TYPE><<<blocks, kThreads, sm, s>>>(blob, stage);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ BF16 GEMM, plain launch
// The plain launch of the tensor-core GEMM is its own persistent kernel: one
// CTA per SM works through the tiles of C (work item i, i + grid, ...), with
// the work split by warp: warp 0 issues the TMA loads of a four-stage ring of
// 64-wide K-slices (A: 128 rows, Bt: 256 rows, 128-byte swizzle), warp 1
// issues the tcgen05.mma instructions (M = 128, N = 256, K = 16; four per
// K-slice) into one of two 256-column accumulators in tensor memory, and warps
// 4-7 read the other accumulator back (tcgen05.ld, warp w owns TMEM lanes
// 32 (w mod 4) ..) and store the finished tile while the next one is being
// multiplied. mbarriers hand each ring stage and each accumulator back and
// forth; every wait is bounded by the device wait limit, after which the
// kernel records KL_EDEVICE_TIMEOUT and every role stops.
// Tile schedule: whole 128 x 256 tiles for as many full waves of the grid as
// there are, then the tiles left over cut into 128 x 128 halves, so the last,
// partial wave takes half as long (512 tiles on 152 SMs: 3 full waves and 56
// tiles, which run as 112 halves at once).
namespace pg {
constexpr uint32_t BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr uint32_t kA = BM * BK * 2;        // 16 KB
constexpr uint32_t kBbox = 64 * BK * 2;     // one 64-row box of Bt (the tensor map's box)
constexpr uint32_t kB = BN * BK * 2;        // 32 KB
constexpr uint32_t kStage = kA + kB;        // 48 KB
constexpr uint32_t kSmem = 1024 + STAGES * kStage + 128;
constexpr uint32_t kTmemCols = 2 * BN;      // two accumulators: all 512 columns of the SM
constexpr uint32_t kIdescFull = tn::idesc_bf16_f32(BM, BN);
constexpr uint32_t kIdescHalf = tn::idesc_bf16_f32(BM, BN / 2);
static_assert(kSmem <= 227u * 1024u, "one CTA per SM");
static_assert(tn::kBfBM == (int)BM && tn::kBfBK == (int)BK && tn::kBfBN == 64, "tensor map boxes: A 64 x 128, Bt 64 x 64");

struct Item {
  uint32_t m0, n0, width;  // rows m0.., columns n0 .. n0 + width of C
  bool valid;              // a half tile wholly beyond N has no work
};
// work item i; nfull = whole tiles scheduled as such (a multiple of the grid)
__device__ __forceinline__ Item item(uint32_t i, uint32_t tiles_n, uint32_t nfull, uint32_t N) {
  uint32_t tile = i, half = 0, width = BN;
  if (i >= nfull) {
    const uint32_t h = i - nfull;
    tile = nfull + (h >> 1);
    half = h & 1u;
    width = BN / 2;
  }
  Item it;
  it.m0 = (tile / tiles_n) * BM;
  it.n0 = (tile % tiles_n) * BN + half * (BN / 2);
  it.width = width;
  it.valid = it.n0 < N;
  return it;
}
__host__ __device__ inline uint32_t nfull_of(uint32_t ntiles, uint32_t grid_ctas) {
  return (ntiles / grid_ctas) * grid_ctas;
}
__host__ __device__ inline uint32_t nitems_of(uint32_t ntiles, uint32_t nfull) { return nfull + 2u * (ntiles - nfull); }
}  // namespace pg

// bounded wait that also gives up once another role of the CTA has failed
__device__ __forceinline__ bool pg_wait(uint32_t bar, uint32_t parity, volatile int* fail, unsigned long long limit) {
  if (tn::mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = tn::tn_gtimer();
  while (!tn::mbar_try_wait(bar, parity)) {
    if (*fail || tn::tn_gtimer() - t0 > limit) {
      *fail = 1;
      return false;
    }
  }
  return true;
}

// sched_ctas: the CTA count the schedule was cut for (the SM count); the
// grid may be smaller when there are fewer work items
__global__ void __launch_bounds__(kThreads, 1) gemm_bf16_plain_kernel(ArgsBlob args, uint32_t sched_ctas,
                                                                     unsigned long long limit) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_fail;
  kl_args_gemm_bf16 a;
  memcpy(&a, args.b, sizeof(a));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tiles_n = tn::cdiv64(a.N, pg::BN), ntiles = tn::cdiv64(a.M, pg::BM) * tiles_n;
  const uint32_t nfull = pg::nfull_of(ntiles, sched_ctas), nitems = pg::nitems_of(ntiles, nfull);
  const uint32_t kt = tn::cdiv64(a.K, pg::BK);
  const uint32_t base = (tn::smem_u32(smem) + 1023u) & ~1023u;
  const uint32_t full0 = base + pg::STAGES * pg::kStage;  // TMA -> MMA, per stage
  const uint32_t empty0 = full0 + 8u * pg::STAGES;        // MMA -> TMA, per stage
  const uint32_t tfull0 = empty0 + 8u * pg::STAGES;       // MMA -> epilogue, per accumulator
  const uint32_t tempty0 = tfull0 + 16u;                  // epilogue -> MMA, per accumulator
  if (tid == 0) {
    for (uint32_t q = 0; q < pg::STAGES; ++q) {
      tn::mbar_init(full0 + 8u * q, 1u);
      tn::mbar_init(empty0 + 8u * q, 1u);
    }
    for (uint32_t q = 0; q < 2; ++q) {
      tn::mbar_init(tfull0 + 8u * q, 1u);
      tn::mbar_init(tempty0 + 8u * q, 4u);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 2) {
    tn::tmem_alloc(tn::smem_u32(&s_tmem), pg::kTmemCols);
    tn::tmem_relinquish();
  }
  tn::tc_fence_before();
  __syncthreads();
  tn::tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (warp == 0 && lane == 0) {
    // producer: K-slices of every work item of this CTA through the ring
    const char* tmA = static_cast<const char*>(a.tmaps);
    const char* tmB = tmA + 128;
    uint32_t s = 0, ph = 0;
    for (uint32_t i = blockIdx.x; i < nitems && !s_fail; i += gridDim.x) {
      const pg::Item it = pg::item(i, tiles_n, nfull, a.N);
      if (!it.valid) continue;
      const uint32_t nb = it.width / 64u;
      for (uint32_t kb = 0; kb < kt; ++kb) {
        if (!pg_wait(empty0 + 8u * s, ph ^ 1u, &s_fail, limit)) break;
        const uint32_t st = base + s * pg::kStage;
        tn::mbar_expect_tx(full0 + 8u * s, pg::kA + nb * pg::kBbox);
        tn::tma_load_2d(st, tmA, (int32_t)(kb * pg::BK), (int32_t)it.m0, full0 + 8u * s);
        for (uint32_t q = 0; q < nb; ++q)
          tn::tma_load_2d(st + pg::kA + q * pg::kBbox, tmB, (int32_t)(kb * pg::BK), (int32_t)(it.n0 + 64u * q),
                          full0 + 8u * s);
        if (++s == pg::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: one accumulator per work item, alternating
    uint32_t s = 0, ph = 0, j = 0;
    for (uint32_t i = blockIdx.x; i < nitems && !s_fail; i += gridDim.x) {
      const pg::Item it = pg::item(i, tiles_n, nfull, a.N);
      if (!it.valid) continue;
      const uint32_t b = j & 1u, use = j >> 1;
      ++j;
      if (!pg_wait(tempty0 + 8u * b, (use & 1u) ^ 1u, &s_fail, limit)) break;
      tn::tc_fence_after();
      const uint32_t d = tmem + b * pg::BN;
      const uint32_t idesc = it.width == pg::BN ? pg::kIdescFull : pg::kIdescHalf;
      bool ok = true;
      for (uint32_t kb = 0; kb < kt; ++kb) {
        if (!pg_wait(full0 + 8u * s, ph, &s_fail, limit)) {
          ok = false;
          break;
        }
        tn::tc_fence_after();
        const uint32_t sa = base + s * pg::kStage, sb = sa + pg::kA;
#pragma unroll
        for (uint32_t k = 0; k < pg::BK / 16u; ++k)
          tn::umma_bf16_id(d, tn::umma_desc_sw128(sa + 32u * k), tn::umma_desc_sw128(sb + 32u * k), idesc,
                           (kb | k) != 0u);
        tn::umma_commit(empty0 + 8u * s);  // the stage is free once these MMAs have read it
        if (++s == pg::STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      tn::umma_commit(tfull0 + 8u * b);    // the accumulator is complete
    }
  } else if (warp >= 4) {
    // epilogue: rows 32 (warp mod 4) + lane of the work item
    const uint32_t q = (uint32_t)warp & 3u;
    uint32_t j = 0;
    for (uint32_t i = blockIdx.x; i < nitems; i += gridDim.x) {
      const pg::Item it = pg::item(i, tiles_n, nfull, a.N);
      if (!it.valid) continue;
      const uint32_t b = j & 1u, use = j >> 1;
      ++j;
      if (!pg_wait(tfull0 + 8u * b, use & 1u, &s_fail, limit)) break;
      tn::tc_fence_after();
      const uint32_t row = it.m0 + 32u * q + (uint32_t)lane;
      float* crow = a.C + (uint64_t)row * a.N;
      for (uint32_t c0 = 0; c0 < it.width && it.n0 + c0 < a.N; c0 += 32u) {
        uint32_t r[32];
        tn::tmem_ld32(tmem + ((32u * q) << 16) + b * pg::BN + c0, r);
        if (row < a.M) {
#pragma unroll
          for (uint32_t v = 0; v < 8u; ++v)
            if (it.n0 + c0 + 4u * v < a.N)
              *reinterpret_cast<float4*>(crow + it.n0 + c0 + 4u * v) =
                  make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]), __uint_as_float(r[4 * v + 2]),
                              __uint_as_float(r[4 * v + 3]));
        }
      }
      tn::tc_fence_before();
      __syncwarp();
      if (lane == 0) tn::mbar_arrive(tempty0 + 8u * b);
    }
  }
  tn::tc_fence_before();
  __syncthreads();
  tn::tc_fence_after();
  if (s_fail && tid == 0) atomicCAS(&g_native_error, 0, (int)KL_EDEVICE_TIMEOUT);
  if (warp == 2) tn::tmem_dealloc(tmem, pg::kTmemCols);
}

static cudaError_t launch_gemm_bf16_plain(const void* args, cudaStream_t s) {
  static int n_sm = 0;
  static bool attr = false;
  if (!attr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_bf16_plain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pg::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  ArgsBlob blob;
  memcpy(blob.b, args, KL_MAX_ARGS_BYTES);
  const kl_args_gemm_bf16* g = static_cast<const kl_args_gemm_bf16*>(args);
  const uint32_t ntiles = tn::cdiv64(g->M, pg::BM) * tn::cdiv64(g->N, pg::BN);
  const uint32_t nitems = pg::nitems_of(ntiles, pg::nfull_of(ntiles, (uint32_t)n_sm));
  const uint32_t grid = nitems < (uint32_t)n_sm ? nitems : (uint32_t)n_sm;
  gemm_bf16_plain_kernel<<<grid, kThreads, pg::kSmem, s>>>(blob, (uint32_t)n_sm, 2000000000ull);
  return cudaGetLastError();
}

// Launch every stage of one tenant on stream s (stage order = stream order).
int native_launch_tenant(uint32_t type, const void* args, cudaStream_t s) {
  const uint32_t ns = tn::nstages(type, args);
  for (uint32_t st = 0; st < ns; ++st) {
    const uint32_t nb = tn::stage_blocks(type, args, st);
    if (nb == 0) continue;
    cudaError_t e;
    switch (type) {
      case KL_T_GATHER: e = launch_one<KL_T_GATHER>(args, st, nb, s); break;
      case KL_T_BLACKSCHOLES: e = launch_one<KL_T_BLACKSCHOLES>(args, st, nb, s); break;
      case KL_T_GEMM_F32: e = launch_one<KL_T_GEMM_F32>(args, st, nb, s); break;
      case KL_T_SPMV_CSR: e = launch_one<KL_T_SPMV_CSR>(args, st, nb, s); break;
      case KL_T_PCHASE: e = launch_one<KL_T_PCHASE>(args, st, nb, s); break;
      case KL_T_TRIAD: e = launch_one<KL_T_TRIAD>(args, st, nb, s); break;
      case KL_T_HIST256: e = launch_one<KL_T_HIST256>(args, st, nb, s); break;
      case KL_T_ESCAPE: e = launch_one<KL_T_ESCAPE>(args, st, nb, s); break;
      case KL_T_BITONIC: e = launch_one<KL_T_BITONIC>(args, st, nb, s); break;
      case KL_T_MATADD: e = launch_one<KL_T_MATADD>(args, st, nb, s); break;
      case KL_T_GEMM_BF16: e = launch_gemm_bf16_plain(args, s); break;
      case KL_T_TEA: e = launch_one<KL_T_TEA>(args, st, nb, s); break;
      case KL_T_SAD: e = launch_one<KL_T_SAD>(args, st, nb, s); break;
      case KL_T_STENCIL: e = launch_one<KL_T_STENCIL>(args, st, nb, s); break;
      case KL_T_MRIQ: e = launch_one<KL_T_MRIQ>(args, st, nb, s); break;
      case KL_T_TESTMIX: e = launch_one<KL_T_TESTMIX>(args, st, nb, s); break;
      case KL_T_BS255: e = launch_heavy<KL_T_BS255>(args, st, nb, s); break;
      case KL_T_HIST1024: e = launch_heavy<KL_T_HIST1024>(args, st, nb, s); break;
      case KL_T_GEMM_F32_BIG: e = launch_heavy<KL_T_GEMM_F32_BIG>(args, st, nb, s); break;
      default: return -1;
    }
    if (e != cudaSuccess) return -1;
  }
  return 0;
}

}  // namespace kl
