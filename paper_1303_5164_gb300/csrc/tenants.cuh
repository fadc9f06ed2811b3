// Tenant kernels as device functions of a rectified (virtual) block index.
//
// Section 4.1 slices a kernel by running a contiguous range of its thread
// blocks with an offset added to the built-in block index ("index
// rectification"). Here every tenant is written from the start as a function
// run_block(args, vb, smem) of the virtual block index vb, so the same body
// serves the plain launch (vb = blockIdx.x, the serial / multi-stream
// baselines) and the persistent co-scheduler (vb = slice offset + i).
// Blocks of one stage never depend on one another (Section 2.2, assumption 2);
// multi-stage tenants (histogram, bitonic sort) are chains of such grids.
//
// Every body uses 256 threads and no __syncthreads-free assumption about the
// caller: the caller guarantees all 256 threads enter run_block together.
//
// Floating point follows the written definitions bit for bit: explicit
// __f*_rn intrinsics wherever the compiler could otherwise contract or
// reassociate.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>
#include "kernelet.h"

namespace kl {
namespace tn {

// ------------------------------------------------------------------ shapes
// Cumulative block numbering over stages: block g of the tenant belongs to the
// stage s with begin(s) <= g < begin(s+1).

struct Stage {
  uint32_t s;      // stage index
  uint32_t begin;  // first cumulative block of the stage
  uint32_t end;    // one past its last
};

__host__ __device__ inline uint32_t cdiv64(uint64_t a, uint64_t b) {
  return (uint32_t)((a + b - 1) / b);
}

constexpr int kGatherPerBlock = 1024;
constexpr int kBsPerBlock = 256;
constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16;
constexpr int kGemmAStride = kGemmBM + 4;  // k-major A tile row (16-byte aligned, fewer bank conflicts)
constexpr int kSpmvRowsPerBlock = 32;
constexpr int kSpmvLanesPerRow = 8;
constexpr int kChasersPerBlock = 256;
constexpr int kTriadPerBlock = 4096;
constexpr int kHistBytesPerBlock = 32768;
constexpr int kEscapePerBlock = 256;
constexpr int kBitonicTileLog2 = 12;  // 4096 keys per tile
// BF16 tensor-core GEMM: 128x64 tile of C per block, K in steps of 64 (one
// 128-byte swizzle row per operand row), two pipeline stages
constexpr int kBfBM = 128, kBfBN = 64, kBfBK = 64;
constexpr uint32_t kBfStageA = kBfBM * kBfBK * 2u;      // 16 KB
constexpr uint32_t kBfStageB = kBfBN * kBfBK * 2u;      // 8 KB
constexpr uint32_t kBfStage = kBfStageA + kBfStageB;
constexpr uint32_t kBfSmem = 1024u + 2u * kBfStage + 64u;  // alignment slack, stages, barriers
constexpr uint32_t kBfTmemCols = 64;                       // FP32 accumulator: 128 lanes x 64 columns
constexpr int kTeaPerBlock = 512;        // 64-bit blocks (two per thread, one 16-byte load)
constexpr int kSadPerBlock = 256;        // SAD values (one per thread)
constexpr int kStencilPerBlock = 256;    // consecutive points (x fastest) of a block
constexpr int kMriqPerBlock = 256;       // k-samples (stage 0) or image points (stage 1)
// Resource-heavy variants, each run by a resource-class kernel of its own
constexpr int kBs255Threads = 128, kBs255PerThread = 32;
constexpr int kBs255PerBlock = kBs255Threads * kBs255PerThread;  // 4096 options
constexpr int kHist1024Threads = 1024;
constexpr int kHist1024BytesPerBlock = kHist1024Threads * 128;  // 131072
constexpr int kGbBM = 128, kGbBN = 128, kGbBK = 32, kGbStages = 3;
constexpr int kGbAStride = kGbBK + 4;                      // row-major A tile rows, 16-byte aligned
constexpr uint32_t kGbStageFloats = kGbBM * kGbAStride + kGbBK * kGbBN;
constexpr uint32_t kGbSmem = kGbStages * kGbStageFloats * 4u;  // 3 x 32.5 KB = 97.5 KB
constexpr int kTestmixPerBlock = 256;

__host__ __device__ inline uint32_t bitonic_tile_log2(uint32_t L) {
  return L < (uint32_t)kBitonicTileLog2 ? L : (uint32_t)kBitonicTileLog2;
}
constexpr uint32_t kBitonicHigh = 10;  // distances above the tile handled by one pass
__host__ __device__ inline uint32_t bitonic_nstages(uint32_t L) {
  uint32_t P = bitonic_tile_log2(L), n = 1;
  for (uint32_t d = 1; d + P <= L; ++d) n += (d + kBitonicHigh - 1) / kBitonicHigh + 1;
  return n;
}

// Static shape: stages, blocks per stage, dynamic shared memory.
__host__ __device__ inline uint32_t nstages(uint32_t type, const void* a) {
  switch (type) {
    case KL_T_HIST256: return 2;
    case KL_T_HIST1024: return 2;
    case KL_T_MRIQ: return 2;
    case KL_T_BITONIC: return bitonic_nstages(((const kl_args_bitonic*)a)->log2n);
    default: return 1;
  }
}

__host__ __device__ inline uint32_t stage_blocks(uint32_t type, const void* a, uint32_t s) {
  switch (type) {
    case KL_T_GATHER: return cdiv64(((const kl_args_gather*)a)->n, kGatherPerBlock);
    case KL_T_BLACKSCHOLES: return cdiv64(((const kl_args_blackscholes*)a)->n, kBsPerBlock);
    case KL_T_GEMM_F32: {
      const kl_args_gemm_f32* g = (const kl_args_gemm_f32*)a;
      return cdiv64(g->M, kGemmBM) * cdiv64(g->N, kGemmBN);
    }
    case KL_T_SPMV_CSR: return cdiv64(((const kl_args_spmv_csr*)a)->nrows, kSpmvRowsPerBlock);
    case KL_T_PCHASE: return cdiv64(((const kl_args_pchase*)a)->nchasers, kChasersPerBlock);
    case KL_T_TRIAD: return cdiv64(((const kl_args_triad*)a)->n, kTriadPerBlock);
    case KL_T_HIST256: return s == 0 ? 1u : cdiv64(((const kl_args_hist256*)a)->n, kHistBytesPerBlock);
    case KL_T_ESCAPE: {
      const kl_args_escape* e = (const kl_args_escape*)a;
      return cdiv64((uint64_t)e->width * e->height, kEscapePerBlock);
    }
    case KL_T_BITONIC: {
      uint32_t L = ((const kl_args_bitonic*)a)->log2n;
      return 1u << (L - bitonic_tile_log2(L));
    }
    case KL_T_MATADD: {
      uint32_t t = ((const kl_args_matadd*)a)->n / 16;
      return t * t;
    }
    case KL_T_GEMM_BF16: {
      const kl_args_gemm_bf16* g = (const kl_args_gemm_bf16*)a;
      return cdiv64(g->M, kBfBM) * cdiv64(g->N, kBfBN);
    }
    case KL_T_TEA: return cdiv64(((const kl_args_tea*)a)->n, kTeaPerBlock);
    case KL_T_SAD: {
      const kl_args_sad* d = (const kl_args_sad*)a;
      const uint64_t D = 2ull * d->range + 1ull;
      return cdiv64((uint64_t)(d->width / 4) * (d->height / 4) * D * D, kSadPerBlock);
    }
    case KL_T_STENCIL: {
      const kl_args_stencil* t = (const kl_args_stencil*)a;
      return cdiv64((uint64_t)t->nx * t->ny * t->nz, kStencilPerBlock);
    }
    case KL_T_MRIQ: {
      const kl_args_mriq* m = (const kl_args_mriq*)a;
      return s == 0 ? cdiv64(m->numK, kMriqPerBlock) : cdiv64(m->numX, kMriqPerBlock);
    }
    case KL_T_TESTMIX: return cdiv64(((const kl_args_testmix*)a)->nthreads, kTestmixPerBlock);
    case KL_T_BS255: return cdiv64(((const kl_args_blackscholes*)a)->n, kBs255PerBlock);
    case KL_T_HIST1024: return s == 0 ? 1u : cdiv64(((const kl_args_hist256*)a)->n, kHist1024BytesPerBlock);
    case KL_T_GEMM_F32_BIG: {
      const kl_args_gemm_f32* g = (const kl_args_gemm_f32*)a;
      return cdiv64(g->M, kGbBM) * cdiv64(g->N, kGbBN);
    }
    default: return 0;
  }
}

__host__ __device__ inline uint64_t total_blocks(uint32_t type, const void* a) {
  uint32_t ns = nstages(type, a);
  if (type == KL_T_BITONIC) return (uint64_t)ns * stage_blocks(type, a, 0);
  uint64_t t = 0;
  for (uint32_t s = 0; s < ns; ++s) t += stage_blocks(type, a, s);
  return t;
}

// Stage containing cumulative block g (g < total).
__host__ __device__ inline Stage stage_of(uint32_t type, const void* a, uint32_t g) {
  if (type == KL_T_HIST256 || type == KL_T_HIST1024) {
    if (g == 0) return Stage{0, 0, 1};
    return Stage{1, 1, 1 + stage_blocks(type, a, 1)};
  }
  if (type == KL_T_BITONIC) {
    uint32_t nb = stage_blocks(type, a, 0);
    uint32_t s = g / nb;
    return Stage{s, s * nb, (s + 1) * nb};
  }
  if (type == KL_T_MRIQ) {
    const uint32_t n0 = stage_blocks(type, a, 0);
    if (g < n0) return Stage{0, 0, n0};
    return Stage{1, n0, n0 + stage_blocks(type, a, 1)};
  }
  return Stage{0, 0, stage_blocks(type, a, 0)};
}


// Co-scheduler builds. Every tenant body compiled into the persistent kernel
// shares its register budget, so each run uses the build that carries only
// the types it holds:
//   kBuildPlain: the first ten types; 4 CTAs x 256 threads per SM, 64 registers.
//   kBuildFull:  every type (adds the tcgen05 GEMM, TEA, SAD, stencil, MRI-Q).
//   kBuildLight: short memory- or issue-bound bodies that fit 32 registers
//                without shared memory beyond 256 B; 8 CTAs x 256 threads per
//                SM, the 64 warps these kernels reach as plain launches
//                (latency-bound ones such as SpMV and the stencil need them to
//                keep enough loads in flight). Left out although they compile
//                to 32 registers or fewer as plain launches: SAD and MRI-Q (their
//                inner loops spill at 32 registers inside the co-scheduler and
//                ran 7-12% slower than at 4 slots) and the pointer chase (64 long
//                blocks per kernel: a pair and its fill list leave most of 8
//                slots per SM idle).
enum : int { kBuildPlain = 0, kBuildFull = 1, kBuildLight = 2 };
__host__ __device__ constexpr bool in_plain_build(uint32_t type) {
  return type <= KL_T_MATADD || type == KL_T_TESTMIX;
}
__host__ __device__ constexpr bool in_light_build(uint32_t type) {
  return type == KL_T_GATHER || type == KL_T_BLACKSCHOLES || type == KL_T_SPMV_CSR || type == KL_T_TRIAD ||
         type == KL_T_ESCAPE || type == KL_T_MATADD || type == KL_T_TEA || type == KL_T_STENCIL ||
         type == KL_T_TESTMIX;
}
__host__ __device__ constexpr bool in_build(int build, uint32_t type) {
  return build == kBuildFull    ? type < KL_T_MAIN_COUNT
         : build == kBuildLight ? in_light_build(type)
                                : in_plain_build(type);
}
// Resource classes: 0 = the co-scheduler's 256-thread, 64-register slots; the
// heavy variants each run in a persistent kernel of their own (kl_cosched.cu,
// class_kernel) with one CTA per SM beside two co-scheduler slots: each of
// those CTAs takes at most half of the SM's 64 K registers.
enum : int { kClassMain = 0, kClassBs255 = 1, kClassHist1024 = 2, kClassGemmBig = 3, kNumClasses = 4 };
__host__ __device__ constexpr int resource_class(uint32_t type) {
  return type == KL_T_BS255 ? kClassBs255 : type == KL_T_HIST1024 ? kClassHist1024
                                          : type == KL_T_GEMM_F32_BIG ? kClassGemmBig : kClassMain;
}
__host__ __device__ constexpr uint32_t block_threads(uint32_t type) {
  return type == KL_T_BS255 ? (uint32_t)kBs255Threads : type == KL_T_HIST1024 ? (uint32_t)kHist1024Threads : 256u;
}

__host__ __device__ constexpr uint32_t smem_bytes(uint32_t type) {
  switch (type) {
    case KL_T_GEMM_F32: return 2u * (kGemmBK * kGemmAStride + kGemmBK * kGemmBN) * 4u;  // 16.5 KB
    case KL_T_SPMV_CSR: return 256u;                                              // long-row list
    case KL_T_HIST256: return 256u * 32u * 4u;                                    // 32 KB
    case KL_T_BITONIC: return ((1u << kBitonicTileLog2) + (1u << (kBitonicTileLog2 - 5))) * 4u;  // padded tile
    case KL_T_GEMM_BF16: return kBfSmem;                                          // 49.1 KB
    case KL_T_MRIQ: return 4u * kMriqPerBlock * 4u;                               // 4 KB k-sample chunk
    case KL_T_HIST1024: return 256u * 32u * 4u;                                   // 32 KB
    case KL_T_GEMM_F32_BIG: return kGbSmem;                                       // 97.5 KB
    default: return 0;
  }
}
constexpr uint32_t kMaxTenantSmem = kBfSmem;  // largest of the co-scheduler's types (BF16 GEMM)
constexpr uint32_t kMaxLightSmem = 2048;       // the light build's types need at most 256 B (SpMV)
constexpr uint32_t kMinCtaSmem = 2048;         // co-scheduler CTAs always have this much (re-plan scratch)
static_assert(256u * 32u * 4u <= kMaxTenantSmem, "smem bound");
__host__ __device__ constexpr bool light_smem_fits() {
  for (uint32_t t = 0; t < KL_T_MAIN_COUNT; ++t)
    if (in_light_build(t) && smem_bytes(t) > kMaxLightSmem) return false;
  return true;
}
static_assert(light_smem_fits(), "every light-build type fits the light build's shared memory");
static_assert(2u * (kGemmBK * kGemmAStride + kGemmBK * kGemmBN) * 4u <= kMaxTenantSmem, "smem bound");

#ifdef __CUDACC__

// Per-CTA context a tenant body may need besides its arguments: the shared
// word holding the CTA's TMEM address (kernels built with the tensor-core
// tenant), the word that records a device-side error, and the bound on any
// wait.
struct BlockCtx {
  uint32_t* tmem;
  int* err;
  unsigned long long limit_ns;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// exp and log from published methods (no math-library internals), the same
// written recipe the CPU oracle follows independently:
//   exp: Cody-Waite reduction x = n ln2 + r (two-part ln2), degree-7 Taylor
//        polynomial of e^r by Horner with fused multiply-add, scale by 2^n.
//   log: x = 2^e m, m in [sqrt(1/2), sqrt(2)]; log m = 2 atanh t with
//        t = (m-1)/(m+1) as 2t + 2t (t^2/3 + t^4/5 + t^6/7 + t^8/9); + e ln2.
__device__ __forceinline__ float kl_expf(float x) {
  if (x != x) return x;
  if (x > 88.7228394f) return __int_as_float(0x7f800000);
  if (x < -103.972694f) return 0.0f;
  float t = __fmul_rn(x, 1.44269504f);
  float n = rintf(t);
  float r = __fmaf_rn(-n, 0.693145751953125f, x);
  r = __fmaf_rn(-n, 1.42860677e-06f, r);
  float p = 1.98412698e-04f;
  p = __fmaf_rn(p, r, 1.38888889e-03f);
  p = __fmaf_rn(p, r, 8.33333333e-03f);
  p = __fmaf_rn(p, r, 4.16666667e-02f);
  p = __fmaf_rn(p, r, 1.66666667e-01f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  int ni = (int)n;
  if (ni < -126) {
    p = __fmul_rn(p, __int_as_float((127 - 64) << 23));
    ni += 64;
  }
  if (ni > 127) {
    p = __fmul_rn(p, 2.0f);
    ni -= 1;
  }
  return __fmul_rn(p, __int_as_float((ni + 127) << 23));
}

__device__ __forceinline__ float kl_logf(float x) {
  if (x != x) return x;
  if (x < 0.0f) return __int_as_float(0x7fc00000);
  if (x == 0.0f) return __int_as_float(0xff800000);
  if (x == __int_as_float(0x7f800000)) return x;
  int e_adj = 0;
  if (x < 1.17549435e-38f) {
    x = __fmul_rn(x, 16777216.0f);
    e_adj = -24;
  }
  unsigned b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127 + e_adj;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > 1.41421356f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  float num = __fsub_rn(m, 1.0f);
  float den = __fadd_rn(m, 1.0f);
  float t = __fdiv_rn(num, den);
  float t2 = __fmul_rn(t, t);
  float s = 1.11111111e-01f;
  s = __fmaf_rn(s, t2, 1.42857143e-01f);
  s = __fmaf_rn(s, t2, 2.00000000e-01f);
  s = __fmaf_rn(s, t2, 3.33333333e-01f);
  float st2 = __fmul_rn(s, t2);
  float tt = __fadd_rn(t, t);
  float lm = __fmaf_rn(tt, st2, tt);
  float fe = (float)e;
  float res = __fmaf_rn(fe, 1.42860677e-06f, lm);
  return __fmaf_rn(fe, 0.693145751953125f, res);
}

// Cumulative normal distribution, Abramowitz & Stegun 26.2.17 with reflection.
__device__ __forceinline__ float kl_cnd(float d) {
  float ad = fabsf(d);
  float pa = __fmul_rn(0.2316419f, ad);
  float den = __fadd_rn(1.0f, pa);
  float k = __fdiv_rn(1.0f, den);
  float poly = 1.330274429f;
  poly = __fmaf_rn(poly, k, -1.821255978f);
  poly = __fmaf_rn(poly, k, 1.781477937f);
  poly = __fmaf_rn(poly, k, -0.356563782f);
  poly = __fmaf_rn(poly, k, 0.31938153f);
  poly = __fmul_rn(poly, k);
  float hd = __fmul_rn(0.5f, d);
  float e = __fmul_rn(hd, d);
  float ex = kl_expf(-e);
  float phi = __fmul_rn(0.398942280f, ex);
  float c = __fmul_rn(phi, poly);
  return (d > 0.0f) ? __fsub_rn(1.0f, c) : c;
}

// ------------------------------------------------------------------ gather

__device__ __forceinline__ void gather_block(const kl_args_gather& a, uint32_t vb) {
  const uint64_t base = (uint64_t)vb * kGatherPerBlock + (uint64_t)threadIdx.x * 4;
  if (base + 4 <= a.n) {
    int4 ix = __ldcs(reinterpret_cast<const int4*>(a.idx + base));
    int4 o;
    o.x = __ldg(a.a + ix.x);
    o.y = __ldg(a.a + ix.y);
    o.z = __ldg(a.a + ix.z);
    o.w = __ldg(a.a + ix.w);
    __stcs(reinterpret_cast<int4*>(a.out + base), o);
  } else {
    for (uint64_t i = base; i < a.n && i < base + 4; ++i) a.out[i] = a.a[a.idx[i]];
  }
}

// ------------------------------------------------------------------ Black-Scholes

// One option by the written recipe (every operation separately rounded).
__device__ __forceinline__ void bs_option(float s, float k, float rr, float vv, float tt, float& call, float& put) {
  float sqrtT = __fsqrt_rn(tt);
  float vsqrtT = __fmul_rn(vv, sqrtT);
  float q = __fdiv_rn(s, k);
  float lq = kl_logf(q);
  float h = __fmul_rn(0.5f, vv);
  h = __fmul_rn(h, vv);
  float ah = __fadd_rn(rr, h);
  ah = __fmul_rn(ah, tt);
  float num = __fadd_rn(lq, ah);
  float d1 = __fdiv_rn(num, vsqrtT);
  float d2 = __fsub_rn(d1, vsqrtT);
  float c1 = kl_cnd(d1);
  float c2 = kl_cnd(d2);
  float m = __fmul_rn(rr, tt);
  float disc = kl_expf(-m);
  float kd = __fmul_rn(k, disc);
  float t1 = __fmul_rn(s, c1);
  float t2 = __fmul_rn(kd, c2);
  call = __fsub_rn(t1, t2);
  float u2 = __fsub_rn(1.0f, c2);
  float u1 = __fsub_rn(1.0f, c1);
  float p1 = __fmul_rn(kd, u2);
  float p2 = __fmul_rn(s, u1);
  put = __fsub_rn(p1, p2);
}

__device__ __forceinline__ void blackscholes_block(const kl_args_blackscholes& a, uint32_t vb) {
  const uint64_t i = (uint64_t)vb * kBsPerBlock + threadIdx.x;
  if (i >= a.n) return;
  float c, p;
  bs_option(__ldcs(a.S + i), __ldcs(a.K + i), __ldcs(a.r + i), __ldcs(a.v + i), __ldcs(a.T + i), c, p);
  __stcs(a.call + i, c);
  __stcs(a.put + i, p);
}

// Resource-heavy variant (128 threads): 32 options a thread, all inputs loaded
// into registers before any is priced, option j of thread t at block offset
// 128 j + t (coalesced per j). Same arithmetic per option as above.
__device__ __forceinline__ void bs255_block(const kl_args_blackscholes& a, uint32_t vb) {
  const uint64_t base = (uint64_t)vb * kBs255PerBlock + threadIdx.x;
  float s[kBs255PerThread], k[kBs255PerThread], r[kBs255PerThread], v[kBs255PerThread], t[kBs255PerThread];
#pragma unroll
  for (int j = 0; j < kBs255PerThread; ++j) {
    const uint64_t i = base + (uint64_t)j * kBs255Threads;
    const bool ok = i < a.n;
    s[j] = ok ? __ldcs(a.S + i) : 1.0f;
    k[j] = ok ? __ldcs(a.K + i) : 1.0f;
    r[j] = ok ? __ldcs(a.r + i) : 0.0f;
    v[j] = ok ? __ldcs(a.v + i) : 1.0f;
    t[j] = ok ? __ldcs(a.T + i) : 1.0f;
  }
#pragma unroll
  for (int j = 0; j < kBs255PerThread; ++j) {
    const uint64_t i = base + (uint64_t)j * kBs255Threads;
    float c, p;
    bs_option(s[j], k[j], r[j], v[j], t[j], c, p);
    if (i < a.n) {
      __stcs(a.call + i, c);
      __stcs(a.put + i, p);
    }
  }
}

// ------------------------------------------------------------------ FP32 GEMM
// 64x64 tile of C per block; 256 threads as 16x16, each a 4x4 micro-tile (rows
// ty*4..+3, cols tx*4..+3). K advances in 16-wide tiles: B by cp.async into a
// [k][n] shared tile, A through registers into a k-major [k][m] shared tile,
// both double buffered and zero-filled past the edges. Each k step is one
// 128-bit shared load of A and one of B for 16 fused multiply-adds. For every
// C[i][j] the fused multiply-adds run over k = 0,1,2,... in order from +0, so
// the result is the ascending fused chain exactly (zero padding adds exact 0).

__device__ __forceinline__ void gemm_f32_block(const kl_args_gemm_f32& a, uint32_t vb, char* smem) {
  float* As = reinterpret_cast<float*>(smem);            // [2][16][68]  (k-major)
  float* Bs = As + 2 * kGemmBK * kGemmAStride;            // [2][16][64]
  const uint32_t tilesN = (a.N + kGemmBN - 1) / kGemmBN;
  const uint32_t m0 = (vb / tilesN) * kGemmBM;
  const uint32_t n0 = (vb % tilesN) * kGemmBN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const uint32_t ktiles = (a.K + kGemmBK - 1) / kGemmBK;
  // A loader: row m = tid % 64 of the tile, k chunk (tid / 64) * 4; it walks
  // a precomputed pointer so the argument block need not stay in registers
  const uint32_t akc = (tid >> 6) * 4;
  const bool arow_ok = m0 + (tid & 63) < a.M;
  const float* aptr = a.A + (uint64_t)(arow_ok ? m0 + (tid & 63) : 0) * a.K + akc;
  const uint32_t K = a.K;

  auto load_a = [&](uint32_t kt) -> float4 {
    const uint32_t gk = kt * kGemmBK + akc;
    if (arow_ok && gk < K) return __ldg(reinterpret_cast<const float4*>(aptr + kt * kGemmBK));
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store_a = [&](float4 v, int buf) {
    float* d = As + buf * kGemmBK * kGemmAStride + akc * kGemmAStride + (tid & 63);
    d[0] = v.x;
    d[kGemmAStride] = v.y;
    d[2 * kGemmAStride] = v.z;
    d[3 * kGemmAStride] = v.w;
  };
  auto load_b = [&](uint32_t kt, int buf) {
    const int row = tid >> 4, nc = tid & 15;
    const uint32_t gk = kt * kGemmBK + row, gn = n0 + nc * 4;
    const bool ok = gk < a.K && gn < a.N;
    const float* src = ok ? a.B + (uint64_t)gk * a.N + gn : a.B;
    cp_async16(Bs + buf * kGemmBK * kGemmBN + row * kGemmBN + nc * 4, src, ok ? 16 : 0);
    cp_async_commit();
  };

  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  store_a(load_a(0), 0);
  load_b(0, 0);
  for (uint32_t kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    float4 an = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kt + 1 < ktiles) {
      an = load_a(kt + 1);  // lands in registers while this tile is computed
      load_b(kt + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* Ab = As + buf * kGemmBK * kGemmAStride + ty * 4;
    const float* Bb = Bs + buf * kGemmBK * kGemmBN + tx * 4;
#pragma unroll
    for (int k = 0; k < kGemmBK; ++k) {
      const float4 av = *reinterpret_cast<const float4*>(Ab + k * kGemmAStride);
      const float4 bv = *reinterpret_cast<const float4*>(Bb + k * kGemmBN);
      const float ar[4] = {av.x, av.y, av.z, av.w};
      const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(ar[i], br[j], acc[i][j]);
    }
    if (kt + 1 < ktiles) store_a(an, buf ^ 1);
    __syncthreads();
  }
  const uint32_t gn = n0 + tx * 4;
  if (gn < a.N) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t gm = m0 + ty * 4 + i;
      if (gm < a.M)
        *reinterpret_cast<float4*>(a.C + (uint64_t)gm * a.N + gn) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
  }
}

// Resource-heavy variant: one 128 x 128 tile of C per block of 256 threads,
// K in steps of 32 through a three-stage cp.async ring of A (row-major rows,
// padded) and B tiles (97.5 KB of shared memory). Thread (ty, tx) of 16 x 16
// holds rows ty*4 + {0..3} and 64 + ty*4 + {0..3} and the same columns from
// tx: 64 accumulators, each the ascending fused chain over k from +0 of the
// definition (bit-identical to the oracle).
__device__ __forceinline__ void gemm_big_block(const kl_args_gemm_f32& a, uint32_t vb, char* smem) {
  float* sbase = reinterpret_cast<float*>(smem);
  const uint32_t tilesN = (a.N + kGbBN - 1) / kGbBN;
  const uint32_t m0 = (vb / tilesN) * kGbBM, n0 = (vb % tilesN) * kGbBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const uint32_t ktiles = (a.K + kGbBK - 1) / kGbBK;
  auto As = [&](int st) { return sbase + st * kGbStageFloats; };
  auto Bs = [&](int st) { return sbase + st * kGbStageFloats + kGbBM * kGbAStride; };
  auto load = [&](uint32_t kt, int st) {
    // A: 128 rows x 8 chunks of 4 floats; B: 32 rows x 32 chunks; 4 of each a thread
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = tid + u * 256;
      const int ar = c >> 3, ak = (c & 7) * 4;
      const uint32_t gm = m0 + ar, gk = kt * kGbBK + ak;
      const bool aok = gm < a.M && gk < a.K;
      cp_async16(As(st) + ar * kGbAStride + ak, aok ? a.A + (uint64_t)gm * a.K + gk : a.A, aok ? 16 : 0);
      const int br = c >> 5, bn = (c & 31) * 4;
      const uint32_t gk2 = kt * kGbBK + br, gn = n0 + bn;
      const bool bok = gk2 < a.K && gn < a.N;
      cp_async16(Bs(st) + br * kGbBN + bn, bok ? a.B + (uint64_t)gk2 * a.N + gn : a.B, bok ? 16 : 0);
    }
    cp_async_commit();
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  load(0, 0);
  if (ktiles > 1) load(1, 1);
  for (uint32_t kt = 0; kt < ktiles; ++kt) {
    const int st = kt % kGbStages;
    if (kt + 1 < ktiles)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    __syncthreads();  // stage kt landed for everyone; stage kt-1 is no longer read
    if (kt + 2 < ktiles) load(kt + 2, (kt + 2) % kGbStages);
    const float* A0 = As(st) + (ty * 4) * kGbAStride;
    const float* A1 = As(st) + (64 + ty * 4) * kGbAStride;
    const float* B0 = Bs(st) + tx * 4;
#pragma unroll
    for (int k2 = 0; k2 < kGbBK; k2 += 2) {
      float2 ar[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = *reinterpret_cast<const float2*>(A0 + i * kGbAStride + k2);
        ar[4 + i] = *reinterpret_cast<const float2*>(A1 + i * kGbAStride + k2);
      }
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const float4 b0 = *reinterpret_cast<const float4*>(B0 + (k2 + kk) * kGbBN);
        const float4 b1 = *reinterpret_cast<const float4*>(B0 + (k2 + kk) * kGbBN + 64);
        const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float av = kk == 0 ? ar[i].x : ar[i].y;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = __fmaf_rn(av, br[j], acc[i][j]);
        }
      }
    }
  }
  __syncthreads();  // the next block reuses the ring
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gm >= a.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t gn = n0 + h * 64 + tx * 4;
      if (gn < a.N)
        *reinterpret_cast<float4*>(a.C + (uint64_t)gm * a.N + gn) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
    }
  }
}

// ------------------------------------------------------------------ testing kernel (Section 4.3)
// Thread g: `iters` rounds of `mem` streaming loads (consecutive threads read
// consecutive words; each round a fresh stretch of the input) added to acc,
// then `alu` dependent fused multiply-adds acc = c1 acc + c2. The ratio of the
// two sets the kernel's pipeline and memory-bandwidth utilisation.
__device__ __forceinline__ void testmix_block(const kl_args_testmix& a, uint32_t vb) {
  const uint32_t g = vb * kTestmixPerBlock + threadIdx.x;
  if (g >= a.nthreads) return;
  const uint32_t mask = a.n_in - 1u;
  float acc = 0.0f;
  uint32_t idx = g & mask;
  for (uint32_t it = 0; it < a.iters; ++it) {
    for (uint32_t m = 0; m < a.mem; ++m) {
      acc = __fadd_rn(acc, __ldcs(a.in + idx));
      idx = (idx + a.nthreads) & mask;
    }
    for (uint32_t q = 0; q < a.alu; ++q) acc = __fmaf_rn(acc, a.c1, a.c2);
  }
  a.out[g] = acc;
}

// ------------------------------------------------------------------ CSR SpMV
// 32 rows per block. A row of at most 128 non-zeros belongs to 8 lanes: lane l
// sums elements l, l+8, l+16, ... with an ascending fused chain, then a fixed
// xor butterfly (4, 2, 1) adds the 8 partial sums. A longer row (power-law
// rows reach 8192) is summed by all 256 threads of the block: thread t takes
// elements t, t+256, ..., then a fixed butterfly within each warp (16..1) and a
// fixed pairwise tree over the 8 warps. Either way the order of the additions
// depends only on the row's length, never on slicing or scheduling.

constexpr int kSpmvLong = 128;

__device__ __forceinline__ float spmv_chain(const kl_args_spmv_csr& a, int e, int end, int step, float acc) {
  // four elements per round, loads issued before any use (predicated past the
  // row end); the fused chain still runs over e, e+step, e+2*step, ... in order
  for (; e < end; e += 4 * step) {
    int c[4];
    float v[4], x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = e + k * step < end;
      c[k] = ok ? __ldcs(a.col + e + k * step) : 0;
      v[k] = ok ? __ldcs(a.val + e + k * step) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = (e + k * step < end) ? __ldg(a.x + c[k]) : 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (e + k * step < end) acc = __fmaf_rn(v[k], x[k], acc);
  }
  return acc;
}

__device__ __forceinline__ void spmv_csr_block(const kl_args_spmv_csr& a, uint32_t vb, char* smem) {
  uint32_t* list = reinterpret_cast<uint32_t*>(smem);          // [32] long rows
  uint32_t* cnt = list + 32;
  float* red = reinterpret_cast<float*>(list + 40);            // [8] warp partials
  const uint32_t row = vb * kSpmvRowsPerBlock + (threadIdx.x >> 3);
  const int l = threadIdx.x & 7;
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  int beg = 0, end = 0;
  if (row < a.nrows) {
    beg = __ldg(a.rowptr + row);
    end = __ldg(a.rowptr + row + 1);
  }
  const bool is_long = end - beg > kSpmvLong;
  float acc = 0.0f;
  if (!is_long) acc = spmv_chain(a, beg + l, end, 8, 0.0f);
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 4));
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 2));
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 1));
  if (l == 0 && row < a.nrows) {
    if (!is_long)
      a.y[row] = acc;
    else
      list[atomicAdd(cnt, 1u)] = row;
  }
  __syncthreads();
  const uint32_t nlong = *cnt;
  for (uint32_t k = 0; k < nlong; ++k) {
    const uint32_t r = list[k];
    const int b = __ldg(a.rowptr + r), e = __ldg(a.rowptr + r + 1);
    float s = spmv_chain(a, b + threadIdx.x, e, 256, 0.0f);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float p01 = __fadd_rn(red[0], red[1]), p23 = __fadd_rn(red[2], red[3]);
      float p45 = __fadd_rn(red[4], red[5]), p67 = __fadd_rn(red[6], red[7]);
      a.y[r] = __fadd_rn(__fadd_rn(p01, p23), __fadd_rn(p45, p67));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ pointer chase

__device__ __forceinline__ void pchase_block(const kl_args_pchase& a, uint32_t vb) {
  // one chain per thread: the chains of a kernel spread over every SM, whose
  // outstanding-miss capacity bounds how many dependent loads are in flight
  // (four chains per thread, 1024 chasers per block, was measured slower on
  // GB300: a kernel's blocks then cover fewer SMs, and concurrent chase
  // kernels thrash the address translation caches sooner)
  const uint32_t t = vb * kChasersPerBlock + threadIdx.x;
  if (t >= a.nchasers) return;
  int p = __ldg(a.start + t);
  for (uint32_t h = 0; h < a.hops; ++h) p = __ldcg(a.next + p);
  a.end[t] = p;
}

// ------------------------------------------------------------------ triad

__device__ __forceinline__ void triad_block(const kl_args_triad& a, uint32_t vb) {
  const uint64_t base = (uint64_t)vb * kTriadPerBlock;
  if (base + kTriadPerBlock <= a.n) {
    float4 b[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint64_t i = base + ((uint64_t)u * 256 + threadIdx.x) * 4;
      b[u] = __ldcs(reinterpret_cast<const float4*>(a.b + i));
      c[u] = __ldcs(reinterpret_cast<const float4*>(a.c + i));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint64_t i = base + ((uint64_t)u * 256 + threadIdx.x) * 4;
      float4 r;
      r.x = __fmaf_rn(a.s, c[u].x, b[u].x);
      r.y = __fmaf_rn(a.s, c[u].y, b[u].y);
      r.z = __fmaf_rn(a.s, c[u].z, b[u].z);
      r.w = __fmaf_rn(a.s, c[u].w, b[u].w);
      __stcs(reinterpret_cast<float4*>(a.a + i), r);
    }
  } else {
    for (uint64_t i = base + threadIdx.x; i < a.n && i < base + kTriadPerBlock; i += 256)
      a.a[i] = __fmaf_rn(a.s, a.c[i], a.b[i]);
  }
}

// ------------------------------------------------------------------ histogram
// stage 0: one block clears the 256 bins; stage 1: each block counts 32 KB into
// 32 lane-private copies of the histogram in shared memory (word bin*32+lane,
// so the 32 lanes of a warp never share a bank even when they hit the same
// bin), then adds its non-zero bins to the global histogram.

__device__ __forceinline__ void hist256_block(const kl_args_hist256& a, uint32_t stage, uint32_t vb,
                                              char* smem) {
  if (stage == 0) {
    a.hist[threadIdx.x] = 0u;
    return;
  }
  uint32_t* sh = reinterpret_cast<uint32_t*>(smem);  // [256][32]
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < 8; ++w)
    reinterpret_cast<uint4*>(sh)[w * 256 + threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const uint64_t base = (uint64_t)vb * kHistBytesPerBlock;
  if (base + kHistBytesPerBlock <= a.n) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = __ldcs(reinterpret_cast<const uint4*>(a.data + base + ((uint64_t)u * 256 + threadIdx.x) * 16));
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint32_t w4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        atomicAdd(sh + (((w4[q] >> 0) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + (((w4[q] >> 8) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + (((w4[q] >> 16) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + ((w4[q] >> 24) << 5 | lane), 1u);
      }
    }
  } else {
    for (uint64_t i = base + threadIdx.x; i < a.n && i < base + kHistBytesPerBlock; i += 256)
      atomicAdd(sh + ((uint32_t)a.data[i] << 5 | lane), 1u);
  }
  __syncthreads();
  uint32_t sum = 0;
#pragma unroll 8
  for (uint32_t c = 0; c < 32; ++c) sum += sh[threadIdx.x << 5 | ((c + lane) & 31)];
  if (sum) atomicAdd(a.hist + threadIdx.x, sum);
}

// Resource-heavy variant: 1024-thread blocks of 131072 bytes (eight 16-byte
// loads a thread), the same 32 lane-private copies of the 256 bins in shared
// memory (each shared by the 32 warps), then per bin one global add.
__device__ __forceinline__ void hist1024_block(const kl_args_hist256& a, uint32_t stage, uint32_t vb, char* smem) {
  if (stage == 0) {
    if (threadIdx.x < 256) a.hist[threadIdx.x] = 0u;
    return;
  }
  uint32_t* sh = reinterpret_cast<uint32_t*>(smem);  // [256][32]
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < 2; ++w)
    reinterpret_cast<uint4*>(sh)[w * kHist1024Threads + threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const uint64_t base = (uint64_t)vb * kHist1024BytesPerBlock;
  if (base + kHist1024BytesPerBlock <= a.n) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = __ldcs(reinterpret_cast<const uint4*>(a.data + base + ((uint64_t)u * kHist1024Threads + threadIdx.x) * 16));
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint32_t w4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        atomicAdd(sh + (((w4[q] >> 0) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + (((w4[q] >> 8) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + (((w4[q] >> 16) & 0xffu) << 5 | lane), 1u);
        atomicAdd(sh + ((w4[q] >> 24) << 5 | lane), 1u);
      }
    }
  } else {
    for (uint64_t i = base + threadIdx.x; i < a.n && i < base + kHist1024BytesPerBlock; i += kHist1024Threads)
      atomicAdd(sh + ((uint32_t)a.data[i] << 5 | lane), 1u);
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    uint32_t sum = 0;
#pragma unroll 8
    for (uint32_t c = 0; c < 32; ++c) sum += sh[threadIdx.x << 5 | ((c + lane) & 31)];
    if (sum) atomicAdd(a.hist + threadIdx.x, sum);
  }
}

// ------------------------------------------------------------------ escape-time

__device__ __forceinline__ void escape_block(const kl_args_escape& a, uint32_t vb) {
  const uint64_t p = (uint64_t)vb * kEscapePerBlock + threadIdx.x;
  const uint64_t npx = (uint64_t)a.width * a.height;
  if (p >= npx) return;
  const uint32_t i = (uint32_t)(p / a.width), j = (uint32_t)(p % a.width);
  float tj = __fadd_rn((float)j, 0.5f);
  float ti = __fadd_rn((float)i, 0.5f);
  float cx = __fadd_rn(a.x0, __fmul_rn(tj, a.dx));
  float cy = __fadd_rn(a.y0, __fmul_rn(ti, a.dy));
  float x = 0.0f, y = 0.0f;
  uint32_t it = 0;
  while (it < a.max_iter) {
    float x2 = __fmul_rn(x, x);
    float y2 = __fmul_rn(y, y);
    if (__fadd_rn(x2, y2) > 4.0f) break;
    float xy = __fmul_rn(x, y);
    y = __fadd_rn(__fadd_rn(xy, xy), cy);
    x = __fadd_rn(__fsub_rn(x2, y2), cx);
    ++it;
  }
  a.count[p] = it;
}

// ------------------------------------------------------------------ bitonic sort
// Keys n = 2^L in tiles of 2^P keys (P = min(L, 12)); merge size k = 2^lv,
// compare distance j = 2^jl; a compare-exchange (i, i+j) orders ascending iff
// (i & k) == 0 (the standard bitonic network on global indices). Stages:
//   0                 : sort every tile in shared memory (lv = 1..P), in -> out
//   for lv = P+1 .. L : the distances above the tile, jl = lv-1 .. P, in passes
//                       of up to 10 levels: a block gathers the 4096 keys whose
//                       indices differ only in those m distance bits and in
//                       the 12 - m lowest bits (runs of at least 4 contiguous
//                       keys), runs the m levels in shared memory and writes
//                       them back; then one pass for jl = P-1 .. 0 on
//                       contiguous 4096-key tiles.
// Every stage has 2^(L-P) blocks of 4096 (or 2^L) keys.

struct BitonicStep {
  uint32_t kind;   // 0 tile sort, 1 pass over distances above the tile, 2 tile merge
  uint32_t lv;     // log2 k
  uint32_t jhi;    // kind 1: highest level
  uint32_t jlo;    // kind 1: lowest level
};

__host__ __device__ inline BitonicStep bitonic_step(uint32_t L, uint32_t s) {
  const uint32_t P = bitonic_tile_log2(L);
  if (s == 0) return BitonicStep{0, P, 0, 0};
  s -= 1;
  for (uint32_t lv = P + 1; lv <= L; ++lv) {
    const uint32_t d = lv - P, npass = (d + kBitonicHigh - 1) / kBitonicHigh;
    if (s < npass) {
      const uint32_t jhi = lv - 1 - kBitonicHigh * s;
      const uint32_t jlo = jhi + 1 >= P + kBitonicHigh ? jhi + 1 - kBitonicHigh : P;
      return BitonicStep{1, lv, jhi, jlo};
    }
    s -= npass;
    if (s == 0) return BitonicStep{2, lv, 0, 0};
    s -= 1;
  }
  return BitonicStep{3, 0, 0, 0};  // out of range (never produced for s < nstages)
}

__device__ __forceinline__ void cmpx(uint32_t& x, uint32_t& y, bool asc) {
  uint32_t lo = min(x, y), hi = max(x, y);
  x = asc ? lo : hi;
  y = asc ? hi : lo;
}

// shared-memory tile index with one padding word per 32 (power-of-two strides
// then fall into different banks)
__device__ __forceinline__ uint32_t tpad(uint32_t i) { return i + (i >> 5); }

// Shared-memory tile network: merge sizes 2^lv_lo .. 2^lv_hi, distances from
// min(k/2, jcap) down to 1, two distances per barrier where possible.
__device__ __forceinline__ void bitonic_tile(uint32_t* t, uint32_t tile_n, uint64_t gbase, uint32_t lv_lo,
                                             uint32_t lv_hi, uint32_t jcap) {
  for (uint32_t lv = lv_lo; lv <= lv_hi; ++lv) {
    const uint64_t k = 1ull << lv;
    uint32_t jl = lv - 1;
    if ((1u << jl) > jcap) jl = 31 - __clz(jcap);
    for (int32_t j = (int32_t)jl; j >= 0;) {
      if (j >= 1) {
        // distances 2^j and 2^(j-1) together on groups {i, i+h, i+2h, i+3h}
        const uint32_t hl = (uint32_t)j - 1, h = 1u << hl;
        for (uint32_t q = threadIdx.x; q < (tile_n >> 2); q += 256) {
          const uint32_t i = ((q >> hl) << (hl + 2)) | (q & (h - 1));
          const bool asc = ((gbase + i) & k) == 0;
          uint32_t a0 = t[tpad(i)], a1 = t[tpad(i + h)], a2 = t[tpad(i + 2 * h)], a3 = t[tpad(i + 3 * h)];
          cmpx(a0, a2, asc);
          cmpx(a1, a3, asc);
          cmpx(a0, a1, asc);
          cmpx(a2, a3, asc);
          t[tpad(i)] = a0;
          t[tpad(i + h)] = a1;
          t[tpad(i + 2 * h)] = a2;
          t[tpad(i + 3 * h)] = a3;
        }
        j -= 2;
      } else {
        for (uint32_t q = threadIdx.x; q < (tile_n >> 1); q += 256) {
          const uint32_t i = 2 * q;
          const bool asc = ((gbase + i) & k) == 0;
          uint32_t x = t[tpad(i)], y = t[tpad(i + 1)];
          cmpx(x, y, asc);
          t[tpad(i)] = x;
          t[tpad(i + 1)] = y;
        }
        j = -1;
      }
      __syncthreads();
    }
  }
}

// Register passes over a 4096-key tile: each of the 256 threads holds 16 keys
// whose tile positions follow one of three patterns; bit b of the register
// index r then corresponds to a compare distance, so four consecutive levels
// of the network run in registers between shared-memory exchanges:
//   pattern 0: i = t + 256 r                       distances 2048, 1024, 512, 256
//   pattern 1: i = t%16 + 16 r + thread bits 4, 5, 6, 7 as tile bits 9, 8, 10, 11
//                                                   distances 128, 64, 32, 16
//   pattern 2: i = 16 t + r                        distances 8, 4, 2, 1
// In pattern 1 a warp's two halves are 512 words apart, 16 banks once the
// tile is padded by one word per 32 (tpad): every exchange is free of bank
// conflicts (with thread bit 4 as tile bit 8 the halves were 8 banks apart,
// two-way conflicts on a third of the shared-memory traffic).
template <int PAT>
__device__ __forceinline__ uint32_t bt_elem(uint32_t t, uint32_t r) {
  if (PAT == 0) return t + 256u * r;
  if (PAT == 1) return (t & 15u) + 16u * r + (((t >> 4) & 1u) << 9) + (((t >> 5) & 1u) << 8) + ((t >> 6) << 10);
  return 16u * t + r;
}

template <int PAT>
__device__ __forceinline__ void bt_load(uint32_t (&v)[16], const uint32_t* t) {
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = t[tpad(bt_elem<PAT>(threadIdx.x, r))];
}
template <int PAT>
__device__ __forceinline__ void bt_store(const uint32_t (&v)[16], uint32_t* t) {
#pragma unroll
  for (int r = 0; r < 16; ++r) t[tpad(bt_elem<PAT>(threadIdx.x, r))] = v[r];
}

// Levels with register-index bits bhi..blo (descending) at merge size k;
// direction from the global index of each pair. The tile index of a pattern is
// a bit field of (thread bits, register bits), so bit log2(k) of the global
// index is either a register bit (known per r at compile time) or the same for
// all of the thread's keys.
template <int PAT>
__device__ __forceinline__ void bt_levels(uint32_t (&v)[16], int bhi, int blo, uint32_t k, uint32_t gbase) {
  constexpr uint32_t r_lo = PAT == 0 ? 8u : (PAT == 1 ? 4u : 0u);  // lowest tile bit taken from r
  const uint32_t lk = 31u - __clz(k);
  const uint32_t rmask = (lk >= r_lo && lk < r_lo + 4u) ? 1u << (lk - r_lo) : 0u;
  const bool tasc = ((gbase + bt_elem<PAT>(threadIdx.x, 0)) & k) == 0;
#pragma unroll
  for (int b = 3; b >= 0; --b) {
    if (b > bhi || b < blo) continue;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r & (1 << b)) continue;
      const bool asc = rmask ? ((uint32_t)r & rmask) == 0 : tasc;
      cmpx(v[r], v[r | (1 << b)], asc);
    }
  }
}

// Same with one direction for the whole tile (merge sizes above the tile).
template <bool ASC>
__device__ __forceinline__ void bt_levels_dir(uint32_t (&v)[16]) {
#pragma unroll
  for (int b = 3; b >= 0; --b)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r & (1 << b)) continue;
      uint32_t lo = min(v[r], v[r | (1 << b)]), hi = max(v[r], v[r | (1 << b)]);
      v[r] = ASC ? lo : hi;
      v[r | (1 << b)] = ASC ? hi : lo;
    }
}

// Tile merge for k > 4096: all 12 distances 2048 .. 1, direction uniform.
__device__ __forceinline__ void bitonic_tile_merge_regs(uint32_t* out, uint32_t* t, uint32_t gbase, uint32_t k) {
  const bool asc = (gbase & k) == 0;
  uint32_t v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldcg(out + gbase + bt_elem<0>(threadIdx.x, r));
  if (asc) bt_levels_dir<true>(v); else bt_levels_dir<false>(v);
  bt_store<0>(v, t);
  __syncthreads();
  bt_load<1>(v, t);
  if (asc) bt_levels_dir<true>(v); else bt_levels_dir<false>(v);
  bt_store<1>(v, t);
  __syncthreads();
  bt_load<2>(v, t);
  if (asc) bt_levels_dir<true>(v); else bt_levels_dir<false>(v);
  uint4* o = reinterpret_cast<uint4*>(out + gbase + 16u * threadIdx.x);
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// The same levels restricted to register bits >= blo (the others are not
// distances of this pass).
template <bool ASC>
__device__ __forceinline__ void bt_levels_dir_from(uint32_t (&v)[16], int blo) {
#pragma unroll
  for (int b = 3; b >= 0; --b) {
    if (b < blo) continue;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r & (1 << b)) continue;
      uint32_t lo = min(v[r], v[r | (1 << b)]), hi = max(v[r], v[r | (1 << b)]);
      v[r] = ASC ? lo : hi;
      v[r | (1 << b)] = ASC ? hi : lo;
    }
  }
}

// Distances 2^jhi .. 2^jlo (all >= 4096, m = jhi - jlo + 1 <= 10 of them) at
// merge size 2^lv for block vb. Tile position i of the block's 4096 keys has
// bits [0, 12 - m) = the low bits of the global index (a contiguous run of
// 2^(12-m) >= 4 keys) and bits [12 - m, 12) = the distance bits jlo .. jhi;
// the block number supplies the global bits between 12 - m and jlo and those
// above jhi. Bit lv is above jhi, so the direction is the same for the whole
// block. The three register patterns of the tile merge carry tile bits 11..8,
// 7..4 and 3..0; levels whose tile bit is below 12 - m are skipped.
__device__ __forceinline__ void bitonic_high_pass(uint32_t* out, uint32_t* t, uint32_t vb, uint32_t lv, uint32_t jhi,
                                                  uint32_t jlo) {
  const uint32_t m = jhi - jlo + 1, lowb = 12u - m, ab = jlo - lowb;
  const uint32_t A = vb & ((1u << ab) - 1u), B = vb >> ab;
  const uint32_t hi = (jhi + 1u < 32u) ? (B << (jhi + 1u)) : 0u;
  const uint32_t fixed = hi | (A << lowb);
  const uint32_t lowmask = (1u << lowb) - 1u;
  auto gidx = [&](uint32_t i) { return fixed | ((i >> lowb) << jlo) | (i & lowmask); };
  const bool asc = ((fixed >> lv) & 1u) == 0u;
  uint32_t v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldcg(out + gidx(bt_elem<0>(threadIdx.x, r)));
  const int b0 = (int)lowb - 8, b1 = (int)lowb - 4, b2 = (int)lowb;  // lowest register bit in use per pattern
  if (asc) bt_levels_dir_from<true>(v, b0); else bt_levels_dir_from<false>(v, b0);
  bt_store<0>(v, t);
  __syncthreads();
  bt_load<1>(v, t);
  if (asc) bt_levels_dir_from<true>(v, b1); else bt_levels_dir_from<false>(v, b1);
  bt_store<1>(v, t);
  __syncthreads();
  bt_load<2>(v, t);
  if (asc) bt_levels_dir_from<true>(v, b2); else bt_levels_dir_from<false>(v, b2);
  // positions 16t .. 16t + 15: groups of 4 are contiguous (runs of >= 4 keys)
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(out + gidx(16u * threadIdx.x + 4u * q)) =
        make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Full sort of a 4096-key tile (merge sizes 2 .. 4096), keys read from `in`.
__device__ __forceinline__ void bitonic_tile_sort_regs(const uint32_t* in, uint32_t* out, uint32_t* t,
                                                       uint32_t gbase) {
  uint32_t v[16];
  const uint4* src = reinterpret_cast<const uint4*>(in + gbase + 16u * threadIdx.x);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 w = __ldcs(src + q);
    v[4 * q] = w.x;
    v[4 * q + 1] = w.y;
    v[4 * q + 2] = w.z;
    v[4 * q + 3] = w.w;
  }
  // k = 2, 4, 8, 16 inside the thread's 16 consecutive keys
#pragma unroll
  for (int lv = 1; lv <= 4; ++lv) bt_levels<2>(v, lv - 1, 0, 1u << lv, gbase);
  int pat = 2;  // pattern the registers currently follow
  for (uint32_t lv = 5; lv <= 12; ++lv) {
    const uint32_t k = 1u << lv;
    if (lv >= 9) {  // distances 2^(lv-1) .. 256
      bt_store<2>(v, t);
      __syncthreads();
      bt_load<0>(v, t);
      bt_levels<0>(v, (int)lv - 9, 0, k, gbase);
      pat = 0;
    }
    // distances min(2^(lv-1), 128) .. 16
    if (pat == 0) bt_store<0>(v, t); else bt_store<2>(v, t);
    __syncthreads();
    bt_load<1>(v, t);
    bt_levels<1>(v, (int)(lv >= 9 ? 3 : lv - 5), 0, k, gbase);
    bt_store<1>(v, t);
    __syncthreads();
    bt_load<2>(v, t);
    bt_levels<2>(v, 3, 0, k, gbase);
    pat = 2;
    __syncthreads();  // the next exchange overwrites the tile
  }
  uint4* o = reinterpret_cast<uint4*>(out + gbase + 16u * threadIdx.x);
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void bitonic_block(const kl_args_bitonic& a, uint32_t stage, uint32_t vb,
                                              char* smem) {
  const uint32_t L = a.log2n;
  const uint32_t P = bitonic_tile_log2(L);
  const uint32_t tile_n = 1u << P;
  const BitonicStep st = bitonic_step(L, stage);
  uint32_t* t = reinterpret_cast<uint32_t*>(smem);
  if (st.kind == 1) {  // only when L > 12: the tile has 4096 keys
    bitonic_high_pass(a.out, t, vb, st.lv, st.jhi, st.jlo);
    return;
  }
  const uint32_t gbase = vb * tile_n;
  if (tile_n == 4096u) {
    if (st.kind == 0)
      bitonic_tile_sort_regs(a.in, a.out, t, gbase);
    else
      bitonic_tile_merge_regs(a.out, t, gbase, 1u << st.lv);
    return;
  }
  // small sorts (fewer than 4096 keys): one block, shared-memory network
  const uint32_t* src = st.kind == 0 ? a.in : a.out;
  for (uint32_t q = threadIdx.x; q < tile_n; q += 256) t[tpad(q)] = __ldcg(src + gbase + q);
  __syncthreads();
  if (st.kind == 0)
    bitonic_tile(t, tile_n, gbase, 1, P, tile_n);
  else
    bitonic_tile(t, tile_n, gbase, st.lv, st.lv, tile_n >> 1);
  for (uint32_t q = threadIdx.x; q < tile_n; q += 256) a.out[gbase + q] = t[tpad(q)];
}

// ------------------------------------------------------------------ MatrixAdd
// Section 4.1 example: n x n add, blocks of 16x16 threads; virtual block vb is
// (bx, by) = (vb mod n/16, vb div n/16).

__device__ __forceinline__ void matadd_block(const kl_args_matadd& a, uint32_t vb) {
  const uint32_t gx = a.n / 16;
  const uint32_t bx = vb % gx, by = vb / gx;
  const uint32_t tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const uint64_t i = (uint64_t)(by * 16 + ty) * a.n + bx * 16 + tx;
  a.c[i] = __fadd_rn(a.a[i], a.b[i]);
}

// ------------------------------------------------------------------ TEA
// Tiny Encryption Algorithm (Wheeler and Needham, 1994): 32 cycles of the
// Feistel round on the 64-bit block (v0, v1) with the 128-bit key; integer
// arithmetic modulo 2^32. Two blocks per thread from one 16-byte load.

__device__ __forceinline__ void tea_encrypt(uint32_t& v0, uint32_t& v1, const uint32_t (&k)[4]) {
  uint32_t sum = 0u;
#pragma unroll 8
  for (int r = 0; r < 32; ++r) {
    sum += 0x9E3779B9u;  // the cipher's key-schedule constant
    v0 += ((v1 << 4) + k[0]) ^ (v1 + sum) ^ ((v1 >> 5) + k[1]);
    v1 += ((v0 << 4) + k[2]) ^ (v0 + sum) ^ ((v0 >> 5) + k[3]);
  }
}

__device__ __forceinline__ void tea_block(const kl_args_tea& a, uint32_t vb) {
  const uint32_t k[4] = {a.key[0], a.key[1], a.key[2], a.key[3]};
  const uint64_t j = (uint64_t)vb * kTeaPerBlock + 2u * threadIdx.x;  // first of this thread's two blocks
  if (j + 1 < a.n) {
    uint4 w = reinterpret_cast<const uint4*>(a.in)[j >> 1];
    tea_encrypt(w.x, w.y, k);
    tea_encrypt(w.z, w.w, k);
    reinterpret_cast<uint4*>(a.out)[j >> 1] = w;
  } else if (j < a.n) {
    uint32_t v0 = a.in[2 * j], v1 = a.in[2 * j + 1];
    tea_encrypt(v0, v1, k);
    a.out[2 * j] = v0;
    a.out[2 * j + 1] = v1;
  }
}

// ------------------------------------------------------------------ SAD
// Sums of absolute differences for motion estimation: thread o computes the
// SAD of 4x4 block b = o / D^2 of the current frame against the reference
// frame displaced by (dx, dy) = (o mod D - R, (o / D) mod D - R), D = 2R + 1,
// reference coordinates clamped to the frame.

__device__ __forceinline__ void sad_block(const kl_args_sad& a, uint32_t vb) {
  const uint32_t D = 2u * a.range + 1u, D2 = D * D;
  const uint32_t mbw = a.width / 4u;
  const uint64_t o = (uint64_t)vb * kSadPerBlock + threadIdx.x;
  const uint64_t nout = (uint64_t)mbw * (a.height / 4u) * D2;
  if (o >= nout) return;
  const uint32_t b = (uint32_t)(o / D2), d = (uint32_t)(o % D2);
  const int dy = (int)(d / D) - (int)a.range, dx = (int)(d % D) - (int)a.range;
  const int x0 = (int)(4u * (b % mbw)), y0 = (int)(4u * (b / mbw));
  const int W = (int)a.width, H = (int)a.height;
  uint32_t acc = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ry = min(max(y0 + i + dy, 0), H - 1);
    const uint8_t* crow = a.cur + (size_t)(y0 + i) * W + x0;
    const uint8_t* rrow = a.ref + (size_t)ry * W;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rx = min(max(x0 + j + dx, 0), W - 1);
      const int c = __ldg(crow + j), r = __ldg(rrow + rx);
      acc += (uint32_t)abs(c - r);
    }
  }
  a.sad[o] = acc;
}

// ------------------------------------------------------------------ 3-D stencil
// 7-point stencil: an interior point becomes c0 * c + c1 * s with s the sum of
// its six face neighbours added in the order -x, +x, -y, +y, -z, +z (each sum
// rounded, then one fused multiply-add); boundary points are copied.

__device__ __forceinline__ void stencil_block(const kl_args_stencil& a, uint32_t vb) {
  // block vb: the 256 consecutive points [256 vb, 256 vb + 256) of the
  // x-fastest grid, so every thread has a point whatever nx is (the host keeps
  // nx * ny * nz below 2^32)
  const uint32_t i = vb * (uint32_t)kStencilPerBlock + threadIdx.x;
  if (i >= a.nx * a.ny * a.nz) return;
  const uint32_t x = i % a.nx, r = i / a.nx;
  const uint32_t y = r % a.ny, z = r / a.ny;
  const uint32_t sx = 1, sy = a.nx, sz = a.nx * a.ny;
  const float c = __ldg(a.in + i);
  if (x == 0 || y == 0 || z == 0 || x + 1 == a.nx || y + 1 == a.ny || z + 1 == a.nz) {
    a.out[i] = c;
    return;
  }
  float s = __fadd_rn(__ldg(a.in + i - sx), __ldg(a.in + i + sx));
  s = __fadd_rn(s, __ldg(a.in + i - sy));
  s = __fadd_rn(s, __ldg(a.in + i + sy));
  s = __fadd_rn(s, __ldg(a.in + i - sz));
  s = __fadd_rn(s, __ldg(a.in + i + sz));
  a.out[i] = __fmaf_rn(a.c1, s, __fmul_rn(a.c0, c));
}

// ------------------------------------------------------------------ MRI-Q
// Q of an MRI reconstruction: stage 0 phiMag[k] = phiR^2 + phiI^2 (one fused
// multiply-add on the rounded square of phiR); stage 1 for every image point
// x: Qr = sum_k phiMag[k] cos(2 pi (k . x)), Qi = sum_k phiMag[k] sin(...),
// k ascending, each term one fused multiply-add. The dot product is
// kx*x, then fused ky*y and kz*z; the angle is its rounded product with the
// binary32 nearest to 2 pi. Sine and cosine: Cody-Waite reduction by pi/2 with
// a two-part constant, then Taylor polynomials (degree 9 for sine, 8 for
// cosine) on [-pi/4, pi/4] in Horner form with fused multiply-adds, and the
// quadrant's sign and swap.

__device__ __forceinline__ void kl_sincosf(float a, float& sn, float& cs) {
  const float n = rintf(__fmul_rn(a, 0.636619772f));  // a * 2/pi, nearest integer
  float r = __fmaf_rn(-n, 1.57079637f, a);            // pi/2 split: 1.57079637f + (-4.37113900e-8f)
  r = __fmaf_rn(-n, -4.37113900e-8f, r);
  const float r2 = __fmul_rn(r, r);
  float ps = __fmaf_rn(r2, 2.75573192e-6f, -1.98412698e-4f);   // 1/9!, -1/7!
  ps = __fmaf_rn(r2, ps, 8.33333333e-3f);                        // 1/5!
  ps = __fmaf_rn(r2, ps, -1.66666667e-1f);                       // -1/3!
  const float s = __fmaf_rn(__fmul_rn(r, r2), ps, r);
  float pc = __fmaf_rn(r2, 2.48015873e-5f, -1.38888889e-3f);     // 1/8!, -1/6!
  pc = __fmaf_rn(r2, pc, 4.16666667e-2f);                        // 1/4!
  pc = __fmaf_rn(r2, pc, -0.5f);                                 // -1/2!
  const float c = __fmaf_rn(r2, pc, 1.0f);
  const int q = ((int)n) & 3;
  sn = q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
  cs = q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}

__device__ __forceinline__ void mriq_block(const kl_args_mriq& a, uint32_t stage, uint32_t vb, char* smem) {
  if (stage == 0) {
    const uint32_t k = vb * kMriqPerBlock + threadIdx.x;
    if (k < a.numK) {
      const float r = __ldg(a.phiR + k), im = __ldg(a.phiI + k);
      a.phiMag[k] = __fmaf_rn(im, im, __fmul_rn(r, r));
    }
    return;
  }
  float* s_kx = reinterpret_cast<float*>(smem);
  float* s_ky = s_kx + kMriqPerBlock;
  float* s_kz = s_ky + kMriqPerBlock;
  float* s_pm = s_kz + kMriqPerBlock;
  const uint32_t xi = vb * kMriqPerBlock + threadIdx.x;
  const bool live = xi < a.numX;
  const float px = live ? __ldg(a.x + xi) : 0.f, py = live ? __ldg(a.y + xi) : 0.f, pz = live ? __ldg(a.z + xi) : 0.f;
  float qr = 0.f, qi = 0.f;
  for (uint32_t k0 = 0; k0 < a.numK; k0 += kMriqPerBlock) {
    const uint32_t k = k0 + threadIdx.x;
    __syncthreads();
    if (k < a.numK) {
      s_kx[threadIdx.x] = __ldg(a.kx + k);
      s_ky[threadIdx.x] = __ldg(a.ky + k);
      s_kz[threadIdx.x] = __ldg(a.kz + k);
      s_pm[threadIdx.x] = a.phiMag[k];  // written by stage 0 of this kernel: not through the read-only path
    }
    __syncthreads();
    const uint32_t kn = min((uint32_t)kMriqPerBlock, a.numK - k0);
    for (uint32_t j = 0; j < kn; ++j) {
      float t = __fmul_rn(s_kx[j], px);
      t = __fmaf_rn(s_ky[j], py, t);
      t = __fmaf_rn(s_kz[j], pz, t);
      float sn, cs;
      kl_sincosf(__fmul_rn(6.28318548f, t), sn, cs);
      qr = __fmaf_rn(s_pm[j], cs, qr);
      qi = __fmaf_rn(s_pm[j], sn, qi);
    }
  }
  if (live) {
    a.Qr[xi] = qr;
    a.Qi[xi] = qi;
  }
}

// ------------------------------------------------------------------ BF16 GEMM on tensor cores
// C[M][N] = sum_k A[m][k] * Bt[n][k], A and Bt bfloat16 (both K-major), FP32
// accumulation in tensor memory. Per block (one 128x64 tile of C): thread 0
// issues the TMA loads of 128x64 (A) and 64x64 (Bt) K-slices into a two-stage
// ring of 128-byte-swizzled shared memory and the tcgen05.mma instructions
// (M=128, N=64, K=16 each, four per K-slice); tcgen05.commit signals an
// mbarrier when a stage's MMAs have read their operands, which frees the stage
// for the next TMA load. After the last K-slice all eight warps read the
// accumulator with tcgen05.ld (warp w: lanes 32(w mod 4).., columns 32(w/4)..)
// and store their rows of C. Rows and columns outside C are zero-filled by
// the TMA unit and not stored. The caller allocates the TMEM columns when the
// CTA starts (acquire_tmem, BlockCtx::tmem) and frees them at its end. Every
// mbarrier wait is bounded by BlockCtx::limit_ns; a wait that runs out
// records KL_EDEVICE_TIMEOUT in *BlockCtx::err and the block stores nothing.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long tn_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// false when the phase did not complete within limit_ns
static __device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = tn_gtimer();
  while (!mbar_try_wait(bar, parity))
    if (tn_gtimer() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand whose 128-byte rows follow
// the 128-byte swizzle, groups of 8 rows 1024 bytes apart (stride offset);
// the leading offset is unused in this layout; version 1; swizzle mode 2.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// bfloat16 (bits 7-9 = 1, 10-12 = 1), both K-major, N/8 at bit 17, M/16 at 24.
constexpr uint32_t kBfIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBfBN >> 3) << 17) |
                              ((uint32_t)(kBfBM >> 4) << 24);
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(kBfIdesc), "r"(accum)
      : "memory");
}
// the same with the instruction descriptor given (other tile widths)
__device__ __forceinline__ void umma_bf16_id(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 lanes; one lane = one row
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 lanes; one lane = one row
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float4 (&v)[4]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 4; ++q)
    v[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                       __uint_as_float(r[4 * q + 3]));
}

static __device__ void gemm_bf16_block(const kl_args_gemm_bf16& a, uint32_t vb, char* smem, const BlockCtx& cx) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tiles_n = cdiv64(a.N, kBfBN);
  const uint32_t m0 = (vb / tiles_n) * kBfBM, n0 = (vb % tiles_n) * kBfBN;
  const uint32_t kt = cdiv64(a.K, kBfBK);
  const uint32_t base = (smem_u32(smem) + 1023u) & ~1023u;  // swizzled tiles need 1024-byte alignment
  const uint32_t full0 = base + 2u * kBfStage;               // TMA -> MMA, per stage
  const uint32_t freed0 = full0 + 16u;                       // MMA done reading, per stage
  const uint32_t accb = full0 + 32u;                         // all MMAs of the tile done
  volatile uint32_t* flag = reinterpret_cast<volatile uint32_t*>(smem + (full0 + 40u - smem_u32(smem)));
  const uint32_t tmem = *cx.tmem;  // allocated by acquire_tmem when the CTA started
  if (tid == 0) {
    mbar_init(full0, 1u);
    mbar_init(full0 + 8u, 1u);
    mbar_init(freed0, 1u);
    mbar_init(freed0 + 8u, 1u);
    mbar_init(accb, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // earlier blocks wrote this shared memory through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t ok = 1u;
    const char* tmA = static_cast<const char*>(a.tmaps);
    const char* tmB = tmA + 128;
    for (uint32_t s = 0; s < 2u && s < kt; ++s) {
      mbar_expect_tx(full0 + 8u * s, kBfStage);
      tma_load_2d(base + s * kBfStage, tmA, (int32_t)(s * kBfBK), (int32_t)m0, full0 + 8u * s);
      tma_load_2d(base + s * kBfStage + kBfStageA, tmB, (int32_t)(s * kBfBK), (int32_t)n0, full0 + 8u * s);
    }
    for (uint32_t i = 0; i < kt; ++i) {
      const uint32_t s = i & 1u, ph = (i >> 1) & 1u;
      if (!mbar_wait(full0 + 8u * s, ph, cx.limit_ns)) {
        ok = 0u;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base + s * kBfStage, sb = sa + kBfStageA;
#pragma unroll
      for (uint32_t k = 0; k < (uint32_t)kBfBK / 16u; ++k)
        umma_bf16(tmem, umma_desc_sw128(sa + 32u * k), umma_desc_sw128(sb + 32u * k), (i | k) != 0u);
      umma_commit(freed0 + 8u * s);
      if (i + 2u < kt) {
        if (!mbar_wait(freed0 + 8u * s, ph, cx.limit_ns)) {
          ok = 0u;
          break;
        }
        mbar_expect_tx(full0 + 8u * s, kBfStage);
        tma_load_2d(sa, tmA, (int32_t)((i + 2u) * kBfBK), (int32_t)m0, full0 + 8u * s);
        tma_load_2d(sb, tmB, (int32_t)((i + 2u) * kBfBK), (int32_t)n0, full0 + 8u * s);
      }
    }
    if (ok) umma_commit(accb);  // arrives once every MMA issued above has completed
    // the stage-free signals of the last two K-slices were never waited for:
    // collect them so no arrival lands after the barriers are invalidated
    for (uint32_t i = kt > 2u ? kt - 2u : 0u; ok && i < kt; ++i)
      if (!mbar_wait(freed0 + 8u * (i & 1u), (i >> 1) & 1u, cx.limit_ns)) ok = 0u;
    *flag = ok;
  }
  __syncthreads();
  bool ok = *flag != 0u;
  if (ok) ok = mbar_wait(accb, 0u, cx.limit_ns);
  tc_fence_after();
  if (ok) {
    const uint32_t q = (uint32_t)warp & 3u, h = (uint32_t)warp >> 2;
    const uint32_t row = m0 + 32u * q + (uint32_t)lane;
    const uint32_t c0 = n0 + 32u * h;
#pragma unroll
    for (uint32_t half = 0; half < 2u; ++half) {
      float4 v[4];
      tmem_ld16(tmem + ((32u * q) << 16) + 32u * h + 16u * half, v);
      if (row < a.M) {
        float4* dst = reinterpret_cast<float4*>(a.C + (uint64_t)row * a.N + c0 + 16u * half);
#pragma unroll
        for (uint32_t j = 0; j < 4u; ++j)
          if (c0 + 16u * half + 4u * j < a.N) dst[j] = v[j];
      }
    }
  } else if (lane == 0) {
    atomicCAS(cx.err, 0, (int)KL_EDEVICE_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    mbar_inval(full0);
    mbar_inval(full0 + 8u);
    mbar_inval(freed0);
    mbar_inval(freed0 + 8u);
    mbar_inval(accb);
  }
  __syncthreads();
}

// CTA start (all threads): allocate the accumulator's TMEM columns, then give
// up the allocation permit at once. The hardware keeps further CTAs of a
// TMEM-allocating kernel off an SM while a resident CTA still holds its
// permit (measured on GB300: one CTA per SM at a time without the relinquish,
// four with it); at most four CTAs x 64 columns of the SM's 512 are ever
// allocated, so the allocation never waits.
__device__ __forceinline__ void acquire_tmem(const BlockCtx& cx) {
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(smem_u32(cx.tmem), kBfTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// CTA exit (all threads): free the columns acquire_tmem allocated.
__device__ __forceinline__ void release_tmem(const BlockCtx& cx) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(*cx.tmem, kBfTmemCols);
}

// ------------------------------------------------------------------ dispatch
// Runs cumulative block g (of stage st) of a tenant. All 256 threads call it.

template <class A>
__device__ __forceinline__ A load_args(const void* p) {
  return *reinterpret_cast<const A*>(p);
}

// BUILD: which co-scheduler build (kBuildPlain, kBuildFull, kBuildLight) the
// caller is; a type outside it compiles to nothing. Any tcgen05 instruction in
// a kernel makes the CUDA occupancy calculator allow one CTA per SM, and every
// extra body adds register pressure to the shared budget, so only the full
// build carries the tensor-core tenant and the types after it.
template <int BUILD>
__device__ __forceinline__ void run_block(uint32_t type, const void* args, const Stage& st, uint32_t g,
                                          char* smem, const BlockCtx& cx) {
  const uint32_t vb = g - st.begin;
  switch (type) {
    case KL_T_GATHER:
      if constexpr (in_build(BUILD, KL_T_GATHER)) gather_block(load_args<kl_args_gather>(args), vb);
      break;
    case KL_T_BLACKSCHOLES:
      if constexpr (in_build(BUILD, KL_T_BLACKSCHOLES))
        blackscholes_block(load_args<kl_args_blackscholes>(args), vb);
      break;
    case KL_T_GEMM_F32:
      if constexpr (in_build(BUILD, KL_T_GEMM_F32)) gemm_f32_block(load_args<kl_args_gemm_f32>(args), vb, smem);
      break;
    case KL_T_SPMV_CSR:
      if constexpr (in_build(BUILD, KL_T_SPMV_CSR)) spmv_csr_block(load_args<kl_args_spmv_csr>(args), vb, smem);
      break;
    case KL_T_PCHASE:
      if constexpr (in_build(BUILD, KL_T_PCHASE)) pchase_block(load_args<kl_args_pchase>(args), vb);
      break;
    case KL_T_TRIAD:
      if constexpr (in_build(BUILD, KL_T_TRIAD)) triad_block(load_args<kl_args_triad>(args), vb);
      break;
    case KL_T_HIST256:
      if constexpr (in_build(BUILD, KL_T_HIST256)) hist256_block(load_args<kl_args_hist256>(args), st.s, vb, smem);
      break;
    case KL_T_ESCAPE:
      if constexpr (in_build(BUILD, KL_T_ESCAPE)) escape_block(load_args<kl_args_escape>(args), vb);
      break;
    case KL_T_BITONIC:
      if constexpr (in_build(BUILD, KL_T_BITONIC)) bitonic_block(load_args<kl_args_bitonic>(args), st.s, vb, smem);
      break;
    case KL_T_MATADD:
      if constexpr (in_build(BUILD, KL_T_MATADD)) matadd_block(load_args<kl_args_matadd>(args), vb);
      break;
    case KL_T_GEMM_BF16:
      if constexpr (in_build(BUILD, KL_T_GEMM_BF16)) gemm_bf16_block(load_args<kl_args_gemm_bf16>(args), vb, smem, cx);
      break;
    case KL_T_TEA:
      if constexpr (in_build(BUILD, KL_T_TEA)) tea_block(load_args<kl_args_tea>(args), vb);
      break;
    case KL_T_SAD:
      if constexpr (in_build(BUILD, KL_T_SAD)) sad_block(load_args<kl_args_sad>(args), vb);
      break;
    case KL_T_STENCIL:
      if constexpr (in_build(BUILD, KL_T_STENCIL)) stencil_block(load_args<kl_args_stencil>(args), vb);
      break;
    case KL_T_MRIQ:
      if constexpr (in_build(BUILD, KL_T_MRIQ)) mriq_block(load_args<kl_args_mriq>(args), st.s, vb, smem);
      break;
    case KL_T_TESTMIX:
      if constexpr (in_build(BUILD, KL_T_TESTMIX)) testmix_block(load_args<kl_args_testmix>(args), vb);
      break;
    default: break;
  }
}

// Runs cumulative blocks [g, ge) of one stage st of a tenant (a slice, or the
// part of it inside one stage) in a co-scheduler CTA, with the type dispatched
// once per slice. `args` is the CTA's shared-memory copy of the descriptor's
// arguments, made once per slice: a block of the short tenants (the stencil's
// 256 points) is a few hundred instructions, and a dependent global load of
// its arguments ahead of every block was a large share of it. Bodies that use
// shared memory or synchronise inside (BARRIER) keep a CTA barrier between
// blocks; in the others every thread is independent of the rest, so each warp
// goes on to the next block as soon as it is done with this one. All threads
// have finished the slice when run_slice returns.
template <class A, bool BARRIER, class Body>
__device__ __forceinline__ void slice_loop(const void* args, uint32_t v0, uint32_t v1, Body&& body) {
  for (uint32_t vb = v0; vb < v1; ++vb) {
    body(load_args<A>(args), vb);
    if constexpr (BARRIER) {
      if (vb + 1u < v1) __syncthreads();  // shared memory is reused by the next block
    }
  }
}

template <int BUILD>
__device__ __forceinline__ void run_slice(uint32_t type, const void* args, const Stage& st, uint32_t g, uint32_t ge,
                                          char* smem, const BlockCtx& cx) {
  const uint32_t v0 = g - st.begin, v1 = ge - st.begin;
  const uint32_t s = st.s;
  switch (type) {
    case KL_T_GATHER:
      if constexpr (in_build(BUILD, KL_T_GATHER))
        slice_loop<kl_args_gather, false>(args, v0, v1, [&](const kl_args_gather& a, uint32_t vb) { gather_block(a, vb); });
      break;
    case KL_T_BLACKSCHOLES:
      if constexpr (in_build(BUILD, KL_T_BLACKSCHOLES))
        slice_loop<kl_args_blackscholes, false>(
            args, v0, v1, [&](const kl_args_blackscholes& a, uint32_t vb) { blackscholes_block(a, vb); });
      break;
    case KL_T_GEMM_F32:
      if constexpr (in_build(BUILD, KL_T_GEMM_F32))
        slice_loop<kl_args_gemm_f32, true>(
            args, v0, v1, [&](const kl_args_gemm_f32& a, uint32_t vb) { gemm_f32_block(a, vb, smem); });
      break;
    case KL_T_SPMV_CSR:
      if constexpr (in_build(BUILD, KL_T_SPMV_CSR))
      {
        if constexpr (BUILD == kBuildLight) {
          // at 32 registers the body reads its arguments from the CTA's shared
          // copy where it needs them instead of holding a private copy (which
          // spills): 10% faster here, and slower for the other bodies
          for (uint32_t vb = v0; vb < v1; ++vb) {
            spmv_csr_block(*reinterpret_cast<const kl_args_spmv_csr*>(args), vb, smem);
            if (vb + 1u < v1) __syncthreads();  // shared memory is reused by the next block
          }
        } else {
          slice_loop<kl_args_spmv_csr, true>(
              args, v0, v1, [&](const kl_args_spmv_csr& a, uint32_t vb) { spmv_csr_block(a, vb, smem); });
        }
      }
      break;
    case KL_T_PCHASE:
      if constexpr (in_build(BUILD, KL_T_PCHASE))
        slice_loop<kl_args_pchase, false>(args, v0, v1, [&](const kl_args_pchase& a, uint32_t vb) { pchase_block(a, vb); });
      break;
    case KL_T_TRIAD:
      if constexpr (in_build(BUILD, KL_T_TRIAD))
        slice_loop<kl_args_triad, false>(args, v0, v1, [&](const kl_args_triad& a, uint32_t vb) { triad_block(a, vb); });
      break;
    case KL_T_HIST256:
      if constexpr (in_build(BUILD, KL_T_HIST256))
        slice_loop<kl_args_hist256, true>(
            args, v0, v1, [&](const kl_args_hist256& a, uint32_t vb) { hist256_block(a, s, vb, smem); });
      break;
    case KL_T_ESCAPE:
      if constexpr (in_build(BUILD, KL_T_ESCAPE))
        slice_loop<kl_args_escape, false>(args, v0, v1, [&](const kl_args_escape& a, uint32_t vb) { escape_block(a, vb); });
      break;
    case KL_T_BITONIC:
      if constexpr (in_build(BUILD, KL_T_BITONIC))
        slice_loop<kl_args_bitonic, true>(
            args, v0, v1, [&](const kl_args_bitonic& a, uint32_t vb) { bitonic_block(a, s, vb, smem); });
      break;
    case KL_T_MATADD:
      if constexpr (in_build(BUILD, KL_T_MATADD))
        slice_loop<kl_args_matadd, false>(args, v0, v1, [&](const kl_args_matadd& a, uint32_t vb) { matadd_block(a, vb); });
      break;
    case KL_T_GEMM_BF16:
      if constexpr (in_build(BUILD, KL_T_GEMM_BF16))
        slice_loop<kl_args_gemm_bf16, true>(
            args, v0, v1, [&](const kl_args_gemm_bf16& a, uint32_t vb) { gemm_bf16_block(a, vb, smem, cx); });
      break;
    case KL_T_TEA:
      if constexpr (in_build(BUILD, KL_T_TEA))
        slice_loop<kl_args_tea, false>(args, v0, v1, [&](const kl_args_tea& a, uint32_t vb) { tea_block(a, vb); });
      break;
    case KL_T_SAD:
      if constexpr (in_build(BUILD, KL_T_SAD))
        slice_loop<kl_args_sad, false>(args, v0, v1, [&](const kl_args_sad& a, uint32_t vb) { sad_block(a, vb); });
      break;
    case KL_T_STENCIL:
      if constexpr (in_build(BUILD, KL_T_STENCIL))
        slice_loop<kl_args_stencil, false>(args, v0, v1, [&](const kl_args_stencil& a, uint32_t vb) { stencil_block(a, vb); });
      break;
    case KL_T_MRIQ:
      if constexpr (in_build(BUILD, KL_T_MRIQ))
        slice_loop<kl_args_mriq, true>(
            args, v0, v1, [&](const kl_args_mriq& a, uint32_t vb) { mriq_block(a, s, vb, smem); });
      break;
    case KL_T_TESTMIX:
      if constexpr (in_build(BUILD, KL_T_TESTMIX))
        slice_loop<kl_args_testmix, false>(args, v0, v1,
                                           [&](const kl_args_testmix& a, uint32_t vb) { testmix_block(a, vb); });
      break;
    default: break;
  }
  __syncthreads();
}

#endif  // __CUDACC__

}  // namespace tn
}  // namespace kl
