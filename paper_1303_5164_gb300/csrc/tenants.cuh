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
constexpr int kGemmBM = 128, kGemmBN = 64, kGemmBK = 16;
constexpr int kSpmvRowsPerBlock = 32;
constexpr int kSpmvLanesPerRow = 8;
constexpr int kChasersPerBlock = 256;
constexpr int kTriadPerBlock = 4096;
constexpr int kHistBytesPerBlock = 16384;
constexpr int kEscapePerBlock = 256;
constexpr int kBitonicTileLog2 = 12;  // 4096 keys per tile

__host__ __device__ inline uint32_t bitonic_tile_log2(uint32_t L) {
  return L < (uint32_t)kBitonicTileLog2 ? L : (uint32_t)kBitonicTileLog2;
}
__host__ __device__ inline uint32_t bitonic_nstages(uint32_t L) {
  uint32_t P = bitonic_tile_log2(L), d = L - P;
  return 1 + d * (d + 1) / 2 + d;
}

// Static shape: stages, blocks per stage, dynamic shared memory.
__host__ __device__ inline uint32_t nstages(uint32_t type, const void* a) {
  switch (type) {
    case KL_T_HIST256: return 2;
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
  if (type == KL_T_HIST256) {
    if (g == 0) return Stage{0, 0, 1};
    return Stage{1, 1, 1 + stage_blocks(type, a, 1)};
  }
  if (type == KL_T_BITONIC) {
    uint32_t nb = stage_blocks(type, a, 0);
    uint32_t s = g / nb;
    return Stage{s, s * nb, (s + 1) * nb};
  }
  return Stage{0, 0, stage_blocks(type, a, 0)};
}

__host__ __device__ inline uint32_t smem_bytes(uint32_t type) {
  switch (type) {
    case KL_T_GEMM_F32: return 2u * (kGemmBM * kGemmBK + kGemmBK * kGemmBN) * 4u;  // 24 KB
    case KL_T_HIST256: return 8u * 256u * 4u;                                     // 8 KB
    case KL_T_BITONIC: return (1u << kBitonicTileLog2) * 4u;                      // 16 KB
    default: return 0;
  }
}
constexpr uint32_t kMaxTenantSmem = 2u * (kGemmBM * kGemmBK + kGemmBK * kGemmBN) * 4u;

#ifdef __CUDACC__

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

__device__ __forceinline__ void blackscholes_block(const kl_args_blackscholes& a, uint32_t vb) {
  const uint64_t i = (uint64_t)vb * kBsPerBlock + threadIdx.x;
  if (i >= a.n) return;
  float s = __ldcs(a.S + i), k = __ldcs(a.K + i), rr = __ldcs(a.r + i), vv = __ldcs(a.v + i),
        tt = __ldcs(a.T + i);
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
  __stcs(a.call + i, __fsub_rn(t1, t2));
  float u2 = __fsub_rn(1.0f, c2);
  float u1 = __fsub_rn(1.0f, c1);
  float p1 = __fmul_rn(kd, u2);
  float p2 = __fmul_rn(s, u1);
  __stcs(a.put + i, __fsub_rn(p1, p2));
}

// ------------------------------------------------------------------ FP32 GEMM
// 128x64 tile of C per block; 256 threads as 16x16, each an 8x4 micro-tile
// (rows ty*8..+7, cols tx*4..+3). K advances in 16-wide tiles staged in shared
// memory by cp.async (double buffered, zero-filled past the edges). For every
// C[i][j] the fused multiply-adds run over k = 0,1,2,... in order from +0, so
// the result is the ascending fused chain exactly (zero padding adds exact 0).

__device__ __forceinline__ void gemm_f32_block(const kl_args_gemm_f32& a, uint32_t vb, char* smem) {
  float* As = reinterpret_cast<float*>(smem);            // [2][128][16]
  float* Bs = As + 2 * kGemmBM * kGemmBK;                 // [2][16][64]
  const uint32_t tilesN = (a.N + kGemmBN - 1) / kGemmBN;
  const uint32_t m0 = (vb / tilesN) * kGemmBM;
  const uint32_t n0 = (vb % tilesN) * kGemmBN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const uint32_t ktiles = (a.K + kGemmBK - 1) / kGemmBK;

  auto load_tile = [&](uint32_t kt, int buf) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int c = tid + u * 256;
      int row = c >> 2, kc = c & 3;
      uint32_t gm = m0 + row, gk = kt * kGemmBK + kc * 4;
      bool ok = gm < a.M && gk < a.K;
      const float* src = ok ? a.A + (uint64_t)gm * a.K + gk : a.A;
      cp_async16(As + buf * kGemmBM * kGemmBK + row * kGemmBK + kc * 4, src, ok ? 16 : 0);
    }
    {
      int row = tid >> 4, nc = tid & 15;
      uint32_t gk = kt * kGemmBK + row, gn = n0 + nc * 4;
      bool ok = gk < a.K && gn < a.N;
      const float* src = ok ? a.B + (uint64_t)gk * a.N + gn : a.B;
      cp_async16(Bs + buf * kGemmBK * kGemmBN + row * kGemmBN + nc * 4, src, ok ? 16 : 0);
    }
    cp_async_commit();
  };

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  load_tile(0, 0);
  for (uint32_t kt = 0; kt < ktiles; ++kt) {
    if (kt + 1 < ktiles) {
      load_tile(kt + 1, (kt + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* Ab = As + (kt & 1) * kGemmBM * kGemmBK + ty * 8 * kGemmBK;
    const float* Bb = Bs + (kt & 1) * kGemmBK * kGemmBN + tx * 4;
#pragma unroll
    for (int k4 = 0; k4 < kGemmBK / 4; ++k4) {
      float4 b0 = *reinterpret_cast<const float4*>(Bb + (k4 * 4 + 0) * kGemmBN);
      float4 b1 = *reinterpret_cast<const float4*>(Bb + (k4 * 4 + 1) * kGemmBN);
      float4 b2 = *reinterpret_cast<const float4*>(Bb + (k4 * 4 + 2) * kGemmBN);
      float4 b3 = *reinterpret_cast<const float4*>(Bb + (k4 * 4 + 3) * kGemmBN);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float4 av = *reinterpret_cast<const float4*>(Ab + i * kGemmBK + k4 * 4);
        acc[i][0] = __fmaf_rn(av.x, b0.x, acc[i][0]);
        acc[i][1] = __fmaf_rn(av.x, b0.y, acc[i][1]);
        acc[i][2] = __fmaf_rn(av.x, b0.z, acc[i][2]);
        acc[i][3] = __fmaf_rn(av.x, b0.w, acc[i][3]);
        acc[i][0] = __fmaf_rn(av.y, b1.x, acc[i][0]);
        acc[i][1] = __fmaf_rn(av.y, b1.y, acc[i][1]);
        acc[i][2] = __fmaf_rn(av.y, b1.z, acc[i][2]);
        acc[i][3] = __fmaf_rn(av.y, b1.w, acc[i][3]);
        acc[i][0] = __fmaf_rn(av.z, b2.x, acc[i][0]);
        acc[i][1] = __fmaf_rn(av.z, b2.y, acc[i][1]);
        acc[i][2] = __fmaf_rn(av.z, b2.z, acc[i][2]);
        acc[i][3] = __fmaf_rn(av.z, b2.w, acc[i][3]);
        acc[i][0] = __fmaf_rn(av.w, b3.x, acc[i][0]);
        acc[i][1] = __fmaf_rn(av.w, b3.y, acc[i][1]);
        acc[i][2] = __fmaf_rn(av.w, b3.z, acc[i][2]);
        acc[i][3] = __fmaf_rn(av.w, b3.w, acc[i][3]);
      }
    }
    __syncthreads();
  }
  const uint32_t gn = n0 + tx * 4;
  if (gn < a.N) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint32_t gm = m0 + ty * 8 + i;
      if (gm < a.M)
        *reinterpret_cast<float4*>(a.C + (uint64_t)gm * a.N + gn) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
  }
}

// ------------------------------------------------------------------ CSR SpMV
// 32 rows per block, 8 lanes per row: lane l of a row sums elements
// l, l+8, l+16, ... with an ascending fused chain, then a fixed xor butterfly
// (4, 2, 1) adds the 8 partial sums. The order depends only on the row length.

__device__ __forceinline__ void spmv_csr_block(const kl_args_spmv_csr& a, uint32_t vb) {
  const uint32_t row = vb * kSpmvRowsPerBlock + (threadIdx.x >> 3);
  const int l = threadIdx.x & 7;
  float acc = 0.0f;
  if (row < a.nrows) {
    const int beg = __ldg(a.rowptr + row), end = __ldg(a.rowptr + row + 1);
    int e = beg + l;
    for (; e + 24 < end; e += 32) {
      int c0 = __ldcs(a.col + e), c1 = __ldcs(a.col + e + 8), c2 = __ldcs(a.col + e + 16),
          c3 = __ldcs(a.col + e + 24);
      float v0 = __ldcs(a.val + e), v1 = __ldcs(a.val + e + 8), v2 = __ldcs(a.val + e + 16),
            v3 = __ldcs(a.val + e + 24);
      float x0 = __ldg(a.x + c0), x1 = __ldg(a.x + c1), x2 = __ldg(a.x + c2), x3 = __ldg(a.x + c3);
      acc = __fmaf_rn(v0, x0, acc);
      acc = __fmaf_rn(v1, x1, acc);
      acc = __fmaf_rn(v2, x2, acc);
      acc = __fmaf_rn(v3, x3, acc);
    }
    for (; e < end; e += 8) acc = __fmaf_rn(__ldcs(a.val + e), __ldg(a.x + __ldcs(a.col + e)), acc);
  }
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 4));
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 2));
  acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, 1));
  if (l == 0 && row < a.nrows) a.y[row] = acc;
}

// ------------------------------------------------------------------ pointer chase

__device__ __forceinline__ void pchase_block(const kl_args_pchase& a, uint32_t vb) {
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
// stage 0: one block clears the 256 bins; stage 1: each block counts 16 KB into
// eight per-warp shared sub-histograms, then adds its non-zero bins globally.

__device__ __forceinline__ void hist256_block(const kl_args_hist256& a, uint32_t stage, uint32_t vb,
                                              char* smem) {
  if (stage == 0) {
    a.hist[threadIdx.x] = 0u;
    return;
  }
  uint32_t* sh = reinterpret_cast<uint32_t*>(smem);  // [8][256]
#pragma unroll
  for (int w = 0; w < 8; ++w) sh[w * 256 + threadIdx.x] = 0u;
  __syncthreads();
  uint32_t* mine = sh + (threadIdx.x >> 5) * 256;
  const uint64_t base = (uint64_t)vb * kHistBytesPerBlock;
  if (base + kHistBytesPerBlock <= a.n) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = __ldcs(reinterpret_cast<const uint4*>(a.data + base + ((uint64_t)u * 256 + threadIdx.x) * 16));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint32_t w4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        atomicAdd(mine + (w4[q] & 0xffu), 1u);
        atomicAdd(mine + ((w4[q] >> 8) & 0xffu), 1u);
        atomicAdd(mine + ((w4[q] >> 16) & 0xffu), 1u);
        atomicAdd(mine + (w4[q] >> 24), 1u);
      }
    }
  } else {
    for (uint64_t i = base + threadIdx.x; i < a.n && i < base + kHistBytesPerBlock; i += 256)
      atomicAdd(mine + a.data[i], 1u);
  }
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) s += sh[w * 256 + threadIdx.x];
  if (s) atomicAdd(a.hist + threadIdx.x, s);
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
// Keys n = 2^L, tile = 2^P keys (P = min(L, 12)). Stage list:
//   0                 : sort every tile in shared memory (all k <= 2^P), in -> out
//   for lv = P+1 .. L : one global stage per j = 2^(lv-1) .. 2^P (compare
//                       across tiles), then one shared-memory stage finishing
//                       j = 2^(P-1) .. 1 of the merge k = 2^lv
// Direction of a compare-exchange (i, i+j) at merge size k: ascending iff
// (i & k) == 0 (standard bitonic network on global indices).

struct BitonicStep {
  uint32_t kind;   // 0 tile-full, 1 global (k, j), 2 tile-merge (k)
  uint32_t lv;     // log2 k
  uint32_t jl;     // log2 j for global stages
};

__host__ __device__ inline BitonicStep bitonic_step(uint32_t L, uint32_t s) {
  uint32_t P = bitonic_tile_log2(L);
  if (s == 0) return BitonicStep{0, P, 0};
  s -= 1;
  for (uint32_t lv = P + 1; lv <= L; ++lv) {
    uint32_t nglobal = lv - P;
    if (s < nglobal) return BitonicStep{1, lv, lv - 1 - s};
    s -= nglobal;
    if (s == 0) return BitonicStep{2, lv, 0};
    s -= 1;
  }
  return BitonicStep{3, 0, 0};  // out of range (never produced for s < nstages)
}

__device__ __forceinline__ void cmpx(uint32_t& x, uint32_t& y, bool asc) {
  uint32_t lo = min(x, y), hi = max(x, y);
  x = asc ? lo : hi;
  y = asc ? hi : lo;
}

// compare-exchange network on a shared tile for merge sizes k in [k_lo, k_hi]
// with j running from min(k/2, jmax) down to 1
__device__ __forceinline__ void bitonic_tile(uint32_t* t, uint32_t tile_n, uint64_t gbase,
                                             uint32_t lv_lo, uint32_t lv_hi, uint32_t jstart_cap) {
  const uint32_t npairs = tile_n >> 1;
  for (uint32_t lv = lv_lo; lv <= lv_hi; ++lv) {
    const uint64_t k = 1ull << lv;
    uint32_t j = (uint32_t)(k >> 1);
    if (j > jstart_cap) j = jstart_cap;
    for (; j >= 1; j >>= 1) {
      for (uint32_t q = threadIdx.x; q < npairs; q += 256) {
        uint32_t i = (q / j) * 2 * j + (q % j);
        bool asc = ((gbase + i) & k) == 0;
        uint32_t x = t[i], y = t[i + j];
        cmpx(x, y, asc);
        t[i] = x;
        t[i + j] = y;
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void bitonic_block(const kl_args_bitonic& a, uint32_t stage, uint32_t vb,
                                              char* smem) {
  const uint32_t L = a.log2n;
  const uint32_t P = bitonic_tile_log2(L);
  const uint32_t tile_n = 1u << P;
  const BitonicStep st = bitonic_step(L, stage);
  if (st.kind == 1) {
    // global stage: 2048 pairs per block (tile_n/2), 8 per thread, coalesced
    const uint64_t j = 1ull << st.jl, k = 1ull << st.lv;
    const uint64_t q0 = (uint64_t)vb * (tile_n >> 1);
    for (uint32_t q = threadIdx.x; q < (tile_n >> 1); q += 256) {
      uint64_t qq = q0 + q;
      uint64_t i = (qq / j) * 2 * j + (qq % j);
      bool asc = (i & k) == 0;
      uint32_t x = __ldcg(a.out + i), y = __ldcg(a.out + i + j);
      cmpx(x, y, asc);
      a.out[i] = x;
      a.out[i + j] = y;
    }
    return;
  }
  uint32_t* t = reinterpret_cast<uint32_t*>(smem);
  const uint64_t gbase = (uint64_t)vb * tile_n;
  const uint32_t* src = st.kind == 0 ? a.in : a.out;
  for (uint32_t q = threadIdx.x; q < tile_n; q += 256) t[q] = __ldcg(src + gbase + q);
  __syncthreads();
  if (st.kind == 0)
    bitonic_tile(t, tile_n, gbase, 1, P, tile_n);
  else
    bitonic_tile(t, tile_n, gbase, st.lv, st.lv, tile_n >> 1);
  for (uint32_t q = threadIdx.x; q < tile_n; q += 256) a.out[gbase + q] = t[q];
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

// ------------------------------------------------------------------ dispatch
// Runs cumulative block g (of stage st) of a tenant. All 256 threads call it.

template <class A>
__device__ __forceinline__ A load_args(const void* p) {
  return *reinterpret_cast<const A*>(p);
}

__device__ __forceinline__ void run_block(uint32_t type, const void* args, const Stage& st, uint32_t g,
                                          char* smem) {
  const uint32_t vb = g - st.begin;
  switch (type) {
    case KL_T_GATHER: gather_block(load_args<kl_args_gather>(args), vb); break;
    case KL_T_BLACKSCHOLES: blackscholes_block(load_args<kl_args_blackscholes>(args), vb); break;
    case KL_T_GEMM_F32: gemm_f32_block(load_args<kl_args_gemm_f32>(args), vb, smem); break;
    case KL_T_SPMV_CSR: spmv_csr_block(load_args<kl_args_spmv_csr>(args), vb); break;
    case KL_T_PCHASE: pchase_block(load_args<kl_args_pchase>(args), vb); break;
    case KL_T_TRIAD: triad_block(load_args<kl_args_triad>(args), vb); break;
    case KL_T_HIST256: hist256_block(load_args<kl_args_hist256>(args), st.s, vb, smem); break;
    case KL_T_ESCAPE: escape_block(load_args<kl_args_escape>(args), vb); break;
    case KL_T_BITONIC: bitonic_block(load_args<kl_args_bitonic>(args), st.s, vb, smem); break;
    case KL_T_MATADD: matadd_block(load_args<kl_args_matadd>(args), vb); break;
    default: break;
  }
}

#endif  // __CUDACC__

}  // namespace tn
}  // namespace kl
