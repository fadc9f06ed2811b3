// Plain launches of the tenant kernels (one grid per stage, blockIdx.x as the
// block index): the comparators the co-scheduler is measured against — serial
// FIFO on one stream and concurrent multi-stream launches — and the unsliced
// reference execution for the slicing-overhead measurement (Section 5.2).
// One instantiation per type so each gets its own register allocation.
#include <cuda_runtime.h>
#include <stdint.h>

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
      case KL_T_GEMM_BF16: e = launch_one<KL_T_GEMM_BF16>(args, st, nb, s); break;
      case KL_T_TEA: e = launch_one<KL_T_TEA>(args, st, nb, s); break;
      case KL_T_SAD: e = launch_one<KL_T_SAD>(args, st, nb, s); break;
      case KL_T_STENCIL: e = launch_one<KL_T_STENCIL>(args, st, nb, s); break;
      case KL_T_MRIQ: e = launch_one<KL_T_MRIQ>(args, st, nb, s); break;
      default: return -1;
    }
    if (e != cudaSuccess) return -1;
  }
  return 0;
}

}  // namespace kl
