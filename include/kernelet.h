/*
 * kernelet.h — C ABI of a GB300 (sm_103a) runtime for sliced, co-scheduled
 * execution of concurrently submitted GPU kernels ("Kernelet", Zhong & He,
 * arXiv 1303.5164).
 *
 * Problem statement (Section 2.2): tenants submit kernels; a kernel is k thread
 * blocks with IDs 0..k-1 that do not depend on one another (assumption 2); a
 * slice is a contiguous range of block IDs; a co-schedule runs slices of two
 * kernels at the same time; the goal is the minimum total execution time of the
 * pending kernels, re-optimised on the residuals when kernels arrive.
 *
 * How this library realises it on one GPU:
 *   - kl_submit copies a kernel descriptor (type, grid, block, resources,
 *     arguments) into the pending set R (Algorithm 1, "a new kernel comes").
 *   - kl_launch starts ONE persistent co-scheduler kernel over R: every SM
 *     holds `slots` CTAs; for the current co-schedule <K1,K2,size1,size2>
 *     (Algorithm 1) the first size1 slots of each SM run K1 and the other size2
 *     run K2; each CTA pulls a slice (contiguous block range) with one atomic
 *     and runs it with rectified block indices (Section 4.1, index
 *     rectification). When a kernel has handed out its last block the CTA that
 *     sees it re-plans on the device (FindCoSchedule over the pending set, using
 *     the CP table the Markov model of Section 4.4 computed on the host).
 *   - kl_poll / kl_wait / kl_drain report completion.
 *   - kl_model_* and kl_plan are pure host functions: the performance model
 *     (Section 4.4), pruning (Section 4.3) and the greedy plan (Algorithm 1).
 *
 * Conventions for every function:
 *   - Return value: KL_OK (0) or a negative kl_status. Nothing is thrown
 *     across the ABI; no function aborts the process.
 *   - Pointers inside kl_args_* blocks are DEVICE pointers the caller owns
 *     (allocated e.g. with torch). They must stay valid and untouched until the
 *     tenant's handle is DONE or ERROR. All other pointers are host pointers.
 *   - Thread safety: one kl_runtime may be used from several host threads;
 *     calls on it are serialised by an internal mutex. Pure functions are
 *     reentrant.
 *   - Device-side waits are bounded (kl_config.device_wait_limit_ns); an
 *     expired wait ends the run with KL_EDEVICE_TIMEOUT and leaves the context
 *     usable.
 */
#ifndef KERNELET_H
#define KERNELET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KL_ABI_VERSION 2
#define KL_BLOCK_THREADS 256     /* threads of a co-scheduler slot (and of every
                                    tenant block but the resource-heavy variants) */
#define KL_MAX_ARGS_BYTES 96     /* largest kl_args_* block                     */
#define KL_MAX_SLOTS 8           /* per-SM block slots of the co-scheduler      */

typedef enum {
    KL_OK = 0,
    KL_EINVAL = -1,           /* bad argument, descriptor or size              */
    KL_ENOMEM = -2,           /* host or device allocation failed              */
    KL_EAGAIN = -3,           /* queue full / a run is still in flight         */
    KL_ETIMEDOUT = -4,        /* host-side wait expired (work continues)       */
    KL_ECUDA = -5,            /* a CUDA runtime call failed                    */
    KL_EDEVICE_TIMEOUT = -6,  /* a device-side bounded wait expired            */
    KL_ESTATE = -7,           /* call not valid in the current state           */
    KL_ENOTFOUND = -8,        /* unknown handle                                */
    KL_EOVERFLOW = -9         /* a device table (phases, tenants) overflowed   */
} kl_status;

typedef enum { KL_PENDING = 0, KL_RUNNING = 1, KL_DONE = 2, KL_ERROR = 3 } kl_state;

typedef struct kl_runtime kl_runtime;   /* opaque; owned by the library */

/* Tenant kernel types. Each is a hand-written device function that runs one
 * 256-thread block given its rectified (virtual) block index. */
typedef enum {
    KL_T_GATHER = 0,        /* out[i] = a[idx[i]], int32                           */
    KL_T_BLACKSCHOLES = 1,  /* European call/put, binary32                         */
    KL_T_GEMM_F32 = 2,      /* C = A B, binary32, ascending-k fused chain per C[i][j] */
    KL_T_SPMV_CSR = 3,      /* y = A x, CSR, binary32                              */
    KL_T_PCHASE = 4,        /* end[t] = next^hops(start[t]), int32                 */
    KL_T_TRIAD = 5,         /* a = s*c + b (fused), binary32                       */
    KL_T_HIST256 = 6,       /* 256-bin histogram of bytes, uint32 counts            */
    KL_T_ESCAPE = 7,        /* escape-time iteration count per pixel, uint32       */
    KL_T_BITONIC = 8,       /* ascending bitonic sort of 2^log2n uint32 keys        */
    KL_T_MATADD = 9,        /* c = a + b on an n x n matrix, 16x16 blocks (Section 4.1 example) */
    KL_T_GEMM_BF16 = 10,    /* C = A B^T, BF16 inputs, FP32 accumulate, tensor cores */
    KL_T_TEA = 11,          /* Tiny Encryption Algorithm, 32 cycles per 64-bit block */
    KL_T_SAD = 12,          /* sums of absolute differences, 4x4 blocks, motion search */
    KL_T_STENCIL = 13,      /* 7-point stencil on a 3-D grid */
    KL_T_MRIQ = 14,         /* MRI Q matrix: phiMag, then Q over the k-space samples */
    KL_T_TESTMIX = 15,      /* Section 4.3 testing kernel: a tunable mix of streaming loads
                               and dependent fused multiply-adds (PUR / MUR sweep)        */
    /* Resource-heavy variants (their blocks do not fit a co-scheduler slot of
     * 256 threads at 64 registers; each runs in a resource-class kernel of its
     * own, one CTA per SM beside two co-scheduler slots, Section 6's merged-
     * kernel register cost): */
    KL_T_BS255 = 16,        /* Black-Scholes, 128-thread blocks of 16 options a thread
                               held in registers (up to 255 per thread)                 */
    KL_T_HIST1024 = 17,     /* 256-bin histogram with 1024-thread blocks                 */
    KL_T_GEMM_F32_BIG = 18, /* FP32 GEMM, 128x128 tiles staged in 96 KB of shared memory */
    KL_T_COUNT = 19
} kl_tenant_type;
#define KL_T_MAIN_COUNT 16  /* types 0 .. 15 run in the co-scheduler's slots; the
                               planner of Algorithm 1 pairs these                         */

/* ----------------------------------------------------------- tenant arguments
 * Layouts: row-major, densely packed, element types as named. Pointers to
 * arrays that the tenant reads or writes with 16-byte vector accesses must be
 * 16-byte aligned (marked "16B"). */

typedef struct {            /* KL_T_GATHER: 1024 elements per block           */
    const int32_t* a;       /* [n_src]                                         */
    const int32_t* idx;     /* [n] 16B, values in [0, n_src)                   */
    int32_t* out;           /* [n] 16B                                         */
    uint64_t n;
} kl_args_gather;

typedef struct {            /* KL_T_BLACKSCHOLES: 256 options per block       */
    const float *S, *K, *r, *v, *T;   /* [n] spot, strike, rate, volatility, years */
    float *call, *put;                /* [n]                                   */
    uint64_t n;
} kl_args_blackscholes;

typedef struct {            /* KL_T_GEMM_F32: one 64x64 tile of C per block   */
    const float* A;         /* [M][K] 16B                                      */
    const float* B;         /* [K][N] 16B                                      */
    float* C;               /* [M][N] 16B                                      */
    uint32_t M, N, K;       /* N and K multiples of 4                          */
    uint32_t pad;
} kl_args_gemm_f32;

typedef struct {            /* KL_T_SPMV_CSR: 32 rows per block                */
    const int32_t* rowptr;  /* [nrows+1], non-decreasing, rowptr[0] = 0        */
    const int32_t* col;     /* [nnz] values in [0, ncols)                      */
    const float* val;       /* [nnz]                                           */
    const float* x;         /* [ncols]                                         */
    float* y;               /* [nrows]                                         */
    uint32_t nrows, ncols;
} kl_args_spmv_csr;

typedef struct {            /* KL_T_PCHASE: 256 chasers per block              */
    const int32_t* next;    /* [N] values in [0, N)                            */
    const int32_t* start;   /* [nchasers] values in [0, N)                     */
    int32_t* end;           /* [nchasers]                                      */
    uint32_t N, nchasers, hops, pad;
} kl_args_pchase;

typedef struct {            /* KL_T_TRIAD: 4096 elements per block             */
    const float* b;         /* [n] 16B                                         */
    const float* c;         /* [n] 16B                                         */
    float* a;               /* [n] 16B                                         */
    float s;
    uint32_t pad;
    uint64_t n;
} kl_args_triad;

typedef struct {            /* KL_T_HIST256: stage 0 = 1 block clears hist;    */
    const uint8_t* data;    /* [n] 16B   stage 1 = 32768 bytes per block        */
    uint32_t* hist;         /* [256]                                           */
    uint64_t n;
} kl_args_hist256;

typedef struct {            /* KL_T_ESCAPE: 256 pixels (row-major) per block   */
    uint32_t* count;        /* [height][width]                                 */
    uint32_t width, height, max_iter, pad;
    float x0, y0, dx, dy;   /* pixel (i,j) -> c = (x0+(j+.5)dx, y0+(i+.5)dy)    */
} kl_args_escape;

typedef struct {            /* KL_T_BITONIC: 4096-key tiles; stage 0 reads in, */
    const uint32_t* in;     /* [2^log2n]   later stages work in place on out   */
    uint32_t* out;          /* [2^log2n]                                       */
    uint32_t log2n;         /* 1..30                                           */
    uint32_t pad;
} kl_args_bitonic;

typedef struct {            /* KL_T_MATADD: 16x16-thread blocks, (n/16)^2 grid */
    const float* a;
    const float* b;
    float* c;
    uint32_t n;             /* multiple of 16                                  */
    uint32_t pad;
} kl_args_matadd;

typedef struct {            /* KL_T_GEMM_BF16: one 128x64 tile of C per block  */
    const uint16_t* A;      /* [M][K] bfloat16 bits, 16B, K multiple of 8      */
    const uint16_t* Bt;     /* [N][K] bfloat16 bits (B stored column-major)    */
    float* C;               /* [M][N] 16B, N multiple of 4                     */
    const void* tmaps;      /* device copy of the 256 bytes written by
                               kl_gemm_bf16_tensor_maps (64B aligned); caller
                               owned, alive until the kernel is DONE           */
    uint32_t M, N, K, pad;
} kl_args_gemm_bf16;

typedef struct {            /* KL_T_TEA: 512 64-bit blocks per thread block     */
    const uint32_t* in;     /* [2n] words, block j = (in[2j], in[2j+1]), 16B    */
    uint32_t* out;          /* [2n] 16B                                         */
    uint32_t key[4];
    uint64_t n;             /* 64-bit blocks                                    */
} kl_args_tea;

typedef struct {            /* KL_T_SAD: 256 SAD values per block               */
    const uint8_t* cur;     /* [height][width] current frame (8-bit luma)       */
    const uint8_t* ref;     /* [height][width] reference frame                  */
    uint32_t* sad;          /* [height/4 * width/4][(2R+1)^2]: for 4x4 block b
                               (row-major) and displacement (dx, dy) in [-R, R]^2,
                               index (dy+R)(2R+1) + (dx+R); reference pixels
                               outside the frame take the nearest edge pixel    */
    uint32_t width, height; /* multiples of 4                                   */
    uint32_t range;         /* R, 1..16                                         */
    uint32_t pad;
} kl_args_sad;

typedef struct {            /* KL_T_STENCIL: 256 x-points of one (y, z) row per block */
    const float* in;        /* [nz][ny][nx]                                     */
    float* out;             /* [nz][ny][nx]; interior: c0 c + c1 (sum of the 6
                               face neighbours); boundary points copied         */
    uint32_t nx, ny, nz, pad;
    float c0, c1;
} kl_args_stencil;

typedef struct {            /* KL_T_MRIQ: stage 0 = phiMag (256 samples per block),
                               stage 1 = Q (256 points per block)               */
    const float *kx, *ky, *kz;  /* [numK] k-space sample coordinates            */
    const float *phiR, *phiI;   /* [numK]                                        */
    float* phiMag;              /* [numK] written by stage 0                     */
    const float *x, *y, *z;     /* [numX] image-space points                    */
    float *Qr, *Qi;             /* [numX]                                        */
    uint32_t numK, numX;
} kl_args_mriq;

typedef struct {            /* KL_T_TESTMIX: thread g of the grid (256 a block) runs
                               `iters` rounds of `mem` streaming loads
                               acc += in[(g + (i mem + m) nthreads) mod n_in] then
                               `alu` dependent steps acc = fma(acc, c1, c2), and
                               stores out[g] = acc                                     */
    const float* in;        /* [n_in], n_in a power of two                              */
    float* out;             /* [nthreads]                                               */
    uint32_t n_in, nthreads;
    uint32_t iters, mem, alu, pad;
    float c1, c2;
} kl_args_testmix;

/* KL_T_BS255 takes kl_args_blackscholes (128 threads x 16 options = 2048
 * options per block); KL_T_HIST1024 takes kl_args_hist256 (stage 0 clears,
 * stage 1 counts 131072 bytes per 1024-thread block); KL_T_GEMM_F32_BIG takes
 * kl_args_gemm_f32 (one 128 x 128 tile of C per block; N, K multiples of 4). */

/* Launch shape of a tenant as a plain kernel would use it (Section 2.2: a
 * kernel is k thread blocks). Multi-stage tenants (histogram, bitonic sort)
 * are a chain of grids; stage s may start only when stage s-1 has finished. */
typedef struct {
    uint32_t grid[3];       /* blocks of stage 0 (x, y, z)                      */
    uint32_t block[3];      /* {256, 1, 1}; {128, 1, 1} for KL_T_BS255, {1024, 1, 1}
                               for KL_T_HIST1024                                 */
    uint32_t nstages;
    uint32_t smem_bytes;    /* dynamic shared memory per block                  */
    uint64_t total_blocks;  /* summed over stages                               */
} kl_tenant_shape;

/* Descriptor of one submitted kernel. */
typedef struct {
    uint32_t type;              /* kl_tenant_type                                */
    uint32_t grid[3];           /* must equal kl_tenant_shape().grid             */
    uint32_t block[3];          /* must equal kl_tenant_shape().block            */
    uint32_t smem_bytes;        /* resource profile: declared dynamic smem       */
    uint32_t regs_per_thread;   /* resource profile: declared registers (0 = n/a) */
    uint32_t slice_blocks;      /* blocks per slice; 0 = runtime's per-type size */
    const void* args;           /* -> kl_args_<type> (host memory; copied)        */
    uint32_t args_size;         /* sizeof(kl_args_<type>)                        */
    uint32_t flags;             /* reserved, 0                                   */
    uint64_t footprint_bytes;   /* device bytes the kernel touches (admission)   */
} kl_kernel_desc;

typedef uint64_t kl_handle;     /* 0 is never a valid handle */

typedef enum {
    KL_RATIO_BALANCED = 0,      /* min dT (Eq. executiontime), ties -> max CP     */
    KL_RATIO_MAX_CP = 1,        /* max CP over the feasible splits                */
    KL_RATIO_FIXED = 2          /* kl_config.fixed_slots_a slots for K1           */
} kl_ratio_policy;

/* kl_config.flags */
#define KL_CFG_BACKFILL 1u  /* a slot that neither kernel of the current co-schedule
                               can use (stage barrier, spread rule, re-plan in
                               flight) runs a slice of another pending kernel;
                               default on */
#define KL_CFG_FILL_TYPES 2u /* backfill tries the next pending kernels of the two
                               types the co-schedule runs before any other
                               pending kernel; default on */
#define KL_CFG_SERVE_TC 8u   /* serving runs use the full co-scheduler build, which
                               also runs KL_T_GEMM_BF16 (tensor cores) and the
                               types after it; without it a serving run refuses
                               those types (KL_EINVAL). Batch runs pick the build
                               from the kernels they hold. */
#define KL_CFG_WIDE_FILL 16u /* backfill considers two pending kernels per slot
                               of an SM (8 at 4 slots, 16 at 8; both chain-lane
                               kernels, then the lowest pending ones) instead
                               of 4; default on */
#define KL_CFG_LAZY_ARRIVAL 32u /* serving: an arrival re-plans only when no pair is
                               running (idle or solo phase); otherwise the new
                               kernel waits in R for the next re-plan, which
                               comes when a kernel of the pair runs out */
#define KL_CFG_RANDOM_PLAN 64u /* the MC comparison of Section 5.1: every re-plan
                               picks a pair of pending kernel types and a slot
                               split uniformly at random (counter-based SplitMix64
                               of kl_config.plan_seed and the phase number)
                               instead of the largest-CP pair */
#define KL_CFG_LIGHT_BUILD 128u /* a batch run whose kernels are all of the light
                               types (gather, Black-Scholes, SpMV, triad,
                               escape-time, MatrixAdd, TEA, stencil, the testing
                               kernel: short bodies within 32 registers), with no
                               resource-heavy variant, uses the co-scheduler
                               build with 8 CTAs per SM instead of 4, and the CP
                               table for 8 slots; needs slots_per_sm = 0 and no
                               kl_set_cp_table override; default on */
#define KL_CFG_DEEP_FILL 256u /* batch runs: a slot that neither the co-schedule
                               nor the backfill list can use takes a slice of
                               the lowest kernel, in submission order, that
                               still has blocks to hand out, so kernels with
                               fewer slices than the GPU has slots do not leave
                               slots idle; default on */
#define KL_CFG_PHASE_MODEL 512u /* with the chain lane: the planner scores each pair
                               as the phase the device runs, the pair plus the
                               chain lane's kernel (the multi-stage type with
                               the most blocks pending), with the three-kernel
                               chain of kl_model_phase, at the pair's split that
                               maximises that phase's CP; default on */
#define KL_CFG_CHAIN_LANE 4u /* while kernels with more than one stage (chains of
                               dependent grids) are pending outside the current
                               co-schedule, the last slot of every SM takes their
                               slices first, so their stage barriers overlap
                               other work instead of forming the end of the run;
                               default on, kl_config.chain_slots = 2 */

typedef struct {
    int32_t device;                 /* CUDA ordinal (default 0)                     */
    uint32_t slots_per_sm;          /* co-scheduler CTAs per SM; 0 = occupancy limit
                                       of the build a run uses                      */
    uint32_t max_tenants;           /* pending-set capacity per run (default 4096)  */
    uint32_t model_states;          /* 2 or 3 (uncoalesced extension); default 3    */
    uint32_t ratio_policy;          /* kl_ratio_policy                              */
    uint32_t fixed_slots_a;         /* for KL_RATIO_FIXED                           */
    uint64_t device_wait_limit_ns;  /* bound on every device spin (default 2 s)     */
    uint64_t mem_cap_bytes;         /* admission cap on summed footprints (0 = none) */
    double alpha_p, alpha_m;        /* pruning thresholds; negative = no pruning    */
    uint32_t flags;                 /* KL_CFG_* bits                                */
    uint32_t chain_slots;           /* KL_CFG_CHAIN_LANE: slots per SM (the last ones)
                                       that serve multi-stage kernels first; 0 = 1 */
    uint64_t age_limit_ns;          /* serving: a kernel pending longer than this
                                       (device clock, since the device took it in) is
                                       put into the next co-schedule with its best
                                       partner, so poorly pairing kernels are not
                                       starved by new arrivals; 0 = 5 ms; ~0 = off.
                                       Batch runs never age (every kernel is present
                                       from the start). */
    uint64_t plan_seed;             /* KL_CFG_RANDOM_PLAN: seed of the random plans */
} kl_config;

/* Model inputs for one tenant type (Table 1 parameters, measured by profiling
 * a plain launch of the kernel, Section 4.4 "getting the input"). */
typedef struct {
    double R_m;             /* memory instructions / instructions                */
    double f_u;             /* fraction of memory instructions that are uncoalesced */
    double m_c;             /* DRAM sectors per coalesced memory instruction     */
    double m_u;             /* DRAM sectors per uncoalesced memory instruction   */
    double L0;              /* unloaded memory latency, SM cycles                */
    double I_block;         /* warp instructions per thread block                */
    double PUR, MUR;        /* Section 4.3 utilisation ratios (pruning)          */
    uint32_t warps_per_block;
    uint32_t valid;         /* 0 = no profile for this type                      */
    uint32_t slice_blocks;  /* blocks per slice for this type (Section 4.1: the
                               smallest slice whose overhead is within p%,
                               measured with several kernels of the type in
                               one launch); 0 = the runtime's built-in size  */
    uint32_t slice_blocks_alone; /* the same rule with one kernel alone: the
                               least a slice shrinks to when a run has too few
                               slices for its CTAs (0 = 1 block)             */
} kl_profile;

typedef struct {
    uint32_t n_sm;          /* SMs                                               */
    uint32_t n_sched;       /* warp schedulers per SM (virtual-SM divisor)       */
    double f_sm_hz;         /* SM clock used to convert cycles to seconds        */
    double dram_bytes_per_s;
    double sector_bytes;    /* DRAM access granularity (32)                      */
    double a0, b0;          /* linear latency model parameters                   */
} kl_model_params;

typedef struct {
    int32_t A, B;           /* submit indices; B = -1 for a solo phase; A = -1 ends */
    uint32_t slots_a, slots_b;
    double cp;              /* predicted co-scheduling profit (Eq. cp)           */
    uint64_t t_ns;          /* device globaltimer when the phase was published   */
    int32_t trigger;        /* tenant whose exhaustion ended the previous phase  */
    uint32_t n_pending;     /* kernels with blocks left when the phase was chosen */
    uint64_t pending_mask;  /* bit i: kernel i (i < 64) was pending               */
    uint32_t done_a, done_b;          /* blocks finished by A, B at publication    */
    uint32_t prev_done_a, prev_done_b;/* by the previous phase's A, B at that time */
} kl_phase;

typedef struct {
    int32_t state;              /* kl_state                                      */
    int32_t error;              /* kl_status when state == KL_ERROR               */
    uint64_t t_submit_ns;       /* host steady clock at kl_submit                 */
    uint64_t t_start_ns;        /* device: first slice of this kernel started     */
    uint64_t t_end_ns;          /* device: last block finished                    */
    uint64_t t_launch_ns;       /* device: run start (first CTA)                  */
    uint32_t slices;            /* slices pulled                                  */
    uint32_t blocks;            /* blocks executed                                */
    uint64_t t_done_host_ns;    /* host steady clock when the runtime saw the
                                   completion (serving: when it was reaped)       */
} kl_tenant_stats;

typedef struct {
    uint32_t n_tenants;
    uint32_t n_phases;
    int32_t error;              /* kl_status of the run                           */
    uint32_t slots_per_sm;
    uint32_t grid_ctas;
    uint32_t pad;
    uint64_t t_launch_ns;       /* device globaltimer at the first CTA            */
    uint64_t t_end_ns;          /* device globaltimer at the last completion      */
    uint64_t kernel_ns;         /* CUDA-event time of the persistent launch (co-
                                   scheduled run) or of the fork/join (baseline) */
    uint64_t run_ns;            /* CUDA-event time from the run's first copy to
                                   its last (descriptors in, results out)        */
    uint64_t slot_wait_ns;      /* co-scheduled: summed over CTAs, time with no
                                   slice to pull (idle slots)                    */
    uint64_t stage_wait_ns;     /* ... time at a stage barrier inside a slice     */
    uint64_t plan_ns;           /* ... time re-planning (FindCoSchedule)          */
    uint32_t class_ctas[4];     /* per resource class (index 1..3: KL_T_BS255,
                                   KL_T_HIST1024, KL_T_GEMM_F32_BIG): CTAs of its
                                   class kernel that found work; [0] unused      */
} kl_run_stats;

typedef enum {
    KL_BASE_SERIAL = 0,       /* plain launches, one stream                      */
    KL_BASE_MULTISTREAM = 1,  /* plain launches, round-robin over n streams      */
    KL_SERVE_COSCHED = 2      /* kl_serve_start only: the persistent co-scheduler */
} kl_baseline_mode;

/* ------------------------------------------------------------------ runtime */

/* Fill `cfg` with defaults (no counterpart in the paper: library
 * housekeeping). KL_EINVAL on NULL. */
int kl_config_default(kl_config* cfg);

/* Create a runtime: the kernel queue and scheduler of Section 3.2 (Fig.
 * kerneletOverview: kernels are buffered in a queue, the scheduler picks the
 * co-schedules, slices are dispatched to the GPU) for one GPU, cfg->device,
 * launching on `cuda_stream` (a cudaStream_t, may be NULL for the legacy
 * default stream). cfg NULL = kl_config_default. Allocates the device queue
 * (cfg->max_tenants descriptors) and pinned host staging; the runtime owns
 * them until kl_destroy. *out receives the handle (host memory).
 * Errors: KL_EINVAL (NULL out, bad device or sizes), KL_ENOMEM, KL_ECUDA. */
int kl_create(const kl_config* cfg, void* cuda_stream, kl_runtime** out);

/* End of the runtime of Section 3.2: wait for in-flight work (up to the
 * device wait limit; a serving run is stopped first), then free the queue,
 * staging and history. Handles of this runtime become invalid. KL_ESTATE if a
 * run could not be retired (its memory is then left allocated); KL_EINVAL on
 * NULL. */
int kl_destroy(kl_runtime* rt);

/* Tensor maps (two CUtensorMap, 128 bytes each: A then Bt) that the
 * KL_T_GEMM_BF16 tenant's TMA loads read: 2-D tiles of 64 K-elements x 128
 * rows of A and x 64 rows of Bt, 128-byte swizzle, zero fill outside the
 * matrix. Written to out_host (256 bytes, host memory); the caller copies them
 * to device memory and passes that address as kl_args_gemm_bf16.tmaps. Needs
 * the CUDA driver (no device work). KL_EINVAL on misaligned pointers, K not a
 * multiple of 8, or a zero size; KL_ECUDA when the CUDA driver refuses the map. */
int kl_gemm_bf16_tensor_maps(const kl_args_gemm_bf16* args, void* out_host);

/* Launch shape of a tenant (no device work). */
int kl_tenant_shape_of(uint32_t type, const void* args, uint32_t args_size, kl_tenant_shape* out);

/* Add a kernel to the pending set. Validates type, grid/block against the
 * tenant's shape, alignment, and admission (summed footprint <= mem cap).
 * Non-blocking; copies the descriptor and arguments. KL_EAGAIN when the
 * pending set is full or over the memory cap. */
int kl_submit(kl_runtime* rt, const kl_kernel_desc* desc, kl_handle* out);

/* Staged arrival (Algorithm 1, "a new kernel comes", for a burst of kernels):
 * kl_submit_staged admits a kernel like kl_submit but, while serving, does
 * not make it visible to the device: the descriptor is written into the
 * mapped ring (co-scheduled) or held back (plain launches) and the kernel
 * stays KL_PENDING. kl_publish makes every staged kernel visible with one
 * release store of the ring's tail, so the device takes the whole burst in
 * and re-plans once instead of once per kernel; a kl_submit publishes every
 * kernel staged before it too. A serving run stopped (kl_serve_stop) while
 * kernels are still staged never runs them: they end in KL_ERROR (error
 * KL_ESTATE), their buffers untouched. Outside serving, kl_submit_staged is
 * kl_submit (the next kl_launch takes every pending kernel) and kl_publish
 * returns KL_OK. Errors as kl_submit; kl_publish: KL_EINVAL on NULL,
 * KL_ECUDA when a held-back plain launch fails. */
int kl_submit_staged(kl_runtime* rt, const kl_kernel_desc* desc, kl_handle* out);
int kl_publish(kl_runtime* rt);

/* A burst of arrivals in one call (Algorithm 1, "a new kernel comes", for n
 * kernels that arrive together): admits descs[0..n) in order, exactly as n
 * kl_submit_staged calls followed by one kl_publish, and writes their handles
 * to out[0..n) (host arrays of n entries). It stops at the first kernel that
 * kl_submit would refuse: *n_done (host, may be NULL) = kernels admitted
 * before it (those stay admitted and, while serving, are published), and the
 * call returns that kernel's error; on success *n_done = n. Allowed while a
 * batch run is in flight: the kernels join the pending set of the next
 * kl_launch. KL_EINVAL on NULL rt, or on NULL descs / out with n > 0. */
int kl_submit_batch(kl_runtime* rt, const kl_kernel_desc* descs, uint32_t n, kl_handle* out,
                    uint32_t* n_done);

/* Plan and start the pending set as one persistent co-scheduled launch on the
 * runtime's stream (Algorithm 1 over the whole set); returns without waiting.
 * The launch uses the smallest co-scheduler build that holds every pending
 * type: 4 slots per SM (plain; or full when a KL_T_GEMM_BF16, TEA, SAD,
 * stencil or MRI-Q kernel is pending), or 8 slots per SM when every kernel is
 * of a KL_CFG_LIGHT_BUILD type; kl_get_run_stats reports the slots the run
 * used. KL_EAGAIN if a run is in flight. */
int kl_launch(kl_runtime* rt);

/* Serving mode: continuous batching. Algorithm 1 lets kernels join the
 * pending set R at any time; an arrival makes the scheduler choose the next
 * co-schedule again over what is left of the running kernels plus the new
 * ones (Section 2.2, Section 4.2). kl_serve_start(KL_SERVE_COSCHED) launches
 * the persistent kernel and leaves it running; from then on each kl_submit is
 * admitted straight to the running kernel: the descriptor is written into a
 * ring in mapped host memory and the tail published with a release store; a
 * dispatcher CTA on the device copies it in and re-plans. Completions come
 * back through a completion queue in mapped memory while the kernel runs.
 * mode KL_BASE_MULTISTREAM (nstreams streams) / KL_BASE_SERIAL is the plain
 * comparator: each admitted kernel is launched at once on stream
 * seq % nstreams.
 * Admission, in every mode: at most cfg.max_tenants kernels in flight and
 * their summed footprint_bytes within cfg.mem_cap_bytes (0 = no cap); beyond
 * that kl_submit returns KL_EAGAIN and the caller retries later. Kernels still
 * pending from kl_submit before the start are admitted first, in order, and
 * keep their handles.
 * idle_limit_ns (co-scheduled): the device ends the run after that long with
 * no kernel in flight and no arrival (0 = 60 s); kl_submit then returns
 * KL_ESTATE until kl_serve_stop and a new kl_serve_start. While serving,
 * kl_launch, kl_launch_baseline and kl_drain return KL_ESTATE, and kl_poll /
 * kl_wait / kl_get_stats / kl_reap see completions as they happen.
 * The serving kernel occupies the runtime's stream until the run ends: work
 * queued on that stream meanwhile (and a synchronize of it) waits for the end,
 * so a kernel's inputs must be complete before its kl_submit (the device may
 * start it at once) and other work goes on other streams.
 * kl_serve_stop: no new admissions; every admitted kernel finishes, the run
 * ends and is retired (KL_ETIMEDOUT after timeout_ns; call again). Returns the
 * run's status. Errors: KL_ESTATE (not serving / already serving), KL_EAGAIN
 * (a batch run is still in flight), KL_ENOMEM / KL_ECUDA. */
int kl_serve_start(kl_runtime* rt, int mode, uint32_t nstreams, uint64_t idle_limit_ns);
int kl_serve_stop(kl_runtime* rt, uint64_t timeout_ns);

/* Serving: up to `cap` handles of kernels that completed since the last call,
 * in completion order, into out[0..*n). The runtime keeps at most 2^20 such
 * handles; older ones are dropped (their stats stay available). */
int kl_reap(kl_runtime* rt, kl_handle* out, uint32_t cap, uint32_t* n);

/* Execute the pending set with plain kernel launches instead of the
 * co-scheduler: KL_BASE_SERIAL = one stream in submit order; KL_BASE_MULTISTREAM
 * = tenant i on stream i % nstreams (concurrent kernel execution). The runtime
 * stream is forked into the side streams and joined back, so events recorded
 * on it bracket the whole run. Returns without waiting. */
int kl_launch_baseline(kl_runtime* rt, int mode, uint32_t nstreams);

/* Current state of a handle (kl_state) into *state, without blocking.
 * Algorithm 1 removes a kernel from the pending set R once all its thread
 * blocks have executed (Section 2.2: every block occurs in one co-schedule
 * once); DONE is that moment, RUNNING means some of its slices have been
 * dispatched. Retires a finished run as a side effect. KL_ENOTFOUND for a
 * handle this runtime never issued (or whose record was dropped). */
int kl_poll(kl_runtime* rt, kl_handle h, int* state);

/* Block until the handle is DONE or ERROR (the end of that kernel in
 * Algorithm 1's loop), or until timeout_ns elapses: KL_ETIMEDOUT, and the
 * kernel keeps running (timeout_ns = 0 only polls). Returns KL_OK when the
 * kernel completed, its error when it failed, KL_ENOTFOUND for an unknown
 * handle, KL_ESTATE for a kernel still in R that no launch has started
 * (waiting for it would never end). */
int kl_wait(kl_runtime* rt, kl_handle h, uint64_t timeout_ns);

/* Algorithm 1 run to the end: launch whatever is pending (the outer loop
 * "while R != null"), then wait until every kernel of the run is DONE or
 * ERROR, or timeout_ns elapses (KL_ETIMEDOUT; the run continues and a later
 * kl_drain waits again). Returns the run's status (KL_OK, KL_EDEVICE_TIMEOUT,
 * KL_EOVERFLOW, ...); KL_ESTATE while serving. */
int kl_drain(kl_runtime* rt, uint64_t timeout_ns);

/* Wait for the run in flight (co-scheduled or plain launches) to end, up to
 * timeout_ns (KL_ETIMEDOUT; the run continues), WITHOUT launching the pending
 * set: kernels submitted while the run was in flight stay pending for the
 * next kl_launch. This lets a caller overlap building the next batch with the
 * current run (submit, then wait, then launch). Returns the finished run's
 * status (KL_OK when no run was in flight and none has failed); KL_ESTATE
 * while serving, KL_EINVAL on NULL. */
int kl_wait_run(kl_runtime* rt, uint64_t timeout_ns);

/* Per-kernel measurements of a finished or running kernel (host memory out):
 * submit, start and end times, slices pulled and blocks executed. The start
 * and end stamps give the kernel's execution time within the scheduling plan
 * (Section 2.2: the total execution time is the objective). KL_ENOTFOUND for
 * an unknown handle. */
int kl_get_stats(kl_runtime* rt, kl_handle h, kl_tenant_stats* out);

/* Statistics of the last retired run (host memory out): its kernel time, the
 * co-schedules chosen, and the idle, stage-barrier and planning time summed
 * over the CTAs (the scheduling overhead Section 3.1 asks to keep small).
 * KL_EINVAL on NULL. */
int kl_get_run_stats(kl_runtime* rt, kl_run_stats* out);

/* Phase log of the last retired run: the sequence of co-schedules
 * <K1, K2, size1, size2> that Algorithm 1 chose, in order (the scheduling
 * plan of Section 2.2), up to cap entries into out (host memory; may be NULL
 * when cap = 0); *n receives the number of phases the run logged, which may
 * exceed cap. */
int kl_get_phases(kl_runtime* rt, kl_phase* out, uint32_t cap, uint32_t* n);

/* Model inputs. kl_set_profiles: per-type profile (Table 1's R_m, the
 * uncoalesced fraction and sectors per access of Section 4.4 "uncoalesced
 * access", instructions per block, PUR and MUR of Section 4.3), measured by
 * profiling the kernel (Section 4.4, "getting the input"); profiles[t] is
 * type t, n_types <= KL_T_COUNT, copied. kl_set_model_params: the GPU
 * parameters of the virtual SM (Section 4.4, "multiple warp schedulers":
 * schedulers per SM; DRAM bandwidth and clock for B; the linear latency
 * parameters a0, b0 of the latency equation). Changing either invalidates the
 * cached CP table. KL_EINVAL on NULL or out-of-range values. */
int kl_set_profiles(kl_runtime* rt, const kl_profile* profiles, uint32_t n_types);
int kl_set_model_params(kl_runtime* rt, const kl_model_params* params);
int kl_get_model_params(kl_runtime* rt, kl_model_params* out);

/* CP table the device planner uses (Eq. cp from the Section 4.4 model, one
 * entry per type pair, the pruning of Section 4.3 in `allowed`):
 * cp[i*KL_T_COUNT+j] and slots for the first kernel of a (type i, type j)
 * pair at the runtime's slots per SM (the balanced ratio, Eq.
 * executiontime). Arrays of KL_T_COUNT^2 entries, host memory; any may be
 * NULL. */
int kl_get_cp_table(kl_runtime* rt, double* cp, uint32_t* slots_a, uint8_t* allowed);

/* Replace the model's table with given values (the OPT comparison of Section
 * 5.1: the same greedy planner, fed with CPs and slice ratios measured by
 * running every pair at every split). cp and slots_a as in kl_get_cp_table
 * (KL_T_COUNT x KL_T_COUNT, host memory, copied); slots_a entries in
 * [1, slots per SM - 1]; every pair is allowed (no pruning). NULL for both
 * returns to the model's table. KL_EINVAL on a split out of range. */
int kl_set_cp_table(kl_runtime* rt, const double* cp, const uint32_t* slots_a);

/* ------------------------------------------------------------ pure functions */

/* Per-kernel IPC (per SM = virtual-SM IPC x n_sched) of n kernels sharing a
 * virtual SM with warps[k] warps of kernel k (Eqs. modelIPC, ipc_k1, ipc_k2).
 * model_states 2 or 3. At most 4 kernels and 4096 joint states. */
int kl_model_ipc(const kl_model_params* gp, const kl_profile* profiles, const uint32_t* warps,
                 uint32_t n, uint32_t model_states, double* ipc_out);

/* Evaluate every split (a + b = slots, a, b >= 1) of a pair: concurrent IPCs,
 * CP (Eq. cp) and dT (Eq. executiontime), and the split chosen by `policy`.
 * Arrays have slots-1 entries, index a-1. solo_ipc[2] = IPC alone at `slots`. */
int kl_model_pair(const kl_model_params* gp, const kl_profile* pa, const kl_profile* pb,
                  uint32_t slots, uint32_t model_states, uint32_t policy, uint32_t fixed_a,
                  double* cipc_a, double* cipc_b, double* cp, double* dT, double* solo_ipc,
                  uint32_t* best_a);

/* A phase of n kernels (1..4) sharing every SM, kernel k on slots[k] of the
 * total_slots slots per SM (Section 2.2: a co-schedule of n >= 1 slices;
 * Section 4.4: the heterogeneous model handles more than two kernels; the
 * co-scheduler's phases run a pair plus the chain lane's kernel):
 * cipc_out[k] = concurrent IPC per SM, solo_out[k] = IPC alone at
 * total_slots, *cp_out = CP by Eq. cp with n terms. Host arrays of n entries.
 * KL_EINVAL on bad sizes or sum(slots) > total_slots. */
int kl_model_phase(const kl_model_params* gp, const kl_profile* profiles, const uint32_t* slots, uint32_t n,
                   uint32_t total_slots, uint32_t model_states, double* cipc_out, double* solo_out,
                   double* cp_out);

/* Greedy plan (Algorithm 1) of n kernels with types[i] and blocks[i] thread
 * blocks, all pending at time 0, simulated with the model's rates. Writes up
 * to cap phases and the predicted makespan in SM cycles. */
int kl_plan(const kl_model_params* gp, const kl_profile* type_profiles, uint32_t n_types,
            const uint32_t* types, const uint64_t* blocks, uint32_t n, uint32_t slots,
            uint32_t model_states, uint32_t policy, double alpha_p, double alpha_m,
            kl_phase* phases, double* phase_cycles, uint32_t cap, uint32_t* n_phases,
            double* makespan_cycles);

/* Number of pairs of n kernels removed by the pruning rule (Section 4.3). */
int kl_count_pruned(const double* pur, const double* mur, uint32_t n, double alpha_p,
                    double alpha_m, uint32_t* out);

/* ------------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory where they run work: frameworks whose caching
 * allocator has reserved the device memory up front (a raw cudaMalloc then
 * fails or fragments their pool), and latency-critical threads that must not
 * call cudaMalloc / cudaFree because those calls can synchronize the device.
 *
 * kl_run_noalloc runs descs[0..n) as ONE co-scheduled launch of the same
 * persistent kernel as kl_launch on `cuda_stream` (a cudaStream_t, may be
 * NULL) and returns after the run has completed: it synchronizes that stream.
 * It calls no cudaMalloc, cudaFree or other allocating routine: the device
 * queue, run state and phase log live in a fixed file-scope device array of
 * the library (KL_NOALLOC_SCRATCH_BYTES = 97,536 bytes, held by every GPU that
 * loads the library until the process exits), and the host-side descriptor
 * image lives on the caller's stack (about 23.5 KB).
 *   descs, n        kernel descriptors as for kl_submit, of the co-scheduler's
 *                   types (type < KL_T_MAIN_COUNT, else KL_EINVAL); 1 <= n <=
 *                   KL_NOALLOC_MAX_TENANTS, else KL_EOVERFLOW (n = 0: KL_EINVAL);
 *                   slice_blocks = 0 takes the runtime's built-in slice of the
 *                   type (no profiles are loaded here)
 *   cp_table        NULL, or KL_T_COUNT x KL_T_COUNT CP values by (type of the
 *                   lower-index kernel, type of the other) for the device planner;
 *                   NULL = all equal (pairs in submission order)
 *   slots_a_table   NULL, or slots per SM for the lower-index kernel of each
 *                   type pair (clamped to 1..slots-1); NULL = even split
 *   wait_limit_ns   bound of every device-side wait (0 = 2 s)
 *   states          NULL, or n entries receiving KL_DONE / KL_ERROR per kernel;
 *                   left untouched when the call returns an error before the
 *                   run's results are read back (a bad descriptor,
 *                   KL_EOVERFLOW, a failed CUDA call)
 * Returns KL_OK when every kernel completed, else a kl_status.
 * The first call on each device takes the device address of the array
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. Every call shares the array, which keeps the last
 * call's contents (each call rewrites what must start at zero); calls whose
 * GPU work overlaps race on it and must not be issued concurrently. */
#define KL_NOALLOC_MAX_TENANTS 64
#define KL_NOALLOC_SCRATCH_BYTES 97536
int kl_run_noalloc(const kl_kernel_desc* descs, uint32_t n, const double* cp_table,
                   const uint32_t* slots_a_table, void* cuda_stream, uint64_t wait_limit_ns,
                   int32_t* states);

/* Static text for a kl_status (no counterpart in the paper). */
const char* kl_strerror(int code);
/* KL_ABI_VERSION of the library that was loaded (no counterpart in the paper). */
int kl_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KERNELET_H */
