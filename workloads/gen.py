"""Seeded synthetic inputs for every tenant type (SplitMix64, vectorised numpy).

The paper's benchmark suites (CUDA SDK, Parboil, CUSP; Section 5.1, Table 4)
are not available; these generators stand in for them with the shapes and
value distributions listed in the workload tables of the design notes:

* Black-Scholes: S, K ~ U[10,100], r ~ U[0.01,0.05], sigma ~ U[0.1,0.5],
  T ~ U[0.25,2]  (float32, structure-of-arrays)
* gather: a = seeded int32, idx = seeded random permutation
* FP32 GEMM: A, B ~ N(0,1), row-major
* CSR SpMV: row length ~ truncated Pareto (pdf ~ d^-2.5) on [x_m, 8192],
  x_m solved for mean 16; columns stratified-uniform over integer strata (distinct, sorted);
  val, x ~ N(0,1)
* pointer chase: one random N-cycle (random order, each element points to
  its successor); T chasers start at t*floor(N/T)
* triad: b, c ~ N(0,1), s = 3
* histogram: uint8 values, rank k in 1..256 with P ~ k^-1.1, value =
  seeded permutation of the rank
* escape-time: no input (pixel grid over [-2,0.5] x [-1.25,1.25])
* bitonic sort: uint32 ~ U[0, 2^32)

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) is evaluated counter-style: output i of stream s is
mix(s + (i+1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "splitmix64", "stream_seed", "uniform01", "normal_f32",
    "gen_blackscholes", "gen_gather", "gen_gemm_f32", "gen_spmv_csr",
    "gen_pchase", "gen_triad", "gen_hist256", "gen_escape", "gen_bitonic",
    "gen_matadd", "gen_tenant", "TENANT_NAMES", "spmv_xm_for_mean",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

TENANT_NAMES = ["gather", "blackscholes", "gemm_f32", "spmv_csr", "pchase",
                "triad", "hist256", "escape", "bitonic", "matadd"]


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream started at `seed`."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, n, _CHUNK):
            hi = min(n, lo + _CHUNK)
            i = np.arange(offset + lo + 1, offset + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix(s + i * _GOLDEN)
    return out


def stream_seed(config_seed: int, tenant_index: int, tag: str) -> int:
    """Independent stream seed for (config, tenant instance, array tag)."""
    h = 0xCBF29CE484222325
    for ch in f"{config_seed}/{tenant_index}/{tag}".encode():
        h = ((h ^ ch) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        return int(_mix(np.array([h], dtype=np.uint64))[0])


def uniform01(seed: int, n: int) -> np.ndarray:
    """float64 in [0,1) from the top 53 bits."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _uniform_f32(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    u = uniform01(seed, n)
    return (lo + (hi - lo) * u).astype(np.float32)


def normal_f32(seed: int, n: int) -> np.ndarray:
    """N(0,1) by Box-Muller on pairs of SplitMix64 uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[:m]          # (0,1]
    u2 = u[m:]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[:m] = r * np.cos(2.0 * math.pi * u2)
    z[m:] = r * np.sin(2.0 * math.pi * u2)
    return z[:n].astype(np.float32)


def _perm(seed: int, n: int) -> np.ndarray:
    return np.argsort(splitmix64(seed, n), kind="stable").astype(np.int64)


# --------------------------------------------------------------------------- tenants

def gen_blackscholes(cs: int, ti: int, n: int) -> dict:
    return dict(
        S=_uniform_f32(stream_seed(cs, ti, "S"), n, 10.0, 100.0),
        K=_uniform_f32(stream_seed(cs, ti, "K"), n, 10.0, 100.0),
        r=_uniform_f32(stream_seed(cs, ti, "r"), n, 0.01, 0.05),
        v=_uniform_f32(stream_seed(cs, ti, "v"), n, 0.1, 0.5),
        T=_uniform_f32(stream_seed(cs, ti, "T"), n, 0.25, 2.0),
        n=n)


def gen_gather(cs: int, ti: int, n: int) -> dict:
    a = (splitmix64(stream_seed(cs, ti, "a"), n) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    idx = _perm(stream_seed(cs, ti, "idx"), n).astype(np.int32)
    return dict(a=a, idx=idx, n=n)


def gen_gemm_f32(cs: int, ti: int, M: int, N: int, K: int) -> dict:
    A = normal_f32(stream_seed(cs, ti, "A"), M * K).reshape(M, K)
    B = normal_f32(stream_seed(cs, ti, "B"), K * N).reshape(K, N)
    return dict(A=A, B=B, M=M, N=N, K=K)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns of float32 values, round to nearest even (the
    input distribution of the BF16 GEMM: N(0,1) values that bfloat16 holds)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def gen_gemm_bf16(cs: int, ti: int, M: int, N: int, K: int) -> dict:
    """A [M][K] and Bt [N][K] (B column-major) as bfloat16 bits from N(0,1)."""
    A = bf16_bits(normal_f32(stream_seed(cs, ti, "A"), M * K)).reshape(M, K)
    Bt = bf16_bits(normal_f32(stream_seed(cs, ti, "B"), N * K)).reshape(N, K)
    return dict(A=A, Bt=Bt, M=M, N=N, K=K)


def _u32(seed: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def gen_tea(cs: int, ti: int, n: int) -> dict:
    """n 64-bit plaintext blocks (2n uint32 words) and a 128-bit key."""
    return dict(words=_u32(stream_seed(cs, ti, "words"), 2 * n), key=_u32(stream_seed(cs, ti, "key"), 4), n=n)


def gen_sad(cs: int, ti: int, width: int = 1920, height: int = 1072, range: int = 8) -> dict:
    """Two 8-bit frames: random luma, and the same frame moved by one global
    motion vector within the search range plus small noise (so every block has
    a clear SAD minimum, as between consecutive video frames)."""
    cur = (_u32(stream_seed(cs, ti, "cur"), width * height) >> np.uint32(24)).astype(np.uint8).reshape(height, width)
    mv = _u32(stream_seed(cs, ti, "mv"), 2) % np.uint32(2 * range + 1)
    dx, dy = int(mv[0]) - range, int(mv[1]) - range
    noise = (_u32(stream_seed(cs, ti, "noise"), width * height) >> np.uint32(29)).astype(np.int16).reshape(height, width)
    ref = np.clip(np.roll(cur, (dy, dx), axis=(0, 1)).astype(np.int16) + noise - 3, 0, 255).astype(np.uint8)
    return dict(cur=cur, ref=ref, width=width, height=height, range=range, mv=(dx, dy))


def gen_stencil(cs: int, ti: int, nx: int, ny: int, nz: int, c0: float = 0.25, c1: float = 0.125) -> dict:
    """A binary32 grid of N(0,1) values and the stencil's two coefficients."""
    return dict(grid=normal_f32(stream_seed(cs, ti, "grid"), nx * ny * nz).reshape(nz, ny, nx),
                nx=nx, ny=ny, nz=nz, c0=c0, c1=c1)


def gen_mriq(cs: int, ti: int, numK: int, numX: int) -> dict:
    """k-space samples (coordinates U[-1/2, 1/2), phi ~ N(0,1)) and image
    points with coordinates U[-8, 8)."""
    return dict(kx=_uniform_f32(stream_seed(cs, ti, "kx"), numK, -0.5, 0.5),
                ky=_uniform_f32(stream_seed(cs, ti, "ky"), numK, -0.5, 0.5),
                kz=_uniform_f32(stream_seed(cs, ti, "kz"), numK, -0.5, 0.5),
                phiR=normal_f32(stream_seed(cs, ti, "phiR"), numK),
                phiI=normal_f32(stream_seed(cs, ti, "phiI"), numK),
                x=_uniform_f32(stream_seed(cs, ti, "x"), numX, -8.0, 8.0),
                y=_uniform_f32(stream_seed(cs, ti, "y"), numX, -8.0, 8.0),
                z=_uniform_f32(stream_seed(cs, ti, "z"), numX, -8.0, 8.0), numK=numK, numX=numX)


def spmv_xm_for_mean(mean: float = 16.0, alpha: float = 2.5, dmax: int = 8192) -> float:
    """Lower bound x_m of a Pareto(pdf ~ x^-alpha) truncated at dmax+1 such
    that E[floor(X)] = mean (bisection on the closed-form expectation)."""
    a1 = alpha - 1.0

    def mean_floor(xm: float) -> float:
        # E[floor X] = sum_{k>=1} P(X >= k) over the truncated law
        top = dmax + 1.0
        norm = xm ** -a1 - top ** -a1
        ks = np.arange(1, dmax + 1, dtype=np.float64)
        surv = np.where(ks <= xm, 1.0, (np.maximum(ks, xm) ** -a1 - top ** -a1) / norm)
        return float(surv.sum())

    lo, hi = 1.0, 200.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if mean_floor(mid) < mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def gen_spmv_csr(cs: int, ti: int, nrows: int, ncols: int | None = None,
                 mean_nnz: float = 16.0, dmax: int = 8192) -> dict:
    ncols = nrows if ncols is None else ncols
    dmax = min(dmax, ncols)
    xm = spmv_xm_for_mean(mean_nnz, 2.5, dmax)
    u = uniform01(stream_seed(cs, ti, "deg"), nrows)
    a1 = 1.5
    top = dmax + 1.0
    # inverse CDF of the truncated Pareto
    x = (xm ** -a1 - u * (xm ** -a1 - top ** -a1)) ** (-1.0 / a1)
    deg = np.clip(np.floor(x), 1, dmax).astype(np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    nnz = int(rowptr[-1])
    row_of = np.repeat(np.arange(nrows, dtype=np.int64), deg)
    j = np.arange(nnz, dtype=np.int64) - rowptr[row_of]
    uc = uniform01(stream_seed(cs, ti, "col"), nnz)
    d = deg[row_of]
    # integer strata [floor(j n/d), floor((j+1) n/d)) are disjoint and non-empty
    lo = (j * ncols) // d
    hi = ((j + 1) * ncols) // d
    col = lo + np.floor(uc * (hi - lo)).astype(np.int64)
    col = np.minimum(col, hi - 1)
    val = normal_f32(stream_seed(cs, ti, "val"), nnz)
    xv = normal_f32(stream_seed(cs, ti, "x"), ncols)
    return dict(rowptr=rowptr.astype(np.int32), col=col.astype(np.int32), val=val,
                x=xv, nrows=nrows, ncols=ncols, nnz=nnz)


def gen_pchase(cs: int, ti: int, N: int, nchasers: int, hops: int) -> dict:
    order = _perm(stream_seed(cs, ti, "cycle"), N)
    nxt = np.empty(N, dtype=np.int32)
    nxt[order] = np.roll(order, -1).astype(np.int32)
    stride = N // nchasers if nchasers <= N else 1
    start = ((np.arange(nchasers, dtype=np.int64) * stride) % N).astype(np.int32)
    return dict(next=nxt, start=start, N=N, nchasers=nchasers, hops=hops)


def gen_triad(cs: int, ti: int, n: int, s: float = 3.0) -> dict:
    return dict(b=normal_f32(stream_seed(cs, ti, "b"), n),
                c=normal_f32(stream_seed(cs, ti, "c"), n), s=np.float32(s), n=n)


def gen_hist256(cs: int, ti: int, n: int, zipf_s: float = 1.1) -> dict:
    ranks = np.arange(1, 257, dtype=np.float64)
    p = ranks ** -zipf_s
    cdf = np.cumsum(p / p.sum())
    cdf[-1] = 1.0
    u = uniform01(stream_seed(cs, ti, "data"), n)
    rank = np.minimum(np.searchsorted(cdf, u, side="right"), 255)
    value_of_rank = _perm(stream_seed(cs, ti, "map"), 256).astype(np.uint8)
    return dict(data=value_of_rank[rank], n=n)


def gen_escape(cs: int, ti: int, width: int = 2048, height: int = 2048,
               max_iter: int = 256) -> dict:
    # window [-2, 0.5] x [-1.25, 1.25]; pixel centres at (j+0.5)*dx
    return dict(width=width, height=height, max_iter=max_iter,
                x0=np.float32(-2.0), y0=np.float32(-1.25),
                dx=np.float32(2.5 / width), dy=np.float32(2.5 / height))


def gen_bitonic(cs: int, ti: int, log2n: int) -> dict:
    n = 1 << log2n
    keys = (splitmix64(stream_seed(cs, ti, "keys"), n) >> np.uint64(32)).astype(np.uint32)
    return dict(data=keys, log2n=log2n, n=n)


def gen_matadd(cs: int, ti: int, n: int = 256) -> dict:
    return dict(a=normal_f32(stream_seed(cs, ti, "a"), n * n).reshape(n, n),
                b=normal_f32(stream_seed(cs, ti, "b"), n * n).reshape(n, n), n=n)


def gen_testmix(cs: int, ti: int, log2_in: int, nthreads: int, iters: int, mem: int, alu: int,
                c1: float = 0.999, c2: float = 0.001) -> dict:
    """Input of the tunable testing kernel: 2^log2_in values N(0,1) and the
    loop counts and coefficients that set its memory / arithmetic mix."""
    n_in = 1 << log2_in
    return dict(data=normal_f32(stream_seed(cs, ti, "in"), n_in), n_in=n_in, nthreads=nthreads, iters=iters,
                mem=mem, alu=alu, c1=np.float32(c1), c2=np.float32(c2))


def gen_tenant(name: str, cs: int, ti: int, **size) -> dict:
    # the resource-heavy variants take the inputs of the kernel they vary
    fn = {"gather": gen_gather, "blackscholes": gen_blackscholes,
          "gemm_f32": gen_gemm_f32, "spmv_csr": gen_spmv_csr, "pchase": gen_pchase,
          "triad": gen_triad, "hist256": gen_hist256, "escape": gen_escape,
          "bitonic": gen_bitonic, "matadd": gen_matadd, "gemm_bf16": gen_gemm_bf16, "tea": gen_tea,
          "sad": gen_sad, "stencil": gen_stencil, "mriq": gen_mriq, "testmix": gen_testmix,
          "bs255": gen_blackscholes, "hist1024": gen_hist256, "gemm_f32_big": gen_gemm_f32}[name]
    return fn(cs, ti, **size)
