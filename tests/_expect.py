"""Expected tenant outputs from the CPU oracle, and the comparisons the parity
tests use (bit-exact except the SpMV reduction, whose tolerance is derived
from its summation depth)."""
import math

import numpy as np

from oracle import tenants as OT

U = 2.0 ** -24    # unit roundoff of binary32


# the resource-heavy variants compute their base kernel's definition
BASE = {"bs255": "blackscholes", "hist1024": "hist256", "gemm_f32_big": "gemm_f32"}


def expected(name: str, inp: dict) -> dict:
    name = BASE.get(name, name)
    if name == "testmix":
        return {"out": OT.testmix(inp)}
    if name == "gather":
        return {"out": OT.gather(inp["a"], inp["idx"])}
    if name == "blackscholes":
        c, p = OT.blackscholes(inp["S"], inp["K"], inp["r"], inp["v"], inp["T"])
        return {"call": c, "put": p}
    if name == "gemm_f32":
        return {"C": OT.gemm_f32(inp["A"], inp["B"])}
    if name == "spmv_csr":
        y32, y64, asum = OT.spmv_csr(inp["rowptr"], inp["col"], inp["val"], inp["x"])
        return {"y": y32, "_y64": y64, "_asum": asum}
    if name == "pchase":
        return {"end": OT.pchase(inp["next"], inp["start"], inp["hops"])}
    if name == "triad":
        return {"a": OT.triad(inp["b"], inp["c"], inp["s"])}
    if name == "hist256":
        return {"hist": OT.hist256(inp["data"])}
    if name == "escape":
        return {"count": OT.escape(inp["width"], inp["height"], inp["max_iter"], inp["x0"], inp["y0"],
                                   inp["dx"], inp["dy"])}
    if name == "bitonic":
        return {"out": OT.sort_u32(inp["data"])}
    if name == "matadd":
        return {"c": OT.matadd(inp["a"], inp["b"])}
    if name == "gemm_bf16":
        c64, cabs = OT.gemm_bf16(inp["A"], inp["Bt"])
        return {"_C64": c64, "_Cabs": cabs}
    if name == "tea":
        return {"out": OT.tea(inp["words"], inp["key"], inp["n"])}
    if name == "sad":
        return {"sad": OT.sad(inp["cur"], inp["ref"], inp["width"], inp["height"], inp["range"])}
    if name == "stencil":
        return {"out": OT.stencil7(inp["grid"], inp["nx"], inp["ny"], inp["nz"], inp["c0"], inp["c1"])}
    if name == "mriq":
        pm, qr, qi = OT.mriq(inp)
        return {"phiMag": pm, "Qr": qr, "Qi": qi}
    raise ValueError(name)


LARGE_GEMM_FLOPS = 1 << 28   # FP32 GEMMs above this go through check_gemm_f32_large


def expected_for_job(job):
    """Worker of a process pool: the oracle's outputs for one job
    (name, config seed, tenant index, size), regenerating its seeded inputs;
    None for FP32 GEMMs above LARGE_GEMM_FLOPS (checked in the parent)."""
    from workloads import gen
    name, cs, ti, size = job
    if name in ("gemm_f32", "gemm_f32_big") and 2 * size["M"] * size["N"] * size["K"] > LARGE_GEMM_FLOPS:
        return None
    OT.build()
    return expected(name, gen.gen_tenant(name, cs, ti, **size))


def gemm_bf16_bound(K, cabs):
    """|C_gpu - C_exact| <= K * 2^-23 * sum_k |a b|: the products of bfloat16
    values are exact in binary32, and each of the at most K binary32 additions
    of the accumulation (whatever order and grouping the tensor cores use, and
    whether they round to nearest or truncate) errs by less than one ulp of a
    partial sum, itself at most sum_k |a b|."""
    return K * 2.0 ** -23 * cabs


SPMV_LONG = 128


def spmv_bound(rowptr, asum):
    """|y_gpu - y_exact| <= depth * u * sum|a x| per row (Higham's bound for a
    summation tree of that depth): rows up to 128 non-zeros run 8 fused chains
    of ceil(len/8) terms and 3 butterfly adds; longer rows run 256 chains of
    ceil(len/256) terms, a 5-level warp butterfly and a 3-level tree."""
    deg = np.diff(rowptr.astype(np.int64))
    depth = np.where(deg > SPMV_LONG, np.ceil(deg / 256.0) + 9.0, np.ceil(deg / 8.0) + 4.0)
    return depth * U * asum


def same_bits(a, b) -> bool:
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    if a.shape != b.shape:
        return False
    if a.dtype.kind == "f":
        return np.array_equal(a.view(np.uint32 if a.itemsize == 4 else np.uint64),
                              b.astype(a.dtype).view(np.uint32 if a.itemsize == 4 else np.uint64))
    return np.array_equal(a, b.astype(a.dtype) if a.dtype != b.dtype else b)


def check_gemm_f32_large(inp: dict, got_C, n_samples: int = 256, seed: int = 0, exact=None):
    """An FP32 GEMM too large for the chain oracle's loop: every entry within
    K 2^-24 sum|ab| of the binary64 value of the definition, and sampled
    entries (every tile corner of the first and last tile rows and columns,
    plus random ones) bit for bit against the chain oracle. `exact`: the
    (value, scale) pair of OT.gemm_f32_exact when already computed."""
    A, B = inp["A"], inp["B"]
    M, K = A.shape
    N = B.shape[1]
    c = np.asarray(got_C, dtype=np.float32).reshape(M, N)
    c64, cabs = exact if exact is not None else OT.gemm_f32_exact(A, B)
    err = np.abs(c.astype(np.float64) - c64)
    bad = np.argwhere(err > K * U * cabs)
    assert len(bad) == 0, f"gemm_f32 entries over the chain bound: {bad[:5].tolist()}"
    rng = np.random.default_rng(seed)
    ii = [0, M - 1, min(63, M - 1), min(64, M - 1), M - 1]
    jj = [0, N - 1, min(63, N - 1), min(64, N - 1), 0]
    ii = np.concatenate([ii, rng.integers(0, M, n_samples)]).astype(np.int64)
    jj = np.concatenate([jj, rng.integers(0, N, n_samples)]).astype(np.int64)
    want = OT.gemm_f32_sample(A, B, ii, jj)
    assert same_bits(c[ii, jj], want), "gemm_f32 sampled entries differ from the chain oracle"


def check(name: str, inp: dict, got: dict, exp: dict):
    """Raises AssertionError with a short reason when `got` misses the bar."""
    name = BASE.get(name, name)
    if name == "gemm_bf16":
        c = got["C"].astype(np.float64).reshape(exp["_C64"].shape)
        err = np.abs(c - exp["_C64"])
        bound = gemm_bf16_bound(inp["K"], exp["_Cabs"])
        bad = np.argwhere(err > bound)
        assert len(bad) == 0, f"gemm_bf16 entries over bound: {bad[:5].tolist()} err {err[tuple(bad[:5].T)]}"
        return
    if name == "spmv_csr":
        y = got["y"].astype(np.float64)
        bound = spmv_bound(inp["rowptr"], exp["_asum"])
        err = np.abs(y - exp["_y64"])
        bad = np.nonzero(err > bound)[0]
        assert len(bad) == 0, f"spmv rows over bound: {bad[:5]} err {err[bad[:5]]} bound {bound[bad[:5]]}"
        return
    for k, v in exp.items():
        g = got[k].reshape(v.shape) if got[k].size == v.size else got[k]
        if not same_bits(g, v):
            gg = np.asarray(g).ravel()
            vv = np.asarray(v).ravel()
            diff = np.nonzero(gg != vv)[0] if gg.shape == vv.shape else []
            raise AssertionError(f"{name}.{k}: {len(diff)} elements differ, first {list(diff[:5])}: "
                                 f"got {gg[diff[:3]] if len(diff) else gg.shape} want "
                                 f"{vv[diff[:3]] if len(diff) else vv.shape}")
