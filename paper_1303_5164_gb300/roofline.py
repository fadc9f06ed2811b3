"""Algorithmic work per tenant instance, for roofline fractions.

Bytes are the DRAM traffic the computation cannot avoid (every input read
once, every output written once); FLOPs count the binary32 operations of the
tenant's written definition. Measured traffic well above these means re-reads.
"""
from __future__ import annotations

import numpy as np

# binary32 operations per Black-Scholes option in the written recipe (two CND
# evaluations, one exp and one log of the Cody-Waite / atanh recipes)
BS_FLOPS_PER_OPTION = 93
ESCAPE_FLOPS_PER_ITER = 7


# the resource-heavy variants do their base kernel's work
BASE = {"bs255": "blackscholes", "hist1024": "hist256", "gemm_f32_big": "gemm_f32"}


def algo_bytes(name: str, inp: dict) -> int:
    name = BASE.get(name, name)
    if name == "testmix":
        return 4 * inp["iters"] * inp["mem"] * inp["nthreads"] + 4 * inp["nthreads"]
    if name == "gather":
        return 12 * inp["n"]
    if name == "blackscholes":
        return 28 * inp["n"]
    if name == "gemm_f32":
        return 4 * (inp["M"] * inp["K"] + inp["K"] * inp["N"] + inp["M"] * inp["N"])
    if name == "spmv_csr":
        return 8 * inp["nnz"] + 4 * (inp["nrows"] + 1) + 4 * inp["nrows"] + 4 * inp["ncols"]
    if name == "pchase":
        return 4 * inp["hops"] * inp["nchasers"] + 8 * inp["nchasers"]
    if name == "triad":
        return 12 * inp["n"]
    if name == "hist256":
        return inp["n"] + 1024
    if name == "escape":
        return 4 * inp["width"] * inp["height"]
    if name == "bitonic":
        return 8 * inp["n"]
    if name == "matadd":
        return 12 * inp["n"] * inp["n"]
    if name == "gemm_bf16":
        return 2 * (inp["M"] * inp["K"] + inp["N"] * inp["K"]) + 4 * inp["M"] * inp["N"]
    if name == "tea":
        return 16 * inp["n"]                      # 8 bytes in, 8 out per 64-bit block
    if name == "sad":
        D = 2 * inp["range"] + 1
        return 2 * inp["width"] * inp["height"] + 4 * (inp["width"] // 4) * (inp["height"] // 4) * D * D
    if name == "stencil":
        return 8 * inp["nx"] * inp["ny"] * inp["nz"]  # neighbours come from cache
    if name == "mriq":
        return 24 * inp["numK"] + 20 * inp["numX"]
    raise ValueError(name)


def _base(name):
    return BASE.get(name, name)


def tensor_flops(name: str, inp: dict) -> int:
    """Operations on the tensor cores (the BF16 GEMM: 2 M N K)."""
    if name == "gemm_bf16":
        return 2 * inp["M"] * inp["N"] * inp["K"]
    return 0


def fp32_flops(name: str, inp: dict, escape_iters: int | None = None) -> int:
    """binary32 operations on the FP32 pipe (integer tenants: 0)."""
    name = _base(name)
    if name == "testmix":
        return inp["iters"] * (inp["mem"] + 2 * inp["alu"]) * inp["nthreads"]
    if name == "gemm_f32":
        return 2 * inp["M"] * inp["N"] * inp["K"]
    if name == "blackscholes":
        return BS_FLOPS_PER_OPTION * inp["n"]
    if name == "spmv_csr":
        return 2 * inp["nnz"]
    if name == "triad":
        return 2 * inp["n"]
    if name == "escape":
        return ESCAPE_FLOPS_PER_ITER * int(escape_iters or 0)
    if name == "matadd":
        return inp["n"] * inp["n"]
    if name == "stencil":
        return 8 * inp["nx"] * inp["ny"] * inp["nz"]
    if name == "mriq":
        # per (point, sample): dot product 5, angle 1, reduction 4, polynomials 16, accumulation 4
        return 30 * inp["numK"] * inp["numX"]
    return 0


# lane operations (one issue slot of one of the SM's 128 lanes) per unit of work
ESCAPE_OPS_PER_ITER = 9          # x*x, y*y, x2+y2, compare, 2*x, *y, +cy, x2-y2, +cx
BITONIC_OPS_PER_EXCHANGE = 2     # min and max of the pair


def lane_ops(name: str, inp: dict, escape_iters: int | None = None) -> int:
    """Issue slots of the written definition, counted per lane: each binary32
    operation (a fused multiply-add once), integer min/max, shared-memory
    atomic, or load of a dependent chain takes one slot of one of the 128
    lanes of an SM. Set against numSM x 128 x f_SM slots per second this is
    the issue-bound time of tenants that are neither HBM- nor FFMA-bound
    (Black-Scholes, escape-time, the bitonic passes, TEA)."""
    name = _base(name)
    if name == "testmix":
        return inp["iters"] * (inp["mem"] + inp["alu"]) * inp["nthreads"]
    if name == "gemm_f32":
        return inp["M"] * inp["N"] * inp["K"]
    if name == "blackscholes":
        return BS_FLOPS_PER_OPTION * inp["n"]
    if name == "spmv_csr":
        return inp["nnz"]
    if name == "triad":
        return inp["n"]
    if name == "escape":
        return ESCAPE_OPS_PER_ITER * int(escape_iters or 0)
    if name == "bitonic":
        L = inp["log2n"]
        return BITONIC_OPS_PER_EXCHANGE * (inp["n"] // 2) * (L * (L + 1) // 2)
    if name == "hist256":
        return inp["n"]
    if name == "pchase":
        return inp["hops"] * inp["nchasers"]
    if name == "gather":
        return inp["n"]
    if name == "matadd":
        return inp["n"] * inp["n"]
    if name == "tea":
        return 32 * 10 * inp["n"]      # 32 cycles of two 5-operation Feistel rounds
    if name == "stencil":
        return 8 * inp["nx"] * inp["ny"] * inp["nz"]
    if name == "mriq":
        return 30 * inp["numK"] * inp["numX"]
    if name == "sad":
        D = 2 * inp["range"] + 1
        return 3 * 16 * (inp["width"] // 4) * (inp["height"] // 4) * D * D  # sub, abs, add per pixel
    return 0


def lane_peak(n_sm: int, f_sm_hz: float) -> float:
    """Issue slots per second: 4 schedulers x 32 lanes per SM per cycle."""
    return n_sm * 128 * f_sm_hz


def fp32_peak_flops(n_sm: int, f_sm_hz: float) -> float:
    """FFMA peak: 128 binary32 lanes per SM, 2 operations per fused multiply-add."""
    return n_sm * 128 * 2 * f_sm_hz
