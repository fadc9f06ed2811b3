"""ctypes front end of the C tenant oracle (oracle/tenants.c). Test infrastructure.

`build()` compiles tenants.c with the host C compiler (plain -O2, no FP
contraction, no fast-math) into oracle/_build/liboracle_tenants.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tenants.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_tenants.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L = C.c_int64
        _lib.or_expf.argtypes = [C.c_float]; _lib.or_expf.restype = C.c_float
        _lib.or_logf.argtypes = [C.c_float]; _lib.or_logf.restype = C.c_float
        _lib.or_blackscholes.argtypes = [f32p] * 7 + [L]
        _lib.or_gather.argtypes = [i32p, i32p, i32p, L, L]
        _lib.or_testmix.argtypes = [f32p, f32p, L, L, L, L, L, C.c_float, C.c_float]
        _lib.or_gemm_f32.argtypes = [f32p, f32p, f32p, L, L, L]
        _lib.or_gemm_f32_sample.argtypes = [f32p, f32p, i64p, i64p, f32p, L, L, L]
        _lib.or_spmv_csr.argtypes = [i32p, i32p, f32p, f32p, f32p, f64p, f64p, L]
        _lib.or_pchase.argtypes = [i32p, i32p, i32p, L, L]
        _lib.or_triad.argtypes = [f32p, f32p, f32p, C.c_float, L, L]
        _lib.or_hist256.argtypes = [u8p, u32p, L]
        _lib.or_escape.argtypes = [u32p, L, L, L, C.c_float, C.c_float, C.c_float, C.c_float, L, L]
        _lib.or_sort_u32.argtypes = [u32p, u32p, L]
        _lib.or_matadd.argtypes = [f32p, f32p, f32p, L]
        _lib.or_tea.argtypes = [u32p, u32p, u32p, L]
        _lib.or_sad.argtypes = [u8p, u8p, u32p, L, L, L]
        _lib.or_stencil7.argtypes = [f32p, f32p, L, L, L, C.c_float, C.c_float]
        fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        _lib.or_sincosf.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        _lib.or_mriq.argtypes = [f32p] * 11 + [L, i64p, L]
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def expf(x: float) -> float:
    return lib().or_expf(float(x))


def logf(x: float) -> float:
    return lib().or_logf(float(x))


def blackscholes(S, K, r, v, T):
    n = len(S)
    call = np.empty(n, np.float32)
    put = np.empty(n, np.float32)
    lib().or_blackscholes(_c(S, np.float32), _c(K, np.float32), _c(r, np.float32),
                          _c(v, np.float32), _c(T, np.float32), call, put, n)
    return call, put


def testmix(inp):
    """The Section 4.3 testing kernel's definition (oracle/tenants.c or_testmix)."""
    out = np.empty(inp["nthreads"], np.float32)
    lib().or_testmix(_c(inp["data"], np.float32), out, inp["n_in"], inp["nthreads"], inp["iters"], inp["mem"],
                     inp["alu"], float(inp["c1"]), float(inp["c2"]))
    return out


def gather(a, idx, lo=0, hi=None, out=None):
    n = len(idx)
    hi = n if hi is None else hi
    out = np.zeros(n, np.int32) if out is None else out
    lib().or_gather(_c(a, np.int32), _c(idx, np.int32), out, lo, hi)
    return out


def gemm_f32(A, B):
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Cm = np.empty((M, N), np.float32)
    lib().or_gemm_f32(_c(A, np.float32), _c(B, np.float32), Cm, M, N, K)
    return Cm


def gemm_f32_sample(A, B, ii, jj):
    M, K = A.shape
    N = B.shape[1]
    out = np.empty(len(ii), np.float32)
    lib().or_gemm_f32_sample(_c(A, np.float32), _c(B, np.float32), _c(ii, np.int64),
                             _c(jj, np.int64), out, len(ii), N, K)
    return out


def gemm_f32_exact(A, B):
    """The definition's exact value C = A B for binary32 inputs, in binary64
    (one library matmul; each product of two binary32 values is exact in
    binary64), and sum_k |a_ik b_kj|, the scale of the binary32 chain's
    rounding error: |C_chain - C| <= K 2^-24 sum_k |a_ik b_kj| per entry.
    For checking GEMMs too large for the chain loop, entry by entry."""
    a = np.asarray(A, dtype=np.float64)
    b = np.asarray(B, dtype=np.float64)
    return a @ b, np.abs(a) @ np.abs(b)


def bf16_to_f64(bits):
    """Value of bfloat16 bit patterns: the upper half of a binary32 word."""
    b = np.ascontiguousarray(bits, dtype=np.uint16)
    return (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def gemm_bf16(A, Bt):
    """C = A B^T of bfloat16 inputs, by definition in binary64 (a product of
    two bfloat16 values is exact in binary64; the sum is one library matmul).
    Also returns sum_k |a_ik b_jk|, the scale of the accumulation error bound."""
    a = bf16_to_f64(A)
    b = bf16_to_f64(Bt)
    return a @ b.T, np.abs(a) @ np.abs(b).T


def gemm_bf16_sample(A, Bt, ii, jj):
    """Entries (ii[t], jj[t]) of gemm_bf16, each a binary64 dot product."""
    c = np.empty(len(ii))
    s = np.empty(len(ii))
    for t, (i, j) in enumerate(zip(ii, jj)):
        a = bf16_to_f64(A[i])
        b = bf16_to_f64(Bt[j])
        c[t] = float(np.dot(a, b))
        s[t] = float(np.dot(np.abs(a), np.abs(b)))
    return c, s


def spmv_csr(rowptr, col, val, x):
    n = len(rowptr) - 1
    y32 = np.empty(n, np.float32)
    y64 = np.empty(n, np.float64)
    asum = np.empty(n, np.float64)
    lib().or_spmv_csr(_c(rowptr, np.int32), _c(col, np.int32), _c(val, np.float32),
                      _c(x, np.float32), y32, y64, asum, n)
    return y32, y64, asum


def pchase(nxt, start, hops):
    end = np.empty(len(start), np.int32)
    lib().or_pchase(_c(nxt, np.int32), _c(start, np.int32), end, len(start), hops)
    return end


def triad(b, c, s, lo=0, hi=None, out=None):
    n = len(b)
    hi = n if hi is None else hi
    out = np.zeros(n, np.float32) if out is None else out
    lib().or_triad(_c(b, np.float32), _c(c, np.float32), out, float(s), lo, hi)
    return out


def hist256(data):
    h = np.empty(256, np.uint32)
    lib().or_hist256(_c(data, np.uint8), h, len(data))
    return h


def escape(width, height, max_iter, x0, y0, dx, dy, row_lo=0, row_hi=None, out=None):
    row_hi = height if row_hi is None else row_hi
    out = np.zeros(width * height, np.uint32) if out is None else out
    lib().or_escape(out, width, height, max_iter, float(x0), float(y0), float(dx), float(dy),
                    row_lo, row_hi)
    return out


def sort_u32(data):
    out = np.empty(len(data), np.uint32)
    lib().or_sort_u32(_c(data, np.uint32), out, len(data))
    return out


def matadd(a, b):
    n = a.shape[0]
    c = np.empty((n, n), np.float32)
    lib().or_matadd(_c(a, np.float32), _c(b, np.float32), c, n)
    return c


def tea(words, key, n):
    out = np.empty(2 * n, np.uint32)
    lib().or_tea(_c(words, np.uint32), out, _c(key, np.uint32), n)
    return out


def sad(cur, ref, width, height, rng):
    D = 2 * rng + 1
    out = np.empty((width // 4) * (height // 4) * D * D, np.uint32)
    lib().or_sad(_c(cur, np.uint8), _c(ref, np.uint8), out, width, height, rng)
    return out


def stencil7(grid, nx, ny, nz, c0, c1):
    out = np.empty(nx * ny * nz, np.float32)
    lib().or_stencil7(_c(grid, np.float32), out, nx, ny, nz, float(c0), float(c1))
    return out


def sincosf(a):
    s, c = C.c_float(), C.c_float()
    lib().or_sincosf(float(a), C.byref(s), C.byref(c))
    return s.value, c.value


def mriq(inp, points=None):
    """phiMag for every sample and (Qr, Qi) at `points` (default: every point)."""
    numK, numX = inp["numK"], inp["numX"]
    pts = np.arange(numX, dtype=np.int64) if points is None else np.asarray(points, np.int64)
    pm = np.empty(numK, np.float32)
    qr = np.empty(len(pts), np.float32)
    qi = np.empty(len(pts), np.float32)
    f = lambda k: _c(inp[k], np.float32)
    lib().or_mriq(f("kx"), f("ky"), f("kz"), f("phiR"), f("phiI"), pm, f("x"), f("y"), f("z"), qr, qi, numK,
                  _c(pts, np.int64), len(pts))
    return pm, qr, qi
