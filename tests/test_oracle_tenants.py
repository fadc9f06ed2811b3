"""Pins for the tenant oracle (oracle/tenants.c) against closed forms,
textbook values, invariants and independent library routines."""
import math

import numpy as np
import pytest

from workloads import gen


def _ulp32(x: float) -> float:
    x = abs(np.float32(x))
    return float(np.spacing(x))


def test_expf_against_binary64(oracle_tenants):
    # the Cody-Waite + Taylor recipe is within 2 ulp of the correctly rounded value
    xs = np.concatenate([np.linspace(-87.0, 88.0, 20001), np.linspace(-1.0, 1.0, 5001),
                         np.linspace(-0.5, 0.0, 1001)]).astype(np.float32)
    worst = 0.0
    for x in xs:
        got = oracle_tenants.expf(float(x))
        ref = math.exp(float(x))
        worst = max(worst, abs(got - ref) / _ulp32(ref))
    assert worst <= 2.0, worst
    assert oracle_tenants.expf(0.0) == 1.0
    assert oracle_tenants.expf(-200.0) == 0.0
    assert math.isinf(oracle_tenants.expf(100.0))
    # subnormal range keeps a sensible value
    assert abs(oracle_tenants.expf(-95.0) - math.exp(-95.0)) <= 2 * 2.0 ** -149


def test_logf_against_binary64(oracle_tenants):
    xs = np.concatenate([np.geomspace(1e-30, 1e30, 20001), np.linspace(0.05, 12.0, 20001)]).astype(np.float32)
    worst = 0.0
    for x in xs:
        got = oracle_tenants.logf(float(x))
        ref = math.log(float(x))
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / _ulp32(ref))
    assert worst <= 2.0, worst
    assert oracle_tenants.logf(1.0) == 0.0
    assert math.isinf(oracle_tenants.logf(0.0))


def test_blackscholes_textbook_value(oracle_tenants):
    # S = K = 100, r = 5%, sigma = 20%, T = 1 year: call 10.4506, put 5.5735
    one = lambda v: np.array([v], np.float32)
    c, p = oracle_tenants.blackscholes(one(100), one(100), one(0.05), one(0.2), one(1.0))
    assert abs(c[0] - 10.4506) < 1e-3
    assert abs(p[0] - 5.5735) < 1e-3


def test_blackscholes_closed_form_and_parity(oracle_tenants):
    d = gen.gen_blackscholes(1, 0, 4096)
    c, p = oracle_tenants.blackscholes(d["S"], d["K"], d["r"], d["v"], d["T"])
    S, K, r, v, T = (d[k].astype(np.float64) for k in "SKrvT")
    # binary64 closed form with the exact normal CDF
    d1 = (np.log(S / K) + (r + 0.5 * v * v) * T) / (v * np.sqrt(T))
    d2 = d1 - v * np.sqrt(T)
    N = lambda x: 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    c64 = S * N(d1) - K * np.exp(-r * T) * N(d2)
    p64 = K * np.exp(-r * T) * N(-d2) - S * N(-d1)
    # A&S 26.2.17 error 7.5e-8 times S, K <= 100, plus binary32 rounding
    assert np.max(np.abs(c - c64)) < 2e-4
    assert np.max(np.abs(p - p64)) < 2e-4
    # put-call parity C - P = S - K e^{-rT}
    par = (c.astype(np.float64) - p) - (S - K * np.exp(-r * T))
    assert np.max(np.abs(par)) < 1e-4 * 100


def test_gather_permutation_invariants(oracle_tenants):
    d = gen.gen_gather(1, 1, 1 << 14)
    out = oracle_tenants.gather(d["a"], d["idx"])
    assert np.array_equal(np.sort(out), np.sort(d["a"]))        # permutation of a
    back = np.empty_like(out)
    back[d["idx"]] = out                                          # scatter recovers a
    assert np.array_equal(back, d["a"])


def test_gemm_identity_integer_and_error_bound(oracle_tenants):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((37, 29)).astype(np.float32)
    I = np.eye(29, dtype=np.float32)
    assert np.array_equal(oracle_tenants.gemm_f32(A, I), A)      # identity B gives A exactly
    Ai = rng.integers(-8, 9, (33, 70)).astype(np.float32)
    Bi = rng.integers(-8, 9, (70, 41)).astype(np.float32)
    assert np.array_equal(oracle_tenants.gemm_f32(Ai, Bi),
                          (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float32))
    d = gen.gen_gemm_f32(2, 0, 64, 48, 300)
    C = oracle_tenants.gemm_f32(d["A"], d["B"])
    C64 = d["A"].astype(np.float64) @ d["B"].astype(np.float64)
    bound = 300 * 2.0 ** -24 * (np.abs(d["A"]).astype(np.float64) @ np.abs(d["B"]).astype(np.float64))
    assert np.all(np.abs(C - C64) <= bound)
    ii = np.array([0, 63, 17]); jj = np.array([0, 47, 5])
    assert np.array_equal(oracle_tenants.gemm_f32_sample(d["A"], d["B"], ii, jj), C[ii, jj])


def test_spmv_small_integers_exact_and_bound(oracle_tenants):
    d = gen.gen_spmv_csr(2, 0, 3000)
    rowptr, col = d["rowptr"], d["col"]
    rng = np.random.default_rng(1)
    vi = rng.integers(-4, 5, len(col)).astype(np.float32)
    xi = rng.integers(-4, 5, d["ncols"]).astype(np.float32)
    y32, y64, asum = oracle_tenants.spmv_csr(rowptr, col, vi, xi)
    # dense reference through scipy-free construction
    dense_rows = np.repeat(np.arange(d["nrows"]), np.diff(rowptr))
    ref = np.zeros(d["nrows"])
    np.add.at(ref, dense_rows, vi.astype(np.float64) * xi[col])
    assert np.array_equal(y32.astype(np.float64), ref)
    y32, y64, asum = oracle_tenants.spmv_csr(rowptr, col, d["val"], d["x"])
    deg = np.diff(rowptr).astype(np.float64)
    assert np.all(np.abs(y32 - y64) <= deg * 2.0 ** -24 * asum + 1e-30)
    # structure of the synthetic matrix: mean ~16, bounds, sorted distinct columns
    assert 14.0 < deg.mean() < 18.0 and deg.min() >= 1 and deg.max() <= 8192
    same_row = dense_rows[1:] == dense_rows[:-1]
    assert np.all(np.diff(col)[same_row] > 0)


def test_pchase_cycle_positions(oracle_tenants):
    d = gen.gen_pchase(2, 0, 1 << 16, 512, 300)
    nxt = d["next"]
    # one cycle: walking from 0 visits every element once
    pos = np.full(len(nxt), -1, np.int64)
    cyc = np.empty(len(nxt), np.int64)
    p = 0
    for k in range(len(nxt)):
        assert pos[p] == -1
        pos[p] = k
        cyc[k] = p
        p = nxt[p]
    assert p == 0
    end = oracle_tenants.pchase(nxt, d["start"], d["hops"])
    expect = cyc[(pos[d["start"]] + d["hops"]) % len(nxt)]
    assert np.array_equal(end, expect)


def test_triad_exact(oracle_tenants):
    d = gen.gen_triad(2, 0, 1 << 14)
    a = oracle_tenants.triad(d["b"], d["c"], d["s"])
    ref64 = 3.0 * d["c"].astype(np.float64) + d["b"]
    # fused: one rounding of the exact value; binary64 holds s*c+b exactly here
    # unless the exponents are 27+ bits apart (then allow the 1-ulp double rounding)
    assert np.all(np.abs(a - ref64) <= 0.5 * np.spacing(np.abs(a)) + 1e-45)
    bi = np.arange(-50, 50, dtype=np.float32)
    ci = np.arange(100, dtype=np.float32)
    assert np.array_equal(oracle_tenants.triad(bi, ci, 3.0), bi + 3 * ci)


def test_hist256_counts(oracle_tenants):
    d = gen.gen_hist256(2, 0, 1 << 18)
    h = oracle_tenants.hist256(d["data"])
    assert int(h.sum()) == len(d["data"])
    vals, runs = np.unique(np.sort(d["data"]), return_counts=True)
    full = np.zeros(256, np.int64)
    full[vals] = runs
    assert np.array_equal(h.astype(np.int64), full)
    # Zipf(1.1): the most frequent value carries about 20% of the bytes
    assert 0.15 < h.max() / h.sum() < 0.25


def test_escape_time_pins(oracle_tenants):
    e = gen.gen_escape(2, 0, 64, 64, 256)
    cnt = oracle_tenants.escape(64, 64, 256, e["x0"], e["y0"], e["dx"], e["dy"]).reshape(64, 64)
    # vertical mirror symmetry: cy(i) = -cy(63-i) exactly on this grid
    assert np.array_equal(cnt, cnt[::-1, :])
    # single-point pins: c = 0 never escapes; c = 1 escapes after 3 steps (0 -> 1 -> 2 -> 5)
    one = oracle_tenants.escape(1, 1, 256, -0.5, -0.5, 1.0, 1.0)   # cx = cy = 0
    assert one[0] == 256
    one = oracle_tenants.escape(1, 1, 256, 0.5, -0.5, 1.0, 1.0)    # cx = 1, cy = 0
    assert one[0] == 3
    # brute-force pure-Python iteration on a few pixels
    for (i, j) in [(0, 0), (31, 20), (40, 50), (10, 63)]:
        cx = np.float32(e["x0"] + np.float32(np.float32(j + 0.5) * e["dx"]))
        cy = np.float32(e["y0"] + np.float32(np.float32(i + 0.5) * e["dy"]))
        x = y = np.float32(0.0)
        it = 0
        while it < 256:
            x2, y2 = np.float32(x * x), np.float32(y * y)
            if np.float32(x2 + y2) > 4.0:
                break
            xy = np.float32(x * y)
            y = np.float32(np.float32(xy + xy) + cy)
            x = np.float32(np.float32(x2 - y2) + cx)
            it += 1
        assert cnt[i, j] == it


def test_sort_definition(oracle_tenants):
    d = gen.gen_bitonic(2, 0, 14)
    out = oracle_tenants.sort_u32(d["data"])
    assert np.array_equal(out, np.sort(d["data"]))
    assert np.all(out[1:] >= out[:-1])


def test_matadd_and_sliced_invariance(oracle_tenants):
    # Section 4.1 example: 256x256 add, 16x16 blocks of 16x16 threads, slices of 8 blocks
    d = gen.gen_matadd(2, 0, 256)
    c = oracle_tenants.matadd(d["a"], d["b"])
    assert np.array_equal(c, d["a"] + d["b"])
    # slicing never changes a result: run the elementwise tenants slice by slice
    # in a shuffled slice order with rectified offsets
    rng = np.random.default_rng(3)
    g = gen.gen_gather(2, 1, 5000)
    t = gen.gen_triad(2, 1, 5000)
    full_g = oracle_tenants.gather(g["a"], g["idx"])
    full_t = oracle_tenants.triad(t["b"], t["c"], t["s"])
    for block, slice_blocks in [(256, 1), (256, 7), (1024, 3), (5000, 1)]:
        nblocks = -(-5000 // block)
        starts = list(range(0, nblocks, slice_blocks))
        rng.shuffle(starts)
        og = np.zeros(5000, np.int32)
        ot = np.zeros(5000, np.float32)
        for s0 in starts:
            lo = s0 * block
            hi = min(5000, (s0 + slice_blocks) * block)
            oracle_tenants.gather(g["a"], g["idx"], lo, hi, og)
            oracle_tenants.triad(t["b"], t["c"], t["s"], lo, hi, ot)
        assert np.array_equal(og, full_g) and np.array_equal(ot, full_t)
    e = gen.gen_escape(2, 0, 48, 40, 64)
    full_e = oracle_tenants.escape(48, 40, 64, e["x0"], e["y0"], e["dx"], e["dy"])
    oe = np.zeros_like(full_e)
    rows = list(range(40))
    rng.shuffle(rows)
    for r0 in rows:
        oracle_tenants.escape(48, 40, 64, e["x0"], e["y0"], e["dx"], e["dy"], r0, r0 + 1, oe)
    assert np.array_equal(oe, full_e)


# ---------------------------------------------------------------- BF16 GEMM (C = A B^T)

def test_bf16_bits_round_to_nearest_even():
    from workloads.gen import bf16_bits
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.0, 1.0 + 2 ** -7 + 2 ** -8], np.float32)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: to the even one (1.0);
    # 1 + 2^-7 + 2^-8 lies halfway between mantissas 1 (odd) and 2: to 2
    assert bf16_bits(x).tolist() == [0x3F80, 0x3F80, 0x3F81, 0xC000, 0x3F82]


def test_bf16_decode_known_values(oracle_tenants):
    OT = oracle_tenants
    v = OT.bf16_to_f64(np.array([0x3F80, 0xC000, 0x3F81, 0x0000, 0x4049], np.uint16))
    assert v.tolist() == [1.0, -2.0, 1.0078125, 0.0, 3.140625]


def _bf16_of_ints(a):
    from workloads.gen import bf16_bits
    return bf16_bits(np.asarray(a, np.float32))


def test_gemm_bf16_small_integers_exact_and_orientation(oracle_tenants):
    OT = oracle_tenants
    rng = np.random.default_rng(11)
    A = rng.integers(-8, 9, (5, 24))
    B = rng.integers(-8, 9, (7, 24))          # stored as Bt: row j is column j of B
    C, S = OT.gemm_bf16(_bf16_of_ints(A), _bf16_of_ints(B))
    assert C.shape == (5, 7)
    assert np.array_equal(C, (A @ B.T).astype(np.float64))
    assert np.array_equal(S, (np.abs(A) @ np.abs(B).T).astype(np.float64))
    eye = _bf16_of_ints(np.eye(24))
    C2, _ = OT.gemm_bf16(_bf16_of_ints(A), eye)
    assert np.array_equal(C2, A.astype(np.float64))


def test_gemm_bf16_matches_fp32_chain_within_its_bound(oracle_tenants):
    OT = oracle_tenants
    # the FP32 oracle's fused chain over bfloat16-valued inputs differs from the
    # exact sum by at most K u sum|ab| (u = 2^-24)
    inp = gen.gen_gemm_bf16(3, 1, 33, 20, 64)
    a = OT.bf16_to_f64(inp["A"]).astype(np.float32)
    b = OT.bf16_to_f64(inp["Bt"]).astype(np.float32)
    c32 = OT.gemm_f32(a, np.ascontiguousarray(b.T)).astype(np.float64)
    c64, s = OT.gemm_bf16(inp["A"], inp["Bt"])
    assert np.all(np.abs(c32 - c64) <= 64 * 2.0 ** -24 * s)
    ii = np.array([0, 5, 32, 17]); jj = np.array([0, 19, 3, 11])
    cs, ss = OT.gemm_bf16_sample(inp["A"], inp["Bt"], ii, jj)
    assert np.allclose(cs, c64[ii, jj], rtol=0, atol=1e-12) and np.allclose(ss, s[ii, jj], rtol=0, atol=1e-12)
