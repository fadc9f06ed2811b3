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


def test_gemm_exact_value_and_chain_bound(oracle_tenants):
    rng = np.random.default_rng(3)
    Ai = rng.integers(-50, 51, (45, 130)).astype(np.float32)
    Bi = rng.integers(-50, 51, (130, 27)).astype(np.float32)
    c64, cabs = oracle_tenants.gemm_f32_exact(Ai, Bi)
    assert np.array_equal(c64, (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64))
    assert np.array_equal(cabs, (np.abs(Ai).astype(np.int64) @ np.abs(Bi).astype(np.int64)).astype(np.float64))
    # the chain oracle lies within K 2^-24 sum|ab| of the exact value, and the
    # bound is tight enough that a wrong operand (B's rows reversed) fails it
    # almost everywhere
    d = gen.gen_gemm_f32(2, 1, 96, 96, 257)
    C = oracle_tenants.gemm_f32(d["A"], d["B"])
    c64, cabs = oracle_tenants.gemm_f32_exact(d["A"], d["B"])
    bound = 257 * 2.0 ** -24 * cabs
    assert np.all(np.abs(C - c64) <= bound)
    wrong, _ = oracle_tenants.gemm_f32_exact(d["A"], d["B"][::-1].copy())
    assert np.mean(np.abs(wrong - c64) > bound) > 0.99


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


# ---------------------------------------------------------------- TEA, SAD, stencil, MRI-Q

def test_tea_known_answer_and_inverse(oracle_tenants):
    OT = oracle_tenants
    # the cipher's published test vector: zero key, zero block
    assert OT.tea(np.zeros(2, np.uint32), np.zeros(4, np.uint32), 1).tolist() == [0x41EA3A0A, 0x94BAA940]
    inp = gen.gen_tea(4, 0, 257)
    ct = OT.tea(inp["words"], inp["key"], inp["n"])
    # decryption runs the cycles backwards (sum from 32 * delta down); it must
    # give back every plaintext block
    k = [int(x) for x in inp["key"]]
    v0 = ct[0::2].astype(np.uint64)
    v1 = ct[1::2].astype(np.uint64)
    M = np.uint64(0xFFFFFFFF)
    s = np.uint64((0x9E3779B9 * 32) & 0xFFFFFFFF)
    for _ in range(32):
        v1 = (v1 - ((((v0 << np.uint64(4)) & M) + np.uint64(k[2])) ^ ((v0 + s) & M) ^ ((v0 >> np.uint64(5)) + np.uint64(k[3])))) & M
        v0 = (v0 - ((((v1 << np.uint64(4)) & M) + np.uint64(k[0])) ^ ((v1 + s) & M) ^ ((v1 >> np.uint64(5)) + np.uint64(k[1])))) & M
        s = (s + np.uint64((1 << 32) - 0x9E3779B9)) & M  # s - delta modulo 2^32
    assert np.array_equal(v0.astype(np.uint32), inp["words"][0::2])
    assert np.array_equal(v1.astype(np.uint32), inp["words"][1::2])


def test_sad_shifted_frame_and_brute_force(oracle_tenants):
    OT = oracle_tenants
    W, H, R = 40, 24, 3
    cur = (np.arange(W * H, dtype=np.uint64) * np.uint64(2654435761) >> np.uint64(13)).astype(np.uint8).reshape(H, W)
    dx, dy = 2, -1
    ref = np.roll(cur, (dy, dx), axis=(0, 1))
    sad = OT.sad(cur, ref, W, H, R).reshape(H // 4, W // 4, 2 * R + 1, 2 * R + 1)
    # interior blocks (no wrap, no clamping) match exactly at the true motion
    for by in range(1, H // 4 - 1):
        for bx in range(1, W // 4 - 1):
            assert sad[by, bx, dy + R, dx + R] == 0
            assert sad[by, bx].min() == 0
    # identical frames: zero at displacement 0 everywhere
    assert np.all(OT.sad(cur, cur, W, H, R).reshape(-1, (2 * R + 1) ** 2)[:, R * (2 * R + 1) + R] == 0)
    # brute force with numpy clipping on a few (block, displacement) pairs
    rng = np.random.default_rng(0)
    full = OT.sad(cur, ref, W, H, R)
    for _ in range(50):
        by, bx = rng.integers(0, H // 4), rng.integers(0, W // 4)
        ddy, ddx = rng.integers(-R, R + 1), rng.integers(-R, R + 1)
        ys = np.clip(np.arange(4 * by, 4 * by + 4) + ddy, 0, H - 1)
        xs = np.clip(np.arange(4 * bx, 4 * bx + 4) + ddx, 0, W - 1)
        want = np.abs(cur[4 * by:4 * by + 4, 4 * bx:4 * bx + 4].astype(int) - ref[np.ix_(ys, xs)].astype(int)).sum()
        o = ((by * (W // 4) + bx) * (2 * R + 1) + ddy + R) * (2 * R + 1) + ddx + R
        assert full[o] == want


def test_stencil_closed_forms(oracle_tenants):
    OT = oracle_tenants
    nx, ny, nz = 9, 7, 5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inner = (x > 0) & (y > 0) & (z > 0) & (x < nx - 1) & (y < ny - 1) & (z < nz - 1)
    const = np.full((nz, ny, nx), 1.5, np.float32)
    out = OT.stencil7(const, nx, ny, nz, 0.25, 0.125).reshape(nz, ny, nx)
    assert np.all(out[inner] == np.float32(1.5 * (0.25 + 6 * 0.125)))
    assert np.all(out[~inner] == 1.5)                           # faces are copied
    lin = (3 * x - 2 * y + 5 * z).astype(np.float32)            # discrete Laplacian of a linear field is 0
    out = OT.stencil7(lin, nx, ny, nz, -6.0, 1.0).reshape(nz, ny, nx)
    assert np.all(out[inner] == 0.0)
    quad = (x * x).astype(np.float32)                           # ... of x^2 is 2
    out = OT.stencil7(quad, nx, ny, nz, -6.0, 1.0).reshape(nz, ny, nx)
    assert np.all(out[inner] == 2.0)


def test_sincosf_against_binary64(oracle_tenants):
    OT = oracle_tenants
    xs = np.linspace(-80.0, 80.0, 20001).astype(np.float32)
    for a in xs[::7]:
        s, c = OT.sincosf(float(a))
        a64 = float(a)
        # a few units of 2^-24 of the result's scale: the reduction's error
        # grows with the quadrant number |n| <= 51 here
        tol = 6e-8 * (4 + abs(a64) / 8)
        assert abs(s - np.sin(a64)) <= tol and abs(c - np.cos(a64)) <= tol, (a, s, c)
    assert OT.sincosf(0.0) == (0.0, 1.0)


def test_mriq_against_binary64(oracle_tenants):
    OT = oracle_tenants
    inp = gen.gen_mriq(5, 1, 96, 40)
    pm, qr, qi = OT.mriq(inp)
    k = {n: inp[n].astype(np.float64) for n in ("kx", "ky", "kz", "phiR", "phiI", "x", "y", "z")}
    pm64 = k["phiR"] ** 2 + k["phiI"] ** 2
    assert np.all(np.abs(pm - pm64) <= 2 * 2.0 ** -24 * pm64)
    t = np.outer(k["x"], k["kx"]) + np.outer(k["y"], k["ky"]) + np.outer(k["z"], k["kz"])
    ang = 2 * np.pi * t
    qr64 = (np.cos(ang) * pm64).sum(axis=1)
    qi64 = (np.sin(ang) * pm64).sum(axis=1)
    # per term: angle error ~ 6 u |2 pi t|-scale plus the sine/cosine's own few
    # u; the sum of numK binary32 terms adds numK u sum(pm)
    u = 2.0 ** -24
    scale = np.abs(np.outer(k["x"], k["kx"])) + np.abs(np.outer(k["y"], k["ky"])) + np.abs(np.outer(k["z"], k["kz"]))
    bound = (pm64 * (6 * u * 2 * np.pi * scale + 8 * u + 6e-8 * (4 + np.abs(ang) / 8))).sum(axis=1) \
        + inp["numK"] * u * pm64.sum()
    assert np.all(np.abs(qr - qr64) <= bound) and np.all(np.abs(qi - qi64) <= bound)


def test_testmix_index_sequence_sums_and_recurrence(oracle_tenants):
    # Section 4.3 testing kernel. Small-integer inputs with c1 = 1, c2 = 0 give
    # exact sums: each thread's total over its index sequence (g + j nthreads)
    # mod n_in, j = 0 .. iters*mem - 1, computed here by numpy fancy indexing
    rng = np.random.default_rng(4)
    n_in, nth, iters, mem = 1 << 10, 300, 7, 3
    data = rng.integers(-3, 4, n_in).astype(np.float32)
    inp = dict(data=data, n_in=n_in, nthreads=nth, iters=iters, mem=mem, alu=5, c1=np.float32(1.0),
               c2=np.float32(0.0))
    j = np.arange(iters * mem)
    idx = (np.arange(nth)[:, None] + j[None, :] * nth) % n_in
    assert np.array_equal(oracle_tenants.testmix(inp), data[idx].astype(np.int64).sum(axis=1).astype(np.float32))
    # no loads: iters*alu steps of acc = acc*1 + 1 from 0 count exactly
    inp.update(mem=0, alu=11, c2=np.float32(1.0))
    assert np.all(oracle_tenants.testmix(inp) == np.float32(iters * 11))
    # one load then acc = 0.5 acc (exact scaling) each round: brute force in
    # binary32 arithmetic round by round
    d = rng.standard_normal(n_in).astype(np.float32)
    inp = dict(data=d, n_in=n_in, nthreads=nth, iters=9, mem=1, alu=1, c1=np.float32(0.5), c2=np.float32(0.0))
    acc = np.zeros(nth, np.float32)
    for i in range(9):
        acc = (acc + d[(np.arange(nth) + i * nth) % n_in]).astype(np.float32)
        acc = (acc * np.float32(0.5)).astype(np.float32)
    assert np.array_equal(oracle_tenants.testmix(inp), acc)
