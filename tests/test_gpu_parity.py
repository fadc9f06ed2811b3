"""GPU parity: every tenant through the C ABI (co-scheduled with several slice
sizes, and as plain launches) against the CPU oracle; the two-tenant pair at
slot ratios 1:3, 1:1, 3:1; a mixed queue where every result equals its
alone-run and every device co-schedule decision equals the oracle's."""
import numpy as np
import pytest

from tests import _expect as X
from workloads import gen

pytestmark = pytest.mark.gpu

CASES = {
    # sizes span several blocks/tiles and end in a ragged tail
    "gather": dict(n=5000),
    "blackscholes": dict(n=70001),
    "gemm_f32": dict(M=200, N=132, K=100),
    "spmv_csr": dict(nrows=5003),
    "pchase": dict(N=100003, nchasers=1001, hops=37),
    "triad": dict(n=3 * 4096 + 7),
    "hist256": dict(n=3 * 32768 + 5),
    "escape": dict(width=300, height=170, max_iter=64),
    "bitonic": dict(log2n=14),
    "matadd": dict(n=256),
    # 2 x 3 tiles of 128 x 64 with ragged M and N, 3 K-slices of 64 with a ragged 8
    "gemm_bf16": dict(M=200, N=132, K=136),
    "tea": dict(n=3 * 512 + 7),                                 # odd leftover block
    "sad": dict(width=64, height=36, range=3),                  # 7056 values: 28 blocks, ragged
    "stencil": dict(nx=300, ny=17, nz=9),                       # 45,900 points: 180 blocks, the last ragged
    "mriq": dict(numK=300, numX=1000),                          # two sample chunks, ragged point block
    # the Section 4.3 testing kernel: 3 blocks and a ragged tail, 14 rounds of 2 loads and 7 fused steps
    "testmix": dict(log2_in=16, nthreads=3 * 256 + 5, iters=14, mem=2, alu=7),
    # resource-heavy variants (resource-class kernels beside the co-scheduler)
    "bs255": dict(n=3 * 4096 + 1001),                          # 4 blocks of 4096 options, ragged
    "hist1024": dict(n=3 * 131072 + 5),                         # 4 counting blocks, ragged
    "gemm_f32_big": dict(M=300, N=260, K=100),                  # 3 x 3 tiles of 128 x 128, ragged
}


@pytest.fixture(scope="module")
def K():
    from paper_1303_5164_gb300 import build, kernelet
    build.build()
    return kernelet


@pytest.fixture(scope="module")
def T():
    from paper_1303_5164_gb300 import tenants
    return tenants


def _runtime(K, **cfg):
    c = K.config_default()
    for k, v in cfg.items():
        setattr(c, k, v)
    return K.Runtime(c)


def _run_alone(K, rt, ten, slice_blocks=0, baseline=None):
    import torch
    for v in ten.outputs:
        ten.bufs[v].fill_(-1)       # poison the outputs
    torch.cuda.synchronize()
    h = rt.submit(ten.type, ten.args, slice_blocks=slice_blocks)
    if baseline is None:
        rt.launch()
    else:
        rt.launch_baseline(baseline, 4)
    rc = rt.drain()
    assert rc == 0, K.lib().kl_strerror(rc)
    assert rt.poll(h) == K.KL_DONE
    return ten.fetch()


@pytest.mark.parametrize("name", list(CASES))
def test_tenant_alone_matches_oracle(K, T, name):
    inp = gen.gen_tenant(name, 7, 0, **CASES[name])
    exp = X.expected(name, inp)
    rt = _runtime(K)
    ten = T.make(name, inp)
    total = ten.shape().total_blocks
    outs = []
    for sl in sorted({1, 7, max(1, total // 4), int(total)}):
        got = _run_alone(K, rt, ten, slice_blocks=sl)
        X.check(name, inp, got, exp)
        outs.append(got)
    for mode in (K.KL_BASE_SERIAL, K.KL_BASE_MULTISTREAM):
        got = _run_alone(K, rt, ten, baseline=mode)
        X.check(name, inp, got, exp)
        outs.append(got)
    # slicing never changes a result: every run is bit-identical to the first
    for o in outs[1:]:
        for k in o:
            assert X.same_bits(o[k], outs[0][k]), (name, k)
    rt.close()


@pytest.mark.parametrize("log2n", [1, 5, 12, 13, 16])
def test_bitonic_sizes(K, T, log2n):
    inp = gen.gen_bitonic(7, 1, log2n)
    rt = _runtime(K)
    got = _run_alone(K, rt, T.make("bitonic", inp))
    X.check("bitonic", inp, got, X.expected("bitonic", inp))
    rt.close()


def test_matadd_slices_of_eight(K, T):
    # Section 4.1: 256x256 add, 16x16 blocks of 16x16 threads, slices of 8 blocks
    inp = gen.gen_matadd(7, 2, 256)
    rt = _runtime(K)
    ten = T.make("matadd", inp)
    assert tuple(ten.shape().grid) == (256, 1, 1)
    h = rt.submit(ten.type, ten.args, slice_blocks=8)
    assert rt.drain() == 0
    X.check("matadd", inp, ten.fetch(), X.expected("matadd", inp))
    assert rt.stats(h).slices == 32 and rt.stats(h).blocks == 256
    rt.close()


@pytest.mark.parametrize("slots_a", [1, 2, 3])
def test_pair_blackscholes_gather_ratios(K, T, slots_a):
    # 65,536 options and a 2^20 gather, each cut into 4 slices, at 1:3, 1:1, 3:1
    bs_in = gen.gen_blackscholes(1, 0, 65536)
    ga_in = gen.gen_gather(1, 1, 1 << 20)
    rt = _runtime(K, ratio_policy=K.KL_RATIO_FIXED, fixed_slots_a=slots_a, slots_per_sm=4)
    bs, ga = T.make("blackscholes", bs_in), T.make("gather", ga_in)
    h0 = rt.submit(bs.type, bs.args, slice_blocks=bs.shape().total_blocks // 4)
    h1 = rt.submit(ga.type, ga.args, slice_blocks=ga.shape().total_blocks // 4)
    assert rt.drain() == 0
    X.check("blackscholes", bs_in, bs.fetch(), X.expected("blackscholes", bs_in))
    X.check("gather", ga_in, ga.fetch(), X.expected("gather", ga_in))
    ph = rt.phases()
    assert (ph[1].A, ph[1].B, ph[1].slots_a, ph[1].slots_b) == (0, 1, slots_a, 4 - slots_a)
    assert ph[-1].A == -1
    assert rt.stats(h0).slices == 4 and rt.stats(h1).slices == 4
    rt.close()


MIX_SMALL = {
    "gemm_f32": dict(M=256, N=192, K=128),
    "spmv_csr": dict(nrows=20000),
    "blackscholes": dict(n=100000),
    "pchase": dict(N=1 << 18, nchasers=4096, hops=64),
    "triad": dict(n=1 << 20),
    "hist256": dict(n=1 << 20),
    "escape": dict(width=256, height=256, max_iter=256),
    "bitonic": dict(log2n=16),
}


def _oracle_profiles(K, rt):
    from oracle import markov as mk
    mp = rt.model_params()
    gpu = mk.GPUParams(n_sm=mp.n_sm, n_sched=mp.n_sched, f_sm_hz=mp.f_sm_hz,
                       dram_bytes_per_s=mp.dram_bytes_per_s, sector_bytes=int(mp.sector_bytes),
                       a0=mp.a0, b0=mp.b0)
    return gpu


@pytest.mark.parametrize("alpha", [None, (0.25, 0.12), "refit"])
def test_mix_alone_equals_in_mix_and_decisions_match_oracle(K, T, alpha):
    # alpha: pruning thresholds (alpha_p, alpha_m) of Section 4.3 on the device
    # planner and the oracle alike; with (0.25, 0.12) every pair of types
    # fewer than three apart below is pruned (their PUR and MUR gaps are both
    # small), same-type pairs included; "refit": the thresholds re-fit on
    # GB300 from the testing kernels (profiles_gb300.json)
    if alpha == "refit":
        import json
        import os
        doc = json.load(open(os.path.join(os.path.dirname(K.__file__), "profiles_gb300.json")))
        alpha = (doc["pruning"]["alpha_p"], doc["pruning"]["alpha_m"])
    from oracle import markov as mk
    from oracle import schedule as sc
    rng = np.random.default_rng(2)
    order = [t for t in MIX_SMALL for _ in range(2)]
    rng.shuffle(order)
    inps = [gen.gen_tenant(nm, 2, i, **MIX_SMALL[nm]) for i, nm in enumerate(order)]
    ap, am = alpha if alpha else (-1.0, -1.0)
    # the pair model of Algorithm 1's FindCoSchedule (the phase model scores
    # pairs with the chain-lane kernel; its decisions are checked below)
    rt = _runtime(K, slots_per_sm=4, alpha_p=ap, alpha_m=am,
                  flags=K.config_default().flags & ~K.KL_CFG_PHASE_MODEL)
    # known model inputs on both sides
    profs = []
    for t in range(K.KL_T_COUNT):
        p = K.kl_profile()
        p.R_m, p.f_u, p.m_c, p.m_u = 0.02 + 0.03 * t, (0.1 * t) % 0.7, 4.0, 32.0
        p.L0, p.I_block, p.warps_per_block, p.valid = 500.0 + 40 * t, 300.0 * (t + 1), 8, 1
        p.PUR, p.MUR = 0.1 * t, 0.05 * (9 - t)
        profs.append(p)
    rt.set_profiles(profs)
    tens = [T.make(nm, x) for nm, x in zip(order, inps)]
    handles = [rt.submit(t.type, t.args) for t in tens]
    assert rt.drain() == 0
    ph = rt.phases()
    for nm, x, t, h in zip(order, inps, tens, handles):
        assert rt.poll(h) == K.KL_DONE
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    in_mix = [t.fetch() for t in tens]
    # each tenant alone on a fresh runtime gives the same bits
    for t, got in zip(tens, in_mix):
        alone = _run_alone(K, rt, t)
        for k in got:
            assert X.same_bits(alone[k], got[k]), (t.name, k)
    # replay every device decision through the oracle's FindCoSchedule
    gpu = _oracle_profiles(K, rt)
    okp = {t: mk.KernelProfile(R_m=p.R_m, L0=p.L0, m_c=p.m_c, m_u=p.m_u, f_u=p.f_u, I_block=p.I_block,
                               warps_per_block=p.warps_per_block) for t, p in enumerate(profs)}
    model = sc.PairModel(gpu, rt.run_stats().slots_per_sm, three_state=True)
    ot = [sc.Tenant(okp[t.type], 1, PUR=profs[t.type].PUR, MUR=profs[t.type].MUR) for t in tens]
    assert ph[-1].A == -1 and ph[-1].n_pending == 0
    for p in ph[1:-1]:
        R = [i for i in range(len(tens)) if (p.pending_mask >> i) & 1]
        assert len(R) == p.n_pending
        cs = sc.find_coschedule(R, ot, model, *(alpha or (None, None)))
        if alpha and len(R) > 1:
            # the device kept to the unpruned pairs whenever there was one
            kept = sc.prune_pairs([(i, j) for i in R for j in R if i < j], ot, *alpha)
            assert (p.A, p.B) in kept
        if (cs.A, cs.B) != (p.A, p.B if p.B >= 0 else None):
            # only a floating-point near-tie may differ
            assert abs(cs.cp - p.cp) < 1e-9, ((cs.A, cs.B, cs.cp), (p.A, p.B, p.cp))
        else:
            assert (cs.bA, cs.bB) == (p.slots_a, p.slots_b)
            assert abs(cs.cp - p.cp) < 1e-9 * max(1.0, abs(cs.cp))
    rt.close()


def test_gemm_bf16_full_size_sampled(K, T):
    # 4096^3 (the resource-heavy workload's tensor-core GEMM): 512 sampled
    # entries, tile corners included, against binary64 dot products
    from oracle import tenants as OT
    inp = gen.gen_gemm_bf16(5, 0, 4096, 4096, 4096)
    rt = _runtime(K)
    got = _run_alone(K, rt, T.make("gemm_bf16", inp))["C"]
    rng = np.random.default_rng(0)
    ii = np.concatenate([[0, 127, 128, 4095, 4095, 2047], rng.integers(0, 4096, 506)])
    jj = np.concatenate([[0, 63, 64, 4095, 0, 2048], rng.integers(0, 4096, 506)])
    c, sabs = OT.gemm_bf16_sample(inp["A"], inp["Bt"], ii, jj)
    err = np.abs(got[ii, jj].astype(np.float64) - c)
    assert np.all(err <= X.gemm_bf16_bound(4096, sabs)), err.max()
    rt.close()


def test_tensor_core_build_coschedules_bf16_with_others(K, T):
    # a run holding a BF16 GEMM uses the co-scheduler build with the tensor-core
    # tenant; it keeps 4 slots per SM and pairs the GEMM with other kernels
    items = [("gemm_bf16", dict(M=1024, N=512, K=1024)), ("blackscholes", dict(n=300000)),
             ("triad", dict(n=1 << 22)), ("pchase", dict(N=1 << 20, nchasers=8192, hops=128)),
             ("gemm_bf16", dict(M=256, N=256, K=2048))]
    inps = [(nm, gen.gen_tenant(nm, 12, i, **sz)) for i, (nm, sz) in enumerate(items)]
    rt = _runtime(K, slots_per_sm=4)
    tens = [T.make(nm, x) for nm, x in inps]
    hs = [rt.submit(t.type, t.args) for t in tens]
    assert rt.drain() == 0
    assert rt.run_stats().slots_per_sm == 4
    ph = rt.phases()
    pairs = [p for p in ph if p.A >= 0 and p.B >= 0]
    assert pairs and all(p.slots_a + p.slots_b == 4 for p in pairs)
    assert any(0 in (p.A, p.B) or 4 in (p.A, p.B) for p in pairs)
    got = [t.fetch() for t in tens]
    for (nm, x), g, h in zip(inps, got, hs):
        assert rt.poll(h) == K.KL_DONE
        X.check(nm, x, g, X.expected(nm, x))
    for t, g in zip(tens, got):
        alone = _run_alone(K, rt, t)
        for k in g:
            assert X.same_bits(alone[k], g[k]), (t.name, k)
    rt.close()


LIGHT = ["gather", "blackscholes", "spmv_csr", "triad", "escape", "matadd", "tea", "stencil"]


def test_light_build_runs_light_types_at_eight_slots(K, T):
    # a run of light types only uses the 8-CTA build; every result equals the
    # oracle and the bits of the same kernel run alone in the 4-CTA builds
    inps = [(nm, gen.gen_tenant(nm, 31, i, **CASES[nm])) for i, nm in enumerate(LIGHT + LIGHT[::-1])]
    rt = _runtime(K)
    tens = [T.make(nm, x) for nm, x in inps]
    hs = [rt.submit(t.type, t.args, slice_blocks=2) for t in tens]
    assert rt.drain() == 0
    S = rt.run_stats().slots_per_sm
    assert S == 8
    pairs = [p for p in rt.phases() if p.A >= 0 and p.B >= 0]
    assert pairs and all(p.slots_a + p.slots_b == S for p in pairs)
    got = [t.fetch() for t in tens]
    for (nm, x), g, h in zip(inps, got, hs):
        assert rt.poll(h) == K.KL_DONE
        X.check(nm, x, g, X.expected(nm, x))
    rt.close()
    rt4 = _runtime(K, flags=K.config_default().flags & ~K.KL_CFG_LIGHT_BUILD)
    for t, g in zip(tens, got):
        alone = _run_alone(K, rt4, t)
        assert rt4.run_stats().slots_per_sm == 4
        for k in g:
            assert X.same_bits(alone[k], g[k]), (t.name, k)
    # one kernel outside the light set puts the whole run on 4 slots
    extra = T.make("gemm_f32", gen.gen_tenant("gemm_f32", 31, 99, **CASES["gemm_f32"]))
    rt = _runtime(K)
    for t in tens[:4] + [extra]:
        rt.submit(t.type, t.args)
    assert rt.drain() == 0
    assert rt.run_stats().slots_per_sm == 4
    for t, g in zip(tens[:4], got[:4]):
        f = t.fetch()
        for k in g:
            assert X.same_bits(f[k], g[k]), (t.name, k)
    rt.close()


def test_deep_fill_many_small_kernels(K, T):
    # 96 kernels of 2-4 slices each leave most slots to deep fill; with it on
    # and off every result equals the oracle, bit for bit the same
    specs = [("triad", dict(n=4 * 4096 + 3)), ("gather", dict(n=3 * 1024 + 5)), ("blackscholes", dict(n=2 * 256 + 1)),
             ("matadd", dict(n=64))]
    inps = [(nm, gen.gen_tenant(nm, 41, i, **sz)) for i in range(24) for nm, sz in specs]
    tens = [T.make(nm, x) for nm, x in inps]
    got = {}
    for deep in (True, False):
        c = K.config_default()
        if not deep:
            c.flags &= ~K.KL_CFG_DEEP_FILL
        rt = K.Runtime(c)
        hs = [rt.submit(t.type, t.args) for t in tens]
        assert rt.drain() == 0
        got[deep] = [t.fetch() for t in tens]
        for (nm, x), t, g, h in zip(inps, tens, got[deep], hs):
            assert rt.poll(h) == K.KL_DONE
            X.check(nm, x, g, X.expected(nm, x))
            assert rt.stats(h).blocks == t.shape().total_blocks
        rt.close()
    for a, b in zip(got[True], got[False]):
        for k in a:
            assert X.same_bits(a[k], b[k])


def test_claim_ahead_counts_every_slice_once(K, T):
    # a triad of 4096 one-block slices (more than 2 x slots x SMs: the slots
    # running it claim their next slice ahead) beside kernels that force
    # re-plans; every block runs once and every slice is counted once
    big_in = gen.gen_triad(43, 0, 4096 * 4096)
    big = T.make("triad", big_in)
    others = [(nm, gen.gen_tenant(nm, 43, i + 1, **MIX_SMALL[nm])) for i, nm in
              enumerate(["blackscholes", "escape", "pchase", "spmv_csr"])]
    oth = [T.make(nm, x) for nm, x in others]
    rt = _runtime(K)
    h = rt.submit(big.type, big.args, slice_blocks=1)
    hs = [rt.submit(t.type, t.args) for t in oth]
    assert rt.drain() == 0
    st = rt.stats(h)
    assert st.blocks == 4096 and st.slices == 4096
    X.check("triad", big_in, big.fetch(), X.expected("triad", big_in))
    for (nm, x), t, hh in zip(others, oth, hs):
        assert rt.poll(hh) == K.KL_DONE
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    rt.close()


@pytest.mark.parametrize("planner", ["random", "table", "phase"])
def test_other_planners_keep_results(K, T, planner):
    # the MC comparison's random plans and an overridden CP table change only
    # the order and sharing of kernels: every result still equals the oracle
    names = list(MIX_SMALL)
    inps = [(nm, gen.gen_tenant(nm, 21, i, **MIX_SMALL[nm])) for i, nm in enumerate(names)]
    c = K.config_default()
    if planner == "random":
        c.flags |= K.KL_CFG_RANDOM_PLAN
        c.plan_seed = 7
    if planner == "phase":
        c.flags |= K.KL_CFG_PHASE_MODEL | K.KL_CFG_CHAIN_LANE
        c.alpha_p = c.alpha_m = -1.0   # no pruning: every pair of pending types is a candidate
    rt = K.Runtime(c)
    if planner == "table":
        n = K.KL_T_COUNT
        rt.set_cp_table([0.01 * ((i * 7 + j * 3) % 11) for i in range(n) for j in range(n)],
                        [1 + (i + j) % 3 for i in range(n) for j in range(n)])
        cp, sa, _ = rt.cp_table()
        assert sa[1 * n + 2] == 1 + 3 % 3 and abs(cp[2 * n + 5] - 0.01 * ((14 + 15) % 11)) < 1e-15
    tens = [T.make(nm, x) for nm, x in inps]
    hs = [rt.submit(t.type, t.args) for t in tens]
    assert rt.drain() == 0
    ph = rt.phases()
    assert any(p.B >= 0 for p in ph)
    for (nm, x), t, h in zip(inps, tens, hs):
        assert rt.poll(h) == K.KL_DONE
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    if planner == "phase":
        # every device decision is the largest-CP pair of pending kernel types
        # (the lowest kernel of each type) in the table the runtime reports:
        # the phase model's table, scored with the chain-lane kernel
        cp, sa, _ = rt.cp_table()
        n = K.KL_T_COUNT
        for p in ph[1:-1]:
            if p.B < 0:
                continue
            pend = [i for i in range(len(tens)) if (p.pending_mask >> i) & 1]
            low = {}
            for i in pend:
                low.setdefault(tens[i].type, []).append(i)
            cands = []
            for ta in low:
                for tb in low:
                    if ta < tb:
                        i, j = sorted((low[ta][0], low[tb][0]))
                    elif ta == tb and len(low[ta]) > 1:
                        i, j = low[ta][0], low[ta][1]
                    else:
                        continue
                    cands.append(cp[tens[i].type * n + tens[j].type])   # (lower index, higher index)
            best = max(cands)
            got = cp[tens[p.A].type * n + tens[p.B].type]
            assert got >= best - 1e-12, (p.A, p.B, got, best)
    if planner == "table":
        rt.set_cp_table(None)
    rt.close()
