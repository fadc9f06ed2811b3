"""Markov model vs measured co-scheduled IPC on the GPU (Section 5.3:
single-kernel and concurrent-kernel IPC prediction, CP prediction).

Every kernel type runs alone in the co-scheduler, then every pair of types
runs co-scheduled at the model's balanced slot split (Eq. executiontime), 8
copies of each kernel per run with backfill and the chain lane off, so that
the phases are pure pairs in steady state. The measured IPC of a type is its
blocks finished during the phases that run exactly that pair (from the phase
log) times its instructions per block (measured with ncu) over those phases'
cycles on all SMs. The model's numbers come from the runtime's own model with
the measured per-type profiles.

The two-tenant case (Black-Scholes 65,536 options + int32 gather 2^20, each
in 4 slices) is repeated 1000 times inside one persistent launch at fixed slot
ratios 1:3, 1:1 and 3:1 and at the model's split, and against the same 2000
kernels as plain launches on 2 streams.

    python -m paper_1303_5164_gb300.validate_pairs --out pairs.json
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TYPES = ["gemm_f32", "spmv_csr", "blackscholes", "pchase", "triad", "hist256", "escape", "bitonic"]
COPIES = 8


def _profiles(K):
    path = os.path.join(ROOT, "paper_1303_5164_gb300", "profiles_gb300.json")
    with open(path) as f:
        doc = json.load(f)
    profs = []
    for name in K.TYPE_NAMES:
        p = K.kl_profile()
        e = doc["types"].get(name)
        if e:
            for k in ("R_m", "f_u", "m_c", "m_u", "L0", "I_block", "PUR", "MUR"):
                setattr(p, k, float(e[k]))
            p.warps_per_block = 8
            # steady-state pair rates are read between phases: the alone-tuned
            # slices, small enough that blocks finish inside every phase (the
            # table tuned in company hands 8 copies one slice per CTA)
            alone = doc.get("slice_autotune_alone", {}).get("slices", {})
            p.slice_blocks = int(alone.get(name, doc.get("slices", {}).get(name, 0)))
            p.valid = 1
        profs.append(p)
    return profs, doc


def _phase_ipc(ph, i, tens, profs, mp):
    """Measured per-SM IPC of the kernels of phase i (ends at phase i+1)."""
    p, q = ph[i], ph[i + 1]
    cycles = (q.t_ns - p.t_ns) * 1e-9 * mp.f_sm_hz
    out = []
    for who, d0, d1 in ((p.A, p.done_a, q.prev_done_a), (p.B, p.done_b, q.prev_done_b)):
        if who < 0:
            out.append(None)
            continue
        ib = profs[tens[who].type].I_block
        out.append((d1 - d0) * ib / (cycles * mp.n_sm) if cycles > 0 else None)
    return out, (q.t_ns - p.t_ns) / 1e3


def run(out_path, reps=3):
    import torch
    from workloads import gen
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    profs, doc = _profiles(K)
    cfg = K.config_default()
    cfg.slots_per_sm = 4
    rt = K.Runtime(cfg)
    mp = rt.model_params()
    mp.a0, mp.b0 = doc.get("a0", 1.0), doc.get("b0", 0.0)
    mp.dram_bytes_per_s = doc.get("dram_bytes_per_s", mp.dram_bytes_per_s)
    rt.set_model_params(mp)
    rt.set_profiles(profs)
    S = rt.run_stats().slots_per_sm
    tens = {t: T.make(t, gen.gen_tenant(t, 9, i, **T.SIZES_MIX[t])) for i, t in enumerate(TYPES)}
    res = {"slots_per_sm": S, "f_sm_hz": mp.f_sm_hz, "n_sm": mp.n_sm, "solo": {}, "pairs": {}}

    # 8 copies of each kernel per run (inputs shared, outputs replicated) and
    # no backfill or chain lane: every phase is a pure pair (or a solo phase)
    # and the pair persists across phases until one type runs out
    reps_of = {nm: [tens[nm]] + [tens[nm].replica() for _ in range(COPIES - 1)] for nm in TYPES}

    def go(names):
        c2 = K.config_default()
        c2.slots_per_sm = S
        c2.flags = 0
        c2.max_tenants = 4096
        # prune only pairs with identical PUR and MUR (two copies of one type):
        # while both types are pending the pair (a, b) runs; once one type is
        # left its copies pair with each other (every pair pruned -> unpruned set)
        c2.alpha_p = c2.alpha_m = 1e-9
        r2 = K.Runtime(c2)
        r2.set_model_params(mp)
        r2.set_profiles(profs)
        best = None
        for _ in range(reps):
            order = [nm for k in range(COPIES) for nm in names]
            for k, nm in enumerate(order):
                t = reps_of[nm][k // len(names)]
                r2.submit(t.type, t.args)
            r2.launch()
            assert r2.drain() == 0
            ker = r2.run_stats().kernel_ns / 1e3
            if best is None or ker < best[1]:
                best = (r2.phases(), ker, order)
        r2.close()
        return best

    def steady_ipc(ph, order, names):
        """Per-type IPC per SM summed over the phases that run exactly the
        types in `names` (both of a pair, or the one type alone): blocks each
        role finished during the phase x instructions per block over the
        phase's cycles on all SMs."""
        want = sorted(names)
        blocks = {nm: 0 for nm in names}
        cyc = 0.0
        splits = []
        for k in range(1, len(ph) - 1):
            p, q = ph[k], ph[k + 1]
            if p.A < 0:
                continue
            types = sorted([order[p.A]] + ([order[p.B]] if p.B >= 0 else []))
            if (len(want) == 1 and set(types) != set(want)) or (len(want) == 2 and types != want):
                continue
            c = (q.t_ns - p.t_ns) * 1e-9 * mp.f_sm_hz
            if c <= 0:
                continue
            cyc += c
            blocks[order[p.A]] += q.prev_done_a - p.done_a
            if p.B >= 0:
                blocks[order[p.B]] += q.prev_done_b - p.done_b
            splits.append(p.slots_a if order[p.A] == names[0] else S - p.slots_a)
        if cyc <= 0:
            return [None] * len(names), 0.0, None
        ipc = [blocks[nm] * profs[tens[nm].type].I_block / (cyc * mp.n_sm) for nm in names]
        sa = max(set(splits), key=splits.count) if splits and len(names) == 2 else None
        return ipc, cyc / mp.f_sm_hz * 1e6, sa

    # solo IPC of each type at the co-scheduler's full occupancy
    for nm in TYPES:
        ph, ker, order = go([nm])
        (ipc,), dur, _ = steady_ipc(ph, order, [nm])
        w = max(1, int(round(S * 8 / 4)))
        pred = K.model_ipc(mp, [profs[tens[nm].type]], [w], 3)[0]
        res["solo"][nm] = {"ipc_measured": ipc, "ipc_predicted": pred, "phases_us": dur, "kernel_us": ker}
        print("solo", nm, res["solo"][nm], flush=True)

    # all pairs at the model's balanced split
    for a, b in itertools.combinations(TYPES, 2):
        ph, ker, order = go([a, b])
        (ca, cb), dur, sa = steady_ipc(ph, order, [a, b])
        if sa is None:
            sa = ph[1].slots_a if ph[1].A >= 0 and order[ph[1].A] == a else S - ph[1].slots_a
        pr = K.model_pair(mp, profs[tens[a].type], profs[tens[b].type], S, 3)
        pa, pb = pr["cipc_a"][sa - 1], pr["cipc_b"][sa - 1]
        ia, ib = res["solo"][a]["ipc_measured"], res["solo"][b]["ipc_measured"]
        cp_meas = 1.0 - 1.0 / (ca / ia + cb / ib) if ca and cb and ia and ib else None
        res["pairs"][f"{a}+{b}"] = {
            "slots_a": sa, "slots_b": S - sa, "cipc_measured": [ca, cb], "cipc_predicted": [pa, pb],
            "ipc_sum_measured": (ca or 0) + (cb or 0), "ipc_sum_predicted": pa + pb,
            "cp_predicted": pr["cp"][sa - 1], "cp_measured": cp_meas, "pair_phases_us": dur, "kernel_us": ker}
        print("pair", a, b, json.dumps(res["pairs"][f"{a}+{b}"]), flush=True)
    del reps_of
    torch.cuda.empty_cache()

    # the two-tenant case (configs: Black-Scholes 65,536 + gather 2^20, 4 slices
    # each) repeated 1000 times inside ONE persistent launch, at slot ratios
    # 1:3, 1:1, 3:1 and at the model's balanced split; against the same 2000
    # kernels as plain launches on 2 streams. Per-pair time = run time / 1000;
    # measured cIPC of each kernel = its blocks x instructions per block over
    # the run's cycles on all SMs.
    n_pairs = 1000
    bs = T.make("blackscholes", gen.gen_blackscholes(1, 0, 65536))
    ga = T.make("gather", gen.gen_gather(1, 1, 1 << 20))
    bss = [bs] + [bs.replica() for _ in range(n_pairs - 1)]
    gas = [ga] + [ga.replica() for _ in range(n_pairs - 1)]
    sl = [bs.shape().total_blocks // 4, ga.shape().total_blocks // 4]
    ib_bs, ib_ga = profs[bs.type].I_block, profs[ga.type].I_block
    c1 = {"pairs_per_launch": n_pairs, "slices": sl}

    def c1_run(policy, fixed):
        c2 = K.config_default()
        c2.slots_per_sm, c2.ratio_policy, c2.fixed_slots_a, c2.max_tenants = S, policy, fixed, 4096
        r2 = K.Runtime(c2)
        r2.set_model_params(mp)
        r2.set_profiles(profs)
        best = None
        for _ in range(reps):
            for b_, g_ in zip(bss, gas):
                r2.submit(b_.type, b_.args, slice_blocks=sl[0])
                r2.submit(g_.type, g_.args, slice_blocks=sl[1])
            r2.launch()
            assert r2.drain() == 0
            ker = r2.run_stats().kernel_ns / 1e3
            if best is None or ker < best[0]:
                ph = r2.phases()
                split = ph[1].slots_a if len(ph) > 1 else None
                best = (ker, split)
        r2.close()
        ker, split = best
        cyc = ker * 1e-6 * mp.f_sm_hz * mp.n_sm
        ipc = [n_pairs * 256 * ib_bs / cyc if ib_bs else None, n_pairs * 4096 * ib_ga / cyc if ib_ga else None]
        return ker, split, ipc

    for sa in (1, 2, 3):
        ker, split, ipc = c1_run(K.KL_RATIO_FIXED, sa)
        pr = K.model_pair(mp, profs[bs.type], profs[ga.type], S, 3, K.KL_RATIO_FIXED, sa)
        c1[f"{sa}:{S - sa}"] = {"per_pair_us": ker / n_pairs, "run_us": ker, "cipc_measured": ipc,
                                "cipc_predicted": [pr["cipc_a"][sa - 1], pr["cipc_b"][sa - 1]],
                                "cp_predicted": pr["cp"][sa - 1], "dT_predicted": pr["dT"][sa - 1]}
        print("c1", sa, c1[f"{sa}:{S - sa}"], flush=True)
    ker, split, ipc = c1_run(K.KL_RATIO_BALANCED, 2)
    c1["balanced"] = {"slots_a": split, "per_pair_us": ker / n_pairs, "run_us": ker, "cipc_measured": ipc}
    print("c1 balanced", c1["balanced"], flush=True)
    r2 = K.Runtime(K.config_default())
    times = []
    for _ in range(reps):
        for b_, g_ in zip(bss, gas):
            r2.submit(b_.type, b_.args)
            r2.submit(g_.type, g_.args)
        r2.launch_baseline(K.KL_BASE_MULTISTREAM, 2)
        assert r2.drain() == 0
        times.append(r2.run_stats().kernel_ns / 1e3)
    c1["two_streams_per_pair_us"] = min(times) / n_pairs
    res["c1_pair"] = c1
    r2.close()
    del bss, gas
    torch.cuda.empty_cache()

    errs = [abs(v["ipc_sum_measured"] - v["ipc_sum_predicted"]) for v in res["pairs"].values()]
    per = [abs(m - p) for v in res["pairs"].values() for m, p in zip(v["cipc_measured"], v["cipc_predicted"])
           if m is not None]
    solo_err = [abs(v["ipc_measured"] - v["ipc_predicted"]) for v in res["solo"].values() if v["ipc_measured"]]
    res["summary"] = {"pair_ipc_sum_mae_per_sm": statistics.mean(errs), "pair_cipc_mae_per_sm": statistics.mean(per),
                      "solo_ipc_mae_per_sm": statistics.mean(solo_err), "ipc_peak_per_sm": 4.0,
                      "pairs_within_20pct_of_peak": sum(e <= 0.8 for e in errs), "pairs": len(errs)}
    print(json.dumps(res["summary"]))
    rt.close()
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    run(a.out)


if __name__ == "__main__":
    main()
