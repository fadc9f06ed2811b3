"""Greedy plan vs OPT vs MC(s) on the 64-kernel mix (Section 5.1 comparisons).

Kernelet: the greedy planner (Algorithm 1) on the Markov model's CP table.
OPT: the same greedy planner on CPs measured on the GPU by running every pair
of kernel types at every slot split (steady state: 8 copies of each kernel,
no backfill, so every phase is the pair), each pair at its best measured split.
MC(s): s runs in which every re-plan picks a random pair of pending kernel
types and a random split (KL_CFG_RANDOM_PLAN, seeds 1..s).

Each planner runs the mix with the library's default flags (backfill, chain
lane: what the bench runs) and with flags 0 (pure pairs: the planner alone
decides what shares the GPU). Reported: co-scheduler kernel time (median of
runs for Kernelet and OPT; every run for MC), and where Kernelet falls in the
MC distribution. Every run's outputs are compared bit for bit with the
kernels' plain launches.

    python -m paper_1303_5164_gb300.compare_plans --out plans.json [--mc 1000]
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

COPIES = 8


def run(out_path, mc=1000, mc_pure=200, reps=5, extra_flags=0):
    import torch
    import bench
    from workloads import gen
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    profs, doc = bench._load_profiles(K)
    mix = bench.mix_jobs()
    inputs = bench.generate(mix, min(16, os.cpu_count() or 1))
    names = [j[0] for j in mix]
    tens = [T.make(nm, x) for nm, x in zip(names, inputs)]
    types = T.MIX_TYPES
    one = {nm: tens[names.index(nm)] for nm in types}
    copies = {nm: [one[nm]] + [one[nm].replica() for _ in range(2 * COPIES - 1)] for nm in types}
    torch.cuda.synchronize()

    def runtime(flags=None, table=None, seed=0, policy=K.KL_RATIO_BALANCED, fixed=2, alpha=None):
        c = K.config_default()
        c.max_tenants = 1024
        if flags is not None:
            c.flags = flags
        c.plan_seed = seed
        c.ratio_policy = policy
        c.fixed_slots_a = fixed
        if alpha is not None:
            c.alpha_p = c.alpha_m = alpha
        rt = K.Runtime(c)
        rt.set_profiles(profs)
        if table is not None:
            rt.set_cp_table(*table)
        return rt

    S = runtime().run_stats().slots_per_sm
    f_hz = doc.get("f_sm_hz", 2.07e9)
    n_sm = doc.get("n_sm", 152)

    # ---- measured cIPC of every pair of types at every split (steady state)
    def pair_ipc(a, b, sa):
        rt = runtime(flags=0, policy=K.KL_RATIO_FIXED, fixed=sa, alpha=1e-9)
        # every copy of a first, then b: while both types are pending, the
        # lowest pending kernel (first role, sa slots) is of type a
        order = [(a, copies[a][k]) for k in range(COPIES)]
        order += [(b, copies[b][COPIES + k if a == b else k]) for k in range(COPIES)]
        best = None
        for _ in range(2):
            # slices small enough that blocks finish inside every phase: the
            # alone-tuned sizes (the run-level table hands a few copies one
            # slice per CTA, and a phase would then count no finished block)
            for _, t in order:
                rt.submit(t.type, t.args, slice_blocks=int(profs[t.type].slice_blocks_alone))
            rt.launch()
            assert rt.drain() == 0
            ph = rt.phases()
            ker = rt.run_stats().kernel_ns
            if best is None or ker < best[0]:
                best = (ker, ph)
        rt.close()
        ph = best[1]
        blk_a = blk_b = 0
        cyc = 0.0
        for k in range(1, len(ph) - 1):
            p, q = ph[k], ph[k + 1]
            if p.A < 0 or p.B < 0 or p.slots_a != sa:
                continue
            if (order[p.A][0], order[p.B][0]) != (a, b):
                continue
            c = (q.t_ns - p.t_ns) * 1e-9 * f_hz
            if c <= 0:
                continue
            blk_a += q.prev_done_a - p.done_a
            blk_b += q.prev_done_b - p.done_b
            cyc += c
        if cyc <= 0:
            return None
        ia, ib = profs[one[a].type].I_block, profs[one[b].type].I_block
        return blk_a * ia / (cyc * n_sm), blk_b * ib / (cyc * n_sm)

    meas = {}
    for a, b in itertools.combinations_with_replacement(types, 2):
        for sa in range(1, S):
            meas[(a, b, sa)] = pair_ipc(a, b, sa)
        print("pair", a, b, [meas[(a, b, sa)] for sa in range(1, S)], flush=True)
    solo = {}
    for a in types:
        v = meas[(a, a, S // 2)]
        solo[a] = (v[0] + v[1]) if v else None
    cp_meas = {}
    for (a, b, sa), v in meas.items():
        if v and solo[a] and solo[b] and v[0] / solo[a] + v[1] / solo[b] > 0:
            cp_meas[(a, b, sa)] = 1.0 - 1.0 / (v[0] / solo[a] + v[1] / solo[b])
    # OPT table: each type pair at its best measured split (both orientations)
    TC = K.KL_T_COUNT
    cp = [0.0] * (TC * TC)
    sl = [max(1, S // 2)] * (TC * TC)
    for a, b in itertools.combinations_with_replacement(types, 2):
        cands = [(cp_meas[(a, b, sa)], sa) for sa in range(1, S) if (a, b, sa) in cp_meas]
        if not cands:
            continue
        c, sa = max(cands)
        ta, tb = one[a].type, one[b].type
        cp[ta * TC + tb], sl[ta * TC + tb] = c, sa
        cp[tb * TC + ta], sl[tb * TC + ta] = c, S - sa
    # the model's table, for the record
    cp_model, sl_model, _ = runtime().cp_table()

    # ---- the mix under each planner; every planner must leave every output
    # equal (on the device, bit for bit) to the kernel's plain launch
    rt = runtime()
    for t in tens:
        for k in t.outputs:
            t.bufs[k].fill_(-1)
        rt.submit(t.type, t.args)
    rt.launch_baseline(K.KL_BASE_SERIAL, 1)
    assert rt.drain() == 0
    rt.close()
    ref = [{k: t.bufs[k].clone() for k in t.outputs} for t in tens]

    def mix_time(rt, n=reps):
        ts = []
        for _ in range(n):
            for t in tens:
                for k in t.outputs:
                    t.bufs[k].fill_(-1)
                rt.submit(t.type, t.args)
            rt.launch()
            assert rt.drain() == 0
            ts.append(rt.run_stats().kernel_ns / 1e6)
            for t, r in zip(tens, ref):
                for k, v in r.items():
                    if not torch.equal(t.bufs[k], v):
                        raise AssertionError(f"{t.name}.{k}: output differs from the plain launch")
        return ts

    res = {"slots_per_sm": S, "cp_measured": {f"{a}+{b}@{sa}": v for (a, b, sa), v in cp_meas.items()},
           "solo_ipc_measured": solo,
           "opt_table": {f"{a}+{b}": (cp[one[a].type * TC + one[b].type], sl[one[a].type * TC + one[b].type])
                         for a, b in itertools.combinations_with_replacement(types, 2)},
           "model_table": {f"{a}+{b}": (cp_model[one[a].type * TC + one[b].type],
                                        sl_model[one[a].type * TC + one[b].type])
                           for a, b in itertools.combinations_with_replacement(types, 2)}}
    res["extra_flags"] = extra_flags
    for label, flags, n_mc in (("default_flags", K.config_default().flags, mc), ("pure_pairs", 0, mc_pure)):
        flags |= extra_flags
        rt = runtime(flags=flags)
        kern = mix_time(rt)
        rt.close()
        rt = runtime(flags=flags, table=(cp, sl))
        opt = mix_time(rt)
        rt.close()
        alt = None
        if flags & K.KL_CFG_CHAIN_LANE:
            # the other reading of Section 4.4: the pair model alone, or the
            # phase the device runs (pair + chain-lane kernel) scored together
            rt = runtime(flags=flags ^ K.KL_CFG_PHASE_MODEL)
            alt = mix_time(rt)
            rt.close()
        alt_name = "phase_model" if not (flags & K.KL_CFG_PHASE_MODEL) else "pair_model"
        base_flags = flags
        mcs = []
        for seed in range(1, n_mc + 1):
            rt = runtime(flags=base_flags | K.KL_CFG_RANDOM_PLAN, seed=seed)
            mcs.append(mix_time(rt, 1)[0])
            rt.close()
        k_med, o_med = statistics.median(kern), statistics.median(opt)
        mcs_sorted = sorted(mcs)
        res[label] = {"kernelet_ms": kern, "opt_ms": opt, "kernelet_median_ms": k_med, "opt_median_ms": o_med,
                      "kernelet_vs_opt": k_med / o_med - 1.0, "mc_runs": len(mcs),
                      "mc_min_ms": mcs_sorted[0], "mc_median_ms": statistics.median(mcs),
                      "mc_max_ms": mcs_sorted[-1],
                      "mc_fraction_faster_than_kernelet": sum(x < k_med for x in mcs) / len(mcs),
                      "kernelet_uses": "phase_model" if flags & K.KL_CFG_PHASE_MODEL else "pair_model",
                      f"kernelet_{alt_name}_median_ms": statistics.median(alt) if alt else None,
                      f"mc_fraction_faster_than_{alt_name}":
                          sum(x < statistics.median(alt) for x in mcs) / len(mcs) if alt else None,
                      "mc_cdf_ms": [mcs_sorted[int(q * (len(mcs) - 1))] for q in
                                    (0.0, 0.01, 0.05, 0.1, 0.25, 0.5, 0.75, 0.9, 0.95, 0.99, 1.0)]}
        print(label, json.dumps({k: v for k, v in res[label].items() if k not in ("kernelet_ms", "opt_ms")}),
              flush=True)
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--mc", type=int, default=1000)
    ap.add_argument("--mc-pure", type=int, default=200)
    ap.add_argument("--extra-flags", type=int, default=0, help="kl_config.flags bits added to every arm")
    a = ap.parse_args(argv)
    run(a.out, a.mc, a.mc_pure, extra_flags=a.extra_flags)


if __name__ == "__main__":
    main()
