"""The testing kernels of Section 4.3 on the GPU: PUR and MUR against the
co-scheduling profit, and the pruning thresholds re-fit for GB300.

A testing kernel (KL_T_TESTMIX) mixes streaming loads and dependent fused
multiply-adds in a ratio set by its arguments; VARIANTS span memory-bound to
issue-bound kernels. Steps:

1. Counters of each variant as a plain launch (after the same command ran
   without ncu):
       ncu --metrics gpu__time_duration.sum,sm__cycles_elapsed.avg,smsp__inst_executed.sum,\
dram__bytes_read.sum,dram__bytes_write.sum --clock-control none -s 12 --csv --page raw \
           --log-file tk.csv python -m paper_1303_5164_gb300.testing_kernels --mode native
   PUR = warp instructions / (cycles x 4 schedulers x SMs); MUR = DRAM bytes /
   (time x measured HBM bandwidth) (reading Q14 of the two ratios).
2. Every pair of variants co-scheduled, pure pairs (no backfill), at each of
   the three slot splits, each variant also paired with a copy of itself.
   The sequential time of a and b is half of a's self-pair time plus half of
   b's (two kernels in one run amortise their launch and tail the same way
   whichever they are), and the pair's measured CP = 1 - T_pair / T_seq at
   its best split, so a self-pair has CP 0 (the variants are sized to run
   equally long alone):
       python -m paper_1303_5164_gb300.testing_kernels --mode pairs --counters tk.csv --out tk.json
3. The Section 4.3 regression of CP on |dPUR| and |dMUR|, and the largest
   thresholds (alpha_p, alpha_m) whose AND rule prunes no pair that gains
   more than CP_KEEP.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (loads per round, dependent fused multiply-adds per round)
VARIANTS = [(8, 0), (4, 0), (2, 0), (1, 0), (1, 1), (1, 2), (1, 4), (1, 8), (1, 16), (1, 32), (1, 64), (1, 256)]
NTHREADS = 1 << 20          # 4096 blocks of 256 threads
LOG2_IN = 26                # 256 MiB of input: every round streams from HBM
NATIVE_ITERS = 32
TARGET_US = 250.0           # each variant alone in the co-scheduler, about this long
CP_KEEP = 0.05              # pairs gaining more than this must survive pruning


def _inputs(iters_of):
    from workloads import gen
    return [gen.gen_testmix(9, i, log2_in=LOG2_IN, nthreads=NTHREADS, iters=iters_of(i), mem=m, alu=a)
            for i, (m, a) in enumerate(VARIANTS)]


def _tenant(T, inp, shared=None):
    """Device tenant; `shared` reuses another variant's input buffer (same data)."""
    import torch
    from paper_1303_5164_gb300 import kernelet as K
    if shared is None:
        return T.make("testmix", inp)
    b = {"in_": shared.bufs["in_"], "out": torch.empty(inp["nthreads"], dtype=torch.float32, device="cuda")}
    args = K.kl_args_testmix(b["in_"].data_ptr(), b["out"].data_ptr(), inp["n_in"], inp["nthreads"],
                             inp["iters"], inp["mem"], inp["alu"], 0, float(inp["c1"]), float(inp["c2"]))
    return T.Tenant("testmix", K.KL_T_TESTMIX, args, b, ["out"], 0)


def run_native(reps=2):
    """Every variant as a plain launch (warm-up pass first: skip it in ncu with -s 12)."""
    import torch
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    inps = _inputs(lambda i: NATIVE_ITERS)
    first = _tenant(T, inps[0])
    tens = [first] + [_tenant(T, x, first) for x in inps[1:]]
    rt = K.Runtime()
    for _ in range(1 + reps):
        for t in tens:
            rt.submit(t.type, t.args)
            rt.launch_baseline(K.KL_BASE_SERIAL, 1)
            assert rt.drain() == 0
        torch.cuda.synchronize()
    rt.close()
    print("native launches:", len(tens), "variants x", 1 + reps)


def counters(csv_path, hbm_gbs, n_sm):
    """PUR and MUR per variant from the ncu launches (variant order, after the warm-up pass)."""
    from paper_1303_5164_gb300.profile_tenants import _num, _read_ncu_csv
    rows = [r for r in _read_ncu_csv(csv_path) if "native_kernel<15>" in r.get("Kernel Name", "").replace(" ", "")]
    per = [[] for _ in VARIANTS]
    for k, r in enumerate(rows):
        per[k % len(VARIANTS)].append(r)
    out = []
    for rs in per:
        inst = sum(_num(r["smsp__inst_executed.sum"]) for r in rs)
        cyc = sum(_num(r["sm__cycles_elapsed.avg"]) for r in rs)
        dram = sum(_num(r["dram__bytes_read.sum"]) + _num(r["dram__bytes_write.sum"]) for r in rs)
        dur = sum(_num(r["gpu__time_duration.sum"]) * {"ns": 1, "nsecond": 1, "us": 1e3, "usecond": 1e3, "ms": 1e6,
                                                        "msecond": 1e6}.get(r.get("gpu__time_duration.sum_unit", "ns"), 1)
                  for r in rs)
        out.append({"PUR": inst / (cyc * 4.0 * n_sm) if cyc else None,
                    "MUR": dram / (dur * 1e-9 * hbm_gbs * 1e9) if dur else None, "launches": len(rs)})
    return out


def regression(pairs):
    """Least squares CP = b0 + bp |dPUR| + bm |dMUR| over the pairs, R^2, and the
    correlation of CP with each gap (Fig. pur_mur)."""
    import numpy as np
    X = np.array([[1.0, p["dPUR"], p["dMUR"]] for p in pairs])
    y = np.array([p["cp"] for p in pairs])
    beta, *_ = np.linalg.lstsq(X, y, rcond=None)
    res = y - X @ beta
    r2 = 1.0 - float(res @ res) / float(((y - y.mean()) ** 2).sum())
    corr = {k: float(np.corrcoef(X[:, i], y)[0, 1]) for i, k in ((1, "dPUR"), (2, "dMUR"))}
    return {"b0": float(beta[0]), "b_pur": float(beta[1]), "b_mur": float(beta[2]), "r2": r2, "corr": corr}


def refit_alpha(pairs, keep=CP_KEEP):
    """The thresholds of the AND rule (Section 4.3, reading Q5) that prune the
    most pairs while pruning none whose measured CP exceeds `keep`; ties to the
    smaller alpha_p + alpha_m."""
    best = None
    grid = [round(0.01 * k, 2) for k in range(0, 101)]
    for ap in grid:
        for am in grid:
            pr = [p for p in pairs if p["dPUR"] < ap and p["dMUR"] < am]
            if any(p["cp"] > keep for p in pr):
                continue
            key = (len(pr), -(ap + am))
            if best is None or key > best[0]:
                best = (key, ap, am, pr)
    (_, _), ap, am, pr = best
    return {"alpha_p": ap, "alpha_m": am, "pruned": len(pr), "pairs": len(pairs), "cp_keep": keep,
            "max_cp_pruned": max((p["cp"] for p in pr), default=None)}


def run_pairs(csv_path, out_path, reps=2):
    import statistics
    import torch
    import bench
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    hbm_gbs, _ = bench._measured_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    cnt = counters(csv_path, hbm_gbs, n_sm) if csv_path else [{} for _ in VARIANTS]

    def runtime(policy=None, sa=2):
        c = K.config_default()
        c.slots_per_sm = 4
        c.flags = 0                         # pure pairs: no backfill, chain lane or deep fill
        if policy is not None:
            c.ratio_policy = policy
            c.fixed_slots_a = sa
        return K.Runtime(c)

    def timed(rt, tens):
        ts = []
        for _ in range(reps + 1):
            for t in tens:
                rt.submit(t.type, t.args)
            rt.launch()
            assert rt.drain() == 0
            ts.append(rt.run_stats().kernel_ns / 1e3)
        return statistics.median(ts[1:])

    # calibrate the rounds so every variant runs about TARGET_US alone
    probe = _inputs(lambda i: 16)
    shared = _tenant(T, probe[0])
    rt = runtime()
    t16 = [timed(rt, [_tenant(T, x, shared)]) for x in probe]
    rt.close()
    iters = [max(2, int(round(16 * TARGET_US / t))) for t in t16]
    inps = _inputs(lambda i: iters[i])
    # two tenants per variant (a pair of one variant with itself needs two outputs)
    tens = [(_tenant(T, x, shared), _tenant(T, x, shared)) for x in inps]
    torch.cuda.synchronize()
    rt = runtime()
    solo = [timed(rt, [a]) for a, _ in tens]
    rt.close()
    tpair = {}
    for i, j in itertools.combinations_with_replacement(range(len(VARIANTS)), 2):
        tp = {}
        for sa in (1, 2, 3):
            rt = runtime(K.KL_RATIO_FIXED, sa)
            tp[sa] = timed(rt, [tens[i][0], tens[j][1]])
            rt.close()
        tpair[(i, j)] = tp
    pairs = []
    for (i, j), tp in tpair.items():
        best_sa = min(tp, key=tp.get)
        t_seq = 0.5 * min(tpair[(i, i)].values()) + 0.5 * min(tpair[(j, j)].values())
        cp = 1.0 - tp[best_sa] / t_seq
        e = {"a": i, "b": j, "t_pair_us": tp, "best_slots_a": best_sa, "cp": cp, "cp_vs_solo": 1.0 - tp[best_sa] / (solo[i] + solo[j])}
        if cnt[i].get("PUR") is not None and cnt[j].get("PUR") is not None:
            e["dPUR"] = abs(cnt[i]["PUR"] - cnt[j]["PUR"])
            e["dMUR"] = abs(cnt[i]["MUR"] - cnt[j]["MUR"])
        pairs.append(e)
        print("pair", i, j, json.dumps({k: v for k, v in e.items() if k != "t_pair_us"}), flush=True)
    res = {"variants": [{"mem": m, "alu": a, "iters": it, "solo_us": s, **c}
                        for (m, a), it, s, c in zip(VARIANTS, iters, solo, cnt)],
           "nthreads": NTHREADS, "n_in": 1 << LOG2_IN, "pairs": pairs}
    fit = [p for p in pairs if "dPUR" in p and p["a"] != p["b"]]
    if fit:
        res["regression"] = regression(fit)
        res["alpha"] = refit_alpha(fit)
        print("regression", json.dumps(res["regression"]), "alpha", json.dumps(res["alpha"]), flush=True)
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["native", "pairs"], required=True)
    ap.add_argument("--counters", default=None, help="ncu CSV of the native launches")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.mode == "native":
        return run_native()
    return run_pairs(a.counters, a.out)


if __name__ == "__main__":
    main()
