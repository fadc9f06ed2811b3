"""Ablations of the Markov model on GB300 measurements (Section 5.3, "model
optimizations": the uncoalesced-access state and the multiple warp
schedulers; plus the latency each type waits on).

Measured inputs, both from this GPU:
  * profiles_gb300.json: per type, the ncu counters of a plain launch (model
    inputs, solo IPC per SM, average warps per SM);
  * pairs_gb300.json (validate_pairs.py --out): each mix type alone in the
    co-scheduler at 4 slots, and every pair of the eight mix types at the
    model's split, with the measured per-kernel IPCs and CP.

The runtime's own model (kl_model_ipc, kl_model_pair) predicts each of them
under these readings:
  full         three-state chain (coalesced and uncoalesced waits), four
               schedulers per SM (virtual SM), L0 = the L2 latency for working
               sets under half the L2 and the DRAM latency otherwise
  two_state    uncoalesced accesses modelled as coalesced (one waiting state)
  one_sched    one scheduler per SM: the whole SM is one virtual SM (two-state
               chains, as the joint three-state chain of a pair then exceeds
               the evaluator's 4096 states; compare with two_state)
  dram_L0      every type waits the DRAM latency
Reported: mean absolute IPC error per SM (peak 4) for plain-launch solo runs,
co-scheduled solo runs and the kernels of the 28 pairs, and the Spearman rank
correlation of predicted and measured CP over the pairs.

    python -m paper_1303_5164_gb300.model_ablation [--pairs pairs_gb300.json] [--out ablation.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))

VARIANTS = {
    "full": dict(states=3, n_sched=4, dram_l0=False),
    "two_state": dict(states=2, n_sched=4, dram_l0=False),
    "one_sched": dict(states=2, n_sched=1, dram_l0=False),
    "dram_L0": dict(states=3, n_sched=4, dram_l0=True),
}
SLOT_WARPS = 8      # warps of one co-scheduler slot


def _spearman(x, y):
    import numpy as np
    rx = np.argsort(np.argsort(x)).astype(float)
    ry = np.argsort(np.argsort(y)).astype(float)
    return float(np.corrcoef(rx, ry)[0, 1])


def evaluate(doc, pairs_doc=None):
    from paper_1303_5164_gb300 import kernelet as K
    lat = doc["latency"]
    f = doc["f_sm_hz"]
    fit_types = doc["ipc_mae_types"]
    out = {}
    for vname, v in VARIANTS.items():
        mp = K.kl_model_params()
        mp.n_sm, mp.n_sched, mp.f_sm_hz = doc["n_sm"], v["n_sched"], f
        mp.dram_bytes_per_s, mp.sector_bytes, mp.a0, mp.b0 = doc["dram_bytes_per_s"], 32.0, doc["a0"], doc["b0"]

        def prof(name):
            e = doc["types"][name]
            p = K.kl_profile()
            for k in ("R_m", "f_u", "m_c", "m_u", "L0", "I_block", "PUR", "MUR"):
                setattr(p, k, float(e[k]))
            if v["dram_l0"]:
                p.L0 = lat["dram_ns_per_hop"] * 1e-9 * f
            p.warps_per_block, p.valid = 8, 1
            return p

        r = {}
        # plain launches: the measured average warps per SM
        errs = {}
        for name in fit_types:
            e = doc["types"][name]
            w = max(1, min(64 // v["n_sched"], int(round(e["warps_per_sm"] / v["n_sched"]))))
            pred = K.model_ipc(mp, [prof(name)], [w], v["states"])[0]
            errs[name] = pred - e["ipc_measured"]
        r["solo_plain_mae"] = sum(abs(x) for x in errs.values()) / len(errs)
        r["solo_plain_err"] = errs
        if pairs_doc:
            S = pairs_doc["slots_per_sm"]
            errs = {}
            for name, e in pairs_doc["solo"].items():
                if e.get("ipc_measured") is None:
                    continue
                w = max(1, int(round(S * SLOT_WARPS / v["n_sched"])))
                errs[name] = K.model_ipc(mp, [prof(name)], [w], v["states"])[0] - e["ipc_measured"]
            r["solo_cosched_mae"] = sum(abs(x) for x in errs.values()) / len(errs)
            kerr, cps_m, cps_p = [], [], []
            for key, e in pairs_doc["pairs"].items():
                a, b = key.split("+")
                if None in e["cipc_measured"]:
                    continue
                pr = K.model_pair(mp, prof(a), prof(b), S, v["states"])
                sa = e["slots_a"]
                kerr += [abs(pr["cipc_a"][sa - 1] - e["cipc_measured"][0]),
                         abs(pr["cipc_b"][sa - 1] - e["cipc_measured"][1])]
                if e.get("cp_measured") is not None:
                    cps_m.append(e["cp_measured"])
                    cps_p.append(pr["cp"][sa - 1])
            r["pair_kernel_mae"] = sum(kerr) / len(kerr)
            r["cp_spearman"] = _spearman(cps_p, cps_m) if len(cps_m) > 2 else None
            r["pairs"] = len(kerr) // 2
        out[vname] = r
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--profiles", default=os.path.join(HERE, "profiles_gb300.json"))
    ap.add_argument("--pairs", default=os.path.join(HERE, "pairs_gb300.json"))
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from paper_1303_5164_gb300 import build
    build.build()
    doc = json.load(open(a.profiles))
    pairs_doc = json.load(open(a.pairs)) if a.pairs and os.path.exists(a.pairs) else None
    res = evaluate(doc, pairs_doc)
    summary = {k: {m: (round(x, 3) if isinstance(x, float) else x) for m, x in v.items() if not m.endswith("_err")}
               for k, v in res.items()}
    print(json.dumps(summary, indent=1))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
