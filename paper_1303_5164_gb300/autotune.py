"""Slice-size selection (Section 4.1): the smallest slice whose overhead is
within p% (default 2%) of the unsliced execution.

On this runtime a slice is the block range one persistent CTA pulls with one
atomic. Tuning runs in the 4-slot co-scheduler builds (the light 8-slot build
off), where every run that mixes in a heavier type executes. For each type the kernel runs alone in the co-scheduler with slices of
1, 2, 4, ... blocks and with one slice per CTA and stage (the fewest pulls
that still use every slot). The paper's reference is the unsliced run and
assumes the overhead falls as slices grow; here it does not always (very
large slices unbalance the SMs), so T_ns is the fastest of the measured runs,
and the chosen size is the smallest with T_s / T_ns - 1 <= p.

With --copies N the kernel runs as N copies in one launch (the same inputs,
their own outputs), as it does in a co-scheduled run, where other kernels'
slices fill the slots one kernel leaves idle between its stages and at its
end; alone, a kernel with stage barriers favours slices that spread each
stage over every slot, in company the per-slice scheduling cost counts more.

    python -m paper_1303_5164_gb300.autotune --out slices.json [--p 0.02] [--copies 8]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def choose_slice(times, p):
    """Section 4.1's rule with the fastest measured run as the reference: the
    smallest slice size whose time is within a fraction p of the fastest."""
    tns = min(times.values())
    return min(c for c in times if times[c] / tns - 1.0 <= p)


def tune(types, p=0.02, reps=3, seed=6, copies=1):
    import torch
    from workloads import gen
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    # one slice size per type serves every run; mixed runs (every run holding
    # one of the heavier types) use the 4-slot builds, so tune there
    c = K.config_default()
    c.flags &= ~K.KL_CFG_LIGHT_BUILD
    rt = K.Runtime(c)
    n_sm = rt.model_params().n_sm
    out = {"p": p, "n_sm": n_sm, "copies": copies, "slices": {}, "times_us": {}, "overhead": {}, "slots_per_sm": {}}
    for i, ty in enumerate(types):
        inp = gen.gen_tenant(ty, seed, i, **T.SIZES_ALL[ty])
        t = T.make(ty, inp)
        group = [t] + [t.replica() for _ in range(copies - 1)]
        sh = t.shape()
        rt.submit(t.type, t.args)  # slots per SM of the build this type runs in
        rt.launch()
        assert rt.drain() == 0
        S = rt.run_stats().slots_per_sm
        stage_blocks = int(sh.grid[0]) if ty != "hist256" else int(sh.total_blocks - 1)
        ref = max(1, math.ceil(copies * stage_blocks / (n_sm * S)))
        cands = sorted({c for c in (1, 2, 4, 8, 16, 32, 64) if c <= stage_blocks} | {ref})

        def run(sl):
            best = float("inf")
            for _ in range(reps + 1):
                for x in group:
                    rt.submit(x.type, x.args, slice_blocks=sl)
                rt.launch()
                assert rt.drain() == 0
                best = min(best, rt.run_stats().kernel_ns / 1e3)
            return best

        times = {c: run(c) for c in cands}
        tns = min(times.values())
        chosen = choose_slice(times, p)
        out["slices"][ty] = chosen
        out["times_us"][ty] = {str(c): round(v, 2) for c, v in times.items()}
        out["overhead"][ty] = round(times[chosen] / tns - 1.0, 4)
        out["slots_per_sm"][ty] = S
        print(ty, "ref", ref, "chosen", chosen, out["times_us"][ty], flush=True)
        del t, group
        torch.cuda.empty_cache()
    rt.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--p", type=float, default=0.02)
    ap.add_argument("--types", default="gemm_f32,spmv_csr,blackscholes,pchase,triad,hist256,escape,bitonic,gather,"
                                       "tea,sad,stencil,mriq")
    ap.add_argument("--copies", type=int, default=1, help="copies of the kernel in each timed launch")
    a = ap.parse_args(argv)
    res = tune(a.types.split(","), a.p, copies=a.copies)
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
