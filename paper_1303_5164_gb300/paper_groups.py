"""The paper's workload groups (Section 5.1, Table tb:workloads) on the GPU.

CI = BS, MM, TEA, MRIQ (compute-intensive); MI = PC, SPMV, ST, SAD
(memory-intensive); MIX = PC, BS, TEA, SAD; ALL = all eight. Each group is
1000 kernel instances, types drawn uniformly from the group in a seeded order
(equal arrival rates, all pending at once), run as one co-scheduled batch, as
plain launches on 32 streams and on one stream; after each arm every output
equals the same kernel's plain launch bit for bit. Instance sizes are the paper's
inputs scaled down (listed in SIZES) so that a group runs in about a second.
Inputs are shared per type and outputs rotate over 32 replicas per type; all
eight kernels are pure functions of their inputs, so two instances that share
a replica store identical values.

    python -m paper_1303_5164_gb300.paper_groups --out groups.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# paper name -> tenant type
PAPER = {"PC": "pchase", "SAD": "sad", "SPMV": "spmv_csr", "ST": "stencil", "MM": "gemm_f32", "MRIQ": "mriq",
         "BS": "blackscholes", "TEA": "tea"}
GROUPS = {"CI": ["BS", "MM", "TEA", "MRIQ"], "MI": ["PC", "SPMV", "ST", "SAD"], "MIX": ["PC", "BS", "TEA", "SAD"],
          "ALL": ["PC", "SPMV", "ST", "BS", "MM", "TEA", "MRIQ", "SAD"]}
SIZES = {
    "pchase": dict(N=1 << 24, nchasers=16384, hops=256),       # paper: 40 M accesses
    "sad": dict(width=960, height=536, range=8),               # paper: 1920 x 1072
    "spmv_csr": dict(nrows=131072),                            # paper: 131072 rows, 16 nnz/row
    "stencil": dict(nx=128, ny=128, nz=128),                   # paper: 512^3
    "gemm_f32": dict(M=1024, N=512, K=512),                    # paper: 8192 x 2048 x 2048
    "mriq": dict(numK=512, numX=262144),                       # paper: 2 Mi points
    "blackscholes": dict(n=1 << 20),                           # paper: 40 M options
    "tea": dict(n=1 << 21),                                    # paper: 20 Mi blocks
}
INSTANCES = 1000
REPLICAS = 32


def make_base(T):
    """Per type: one tenant on seeded inputs at SIZES and REPLICAS - 1 more
    output replicas on the same inputs."""
    from workloads import gen
    base = {}
    for i, (nm, sz) in enumerate(SIZES.items()):
        t = T.make(nm, gen.gen_tenant(nm, 8, i, **sz))
        base[nm] = [t] + [t.replica() for _ in range(REPLICAS - 1)]
    return base


def group_tenants(base, g):
    """The INSTANCES kernels of group g, in their seeded order, each on the
    next output replica of its type; and how many of each type."""
    import numpy as np
    members = GROUPS[g]
    rng = np.random.default_rng([8, list(GROUPS).index(g)])
    kinds = [PAPER[members[k]] for k in rng.integers(0, len(members), INSTANCES)]
    seen = {nm: 0 for nm in SIZES}
    tens = []
    for nm in kinds:
        tens.append(base[nm][seen[nm] % REPLICAS])
        seen[nm] += 1
    return tens, seen


def group_config(K):
    """Runtime configuration of every arm: defaults with room for the whole group."""
    c = K.config_default()
    c.max_tenants = 4096
    return c


def poison(tens):
    """Overwrite every output of these tenants, so a result must come from the next run."""
    for t in {id(t): t for t in tens}.values():
        for k in t.outputs:
            t.bufs[k].fill_(-1)


def reference_outputs(K, base, profs):
    """Each type's output as one plain launch (serial stream): what every
    replica must hold after any arm (all eight kernels are deterministic)."""
    import torch
    ref = {}
    rt = K.Runtime(group_config(K))
    rt.set_profiles(profs)
    for nm, reps in base.items():
        poison([reps[0]])
        torch.cuda.synchronize()
        rt.submit(reps[0].type, reps[0].args)
        rt.launch_baseline(K.KL_BASE_SERIAL, 1)
        if rt.drain() != 0:
            raise RuntimeError(f"reference launch of {nm} failed")
        ref[nm] = reps[0].fetch()
    rt.close()
    return ref


def assert_outputs(tens, ref):
    """Every replica the group used holds its type's reference output, bit for bit."""
    import numpy as np
    for t in {id(t): t for t in tens}.values():
        got = t.fetch()
        for k, v in ref[t.name].items():
            a, b = np.ascontiguousarray(got[k]), np.ascontiguousarray(v)
            if a.shape != b.shape or a.tobytes() != b.tobytes():
                raise AssertionError(f"{t.name}.{k}: output differs from the plain launch")


def run(out_path, reps=3, nstreams=32):
    import statistics as st
    import torch
    import bench
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    profs, doc = bench._load_profiles(K)
    base = make_base(T)
    torch.cuda.synchronize()
    ref = reference_outputs(K, base, profs)
    res = {"instances": INSTANCES, "sizes": SIZES, "groups": {}}
    for g, members in GROUPS.items():
        tens, seen = group_tenants(base, g)

        def arm(mode):
            rt = K.Runtime(group_config(K))
            rt.set_profiles(profs)
            ts = []
            for _ in range(reps + 1):
                poison(tens)
                for t in tens:
                    rt.submit(t.type, t.args)
                if mode == "cosched":
                    rt.launch()
                elif mode == "multistream":
                    rt.launch_baseline(K.KL_BASE_MULTISTREAM, nstreams)
                else:
                    rt.launch_baseline(K.KL_BASE_SERIAL, 1)
                rc = rt.drain()
                if rc != 0:
                    raise RuntimeError(f"{g} {mode}: {K.lib().kl_strerror(rc).decode()}")
                ts.append(rt.run_stats().kernel_ns / 1e6)
            rt.close()
            assert_outputs(tens, ref)
            return st.median(ts[1:])

        co, ms, se = arm("cosched"), arm("multistream"), arm("serial")
        res["groups"][g] = {"members": members, "cosched_ms": co, "multistream_ms": ms, "serial_ms": se,
                            "speedup_vs_multistream": ms / co, "speedup_vs_serial": se / co,
                            "counts": {nm: n for nm, n in seen.items() if n}, "outputs": "checked"}
        print(g, json.dumps(res["groups"][g]), flush=True)
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    run(a.out)


if __name__ == "__main__":
    main()
