"""Runs tenants as plain launches (one instance per type, after a warm-up) so
that an external profiler (ncu) can measure them; also the driver for the
per-type model inputs of Section 4.4 (R_m, sectors per request, instructions
per block, IPC, PUR/MUR) when run under ncu with --csv.

    python -m paper_1303_5164_gb300.profile_tenants [--types a,b] [--mode native|cosched]
                                                    [--scale 1.0] [--reps 1]

--mode cosched runs each type alone through the persistent co-scheduler
instead (the kernel name is cosched_kernel). --scale shrinks the mix sizes.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def scaled_sizes(name, scale):
    from paper_1303_5164_gb300.tenants import SIZES_MIX
    s = dict(SIZES_MIX[name])
    if scale == 1.0:
        return s
    if name == "gemm_f32":
        m = max(64, int(1024 * scale ** (1 / 3)) // 64 * 64)
        return dict(M=m, N=m, K=m)
    if name == "escape":
        w = max(64, int(2048 * scale ** 0.5))
        return dict(width=w, height=w, max_iter=256)
    if name == "bitonic":
        return dict(log2n=max(12, int(22 + __import__("math").log2(scale))))
    if name == "pchase":
        return dict(N=max(1 << 16, int(s["N"] * scale)), nchasers=max(256, int(65536 * scale)), hops=256)
    key = {"spmv_csr": "nrows", "blackscholes": "n", "triad": "n", "hist256": "n"}[name]
    s[key] = max(4096, int(s[key] * scale))
    return s


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--types", default="gemm_f32,spmv_csr,blackscholes,pchase,triad,hist256,escape,bitonic")
    ap.add_argument("--mode", default="native", choices=["native", "cosched"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--reps", type=int, default=1)
    args = ap.parse_args(argv)
    from workloads import gen
    types = args.types.split(",")
    inputs = [gen.gen_tenant(t, 5, i, **scaled_sizes(t, args.scale)) for i, t in enumerate(types)]
    import torch
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    tens = [T.make(t, x) for t, x in zip(types, inputs)]
    rt = K.Runtime()

    def run(t):
        rt.submit(t.type, t.args)
        if args.mode == "native":
            rt.launch_baseline(K.KL_BASE_SERIAL, 1)
        else:
            rt.launch()
        rc = rt.drain()
        if rc != 0:
            raise RuntimeError(f"{t.name}: {K.lib().kl_strerror(rc).decode()}")

    for t in tens:          # warm-up pass (not of interest to the profiler: use -s)
        run(t)
    torch.cuda.synchronize()
    for _ in range(args.reps):
        for t in tens:
            run(t)
    torch.cuda.synchronize()
    rt.close()
    print("profiled:", ",".join(types), args.mode)


if __name__ == "__main__":
    main()
