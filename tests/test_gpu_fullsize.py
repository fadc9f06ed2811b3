"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the 64-kernel mix (8 each of the FP32 GEMM 1024^3, CSR SpMV
of 1 Mi rows, Black-Scholes 4 Mi, pointer chase over 64 MiB with 65,536
chasers x 256 hops, triad 64 Mi, 256-bin histogram of 64 Mi bytes,
escape-time 2048^2, bitonic sort of 2^22 keys), generated exactly as
bench.py generates it, submitted through the C ABI with the default flags
and the measured profiles, and run as one co-scheduled launch. Every output
of every kernel is compared in full with the CPU oracle (bit-exact; SpMV
within its derived bound)."""
import numpy as np
import pytest

from tests import _expect as X

pytestmark = pytest.mark.gpu


def test_bench_mix_full_size_matches_oracle():
    import bench
    import torch
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    jobs = bench.mix_jobs()
    inputs = bench.generate(jobs, 16)  # spawn pool: safe after CUDA initialisation
    build.build()
    profs, _ = bench._load_profiles(K)
    c = K.config_default()
    c.max_tenants = 1024
    rt = K.Runtime(c)
    rt.set_profiles(profs)
    tens = [T.make(j[0], x) for j, x in zip(jobs, inputs)]
    for t in tens:
        for v in t.outputs:
            t.bufs[v].fill_(-1)  # poison: every output must be written by this run
    torch.cuda.synchronize()
    hs = [rt.submit(t.type, t.args) for t in tens]
    rt.launch()
    assert rt.drain() == 0
    assert rt.run_stats().slots_per_sm == 4  # the mix holds 64-register types: a 4-slot build
    for (nm, _, _, _), x, t, h in zip(jobs, inputs, tens, hs):
        assert rt.poll(h) == K.KL_DONE
        st = rt.stats(h)
        assert st.blocks == t.shape().total_blocks
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    rt.close()
    assert sorted({j[0] for j in jobs}) == sorted(T.MIX_TYPES) and len(jobs) == 64
