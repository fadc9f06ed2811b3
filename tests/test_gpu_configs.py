"""GPU parity for the workloads the measurement scripts time, at their full
sizes and in the launch configuration each script uses, every output of every
kernel compared with the CPU oracle:

* the 512-tenant batch (bench.py --workload batch): types uniform over the
  eight mix kernels, grids log-uniform in [1, 4096] blocks, one persistent
  launch with the benchmark's runtime (default flags, measured profiles);
* the resource-heavy set (validate_heavy.py): the FP32 GEMM 4096^3 with
  96 KB tiles and its BF16 tensor-core variant, Black-Scholes 4 Mi at up to
  255 registers a thread, the histogram of 64 Mi bytes with 1024-thread
  blocks and the pointer chase over a 1 GiB cycle, each alone, every pair
  and all five together (three of them in resource-class kernels beside the
  co-scheduler);
* the paper's ALL group (paper_groups.py, Section 5.1): 1000 instances of the
  eight paper kernels at the group sizes, outputs on 32 replicas per type.

Slicing never changes a kernel's result (Section 2.2: blocks are
independent), so each output must equal the oracle's: bit for bit, SpMV and
the BF16 GEMM within their derived bounds, FP32 GEMMs too large for the chain
loop within the chain's bound everywhere and bit for bit on sampled entries."""
import os

import numpy as np
import pytest

from tests import _expect as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    from paper_1303_5164_gb300 import build, kernelet
    build.build()
    return kernelet


@pytest.fixture(scope="module")
def T():
    from paper_1303_5164_gb300 import tenants
    return tenants


def _poison(tens):
    import torch
    for t in {id(t): t for t in tens}.values():
        for k in t.outputs:
            t.bufs[k].fill_(-1)
    torch.cuda.synchronize()


def _oracle_pool(jobs):
    """Expected outputs of every job, computed in a spawn pool (safe after
    CUDA initialisation): each worker regenerates its job's seeded inputs."""
    import multiprocessing as mp
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(X.expected_for_job, jobs, chunksize=1)


def _check(nm, inp, got, exp):
    if exp is None:
        X.check_gemm_f32_large(inp, got["C"])
    else:
        X.check(nm, inp, got, exp)


def test_batch_512_tenants_full_size(K, T):
    import bench
    import torch
    jobs = bench.batch_jobs()
    assert len(jobs) == 512
    inputs = bench.generate(jobs, os.cpu_count() or 1)
    tens = [T.make(j[0], x) for j, x in zip(jobs, inputs)]
    rt, _, _ = bench.make_runtime(K, 0, torch.cuda.current_stream().cuda_stream)
    _poison(tens)
    hs = [rt.submit(t.type, t.args) for t in tens]
    rt.launch()
    assert rt.drain() == 0
    for t, h in zip(tens, hs):
        assert rt.poll(h) == K.KL_DONE
        assert rt.stats(h).blocks == t.shape().total_blocks
    got = [t.fetch() for t in tens]
    rt.close()
    del tens
    exps = _oracle_pool(jobs)
    for j, x, g, e in zip(jobs, inputs, got, exps):
        _check(j[0], x, g, e)


def test_heavy_set_alone_pairs_and_all(K, T):
    import itertools
    from paper_1303_5164_gb300 import validate_heavy as VH
    inputs = VH.heavy_inputs()
    names = list(VH.HEAVY)
    tens = {nm: T.make(nm, inputs[nm]) for nm in names}
    exp = {nm: X.expected(nm, inputs[nm]) for nm in names if nm != "gemm_f32_big"}
    big = inputs["gemm_f32_big"]
    from oracle import tenants as OT
    big_exact = OT.gemm_f32_exact(big["A"], big["B"])   # 4096^3: the chain oracle only on samples
    cfg, mp, profs = VH.heavy_setup(K)
    runs = [[nm] for nm in names] + [list(p) for p in itertools.combinations(names, 2)] + [names]
    for sel in runs:
        rt = VH.heavy_runtime(K, cfg, mp, profs)
        _poison([tens[nm] for nm in sel])
        hs = [rt.submit(tens[nm].type, tens[nm].args) for nm in sel]
        rt.launch()
        assert rt.drain() == 0, sel
        for nm, h in zip(sel, hs):
            assert rt.poll(h) == K.KL_DONE, (sel, nm)
            assert rt.stats(h).blocks == tens[nm].shape().total_blocks, (sel, nm)
            if nm == "gemm_f32_big":
                X.check_gemm_f32_large(big, tens[nm].fetch()["C"], exact=big_exact)
            else:
                X.check(nm, inputs[nm], tens[nm].fetch(), exp[nm])
        rt.close()


def test_paper_group_all_full_size(K, T):
    import bench
    import torch
    from workloads import gen
    from paper_1303_5164_gb300 import paper_groups as PG
    base = PG.make_base(T)
    tens, seen = PG.group_tenants(base, "ALL")
    assert len(tens) == PG.INSTANCES and all(seen[nm] > 0 for nm in PG.SIZES)
    profs, _ = bench._load_profiles(K)
    rt = K.Runtime(PG.group_config(K))
    rt.set_profiles(profs)
    PG.poison(tens)
    torch.cuda.synchronize()
    hs = [rt.submit(t.type, t.args) for t in tens]
    rt.launch()
    assert rt.drain() == 0
    assert all(rt.poll(h) == K.KL_DONE for h in hs)
    rt.close()
    for i, (nm, sz) in enumerate(PG.SIZES.items()):
        inp = gen.gen_tenant(nm, 8, i, **sz)
        exp = X.expected(nm, inp)
        used = {id(t): t for t in tens if t.name == nm}
        assert len(used) == min(seen[nm], PG.REPLICAS)
        for t in used.values():
            X.check(nm, inp, t.fetch(), exp)
