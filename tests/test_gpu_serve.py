"""GPU tests of serving mode (continuous batching): kernels submitted while
the persistent co-scheduler runs are taken in and co-scheduled with the work
already on the device (Algorithm 1 with arrivals), each result equals the
oracle's and the same kernel run alone; admission by in-flight slots and by
device-memory footprint; kernels pending before the start keep their handles;
the idle limit ends a run by itself; the plain multi-stream comparator."""
import time

import numpy as np
import pytest

from tests import _expect as X
from workloads import gen

pytestmark = pytest.mark.gpu

WAVE = {
    "gemm_f32": dict(M=256, N=192, K=128),
    "spmv_csr": dict(nrows=20000),
    "blackscholes": dict(n=100000),
    "triad": dict(n=1 << 20),
    "hist256": dict(n=1 << 20),
    "escape": dict(width=256, height=256, max_iter=256),
    "bitonic": dict(log2n=16),
    "gather": dict(n=1 << 18),
}
# one long latency-bound kernel (256 chasers x 60,000 dependent loads over
# 64 MB, tens of milliseconds) keeps the device busy while later kernels arrive
LONG = dict(N=1 << 24, nchasers=256, hops=60000)


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


def _alone(K, rt, ten):
    import torch
    for v in ten.outputs:
        ten.bufs[v].fill_(-1)
    torch.cuda.synchronize()
    ten_h = rt.submit(ten.type, ten.args)
    assert rt.drain() == 0
    assert rt.poll(ten_h) == K.KL_DONE
    return ten.fetch()


def test_serve_arrivals_overlap_and_match_alone(K, T):
    rt = _runtime(K, slots_per_sm=4)
    long_in = gen.gen_pchase(5, 99, **LONG)
    long_t = T.make("pchase", long_in)
    waves = []
    for w in range(3):
        names = list(WAVE)
        np.random.default_rng(w).shuffle(names)
        waves.append([(nm, gen.gen_tenant(nm, 5, 10 * w + i, **WAVE[nm])) for i, nm in enumerate(names)])
    tens = [[(nm, x, T.make(nm, x)) for nm, x in wv] for wv in waves]
    import torch
    torch.cuda.synchronize()
    rt.serve_start()
    h_long = rt.submit(long_t.type, long_t.args)
    handles = []
    for wv in tens:
        time.sleep(0.002)  # later waves arrive while earlier kernels run
        handles.append([rt.submit(t.type, t.args) for _, _, t in wv])
    for hs in handles:
        for h in hs:
            assert rt.wait(h, 20_000_000_000) == 0
    assert rt.wait(h_long, 20_000_000_000) == 0
    seen = set()
    for _ in range(100):
        seen.update(rt.reap())
        if len(seen) == 1 + sum(len(hs) for hs in handles):
            break
        time.sleep(0.001)
    assert seen == {h_long, *[h for hs in handles for h in hs]}
    st_long = rt.stats(h_long)
    st = [rt.stats(h) for hs in handles for h in hs]
    assert rt.serve_stop() == 0
    # every kernel ran to completion and the later arrivals shared the device
    # with the long kernel: they started before it ended
    assert all(s.state == K.KL_DONE and s.t_done_host_ns >= s.t_submit_ns for s in st)
    assert sum(s.t_start_ns < st_long.t_end_ns for s in st) >= len(WAVE)
    rs = rt.run_stats()
    assert rs.error == 0 and rs.n_tenants == 1 + len(st) and rs.n_phases >= 2
    # results: the oracle's, and bit-identical to each kernel run alone
    X.check("pchase", long_in, long_t.fetch(), X.expected("pchase", long_in))
    in_serve = [[t.fetch() for _, _, t in wv] for wv in tens]
    for wv, outs in zip(tens, in_serve):
        for (nm, x, t), got in zip(wv, outs):
            X.check(nm, x, got, X.expected(nm, x))
            alone = _alone(K, rt, t)
            for k in got:
                assert X.same_bits(alone[k], got[k]), (nm, k)
    rt.close()


def test_serve_admission_by_slots_and_footprint(K, T):
    rt = _runtime(K, max_tenants=4, mem_cap_bytes=1000)
    long_t = T.make("pchase", gen.gen_pchase(6, 0, **LONG))
    small = [T.make("triad", gen.gen_triad(6, 1 + i, 1 << 16)) for i in range(4)]
    rt.serve_start()
    h0 = rt.try_submit(long_t.type, long_t.args, footprint=600)
    assert h0 is not None
    # over the memory cap while the long kernel is in flight
    assert rt.try_submit(small[0].type, small[0].args, footprint=500) is None
    hs = [rt.try_submit(t.type, t.args, footprint=100) for t in small[:3]]
    assert all(h is not None for h in hs)
    # four kernels in flight: no slot left until one completes
    for h in hs:
        assert rt.wait(h, 10_000_000_000) == 0
    if rt.poll(h0) != K.KL_DONE:
        assert rt.try_submit(small[3].type, small[3].args, footprint=500) is None
    assert rt.wait(h0, 20_000_000_000) == 0
    h4 = rt.try_submit(small[3].type, small[3].args, footprint=500)
    assert h4 is not None and rt.wait(h4, 10_000_000_000) == 0
    assert rt.serve_stop() == 0
    rt.close()


def test_serve_full_slots_reject(K, T):
    rt = _runtime(K, max_tenants=2)
    longs = [T.make("pchase", gen.gen_pchase(7, i, **LONG)) for i in range(2)]
    extra = T.make("triad", gen.gen_triad(7, 5, 1 << 16))
    rt.serve_start()
    hs = [rt.submit(t.type, t.args) for t in longs]
    assert rt.try_submit(extra.type, extra.args) is None or rt.poll(hs[0]) == K.KL_DONE
    for h in hs:
        assert rt.wait(h, 20_000_000_000) == 0
    assert rt.serve_stop() == 0
    rt.close()


def test_serve_pending_keep_handles_and_restart(K, T):
    rt = _runtime(K)
    ins = [("hist256", gen.gen_hist256(8, i, 70000)) for i in range(3)]
    tens = [T.make(nm, x) for nm, x in ins]
    pre = [rt.submit(t.type, t.args) for t in tens]
    rt.serve_start()
    for h in pre:
        assert rt.wait(h, 10_000_000_000) == 0
    with pytest.raises(K.KLError):
        rt.launch()  # batch launches are refused while serving
    assert rt.serve_stop() == 0
    for (nm, x), t in zip(ins, tens):
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    # batch mode works again, and so does a second serving run
    bs_in = gen.gen_blackscholes(8, 9, 5000)
    bs = T.make("blackscholes", bs_in)
    assert rt.poll(rt.submit(bs.type, bs.args)) == K.KL_PENDING
    assert rt.drain() == 0
    X.check("blackscholes", bs_in, bs.fetch(), X.expected("blackscholes", bs_in))
    import torch
    for t in tens:
        t.bufs["hist"].fill_(7)
    # the serving kernel holds the runtime's stream until kl_serve_stop: inputs
    # are made ready before the start, not queued behind it
    torch.cuda.synchronize()
    rt.serve_start()
    hs = [rt.submit(t.type, t.args) for t in tens]
    for h in hs:
        assert rt.wait(h, 10_000_000_000) == 0
    assert rt.serve_stop() == 0
    for (nm, x), t in zip(ins, tens):
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    rt.close()


def test_serve_idle_limit_ends_the_run(K, T):
    rt = _runtime(K)
    rt.serve_start(idle_limit_ns=50_000_000)
    time.sleep(0.5)
    t = T.make("triad", gen.gen_triad(9, 0, 4096))
    with pytest.raises(K.KLError) as e:
        rt.submit(t.type, t.args)
    assert e.value.code == K.KL_ESTATE
    assert rt.serve_stop() == 0
    assert rt.run_stats().n_tenants == 0
    rt.close()


@pytest.mark.parametrize("mode,nstreams", [("multistream", 4), ("serial", 1)])
def test_serve_plain_launch_comparator(K, T, mode, nstreams):
    m = K.KL_BASE_MULTISTREAM if mode == "multistream" else K.KL_BASE_SERIAL
    rt = _runtime(K)
    items = [(nm, gen.gen_tenant(nm, 10, i, **WAVE[nm])) for i, nm in enumerate(WAVE)]
    tens = [T.make(nm, x) for nm, x in items]
    rt.serve_start(m, nstreams)
    hs = [rt.submit(t.type, t.args) for t in tens]
    got = set()
    for _ in range(10000):
        got.update(rt.reap())
        if len(got) == len(hs):
            break
        time.sleep(0.0005)
    assert got == set(hs)
    assert rt.serve_stop() == 0
    for (nm, x), t, h in zip(items, tens, hs):
        assert rt.stats(h).state == K.KL_DONE
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    rt.close()


def test_serve_tensor_core_build(K, T):
    # serving with KL_CFG_SERVE_TC runs the BF16 GEMM among the arrivals;
    # without it the type is refused
    import torch
    g_in = gen.gen_gemm_bf16(13, 0, 512, 256, 1024)
    b_in = gen.gen_blackscholes(13, 1, 200000)
    g, b = T.make("gemm_bf16", g_in), T.make("blackscholes", b_in)
    torch.cuda.synchronize()
    rt = _runtime(K)
    rt.serve_start()
    with pytest.raises(K.KLError) as e:
        rt.submit(g.type, g.args)
    assert e.value.code == K.KL_EINVAL
    assert rt.serve_stop() == 0
    rt.close()
    c = K.config_default()
    c.flags |= K.KL_CFG_SERVE_TC
    rt = K.Runtime(c)
    rt.serve_start()
    hs = [rt.submit(g.type, g.args), rt.submit(b.type, b.args)]
    for h in hs:
        assert rt.wait(h, 20_000_000_000) == 0
    assert rt.serve_stop() == 0
    X.check("gemm_bf16", g_in, g.fetch(), X.expected("gemm_bf16", g_in))
    X.check("blackscholes", b_in, b.fetch(), X.expected("blackscholes", b_in))
    rt.close()
