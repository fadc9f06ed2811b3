"""Failures made on the host, tested without any GPU fault:

* kl_wait with a zero timeout on a kernel that is still running returns
  KL_ETIMEDOUT and leaves it running; kl_wait on a kernel no launch has
  started returns KL_ESTATE;
* eight host threads call kl_submit at the same time (the header promises a
  runtime may be shared by threads): every kernel gets its own handle and,
  after one kl_drain, its correct output;
* serving: a submitter thread stops in the middle of a stream (it has staged a
  descriptor in the mapped ring and never publishes it): kl_serve_stop still
  retires the run cleanly, every published kernel completes with the oracle's
  output, the unpublished one never runs (its output stays untouched) and
  ends in KL_ERROR, and the runtime serves again afterwards;
* a staged burst becomes visible only at kl_publish (Algorithm 1: the burst
  arrives at once and is planned once);
* a batch submitted with kl_submit_batch while a run is in flight joins the
  next run, not the running one: kl_wait_run returns with it still pending,
  the next kl_launch runs it, and both batches match the oracle; a batch with
  a bad descriptor in the middle admits the kernels before it and reports
  how many."""
import ctypes as C
import threading
import time

import numpy as np
import pytest

from tests import _expect as X
from workloads import gen

pytestmark = pytest.mark.gpu

# 256 chasers x 60,000 dependent loads over 64 MB: tens of milliseconds
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


def _still_poisoned(a) -> bool:
    """Every element still holds the -1 that _poison wrote (-1.0 for floats)."""
    a = np.asarray(a)
    return bool(np.all(a == -1.0)) if a.dtype.kind == "f" else bool(np.all(a.view(np.int32) == -1))


def _poison(tens):
    import torch
    for t in tens:
        for k in t.outputs:
            t.bufs[k].fill_(-1)
    torch.cuda.synchronize()


def test_wait_zero_timeout_on_a_running_kernel(K, T):
    rt = K.Runtime()
    x = gen.gen_pchase(21, 0, **LONG)
    t = T.make("pchase", x)
    _poison([t])
    h = rt.submit(t.type, t.args)
    assert rt.wait(h, 0) == K.KL_ESTATE          # still in R: no launch has started it
    rt.launch()
    assert rt.wait(h, 0) == K.KL_ETIMEDOUT       # running: the wait expires at once
    assert rt.poll(h) == K.KL_RUNNING
    assert rt.wait(h, 1000) == K.KL_ETIMEDOUT     # 1 us: still running, still not an error
    assert rt.drain() == 0
    assert rt.wait(h, 0) == 0 and rt.poll(h) == K.KL_DONE
    X.check("pchase", x, t.fetch(), X.expected("pchase", x))
    rt.close()


def test_eight_threads_submit_at_once(K, T):
    names = ["blackscholes", "triad", "hist256", "gather", "escape", "spmv_csr", "bitonic", "gemm_f32"]
    sizes = {"blackscholes": dict(n=50001), "triad": dict(n=200000), "hist256": dict(n=100003),
             "gather": dict(n=70000), "escape": dict(width=200, height=90, max_iter=64),
             "spmv_csr": dict(nrows=7000), "bitonic": dict(log2n=13), "gemm_f32": dict(M=130, N=72, K=40)}
    per_thread = 8
    items = [[(nm, gen.gen_tenant(nm, 22, 100 * k + i, **sizes[nm])) for i, nm in
              enumerate(np.random.default_rng(k).permutation(names))] for k in range(8)]
    tens = [[T.make(nm, x) for nm, x in row] for row in items]
    _poison([t for row in tens for t in row])
    rt = K.Runtime()
    L = K.lib()
    descs = [[K.make_desc(t.type, t.args) for t in row] for row in tens]
    handles = [[0] * per_thread for _ in range(8)]
    codes = [[None] * per_thread for _ in range(8)]
    go = threading.Barrier(8)

    def submitter(k):
        go.wait()
        h = C.c_uint64()
        for i in range(per_thread):
            # ctypes drops the GIL for the call: the eight threads really race
            codes[k][i] = L.kl_submit(rt._h, C.byref(descs[k][i]), C.byref(h))
            handles[k][i] = h.value

    ths = [threading.Thread(target=submitter, args=(k,)) for k in range(8)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert all(c == 0 for row in codes for c in row)
    flat = [h for row in handles for h in row]
    assert len(set(flat)) == 64 and 0 not in flat
    assert rt.drain() == 0
    for row_items, row_tens, row_h in zip(items, tens, handles):
        for (nm, x), t, h in zip(row_items, row_tens, row_h):
            assert rt.poll(h) == K.KL_DONE
            X.check(nm, x, t.fetch(), X.expected(nm, x))
    rt.close()


def test_serving_submitter_stops_mid_stream(K, T):
    import torch
    rt = K.Runtime()
    long_x = gen.gen_pchase(23, 0, **LONG)
    long_t = T.make("pchase", long_x)
    xs = [("triad", gen.gen_triad(23, 1 + i, 1 << 18)) for i in range(6)]
    tens = [T.make(nm, x) for nm, x in xs]
    orphan_x = gen.gen_blackscholes(23, 9, 40000)
    orphan = T.make("blackscholes", orphan_x)
    _poison([long_t, orphan] + tens)
    rt.serve_start()
    h_long = rt.submit(long_t.type, long_t.args)
    out = {}

    def submitter():
        hs = []
        for t in tens:
            hs.append(rt.submit(t.type, t.args))
            time.sleep(0.0005)
        # stops here: the next descriptor is written into the ring but its
        # tail is never published
        out["orphan"] = rt.submit(orphan.type, orphan.args, staged=True)
        out["hs"] = hs

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    assert rt.poll(out["orphan"]) == K.KL_PENDING
    for h in out["hs"] + [h_long]:
        assert rt.wait(h, 20_000_000_000) == 0
    assert rt.serve_stop(20_000_000_000) == 0           # retires cleanly
    assert rt.stats(out["orphan"]).state == K.KL_ERROR
    assert rt.stats(out["orphan"]).error == K.KL_ESTATE
    assert rt.run_stats().error == 0
    # never ran: its outputs still hold the poison
    for k, v in orphan.fetch().items():
        assert _still_poisoned(v), k
    X.check("pchase", long_x, long_t.fetch(), X.expected("pchase", long_x))
    for (nm, x), t in zip(xs, tens):
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    # the runtime serves again; the same kernel runs normally now
    torch.cuda.synchronize()
    rt.serve_start()
    h = rt.submit(orphan.type, orphan.args)
    assert rt.wait(h, 20_000_000_000) == 0
    assert rt.serve_stop() == 0
    X.check("blackscholes", orphan_x, orphan.fetch(), X.expected("blackscholes", orphan_x))
    rt.close()


@pytest.mark.parametrize("mode", ["cosched", "multistream"])
def test_staged_burst_runs_only_after_publish(K, T, mode):
    import torch
    # the serving kernel holds the runtime's stream while it runs: give the
    # runtime a stream of its own (torch's are non-blocking), so the reads
    # of the outputs below, on the default stream, do not wait behind it
    side = torch.cuda.Stream()
    rt = K.Runtime(K.config_default(), stream=side.cuda_stream)
    long_x = gen.gen_pchase(24, 0, **LONG)
    long_t = T.make("pchase", long_x)
    xs = [(nm, gen.gen_tenant(nm, 24, 1 + i, **sz)) for i, (nm, sz) in
          enumerate([("triad", dict(n=1 << 18)), ("hist256", dict(n=300000)), ("blackscholes", dict(n=90000)),
                     ("bitonic", dict(log2n=15))])]
    tens = [T.make(nm, x) for nm, x in xs]
    _poison([long_t] + tens)
    if mode == "cosched":
        rt.serve_start()
    else:
        rt.serve_start(K.KL_BASE_MULTISTREAM, 4)
    hs = [rt.submit(t.type, t.args, staged=True) for t in tens]
    time.sleep(0.05)
    assert all(rt.poll(h) == K.KL_PENDING for h in hs)   # nothing visible to the device yet
    for t in tens:
        for k, v in t.fetch().items():
            assert _still_poisoned(v), (t.name, k)
    rt.publish()
    h_long = rt.submit(long_t.type, long_t.args)
    for h in hs + [h_long]:
        assert rt.wait(h, 20_000_000_000) == 0
    assert rt.serve_stop() == 0
    for (nm, x), t in zip(xs, tens):
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    X.check("pchase", long_x, long_t.fetch(), X.expected("pchase", long_x))
    # outside serving, a staged submit is a plain submit and publish does nothing
    h = rt.submit(tens[0].type, tens[0].args, staged=True)
    rt.publish()
    assert rt.drain() == 0 and rt.poll(h) == K.KL_DONE
    rt.close()


def test_batch_submitted_during_a_run_joins_the_next_run(K, T):
    import ctypes as C
    names = ["blackscholes", "triad", "hist256", "bitonic", "spmv_csr", "gemm_f32"]
    sizes = {"blackscholes": dict(n=50001), "triad": dict(n=200000), "hist256": dict(n=100003),
             "bitonic": dict(log2n=14), "spmv_csr": dict(nrows=7000), "gemm_f32": dict(M=130, N=72, K=40)}
    first = [("pchase", gen.gen_pchase(23, 0, **LONG))] + [
        (nm, gen.gen_tenant(nm, 23, 1 + i, **sizes[nm])) for i, nm in enumerate(names)]
    second = [(nm, gen.gen_tenant(nm, 24, i, **sizes[nm])) for i, nm in enumerate(names)]
    t1 = [T.make(nm, x) for nm, x in first]
    t2 = [T.make(nm, x) for nm, x in second]
    _poison(t1 + t2)
    rt = K.Runtime()
    h1 = list(rt.submit_batch(K.make_descs((t.type, t.args) for t in t1)))
    rt.launch()
    d2 = K.make_descs((t.type, t.args) for t in t2)
    h2 = list(rt.submit_batch(d2))            # the pointer chase keeps the first run busy meanwhile
    assert len(set(h1 + h2)) == len(h1) + len(h2)
    assert rt.poll(h1[0]) in (K.KL_RUNNING, K.KL_PENDING)
    assert rt.wait_run() == 0
    for h in h1:
        assert rt.poll(h) == K.KL_DONE
    for h, t in zip(h2, t2):
        assert rt.poll(h) == K.KL_PENDING and rt.wait(h, 0) == K.KL_ESTATE
        assert all(_still_poisoned(v) for v in t.fetch().values())
    assert rt.wait_run() == 0                  # nothing in flight: returns at once, launches nothing
    assert rt.poll(h2[0]) == K.KL_PENDING
    rt.launch()
    assert rt.wait_run() == 0
    for h in h2:
        assert rt.poll(h) == K.KL_DONE
    for (nm, x), t in zip(first + second, t1 + t2):
        X.check(nm, x, t.fetch(), X.expected(nm, x))

    # a refused descriptor in the middle: the ones before it stay admitted
    bad = K.make_descs((t.type, t.args) for t in t2[:3])
    bad[1].type = 200
    out = (C.c_uint64 * 3)()
    done = C.c_uint32()
    assert K.lib().kl_submit_batch(rt._h, bad, 3, out, C.byref(done)) == K.KL_EINVAL
    assert done.value == 1 and out[0] != 0 and rt.poll(out[0]) == K.KL_PENDING
    assert rt.drain() == 0 and rt.poll(out[0]) == K.KL_DONE
    rt.close()
