"""The allocation-free entry point (kl_run_noalloc) against the regular one.

kl_run_noalloc serves callers that cannot allocate device memory where they
run work (frameworks whose caching allocator already reserved the device
memory, and latency-critical threads that must not call cudaMalloc/cudaFree
because those can synchronize the device): it keeps the co-scheduler's queue
in a fixed device array of the library instead. This test calls it through
the C ABI twice in a row, on two different batches, and checks every output
against the same batch run through kl_submit / kl_drain (the tenants are
bit-reproducible, so the comparison is bit for bit, as in the other tests).
The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

from tests import _expect as X
from workloads import gen

pytestmark = pytest.mark.gpu

BATCHES = [
    [("blackscholes", dict(n=70001)), ("gather", dict(n=300000)), ("hist256", dict(n=200003))],
    [("triad", dict(n=1 << 20)), ("bitonic", dict(log2n=16)), ("spmv_csr", dict(nrows=20000)),
     ("escape", dict(width=300, height=170, max_iter=128)), ("gemm_f32", dict(M=200, N=132, K=100))],
]


def _poison(tens):
    import torch
    for t in tens:
        for k in t.outputs:
            t.bufs[k].fill_(-1)
    torch.cuda.synchronize()


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    L = K.lib()
    for call, batch in enumerate(BATCHES):
        inps = [gen.gen_tenant(nm, 11, call * 10 + i, **sz) for i, (nm, sz) in enumerate(batch)]
        tens = [T.make(nm, x) for (nm, _), x in zip(batch, inps)]
        # reference: the regular entry point
        _poison(tens)
        rt = K.Runtime()
        for t in tens:
            rt.submit(t.type, t.args)
        assert rt.drain() == 0
        ref = [t.fetch() for t in tens]
        rt.close()
        # the allocation-free entry point, same batch
        _poison(tens)
        n = len(tens)
        descs = (K.kl_kernel_desc * n)(*[K.make_desc(t.type, t.args) for t in tens])
        states = (C.c_int32 * n)()
        rc = L.kl_run_noalloc(descs, n, None, None, None, 0, states)
        assert rc == 0, L.kl_strerror(rc)
        assert list(states) == [K.KL_DONE] * n
        torch.cuda.synchronize()
        for (nm, _), x, t, r in zip(batch, inps, tens, ref):
            got = t.fetch()
            for k in r:
                assert X.same_bits(got[k], r[k]), (call, nm, k)
            X.check(nm, x, got, X.expected(nm, x))


def test_noalloc_tensor_core_build_tables_and_stream():
    """A batch holding the BF16 tensor-core GEMM (the co-scheduler build with
    tcgen05), run with caller-supplied CP and slot tables on a torch stream,
    twice in a row: outputs equal the regular entry point's and the oracle."""
    import torch
    from paper_1303_5164_gb300 import build, kernelet as K, tenants as T
    build.build()
    L = K.lib()
    batch = [("gemm_bf16", dict(M=384, N=320, K=256)), ("triad", dict(n=300000)),
             ("pchase", dict(N=1 << 16, nchasers=3000, hops=64)), ("hist256", dict(n=100000))]
    inps = [gen.gen_tenant(nm, 12, i, **sz) for i, (nm, sz) in enumerate(batch)]
    tens = [T.make(nm, x) for (nm, _), x in zip(batch, inps)]
    _poison(tens)
    rt = K.Runtime()
    for t in tens:
        rt.submit(t.type, t.args)
    assert rt.drain() == 0
    ref = [t.fetch() for t in tens]
    rt.close()
    nt = K.KL_T_COUNT
    rng = np.random.default_rng(7)
    cp = (C.c_double * (nt * nt))(*rng.uniform(0.0, 0.5, nt * nt))
    sa = (C.c_uint32 * (nt * nt))(*rng.integers(0, 9, nt * nt))  # out of range entries are clamped
    stream = torch.cuda.Stream()
    n = len(tens)
    descs = (K.kl_kernel_desc * n)(*[K.make_desc(t.type, t.args) for t in tens])
    for _ in range(2):
        _poison(tens)
        states = (C.c_int32 * n)()
        rc = L.kl_run_noalloc(descs, n, cp, sa, C.c_void_p(stream.cuda_stream), 0, states)
        assert rc == 0, L.kl_strerror(rc)
        assert list(states) == [K.KL_DONE] * n
        for (nm, _), x, t, r in zip(batch, inps, tens, ref):
            got = t.fetch()
            if nm == "gemm_bf16":
                X.check(nm, x, got, X.expected(nm, x))
                continue
            for k in r:
                assert X.same_bits(got[k], r[k]), (nm, k)
            X.check(nm, x, got, X.expected(nm, x))


def test_noalloc_rejects_too_many_kernels():
    from paper_1303_5164_gb300 import build, kernelet as K
    build.build()
    n = K.KL_NOALLOC_MAX_TENANTS + 1
    descs = (K.kl_kernel_desc * n)()
    assert K.lib().kl_run_noalloc(descs, n, None, None, None, 0, None) == K.KL_EOVERFLOW
    assert K.lib().kl_run_noalloc(descs, 0, None, None, None, 0, None) == K.KL_EINVAL
