"""Failure detection on the GPU without a fault: every device wait of the
co-scheduler is bounded; with a 2 us limit the waits at stage barriers and of
idle slots run out, the run ends with KL_EDEVICE_TIMEOUT, its kernels are
reported as errors, and the same runtime (and CUDA context) runs the next
batch normally."""
import pytest

from tests import _expect as X
from workloads import gen

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


def test_wait_limit_runs_out_and_the_runtime_recovers(K, T):
    c = K.config_default()
    c.device_wait_limit_ns = 2000
    rt = K.Runtime(c)
    srt = gen.gen_bitonic(11, 0, 20)
    chase = gen.gen_pchase(11, 1, N=1 << 22, nchasers=4096, hops=2048)
    ts = [T.make("bitonic", srt), T.make("pchase", chase)]
    hs = [rt.submit(t.type, t.args) for t in ts]
    rc = rt.drain()
    assert rc == K.KL_EDEVICE_TIMEOUT
    states = [rt.stats(h).state for h in hs]
    assert K.KL_ERROR in states
    rt.close()
    # the context is still usable: a normal limit on a fresh runtime, same buffers
    rt = K.Runtime(K.config_default())
    hs = [rt.submit(t.type, t.args) for t in ts]
    assert rt.drain() == 0
    assert all(rt.poll(h) == K.KL_DONE for h in hs)
    X.check("bitonic", srt, ts[0].fetch(), X.expected("bitonic", srt))
    X.check("pchase", chase, ts[1].fetch(), X.expected("pchase", chase))
    rt.close()
