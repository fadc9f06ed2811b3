"""KL_CFG_L2_BUDGET on the GPU: pointer chases over 64, 16 and 4 MB cycles and
two streaming kernels in one co-scheduled run. Every output equals the oracle,
and at the moment each chase started (its first slice, stamped after it was
admitted) the chases still running plus itself fitted half of the L2, unless
none was running. Without the flag the same kernels give the same outputs."""
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


def _items():
    chases = [(1 << 24), (1 << 24), (1 << 22), (1 << 22), (1 << 22), (1 << 22), (1 << 24), (1 << 20), (1 << 20)]
    items = [("pchase", gen.gen_pchase(41, i, N=N, nchasers=8192, hops=96)) for i, N in enumerate(chases)]
    items.insert(3, ("triad", gen.gen_tenant("triad", 41, 20, n=1 << 22)))
    items.append(("escape", gen.gen_tenant("escape", 41, 21, width=512, height=256, max_iter=128)))
    return items


@pytest.mark.parametrize("budget", [True, False])
def test_chases_start_within_half_the_l2(K, T, budget):
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    budget_kb = l2 // 2 // 1024
    items = _items()
    tens = [T.make(nm, x) for nm, x in items]
    torch.cuda.synchronize()
    c = K.config_default()
    if budget:
        c.flags |= K.KL_CFG_L2_BUDGET
    else:
        c.flags &= ~K.KL_CFG_L2_BUDGET
    rt = K.Runtime(c)
    hs = [rt.submit(t.type, t.args) for t in tens]
    assert rt.drain() == 0
    for (nm, x), t in zip(items, tens):
        X.check(nm, x, t.fetch(), X.expected(nm, x))
    if not budget:
        rt.close()
        return
    chase = [(rt.stats(h), -(-4 * x["N"] // 1024)) for (nm, x), h in zip(items, hs) if nm == "pchase"]
    for i, (si, kbi) in enumerate(chase):
        used = sum(kb for j, (sj, kb) in enumerate(chase)
                   if j != i and sj.t_start_ns <= si.t_start_ns < sj.t_end_ns)
        assert used == 0 or used + kbi <= budget_kb, (i, used, kbi, budget_kb)
    # 64 MB cycles: more than half of any L2 up to 128 MiB, so they ran one at a time
    big = [s for (s, kb) in chase if kb * 2 > budget_kb]
    big.sort(key=lambda s: s.t_start_ns)
    for a, b in zip(big, big[1:]):
        assert b.t_start_ns >= a.t_end_ns
    rt.close()
