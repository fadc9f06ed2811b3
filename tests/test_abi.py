"""CPU checks of the C ABI: the library loads, exports every declared entry
point, rejects bad input without a GPU, and its pure host functions (Markov
model, pair evaluation, greedy plan, pruning) agree with the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import markov as mk
from oracle import schedule as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def K():
    from paper_1303_5164_gb300 import build, kernelet
    build.build()
    return kernelet


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(kl_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(K):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(K.lib_path())
    for n in sorted(names):
        assert hasattr(L, n), n
    bound = {s[0] for s in K.SIGNATURES}
    assert names == bound, names ^ bound


def test_errors_without_gpu(K):
    L = K.lib()
    assert L.kl_abi_version() == 2
    assert L.kl_strerror(K.KL_EINVAL) == b"invalid argument"
    out = C.c_void_p()
    cfg = K.config_default()
    cfg.model_states = 5
    assert L.kl_create(C.byref(cfg), None, C.byref(out)) == K.KL_EINVAL
    assert L.kl_submit(None, None, None) == K.KL_EINVAL
    assert L.kl_drain(None, 0) == K.KL_EINVAL
    assert L.kl_wait_run(None, 0) == K.KL_EINVAL
    done = C.c_uint32(7)
    assert L.kl_submit_batch(None, None, 0, None, C.byref(done)) == K.KL_EINVAL and done.value == 0
    # shape queries are host-only
    a = K.kl_args_triad(16, 32, 48, 3.0, 0, 3 * 4096 + 7)
    sh = K.tenant_shape(K.KL_T_TRIAD, a)
    assert tuple(sh.grid) == (4, 1, 1) and sh.nstages == 1 and sh.total_blocks == 4
    bad = K.kl_args_triad(17, 32, 48, 3.0, 0, 100)          # misaligned pointer
    assert L.kl_tenant_shape_of(K.KL_T_TRIAD, C.byref(bad), C.sizeof(bad), C.byref(sh)) == K.KL_EINVAL
    g = K.kl_args_gemm_f32(16, 32, 48, 128, 130, 64, 0)     # N not a multiple of 4
    assert L.kl_tenant_shape_of(K.KL_T_GEMM_F32, C.byref(g), C.sizeof(g), C.byref(sh)) == K.KL_EINVAL
    b = K.kl_args_bitonic(16, 32, 22, 0)
    sh = K.tenant_shape(K.KL_T_BITONIC, b)
    # 2^22 keys in 4096-key tiles: the tile sort, then for each of the 10 merge
    # sizes above the tile one pass over its distances above the tile (at most
    # 10 of them) and one tile merge: 1 + 10 x 2 stages of 1024 blocks
    assert sh.nstages == 21 and sh.grid[0] == 1024 and sh.total_blocks == 21 * 1024
    b = K.kl_args_bitonic(16, 32, 30, 0)                    # merge sizes 2^23 .. 2^30 need two such passes
    assert K.tenant_shape(K.KL_T_BITONIC, b).nstages == 1 + 10 * 2 + 8 * 3
    h = K.kl_args_hist256(16, 32, (1 << 26))
    sh = K.tenant_shape(K.KL_T_HIST256, h)
    assert sh.nstages == 2 and sh.grid[0] == 1 and sh.total_blocks == 1 + 2048


def test_serving_and_tensor_map_argument_checks_without_gpu(K):
    L = K.lib()
    n = K.U32()
    buf = (K.U64 * 4)()
    assert L.kl_serve_start(None, K.KL_SERVE_COSCHED, 0, 0) == K.KL_EINVAL
    assert L.kl_serve_stop(None, 0) == K.KL_EINVAL
    assert L.kl_reap(None, buf, 4, C.byref(n)) == K.KL_EINVAL
    assert L.kl_run_noalloc(None, 0, None, None, None, 0, None) == K.KL_EINVAL
    maps = (C.c_ubyte * 256)()
    assert L.kl_gemm_bf16_tensor_maps(None, maps) == K.KL_EINVAL
    bad = K.kl_args_gemm_bf16(16, 32, 48, 64, 128, 64, 100, 0)   # K not a multiple of 8
    assert L.kl_gemm_bf16_tensor_maps(C.byref(bad), maps) == K.KL_EINVAL
    sh = K.kl_tenant_shape()
    assert L.kl_tenant_shape_of(K.KL_T_GEMM_BF16, C.byref(bad), C.sizeof(bad), C.byref(sh)) == K.KL_EINVAL
    unaligned_maps = K.kl_args_gemm_bf16(16, 32, 48, 96, 128, 64, 128, 0)  # tensor maps not 64-byte aligned
    assert L.kl_tenant_shape_of(K.KL_T_GEMM_BF16, C.byref(unaligned_maps), C.sizeof(unaligned_maps),
                                C.byref(sh)) == K.KL_EINVAL
    ok = K.kl_args_gemm_bf16(16, 32, 48, 64, 200, 132, 136, 0)
    sh = K.tenant_shape(K.KL_T_GEMM_BF16, ok)
    # 128 x 64 tiles: 2 x 3 with ragged edges, one stage, the largest shared memory of any type
    assert tuple(sh.grid) == (6, 1, 1) and sh.nstages == 1 and sh.smem_bytes >= 48 * 1024
    cfg = K.config_default()
    assert cfg.flags & K.KL_CFG_BACKFILL and cfg.flags & K.KL_CFG_CHAIN_LANE and cfg.flags & K.KL_CFG_WIDE_FILL
    assert cfg.flags & K.KL_CFG_LIGHT_BUILD
    assert cfg.chain_slots == 2 and cfg.age_limit_ns == 0


def test_header_constants_match_the_binding(K):
    # every integer #define of the public header has the same value in the binding
    txt = open(os.path.join(ROOT, "include", "kernelet.h")).read()
    defs = dict(re.findall(r"^#define\s+(KL_\w+)\s+\(?(-?\d+)u?\)?", txt, flags=re.M))
    assert len(defs) >= 10
    for name, v in defs.items():
        if hasattr(K, name):
            assert getattr(K, name) == int(v), name
    flags = [n for n in defs if n.startswith("KL_CFG_")]
    assert all(hasattr(K, n) for n in flags), [n for n in flags if not hasattr(K, n)]


def test_ctypes_structs_match_the_header(K, tmp_path):
    # sizes of the ABI structs as gcc lays them out from include/kernelet.h,
    # against the binding's ctypes declarations
    names = ["kl_config", "kl_kernel_desc", "kl_tenant_shape", "kl_profile", "kl_model_params", "kl_phase",
             "kl_tenant_stats", "kl_run_stats"] + [t.__name__ for t in K.ARGS_TYPES]
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "kernelet.h"\nint main(void) {\n' +
                   "".join(f'  printf("%s %zu\\n", "{n}", sizeof({n}));\n' for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for n in names:
        assert int(got[n]) == C.sizeof(getattr(K, n)), n
    assert all(C.sizeof(t) <= K.KL_MAX_ARGS_BYTES for t in K.ARGS_TYPES)


GPU = mk.GPUParams(n_sm=152, n_sched=4, f_sm_hz=1.9e9, dram_bytes_per_s=6753e9)


def _kp(K, p: mk.KernelProfile, PUR=0.0, MUR=0.0):
    q = K.kl_profile()
    q.R_m, q.f_u, q.m_c, q.m_u, q.L0, q.I_block = p.R_m, p.f_u, p.m_c, p.m_u, p.L0, p.I_block
    q.PUR, q.MUR, q.warps_per_block, q.valid = PUR, MUR, p.warps_per_block, 1
    return q


def _mp(K):
    m = K.kl_model_params()
    m.n_sm, m.n_sched, m.f_sm_hz, m.dram_bytes_per_s = GPU.n_sm, GPU.n_sched, GPU.f_sm_hz, GPU.dram_bytes_per_s
    m.sector_bytes, m.a0, m.b0 = 32.0, GPU.a0, GPU.b0
    return m


def _rand_prof(rng, f_u=True):
    # memory-bound to compute-bound kernels, so CP differs between pairs
    return mk.KernelProfile(R_m=float(rng.choice([0.002, 0.02, 0.1, 0.3])) * float(rng.uniform(0.8, 1.2)),
                            L0=float(rng.uniform(100, 1200)),
                            m_c=4.0, m_u=float(rng.choice([8.0, 16.0, 32.0])),
                            f_u=float(rng.uniform(0.05, 0.9)) if f_u else 0.0,
                            I_block=float(rng.uniform(100, 20000)), warps_per_block=8)


@pytest.mark.parametrize("seed", range(6))
def test_model_ipc_matches_oracle(K, seed):
    rng = np.random.default_rng(seed)
    for states in (2, 3):
        pa, pb = _rand_prof(rng), _rand_prof(rng)
        for warps in ([1], [5], [8], [3, 5], [1, 7], [4, 4]):
            profs = [pa, pb][:len(warps)]
            ref, _, _, _ = mk.model_ipc(profs, warps, GPU, three_state=(states == 3))
            got = K.model_ipc(_mp(K), [_kp(K, p) for p in profs], warps, states)
            assert np.allclose(np.array(got) / GPU.n_sched, ref, rtol=1e-11, atol=1e-14), (got, ref)


@pytest.mark.parametrize("seed", range(4))
def test_model_pair_matches_oracle(K, seed):
    rng = np.random.default_rng(100 + seed)
    pa, pb = _rand_prof(rng), _rand_prof(rng)
    for slots in (2, 4, 6):
        best, evals, (ia, ib) = mk.evaluate_pair(pa, pb, slots, GPU, three_state=True)
        r = K.model_pair(_mp(K), _kp(K, pa), _kp(K, pb), slots, 3)
        assert np.allclose(r["solo"], [ia, ib], rtol=1e-11)
        for e in evals:
            i = e.bA - 1
            assert np.isclose(r["cipc_a"][i], e.cipcA, rtol=1e-11)
            assert np.isclose(r["cipc_b"][i], e.cipcB, rtol=1e-11)
            assert np.isclose(r["cp"][i], e.cp, rtol=1e-10, atol=1e-13)
            assert np.isclose(r["dT"][i], e.dT, rtol=1e-9)
        assert r["best_a"] == best.bA


@pytest.mark.parametrize("seed", range(3))
def test_model_phase_matches_oracle(K, seed):
    # three kernels sharing the SM (a pair plus the chain lane's kernel), and
    # a kernel with no slot at all
    rng = np.random.default_rng(300 + seed)
    ps = [_rand_prof(rng, f_u=bool(k % 2)) for k in range(3)]
    for slots, total, states in (((1, 2, 1), 4, 3), ((2, 1, 1), 4, 2), ((1, 1, 2), 6, 3), ((2, 2, 0), 4, 3)):
        ci, so, cp = K.model_phase(_mp(K), [_kp(K, p) for p in ps], list(slots), total, states)
        oc, osolo, ocp = mk.phase_cp(ps, list(slots), total, GPU, three_state=states == 3)
        assert np.allclose(ci, oc, rtol=1e-11, atol=1e-14)
        assert np.allclose(so, osolo, rtol=1e-11)
        assert np.isclose(cp, ocp, rtol=1e-10, atol=1e-13)
    with pytest.raises(K.KLError):
        K.model_phase(_mp(K), [_kp(K, p) for p in ps], [2, 2, 1], 4, 3)   # more slots than the SM has


def test_count_pruned_table3(K):
    gold = os.path.join(ROOT, "tests", "golden")
    rows = [l.split() for l in open(os.path.join(gold, "c2050_pur_mur.txt")) if not l.startswith("#")]
    pur = [float(r[1]) for r in rows]
    mur = [float(r[2]) for r in rows]
    for am in (0.015, 0.045, 0.06, 0.105, 0.15):
        for ap in (0.1, 0.4, 0.7, 1.0):
            assert K.count_pruned(pur, mur, ap, am) == sc.count_pruned(pur, mur, ap, am)
    assert K.count_pruned(pur, mur, 0.4, 0.015) == 2       # Table 3, first row


@pytest.mark.parametrize("seed", range(4))
def test_plan_matches_oracle_greedy(K, seed):
    rng = np.random.default_rng(200 + seed)
    kinds = [_rand_prof(rng, f_u=bool(k % 2)) for k in range(4)]
    pur = rng.uniform(0, 1, 4)
    mur = rng.uniform(0, 0.3, 4)
    n = 7
    types = [int(rng.integers(4)) for _ in range(n)]
    blocks = [int(rng.integers(20, 5000)) for _ in range(n)]
    for ap, am in ((-1.0, -1.0), (0.3, 0.1)):
        ts = [sc.Tenant(kinds[t], b, PUR=pur[t], MUR=mur[t]) for t, b in zip(types, blocks)]
        model = sc.PairModel(GPU, 4, three_state=True)
        phases, mksp = sc.greedy_plan(ts, model, None if ap < 0 else ap, None if am < 0 else am)
        got, gmk = K.plan(_mp(K), [_kp(K, kinds[t], pur[t], mur[t]) for t in range(4)], types, blocks, 4, 3,
                          alpha_p=ap, alpha_m=am)
        assert len(got) == len(phases)
        for (A, B, sa, sb, cpv, cyc), (cs, dur) in zip(got, phases):
            assert (A, B if B >= 0 else None) == (cs.A, cs.B)
            assert (sa, sb) == (cs.bA, cs.bB)
            assert np.isclose(cyc, dur, rtol=1e-9)
        assert np.isclose(gmk, mksp, rtol=1e-9)
