"""CPU checks of the co-scheduler builds: which tenant types each build
holds, from a host-only compile of the tenant header, against the sets the
public header documents and the runtime relies on."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_5164_gb300", "csrc")
INC = os.path.join(ROOT, "include")
CUDA_INC = "/usr/local/cuda/include"

NAMES = ["gather", "blackscholes", "gemm_f32", "spmv_csr", "pchase", "triad", "hist256", "escape", "bitonic",
         "matadd", "gemm_bf16", "tea", "sad", "stencil", "mriq", "testmix", "bs255", "hist1024", "gemm_f32_big"]
LIGHT = {"gather", "blackscholes", "spmv_csr", "triad", "escape", "matadd", "tea", "stencil", "testmix"}
HEAVY = {"bs255": (1, 128), "hist1024": (2, 1024), "gemm_f32_big": (3, 256)}  # resource class, block threads


@pytest.fixture(scope="module")
def membership(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("builds")
    src = d / "m.cpp"
    src.write_text('#include <cstdio>\n#include "tenants.cuh"\nint main() {\n'
                   '  for (uint32_t t = 0; t < KL_T_COUNT; ++t)\n'
                   '    std::printf("%u %d %d %d %u %d %u\\n", t, (int)kl::tn::in_plain_build(t),\n'
                   '                (int)kl::tn::in_light_build(t), (int)kl::tn::in_build(kl::tn::kBuildFull, t),\n'
                   '                kl::tn::smem_bytes(t), kl::tn::resource_class(t), kl::tn::block_threads(t));\n'
                   '  return 0;\n}\n')
    exe = d / "m"
    subprocess.run([gxx, "-std=c++17", "-I", INC, "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(int, l.split())) for l in out if l.strip()]
    assert [r[0] for r in rows] == list(range(len(NAMES)))
    return {NAMES[r[0]]: dict(plain=bool(r[1]), light=bool(r[2]), full=bool(r[3]), smem=r[4], cls=r[5], threads=r[6])
            for r in rows}


def test_build_sets(membership):
    assert {n for n, m in membership.items() if m["light"]} == LIGHT
    assert {n for n, m in membership.items() if m["plain"]} == set(NAMES[:10]) | {"testmix"}
    # every co-scheduler type is in the full build; no resource-heavy variant is in any build
    assert {n for n, m in membership.items() if m["full"]} == set(NAMES[:16])
    for n, m in membership.items():
        assert (m["cls"], m["threads"]) == HEAVY.get(n, (0, 256)), n
    # a class CTA beside two co-scheduler slots: the 96 KB tiles plus two slots of the largest
    # co-scheduler type (the BF16 GEMM) fit the SM's 228 KB
    assert membership["gemm_f32_big"]["smem"] + 2 * membership["gemm_bf16"]["smem"] <= 228 * 1024 - 3 * 1024
    # the light build runs 8 CTAs per SM with 2 KB of dynamic shared memory
    assert all(m["smem"] <= 2048 for n, m in membership.items() if m["light"])


def test_header_documents_the_light_set(membership):
    txt = open(os.path.join(INC, "kernelet.h")).read()
    doc = re.search(r"#define KL_CFG_LIGHT_BUILD 128u /\*(.*?)\*/", txt, flags=re.S).group(1)
    words = {"gather": "gather", "blackscholes": "Black-Scholes", "spmv_csr": "SpMV", "triad": "triad",
             "escape": "escape-time", "matadd": "MatrixAdd", "tea": "TEA", "stencil": "stencil",
             "testmix": "testing kernel"}
    flat = " ".join(doc.split())
    for n in LIGHT:
        assert words[n] in flat, n


def test_benchmark_mix_needs_a_four_slot_build(membership):
    # the 64-kernel mix holds 64-register types, so it never runs in the light build
    from paper_1303_5164_gb300.tenants import MIX_TYPES
    assert any(not membership[t]["light"] for t in MIX_TYPES)
    assert all(membership[t]["plain"] for t in MIX_TYPES)
