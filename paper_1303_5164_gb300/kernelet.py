"""Thin Python binding of the C ABI in include/kernelet.h (ctypes).

Argument marshalling only: every step of the hot path runs in libkernelet.so
(host runtime + CUDA kernels). Importing this module does not need a GPU; the
library must have been built (paper_1303_5164_gb300.build.build()). There is
no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

KL_BLOCK_THREADS = 256
KL_MAX_ARGS_BYTES = 96
KL_MAX_SLOTS = 8

KL_OK, KL_EINVAL, KL_ENOMEM, KL_EAGAIN, KL_ETIMEDOUT, KL_ECUDA, KL_EDEVICE_TIMEOUT, KL_ESTATE, \
    KL_ENOTFOUND, KL_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
KL_PENDING, KL_RUNNING, KL_DONE, KL_ERROR = 0, 1, 2, 3

(KL_T_GATHER, KL_T_BLACKSCHOLES, KL_T_GEMM_F32, KL_T_SPMV_CSR, KL_T_PCHASE, KL_T_TRIAD,
 KL_T_HIST256, KL_T_ESCAPE, KL_T_BITONIC, KL_T_MATADD, KL_T_GEMM_BF16, KL_T_TEA, KL_T_SAD, KL_T_STENCIL,
 KL_T_MRIQ, KL_T_TESTMIX, KL_T_BS255, KL_T_HIST1024, KL_T_GEMM_F32_BIG) = range(19)
KL_T_COUNT = 19
KL_T_MAIN_COUNT = 16
TYPE_NAMES = ["gather", "blackscholes", "gemm_f32", "spmv_csr", "pchase", "triad", "hist256",
              "escape", "bitonic", "matadd", "gemm_bf16", "tea", "sad", "stencil", "mriq", "testmix",
              "bs255", "hist1024", "gemm_f32_big"]
KL_RATIO_BALANCED, KL_RATIO_MAX_CP, KL_RATIO_FIXED = 0, 1, 2
KL_BASE_SERIAL, KL_BASE_MULTISTREAM, KL_SERVE_COSCHED = 0, 1, 2
KL_CFG_BACKFILL = 1
KL_CFG_FILL_TYPES = 2
KL_CFG_CHAIN_LANE = 4
KL_CFG_SERVE_TC = 8
KL_CFG_WIDE_FILL = 16
KL_CFG_LAZY_ARRIVAL = 32
KL_CFG_RANDOM_PLAN = 64
KL_CFG_LIGHT_BUILD = 128
KL_CFG_DEEP_FILL = 256
KL_CFG_PHASE_MODEL = 512

P = C.c_void_p
U32, U64, I32, F32, F64 = C.c_uint32, C.c_uint64, C.c_int32, C.c_float, C.c_double


class kl_args_gather(C.Structure):
    _fields_ = [("a", P), ("idx", P), ("out", P), ("n", U64)]


class kl_args_blackscholes(C.Structure):
    _fields_ = [("S", P), ("K", P), ("r", P), ("v", P), ("T", P), ("call", P), ("put", P), ("n", U64)]


class kl_args_gemm_f32(C.Structure):
    _fields_ = [("A", P), ("B", P), ("C", P), ("M", U32), ("N", U32), ("K", U32), ("pad", U32)]


class kl_args_spmv_csr(C.Structure):
    _fields_ = [("rowptr", P), ("col", P), ("val", P), ("x", P), ("y", P), ("nrows", U32), ("ncols", U32)]


class kl_args_pchase(C.Structure):
    _fields_ = [("next", P), ("start", P), ("end", P), ("N", U32), ("nchasers", U32), ("hops", U32),
                ("pad", U32)]


class kl_args_triad(C.Structure):
    _fields_ = [("b", P), ("c", P), ("a", P), ("s", F32), ("pad", U32), ("n", U64)]


class kl_args_hist256(C.Structure):
    _fields_ = [("data", P), ("hist", P), ("n", U64)]


class kl_args_escape(C.Structure):
    _fields_ = [("count", P), ("width", U32), ("height", U32), ("max_iter", U32), ("pad", U32),
                ("x0", F32), ("y0", F32), ("dx", F32), ("dy", F32)]


class kl_args_testmix(C.Structure):
    _fields_ = [("in_", P), ("out", P), ("n_in", U32), ("nthreads", U32), ("iters", U32), ("mem", U32),
                ("alu", U32), ("pad", U32), ("c1", F32), ("c2", F32)]


class kl_args_bitonic(C.Structure):
    _fields_ = [("in_", P), ("out", P), ("log2n", U32), ("pad", U32)]


class kl_args_matadd(C.Structure):
    _fields_ = [("a", P), ("b", P), ("c", P), ("n", U32), ("pad", U32)]


class kl_args_gemm_bf16(C.Structure):
    _fields_ = [("A", P), ("Bt", P), ("C", P), ("tmaps", P), ("M", U32), ("N", U32), ("K", U32), ("pad", U32)]


class kl_args_tea(C.Structure):
    _fields_ = [("in_", P), ("out", P), ("key", U32 * 4), ("n", U64)]


class kl_args_sad(C.Structure):
    _fields_ = [("cur", P), ("ref", P), ("sad", P), ("width", U32), ("height", U32), ("range", U32),
                ("pad", U32)]


class kl_args_stencil(C.Structure):
    _fields_ = [("in_", P), ("out", P), ("nx", U32), ("ny", U32), ("nz", U32), ("pad", U32),
                ("c0", F32), ("c1", F32)]


class kl_args_mriq(C.Structure):
    _fields_ = [("kx", P), ("ky", P), ("kz", P), ("phiR", P), ("phiI", P), ("phiMag", P), ("x", P), ("y", P),
                ("z", P), ("Qr", P), ("Qi", P), ("numK", U32), ("numX", U32)]


ARGS_TYPES = [kl_args_gather, kl_args_blackscholes, kl_args_gemm_f32, kl_args_spmv_csr,
              kl_args_pchase, kl_args_triad, kl_args_hist256, kl_args_escape, kl_args_bitonic,
              kl_args_matadd, kl_args_gemm_bf16, kl_args_tea, kl_args_sad, kl_args_stencil, kl_args_mriq,
              kl_args_testmix]


class kl_tenant_shape(C.Structure):
    _fields_ = [("grid", U32 * 3), ("block", U32 * 3), ("nstages", U32), ("smem_bytes", U32),
                ("total_blocks", U64)]


class kl_kernel_desc(C.Structure):
    _fields_ = [("type", U32), ("grid", U32 * 3), ("block", U32 * 3), ("smem_bytes", U32),
                ("regs_per_thread", U32), ("slice_blocks", U32), ("args", P), ("args_size", U32),
                ("flags", U32), ("footprint_bytes", U64)]


class kl_config(C.Structure):
    _fields_ = [("device", I32), ("slots_per_sm", U32), ("max_tenants", U32), ("model_states", U32),
                ("ratio_policy", U32), ("fixed_slots_a", U32), ("device_wait_limit_ns", U64),
                ("mem_cap_bytes", U64), ("alpha_p", F64), ("alpha_m", F64), ("flags", U32),
                ("chain_slots", U32), ("age_limit_ns", U64), ("plan_seed", U64)]


class kl_profile(C.Structure):
    _fields_ = [("R_m", F64), ("f_u", F64), ("m_c", F64), ("m_u", F64), ("L0", F64),
                ("I_block", F64), ("PUR", F64), ("MUR", F64), ("warps_per_block", U32),
                ("valid", U32), ("slice_blocks", U32), ("slice_blocks_alone", U32)]


class kl_model_params(C.Structure):
    _fields_ = [("n_sm", U32), ("n_sched", U32), ("f_sm_hz", F64), ("dram_bytes_per_s", F64),
                ("sector_bytes", F64), ("a0", F64), ("b0", F64)]


class kl_phase(C.Structure):
    _fields_ = [("A", I32), ("B", I32), ("slots_a", U32), ("slots_b", U32), ("cp", F64),
                ("t_ns", U64), ("trigger", I32), ("n_pending", U32), ("pending_mask", U64),
                ("done_a", U32), ("done_b", U32), ("prev_done_a", U32), ("prev_done_b", U32)]


class kl_tenant_stats(C.Structure):
    _fields_ = [("state", I32), ("error", I32), ("t_submit_ns", U64), ("t_start_ns", U64),
                ("t_end_ns", U64), ("t_launch_ns", U64), ("slices", U32), ("blocks", U32),
                ("t_done_host_ns", U64)]


class kl_run_stats(C.Structure):
    _fields_ = [("n_tenants", U32), ("n_phases", U32), ("error", I32), ("slots_per_sm", U32),
                ("grid_ctas", U32), ("pad", U32), ("t_launch_ns", U64), ("t_end_ns", U64),
                ("kernel_ns", U64), ("run_ns", U64), ("slot_wait_ns", U64), ("stage_wait_ns", U64),
                ("plan_ns", U64), ("class_ctas", U32 * 4)]


class KLError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().kl_strerror(code).decode()} ({code})")


_lib = None

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("kl_abi_version", C.c_int, []),
    ("kl_strerror", C.c_char_p, [C.c_int]),
    ("kl_config_default", C.c_int, [C.POINTER(kl_config)]),
    ("kl_create", C.c_int, [C.POINTER(kl_config), P, C.POINTER(P)]),
    ("kl_destroy", C.c_int, [P]),
    ("kl_tenant_shape_of", C.c_int, [U32, P, U32, C.POINTER(kl_tenant_shape)]),
    ("kl_gemm_bf16_tensor_maps", C.c_int, [C.POINTER(kl_args_gemm_bf16), P]),
    ("kl_submit", C.c_int, [P, C.POINTER(kl_kernel_desc), C.POINTER(U64)]),
    ("kl_submit_staged", C.c_int, [P, C.POINTER(kl_kernel_desc), C.POINTER(U64)]),
    ("kl_publish", C.c_int, [P]),
    ("kl_submit_batch", C.c_int, [P, C.POINTER(kl_kernel_desc), U32, C.POINTER(U64), C.POINTER(U32)]),
    ("kl_launch", C.c_int, [P]),
    ("kl_serve_start", C.c_int, [P, C.c_int, U32, U64]),
    ("kl_serve_stop", C.c_int, [P, U64]),
    ("kl_reap", C.c_int, [P, C.POINTER(U64), U32, C.POINTER(U32)]),
    ("kl_launch_baseline", C.c_int, [P, C.c_int, U32]),
    ("kl_poll", C.c_int, [P, U64, C.POINTER(C.c_int)]),
    ("kl_wait", C.c_int, [P, U64, U64]),
    ("kl_drain", C.c_int, [P, U64]),
    ("kl_wait_run", C.c_int, [P, U64]),
    ("kl_get_stats", C.c_int, [P, U64, C.POINTER(kl_tenant_stats)]),
    ("kl_get_run_stats", C.c_int, [P, C.POINTER(kl_run_stats)]),
    ("kl_get_phases", C.c_int, [P, C.POINTER(kl_phase), U32, C.POINTER(U32)]),
    ("kl_set_profiles", C.c_int, [P, C.POINTER(kl_profile), U32]),
    ("kl_set_model_params", C.c_int, [P, C.POINTER(kl_model_params)]),
    ("kl_get_model_params", C.c_int, [P, C.POINTER(kl_model_params)]),
    ("kl_get_cp_table", C.c_int, [P, C.POINTER(F64), C.POINTER(U32), C.POINTER(C.c_uint8)]),
    ("kl_set_cp_table", C.c_int, [P, C.POINTER(F64), C.POINTER(U32)]),
    ("kl_model_ipc", C.c_int, [C.POINTER(kl_model_params), C.POINTER(kl_profile), C.POINTER(U32), U32,
                               U32, C.POINTER(F64)]),
    ("kl_model_pair", C.c_int, [C.POINTER(kl_model_params), C.POINTER(kl_profile), C.POINTER(kl_profile),
                                U32, U32, U32, U32, C.POINTER(F64), C.POINTER(F64), C.POINTER(F64),
                                C.POINTER(F64), C.POINTER(F64), C.POINTER(U32)]),
    ("kl_plan", C.c_int, [C.POINTER(kl_model_params), C.POINTER(kl_profile), U32, C.POINTER(U32),
                          C.POINTER(U64), U32, U32, U32, U32, F64, F64, C.POINTER(kl_phase),
                          C.POINTER(F64), U32, C.POINTER(U32), C.POINTER(F64)]),
    ("kl_count_pruned", C.c_int, [C.POINTER(F64), C.POINTER(F64), U32, F64, F64, C.POINTER(U32)]),
    ("kl_model_phase", C.c_int, [C.POINTER(kl_model_params), C.POINTER(kl_profile), C.POINTER(U32), U32, U32,
                                 U32, C.POINTER(F64), C.POINTER(F64), C.POINTER(F64)]),
    ("kl_run_noalloc", C.c_int, [C.POINTER(kl_kernel_desc), U32, C.POINTER(F64), C.POINTER(U32), P, U64,
                                 C.POINTER(I32)]),
]
KL_NOALLOC_MAX_TENANTS = 64
KL_NOALLOC_SCRATCH_BYTES = 97536


def lib_path() -> str:
    return _build.LIB_PATH


def lib():
    """Load libkernelet.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_1303_5164_gb300.build.build() first "
                               "(no fallback implementation exists)")
        L = C.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code: int, what: str) -> int:
    if code < 0:
        raise KLError(code, what)
    return code


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


# ------------------------------------------------------------------ pure functions

def model_ipc(params: kl_model_params, profiles, warps, states: int = 3):
    n = len(profiles)
    out = (F64 * n)()
    check(lib().kl_model_ipc(C.byref(params), _arr(kl_profile, profiles), _arr(U32, warps), n, states, out),
          "kl_model_ipc")
    return list(out)


def model_pair(params, pa, pb, slots: int, states: int = 3, policy: int = KL_RATIO_BALANCED,
               fixed_a: int = 1):
    m = slots - 1
    ca, cb, cp, dT = (F64 * m)(), (F64 * m)(), (F64 * m)(), (F64 * m)()
    solo = (F64 * 2)()
    best = U32()
    check(lib().kl_model_pair(C.byref(params), C.byref(pa), C.byref(pb), slots, states, policy, fixed_a,
                              ca, cb, cp, dT, solo, C.byref(best)), "kl_model_pair")
    return dict(cipc_a=list(ca), cipc_b=list(cb), cp=list(cp), dT=list(dT), solo=list(solo),
                best_a=best.value)


def model_phase(params, profiles, slots, total_slots: int, states: int = 3):
    """kl_model_phase: (cipc per kernel, solo ipc per kernel, cp) of an n-kernel phase."""
    n = len(profiles)
    c, so, cp = (F64 * n)(), (F64 * n)(), F64()
    check(lib().kl_model_phase(C.byref(params), _arr(kl_profile, profiles), _arr(U32, slots), n, total_slots, states,
                               c, so, C.byref(cp)), "kl_model_phase")
    return list(c), list(so), cp.value


def plan(params, type_profiles, types, blocks, slots: int, states: int = 3,
         policy: int = KL_RATIO_BALANCED, alpha_p: float = -1.0, alpha_m: float = -1.0, cap: int = 4096):
    n = len(types)
    ph = (kl_phase * cap)()
    cyc = (F64 * cap)()
    nph = U32()
    mk = F64()
    check(lib().kl_plan(C.byref(params), _arr(kl_profile, type_profiles), len(type_profiles),
                        _arr(U32, types), _arr(U64, blocks), n, slots, states, policy, alpha_p, alpha_m,
                        ph, cyc, cap, C.byref(nph), C.byref(mk)), "kl_plan")
    k = min(nph.value, cap)
    return [(ph[i].A, ph[i].B, ph[i].slots_a, ph[i].slots_b, ph[i].cp, cyc[i]) for i in range(k)], mk.value


def count_pruned(pur, mur, alpha_p, alpha_m) -> int:
    out = U32()
    check(lib().kl_count_pruned(_arr(F64, pur), _arr(F64, mur), len(pur), alpha_p, alpha_m, C.byref(out)),
          "kl_count_pruned")
    return out.value


def tenant_shape(type_: int, args) -> kl_tenant_shape:
    sh = kl_tenant_shape()
    check(lib().kl_tenant_shape_of(type_, C.byref(args), C.sizeof(args), C.byref(sh)), "kl_tenant_shape_of")
    return sh


def make_desc(type_: int, args, slice_blocks: int = 0, footprint: int = 0) -> kl_kernel_desc:
    """Descriptor of one kernel with the tenant's own launch shape."""
    sh = tenant_shape(type_, args)
    d = kl_kernel_desc()
    d.type = type_
    d.grid[:] = list(sh.grid)
    d.block[:] = list(sh.block)
    d.smem_bytes = sh.smem_bytes
    d.slice_blocks = slice_blocks
    d.args = C.cast(C.byref(args), P)
    d.args_size = C.sizeof(args)
    d.footprint_bytes = footprint
    return d


def make_descs(items) -> "C.Array":
    """Array of descriptors for kl_submit_batch from (type, args) pairs (or
    (type, args, slice_blocks, footprint)); the args structs must outlive it."""
    items = list(items)
    arr = (kl_kernel_desc * len(items))()
    for k, it in enumerate(items):
        arr[k] = make_desc(*it)
    return arr


def config_default() -> kl_config:
    c = kl_config()
    check(lib().kl_config_default(C.byref(c)), "kl_config_default")
    return c


# ------------------------------------------------------------------ runtime

class Runtime:
    """Owns one kl_runtime (one persistent co-scheduler context on one GPU)."""

    def __init__(self, config: kl_config | None = None, stream: int = 0):
        self._h = P()
        cfg = config if config is not None else config_default()
        check(lib().kl_create(C.byref(cfg), P(stream) if stream else None, C.byref(self._h)), "kl_create")

    def close(self):
        if self._h:
            check(lib().kl_destroy(self._h), "kl_destroy")
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, type_: int, args, slice_blocks: int = 0, footprint: int = 0, staged: bool = False) -> int:
        """kl_submit (kl_submit_staged with staged=True)."""
        sh = tenant_shape(type_, args)
        d = kl_kernel_desc()
        d.type = type_
        d.grid[:] = list(sh.grid)
        d.block[:] = list(sh.block)
        d.smem_bytes = sh.smem_bytes
        d.slice_blocks = slice_blocks
        d.args = C.cast(C.byref(args), P)
        d.args_size = C.sizeof(args)
        d.footprint_bytes = footprint
        h = U64()
        fn = lib().kl_submit_staged if staged else lib().kl_submit
        check(fn(self._h, C.byref(d), C.byref(h)), "kl_submit_staged" if staged else "kl_submit")
        return h.value

    def publish(self):
        check(lib().kl_publish(self._h), "kl_publish")

    def submit_batch(self, descs, n: int | None = None):
        """kl_submit_batch of the first n descriptors of a make_descs array
        (all by default); returns the handles (a ctypes array of n uint64)."""
        n = len(descs) if n is None else n
        out = (U64 * max(1, n))()
        done = U32()
        check(lib().kl_submit_batch(self._h, descs, n, out, C.byref(done)), "kl_submit_batch")
        return out

    def submit_desc(self, desc: kl_kernel_desc) -> int:
        h = U64()
        check(lib().kl_submit(self._h, C.byref(desc), C.byref(h)), "kl_submit")
        return h.value

    def launch(self):
        check(lib().kl_launch(self._h), "kl_launch")

    def serve_start(self, mode: int = KL_SERVE_COSCHED, nstreams: int = 0, idle_limit_ns: int = 0):
        check(lib().kl_serve_start(self._h, mode, nstreams, idle_limit_ns), "kl_serve_start")

    def reap(self, cap: int = 4096):
        """Handles completed since the last call (serving mode)."""
        buf = (U64 * cap)()
        n = U32()
        check(lib().kl_reap(self._h, buf, cap, C.byref(n)), "kl_reap")
        return list(buf[: n.value])

    def serve_stop(self, timeout_ns: int = 30_000_000_000) -> int:
        return lib().kl_serve_stop(self._h, timeout_ns)

    def try_submit(self, type_: int, args, slice_blocks: int = 0, footprint: int = 0):
        """Like submit(), but returns None instead of raising on KL_EAGAIN."""
        d = make_desc(type_, args, slice_blocks, footprint)
        h = U64()
        rc = lib().kl_submit(self._h, C.byref(d), C.byref(h))
        if rc == KL_EAGAIN:
            return None
        check(rc, "kl_submit")
        return h.value

    def launch_baseline(self, mode: int, nstreams: int = 32):
        check(lib().kl_launch_baseline(self._h, mode, nstreams), "kl_launch_baseline")

    def poll(self, h: int) -> int:
        s = C.c_int()
        check(lib().kl_poll(self._h, h, C.byref(s)), "kl_poll")
        return s.value

    def wait(self, h: int, timeout_ns: int = 10_000_000_000) -> int:
        return lib().kl_wait(self._h, h, timeout_ns)

    def drain(self, timeout_ns: int = 30_000_000_000) -> int:
        return lib().kl_drain(self._h, timeout_ns)

    def wait_run(self, timeout_ns: int = 30_000_000_000) -> int:
        """kl_wait_run: wait for the run in flight without launching the pending set."""
        return lib().kl_wait_run(self._h, timeout_ns)

    def stats(self, h: int) -> kl_tenant_stats:
        s = kl_tenant_stats()
        check(lib().kl_get_stats(self._h, h, C.byref(s)), "kl_get_stats")
        return s

    def run_stats(self) -> kl_run_stats:
        s = kl_run_stats()
        check(lib().kl_get_run_stats(self._h, C.byref(s)), "kl_get_run_stats")
        return s

    def phases(self, cap: int = 65536):
        buf = (kl_phase * cap)()
        n = U32()
        check(lib().kl_get_phases(self._h, buf, cap, C.byref(n)), "kl_get_phases")
        return [buf[i] for i in range(min(n.value, cap))]

    def set_profiles(self, profiles):
        check(lib().kl_set_profiles(self._h, _arr(kl_profile, profiles), len(profiles)), "kl_set_profiles")

    def set_model_params(self, mp: kl_model_params):
        check(lib().kl_set_model_params(self._h, C.byref(mp)), "kl_set_model_params")

    def model_params(self) -> kl_model_params:
        mp = kl_model_params()
        check(lib().kl_get_model_params(self._h, C.byref(mp)), "kl_get_model_params")
        return mp

    def cp_table(self):
        cp = (F64 * (KL_T_COUNT * KL_T_COUNT))()
        sa = (U32 * (KL_T_COUNT * KL_T_COUNT))()
        al = (C.c_uint8 * (KL_T_COUNT * KL_T_COUNT))()
        check(lib().kl_get_cp_table(self._h, cp, sa, al), "kl_get_cp_table")
        return list(cp), list(sa), list(al)

    def set_cp_table(self, cp=None, slots_a=None):
        """Override the planner's CP / split table (None: back to the model)."""
        if cp is None:
            check(lib().kl_set_cp_table(self._h, None, None), "kl_set_cp_table")
            return
        a = (F64 * (KL_T_COUNT * KL_T_COUNT))(*cp)
        b = (U32 * (KL_T_COUNT * KL_T_COUNT))(*slots_a)
        check(lib().kl_set_cp_table(self._h, a, b), "kl_set_cp_table")
