"""Device buffers and C-ABI argument blocks for each tenant type.

Plumbing only: torch allocates device memory and copies host arrays; the
argument structs point at those tensors. No tenant arithmetic happens here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import kernelet as K

NAME_TO_TYPE = {n: i for i, n in enumerate(K.TYPE_NAMES)}


def _torch():
    import torch
    return torch


def _dev(arr: np.ndarray, device, pin: bool = False):
    torch = _torch()
    a = np.ascontiguousarray(arr)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    t = torch.from_numpy(a)
    return t.to(device, non_blocking=pin)


def _empty(n, dtype, device):
    torch = _torch()
    return torch.empty(n, dtype=dtype, device=device)


def _ptr(t) -> int:
    return t.data_ptr()


@dataclass
class Tenant:
    name: str
    type: int
    args: C.Structure
    bufs: dict
    outputs: list
    footprint: int = 0
    host_inputs: dict = field(default_factory=dict)

    def fetch(self) -> dict:
        """Outputs copied back to host numpy arrays (uint32 outputs as uint32)."""
        out = {}
        for k in self.outputs:
            a = self.bufs[k].cpu().numpy()
            if k in ("hist", "count", "out", "sad") and self.name in ("hist256", "hist1024", "escape", "bitonic",
                                                                        "tea", "sad"):
                a = a.view(np.uint32)
            out[k] = a
        return out

    def shape(self):
        return K.tenant_shape(self.type, self.args)

    def replica(self) -> "Tenant":
        """Another request on the same inputs: shared input buffers, fresh
        output buffers (output buffer names equal the argument fields)."""
        torch = _torch()
        b = dict(self.bufs)
        args = type(self.args).from_buffer_copy(self.args)
        for k in self.outputs:
            b[k] = torch.empty_like(self.bufs[k])
            setattr(args, k, _ptr(b[k]))
        return Tenant(self.name, self.type, args, b, list(self.outputs), self.footprint)


def make(name: str, inp: dict, device="cuda") -> Tenant:
    """Device tenant from the seeded host inputs of workloads.gen.gen_<name>."""
    torch = _torch()
    t = NAME_TO_TYPE[name]
    b = {}
    if name == "gather":
        b["a"], b["idx"] = _dev(inp["a"], device), _dev(inp["idx"], device)
        b["out"] = _empty(inp["n"], torch.int32, device)
        args = K.kl_args_gather(_ptr(b["a"]), _ptr(b["idx"]), _ptr(b["out"]), inp["n"])
        outs = ["out"]
    elif name == "testmix":
        b["in_"] = _dev(inp["data"], device)
        b["out"] = _empty(inp["nthreads"], torch.float32, device)
        args = K.kl_args_testmix(_ptr(b["in_"]), _ptr(b["out"]), inp["n_in"], inp["nthreads"], inp["iters"],
                                 inp["mem"], inp["alu"], 0, float(inp["c1"]), float(inp["c2"]))
        outs = ["out"]
    elif name in ("blackscholes", "bs255"):
        for k in "SKrvT":
            b[k] = _dev(inp[k], device)
        b["call"] = _empty(inp["n"], torch.float32, device)
        b["put"] = _empty(inp["n"], torch.float32, device)
        args = K.kl_args_blackscholes(*[_ptr(b[k]) for k in ["S", "K", "r", "v", "T", "call", "put"]], inp["n"])
        outs = ["call", "put"]
    elif name in ("gemm_f32", "gemm_f32_big"):
        b["A"], b["B"] = _dev(inp["A"], device), _dev(inp["B"], device)
        b["C"] = _empty((inp["M"], inp["N"]), torch.float32, device)
        args = K.kl_args_gemm_f32(_ptr(b["A"]), _ptr(b["B"]), _ptr(b["C"]), inp["M"], inp["N"], inp["K"], 0)
        outs = ["C"]
    elif name == "spmv_csr":
        for k in ("rowptr", "col", "val", "x"):
            b[k] = _dev(inp[k], device)
        b["y"] = _empty(inp["nrows"], torch.float32, device)
        args = K.kl_args_spmv_csr(_ptr(b["rowptr"]), _ptr(b["col"]), _ptr(b["val"]), _ptr(b["x"]),
                                  _ptr(b["y"]), inp["nrows"], inp["ncols"])
        outs = ["y"]
    elif name == "pchase":
        b["next"], b["start"] = _dev(inp["next"], device), _dev(inp["start"], device)
        b["end"] = _empty(inp["nchasers"], torch.int32, device)
        args = K.kl_args_pchase(_ptr(b["next"]), _ptr(b["start"]), _ptr(b["end"]), inp["N"],
                                inp["nchasers"], inp["hops"], 0)
        outs = ["end"]
    elif name == "triad":
        b["b"], b["c"] = _dev(inp["b"], device), _dev(inp["c"], device)
        b["a"] = _empty(inp["n"], torch.float32, device)
        args = K.kl_args_triad(_ptr(b["b"]), _ptr(b["c"]), _ptr(b["a"]), float(inp["s"]), 0, inp["n"])
        outs = ["a"]
    elif name in ("hist256", "hist1024"):
        b["data"] = _dev(inp["data"], device)
        b["hist"] = _empty(256, torch.int32, device)
        args = K.kl_args_hist256(_ptr(b["data"]), _ptr(b["hist"]), inp["n"])
        outs = ["hist"]
    elif name == "escape":
        n = inp["width"] * inp["height"]
        b["count"] = _empty(n, torch.int32, device)
        args = K.kl_args_escape(_ptr(b["count"]), inp["width"], inp["height"], inp["max_iter"], 0,
                                float(inp["x0"]), float(inp["y0"]), float(inp["dx"]), float(inp["dy"]))
        outs = ["count"]
    elif name == "bitonic":
        b["in"] = _dev(inp["data"], device)
        b["out"] = _empty(inp["n"], torch.int32, device)
        args = K.kl_args_bitonic(_ptr(b["in"]), _ptr(b["out"]), inp["log2n"], 0)
        outs = ["out"]
    elif name == "gemm_bf16":
        b["A"] = _dev(inp["A"].view(np.int16), device)
        b["Bt"] = _dev(inp["Bt"].view(np.int16), device)
        b["C"] = _empty((inp["M"], inp["N"]), torch.float32, device)
        args = K.kl_args_gemm_bf16(_ptr(b["A"]), _ptr(b["Bt"]), _ptr(b["C"]), None, inp["M"], inp["N"], inp["K"], 0)
        maps = (C.c_ubyte * 256)()
        K.check(K.lib().kl_gemm_bf16_tensor_maps(C.byref(args), maps), "kl_gemm_bf16_tensor_maps")
        b["tmaps"] = torch.frombuffer(bytearray(bytes(maps)), dtype=torch.uint8).to(device)
        args.tmaps = _ptr(b["tmaps"])
        outs = ["C"]
    elif name == "tea":
        b["in_"] = _dev(inp["words"], device)
        b["out"] = _empty(2 * inp["n"], torch.int32, device)
        args = K.kl_args_tea(_ptr(b["in_"]), _ptr(b["out"]), (K.U32 * 4)(*[int(k) for k in inp["key"]]), inp["n"])
        outs = ["out"]
    elif name == "sad":
        b["cur"] = torch.from_numpy(np.ascontiguousarray(inp["cur"])).to(device)
        b["ref"] = torch.from_numpy(np.ascontiguousarray(inp["ref"])).to(device)
        D = 2 * inp["range"] + 1
        b["sad"] = _empty((inp["width"] // 4) * (inp["height"] // 4) * D * D, torch.int32, device)
        args = K.kl_args_sad(_ptr(b["cur"]), _ptr(b["ref"]), _ptr(b["sad"]), inp["width"], inp["height"],
                             inp["range"], 0)
        outs = ["sad"]
    elif name == "stencil":
        b["in_"] = _dev(inp["grid"], device)
        b["out"] = _empty(inp["nx"] * inp["ny"] * inp["nz"], torch.float32, device)
        args = K.kl_args_stencil(_ptr(b["in_"]), _ptr(b["out"]), inp["nx"], inp["ny"], inp["nz"], 0,
                                 float(inp["c0"]), float(inp["c1"]))
        outs = ["out"]
    elif name == "mriq":
        for k in ("kx", "ky", "kz", "phiR", "phiI", "x", "y", "z"):
            b[k] = _dev(inp[k], device)
        b["phiMag"] = _empty(inp["numK"], torch.float32, device)
        b["Qr"] = _empty(inp["numX"], torch.float32, device)
        b["Qi"] = _empty(inp["numX"], torch.float32, device)
        args = K.kl_args_mriq(*[_ptr(b[k]) for k in ("kx", "ky", "kz", "phiR", "phiI", "phiMag", "x", "y", "z",
                                                     "Qr", "Qi")], inp["numK"], inp["numX"])
        outs = ["phiMag", "Qr", "Qi"]
    elif name == "matadd":
        b["a"], b["b"] = _dev(inp["a"], device), _dev(inp["b"], device)
        b["c"] = _empty((inp["n"], inp["n"]), torch.float32, device)
        args = K.kl_args_matadd(_ptr(b["a"]), _ptr(b["b"]), _ptr(b["c"]), inp["n"], 0)
        outs = ["c"]
    else:
        raise ValueError(name)
    fp = sum(v.numel() * v.element_size() for v in b.values())
    return Tenant(name, t, args, b, outs, fp)


# Sizes of the synthetic workloads (per tenant instance)
SIZES_PAIR = {"blackscholes": dict(n=65536), "gather": dict(n=1 << 20)}
SIZES_MIX = {
    "gemm_f32": dict(M=1024, N=1024, K=1024),
    "spmv_csr": dict(nrows=1 << 20),
    "blackscholes": dict(n=4 * 1024 * 1024),
    "pchase": dict(N=1 << 24, nchasers=65536, hops=256),
    "triad": dict(n=64 * 1024 * 1024),
    "hist256": dict(n=64 * 1024 * 1024),
    "escape": dict(width=2048, height=2048, max_iter=256),
    "bitonic": dict(log2n=22),
}
MIX_TYPES = ["gemm_f32", "spmv_csr", "blackscholes", "pchase", "triad", "hist256", "escape", "bitonic"]
# the other types at the sizes they are profiled and validated at: the
# two-tenant pair's gather, the MatrixAdd example, the 4096^3 tensor-core GEMM
SIZES_OTHER = {"gather": dict(n=1 << 20), "matadd": dict(n=256), "gemm_bf16": dict(M=4096, N=4096, K=4096),
               # the paper's remaining benchmark kernels, at its input sizes (Table tb:description)
               "tea": dict(n=20971520), "sad": dict(width=1920, height=1072, range=8),
               "stencil": dict(nx=256, ny=256, nz=256),  # the paper's grid is 512^3; 256^3 keeps captures small
               "mriq": dict(numK=512, numX=2097152)}
SIZES_ALL = {**SIZES_MIX, **SIZES_OTHER}
