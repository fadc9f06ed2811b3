"""Markov-chain performance model of warp issue (Section 4.4): ORACLE, test infrastructure.

Follows the paper's steps and notation, in binary64:

* Virtual SM (Section 4.4, "multiple warp schedulers"): model one warp
  scheduler; warps and bandwidth of the SM are divided by the scheduler count.
* A warp is ready or idle (two-state model, Fig. "warp state transition"):
  ready -> idle with probability R_m, idle -> ready with probability P_i->r.
  With uncoalesced accesses (Section 4.4, "Uncoalesced Access") idle splits
  into idle-on-coalesced and idle-on-uncoalesced, each with its own latency.
* State S_i = number of idle warps; a time step is one round in which every
  ready warp issues one instruction; round duration = ready warps, or 1 cycle
  when no warp is ready.
* Transition S_i -> S_j sums the probabilities of every (woken, stalled)
  combination with stalled - woken = j - i (Eq. for the constraints on
  N_i->r, N_r->i); warps are independent, so the counts are binomial.
* Steady state pi: eigenvector of P for eigenvalue 1 (Eq. steadyStateVector),
  computed with the GTH (Grassmann-Taqqu-Heyman) elimination.
* IPC = non-idle cycles / all cycles (Eq. modelIPC); for two kernels the state
  is (p, q) and the transition is the product of per-kernel transitions;
  IPC_K1, IPC_K2 use the round duration R(p,q) in the denominator
  (Eqs. ipc_k1, ipc_k2); C = IPC_K1 + IPC_K2 (Eq. ipc).
* CP (Eq. cp) = 1 - 1 / sum_i cIPC_i / IPC_i.
* Balanced slice ratio (Eq. executiontime): minimise
  dT = | I_1 P_1 / IPC_1 - I_2 P_2 / IPC_2 |.

Readings taken where the paper is garbled or silent (each listed in the design
notes):
  latency     L_{k,x}(s) = L0_k + b0 + a0 * m_{k,x} * I(s) / B_v, with I(s) the
              idle warps of state s, m the sectors per memory instruction of the
              class and B_v the virtual SM's DRAM sectors per cycle (processor
              sharing of the bandwidth; the printed L = L0 + B/(a0 S_i) + b0
              divides by zero at S_0 and falls as contention rises).
  wake prob.  P_i->r = min(1, d(s) / L) with d(s) = max(ready warps, 1): the
              printed (W-I)/L makes S_W absorbing and can exceed 1.
  warps       w = floor(blocks * warps_per_block / schedulers + 1/2), at least 1
              when the kernel has a block on the SM.
  IPC_i in CP is the kernel's solo IPC at its full occupancy.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class GPUParams:
    n_sm: int                  # SMs on the GPU
    n_sched: int               # warp schedulers per SM (virtual SM divisor)
    f_sm_hz: float             # SM clock
    dram_bytes_per_s: float    # DRAM bandwidth
    sector_bytes: int = 32
    a0: float = 1.0            # linear latency model parameters
    b0: float = 0.0

    @property
    def B_v(self) -> float:
        """DRAM sectors per cycle available to one virtual SM."""
        per_s = self.dram_bytes_per_s / self.sector_bytes
        return per_s / (self.f_sm_hz * self.n_sm * self.n_sched)


@dataclass
class KernelProfile:
    R_m: float                 # memory instructions / instructions
    L0: float                  # unloaded memory latency, cycles
    m_c: float = 4.0           # sectors per coalesced memory instruction
    m_u: float = 32.0          # sectors per uncoalesced memory instruction
    f_u: float = 0.0           # fraction of memory instructions that are uncoalesced
    I_block: float = 1.0       # warp instructions per thread block
    warps_per_block: int = 8
    name: str = ""


# ----------------------------------------------------------------- linear algebra

def gth_stationary(P: np.ndarray) -> np.ndarray:
    """Stationary distribution of a row-stochastic matrix by GTH elimination."""
    A = np.array(P, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k in range(n - 1, 0, -1):
        s = A[k, :k].sum()
        if s <= 0.0:
            raise ValueError("GTH: state cannot reach lower-numbered states (reducible chain)")
        A[:k, k] /= s
        A[:k, :k] += np.outer(A[:k, k], A[k, :k])
    pi = np.zeros(n)
    pi[0] = 1.0
    for k in range(1, n):
        pi[k] = pi[:k] @ A[:k, k]
    return pi / pi.sum()


def binom_pmf(n: int, p: float) -> np.ndarray:
    """P[X = x] for X ~ Binomial(n, p), x = 0..n."""
    out = np.empty(n + 1)
    for x in range(n + 1):
        out[x] = math.comb(n, x) * (p ** x) * ((1.0 - p) ** (n - x))
    return out


# ----------------------------------------------------------------- warp counts

def warps_on_virtual_sm(blocks_per_sm: int, warps_per_block: int, n_sched: int) -> int:
    if blocks_per_sm <= 0:
        return 0
    w = math.floor(blocks_per_sm * warps_per_block / n_sched + 0.5)
    return max(1, w)


# ----------------------------------------------------------------- the chain

@dataclass
class _Kernel:
    prof: KernelProfile
    w: int
    three_state: bool
    states: list = field(default_factory=list)   # per-kernel states


def _kernel_states(w: int, three_state: bool):
    if three_state:
        return [(ic, iu) for ic in range(w + 1) for iu in range(w + 1 - ic)]
    return [(i, 0) for i in range(w + 1)]


def _kernel_row(kern: _Kernel, st, d: float, I_tot: int, gpu: GPUParams) -> dict:
    """Distribution of the kernel's next state given its state `st` = (ic, iu),
    the round duration d of the SM state and its total idle warps I_tot."""
    p = kern.prof
    ic, iu = st
    r = kern.w - ic - iu
    Lc = p.L0 + gpu.b0 + gpu.a0 * p.m_c * I_tot / gpu.B_v
    qc = min(1.0, d / Lc)
    wake_c = binom_pmf(ic, qc)
    if kern.three_state:
        Lu = p.L0 + gpu.b0 + gpu.a0 * p.m_u * I_tot / gpu.B_v
        qu = min(1.0, d / Lu)
        wake_u = binom_pmf(iu, qu)
        pc = p.R_m * (1.0 - p.f_u)
        pu = p.R_m * p.f_u
        ps = 1.0 - p.R_m
        row = {}
        for yc in range(r + 1):
            for yu in range(r + 1 - yc):
                ys = r - yc - yu
                pm = (math.factorial(r) / (math.factorial(yc) * math.factorial(yu) * math.factorial(ys))
                      * (pc ** yc) * (pu ** yu) * (ps ** ys))
                if pm == 0.0:
                    continue
                for xc in range(ic + 1):
                    for xu in range(iu + 1):
                        pr = pm * wake_c[xc] * wake_u[xu]
                        if pr == 0.0:
                            continue
                        key = (ic - xc + yc, iu - xu + yu)
                        row[key] = row.get(key, 0.0) + pr
        return row
    stall = binom_pmf(r, p.R_m)
    row = {}
    for x in range(ic + 1):
        for y in range(r + 1):
            pr = wake_c[x] * stall[y]
            if pr == 0.0:
                continue
            key = (ic - x + y, 0)
            row[key] = row.get(key, 0.0) + pr
    return row


def build_chain(kernels, gpu: GPUParams):
    """Joint states (tuple of per-kernel states) and the transition matrix."""
    per = [k.states for k in kernels]
    joint = list(itertools.product(*per))
    index = {s: i for i, s in enumerate(joint)}
    n = len(joint)
    P = np.zeros((n, n))
    ready = np.zeros((n, len(kernels)))
    dur = np.zeros(n)
    for si, s in enumerate(joint):
        idle = [ic + iu for (ic, iu) in s]
        rdy = [k.w - i for k, i in zip(kernels, idle)]
        d = float(max(sum(rdy), 1))
        I_tot = sum(idle)
        ready[si] = rdy
        dur[si] = d
        rows = [_kernel_row(k, st, d, I_tot, gpu) for k, st in zip(kernels, s)]
        for combo in itertools.product(*[list(r.items()) for r in rows]):
            prob = 1.0
            for _, pr in combo:
                prob *= pr
            P[si, index[tuple(c[0] for c in combo)]] += prob
    return joint, P, ready, dur


def model_ipc(profiles, warps, gpu: GPUParams, three_state: bool = False):
    """Per-kernel IPC of one virtual SM holding `warps[k]` warps of kernel k.

    Returns (ipc_per_kernel [virtual SM], pi, joint_states, P)."""
    kernels = []
    for prof, w in zip(profiles, warps):
        ts = three_state and prof.f_u > 0.0
        kernels.append(_Kernel(prof, int(w), ts, _kernel_states(int(w), ts)))
    joint, P, ready, dur = build_chain(kernels, gpu)
    pi = gth_stationary(P)
    denom = float(pi @ dur)
    ipc = [float(pi @ ready[:, k]) / denom for k in range(len(kernels))]
    return ipc, pi, joint, P


def homogeneous_ipc(prof: KernelProfile, W: int, gpu: GPUParams, three_state=False) -> float:
    """Eq. modelIPC for one kernel with W warps on the virtual SM."""
    return model_ipc([prof], [W], gpu, three_state)[0][0]


def cp(cipc, ipc_solo) -> float:
    """Co-scheduling profit, Eq. cp."""
    s = sum(c / i for c, i in zip(cipc, ipc_solo))
    return 1.0 - 1.0 / s


@dataclass
class PairEval:
    bA: int
    bB: int
    cipcA: float       # per SM
    cipcB: float
    cp: float
    dT: float


def phase_cp(profiles, slots, total_slots: int, gpu: GPUParams, three_state: bool = False):
    """A phase of n kernels sharing the SM, kernel k on slots[k] block slots
    (Section 2.2: a co-schedule of n slices; Section 4.4: the heterogeneous
    chain of n kernels): per-kernel concurrent IPC per SM, solo IPC per SM at
    `total_slots` (full occupancy), and CP by Eq. cp over the n kernels.
    Kernels with no slot contribute nothing to CP."""
    S = gpu.n_sched
    w = [warps_on_virtual_sm(b, p.warps_per_block, S) for p, b in zip(profiles, slots)]
    conc = model_ipc(profiles, w, gpu, three_state)[0]
    cipc = [c * S for c in conc]
    solo = [homogeneous_ipc(p, warps_on_virtual_sm(total_slots, p.warps_per_block, S), gpu, three_state) * S
            for p in profiles]
    terms = [c / s for c, s in zip(cipc, solo) if s > 0.0]
    return cipc, solo, (1.0 - 1.0 / sum(terms)) if sum(terms) > 0.0 else 0.0


def evaluate_pair(pA: KernelProfile, pB: KernelProfile, slots: int, gpu: GPUParams,
                  three_state: bool = False):
    """Every feasible slot split (bA + bB = slots, both >= 1) of the per-SM
    block slots between A and B: concurrent IPCs, CP and dT; plus the chosen
    balanced split (min dT, then max CP, then larger bA).

    Solo IPC (for CP) is each kernel alone with all `slots` blocks per SM."""
    S = gpu.n_sched
    wA_solo = warps_on_virtual_sm(slots, pA.warps_per_block, S)
    wB_solo = warps_on_virtual_sm(slots, pB.warps_per_block, S)
    ipcA = homogeneous_ipc(pA, wA_solo, gpu, three_state) * S
    ipcB = homogeneous_ipc(pB, wB_solo, gpu, three_state) * S
    evals = []
    for bA in range(1, slots):
        bB = slots - bA
        wA = warps_on_virtual_sm(bA, pA.warps_per_block, S)
        wB = warps_on_virtual_sm(bB, pB.warps_per_block, S)
        (cA, cB), _, _, _ = model_ipc([pA, pB], [wA, wB], gpu, three_state)
        cA *= S
        cB *= S
        PA = bA * gpu.n_sm
        PB = bB * gpu.n_sm
        dT = abs(pA.I_block * PA / cA - pB.I_block * PB / cB)
        evals.append(PairEval(bA, bB, cA, cB, cp([cA, cB], [ipcA, ipcB]), dT))
    best = None
    for e in evals:
        if best is None or better_split(e, best):
            best = e
    return best, evals, (ipcA, ipcB)


CP_TIE = 1e-12      # CP values closer than this are equal
DT_TIE = 1e-9       # dT values closer than this (relative) are equal


def better_split(e: "PairEval", best: "PairEval", policy: str = "balanced") -> bool:
    """Order of slot splits. The paper picks the split with the smallest dT
    (Eq. executiontime) and states no tie rule; ties (within rounding) go to
    the larger CP, then the more even split, then the larger share of K1."""
    if policy == "balanced":
        scale = max(e.dT, best.dT)
        if abs(e.dT - best.dT) > DT_TIE * scale:
            return e.dT < best.dT
    if abs(e.cp - best.cp) > CP_TIE:
        return e.cp > best.cp
    ue, ub = abs(e.bA - e.bB), abs(best.bA - best.bB)
    if ue != ub:
        return ue < ub
    return e.bA > best.bA
