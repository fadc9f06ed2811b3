"""Co-schedule search (Sections 4.2-4.3, Algorithm 1): ORACLE, test infrastructure.

* Pruning (Section 4.3): a candidate pair is removed when the two kernels'
  PUR values AND their MUR values are both closer than the thresholds
  (|dPUR| < alpha_p and |dMUR| < alpha_m). The text says "or"; the paper's
  pruning table (Table 3, built from Table 2) is reproduced by "and" and not by
  "or". When every pair is pruned the unpruned candidate set is used.
* FindCoSchedule (Algorithm 1, procedure): enumerate the N(N-1)/2 pairs of
  pending kernels, prune, evaluate CP of each survivor at its balanced slice
  ratio with the performance model, return the pair with the largest CP
  (CP equal within 1e-12: smallest (i, j) in submission order). One pending
  kernel runs alone.
* Greedy loop (Algorithm 1, main): repeat the chosen co-schedule while the
  pending set is unchanged AND both kernels still have thread blocks; then
  re-plan on the residuals.
* Plan simulation: a kernel k in a phase advances at cIPC_k * n_sm / I_k
  blocks per cycle; the phase lasts until the first of the two runs out.
* Brute force: every sequence of pairs and slot splits for tiny queues.
* MC(s) (Section 5.1): s random schedules (random pair, random split).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .markov import CP_TIE, GPUParams, KernelProfile, evaluate_pair, homogeneous_ipc, warps_on_virtual_sm


@dataclass
class Tenant:
    prof: KernelProfile
    blocks: int
    PUR: float = 0.0
    MUR: float = 0.0


def prune_pairs(pairs, tenants, alpha_p, alpha_m):
    """Pairs surviving the PUR/MUR rule; the full list if none survives."""
    if alpha_p is None or alpha_m is None:
        return list(pairs)
    keep = [(i, j) for (i, j) in pairs
            if not (abs(tenants[i].PUR - tenants[j].PUR) < alpha_p
                    and abs(tenants[i].MUR - tenants[j].MUR) < alpha_m)]
    return keep if keep else list(pairs)


def count_pruned(purs, murs, alpha_p, alpha_m) -> int:
    """Number of the N(N-1)/2 kernel pairs removed by the pruning rule."""
    n = len(purs)
    c = 0
    for i in range(n):
        for j in range(i + 1, n):
            if abs(purs[i] - purs[j]) < alpha_p and abs(murs[i] - murs[j]) < alpha_m:
                c += 1
    return c


class PairModel:
    """Caches the performance model per (profile A, profile B)."""

    def __init__(self, gpu: GPUParams, slots: int, three_state: bool = False):
        self.gpu, self.slots, self.three_state = gpu, slots, three_state
        self._pair = {}
        self._solo = {}

    def pair(self, pa: KernelProfile, pb: KernelProfile):
        key = (id(pa), id(pb))
        if key not in self._pair:
            self._pair[key] = evaluate_pair(pa, pb, self.slots, self.gpu, self.three_state)
        return self._pair[key]

    def solo_ipc(self, p: KernelProfile) -> float:
        if id(p) not in self._solo:
            w = warps_on_virtual_sm(self.slots, p.warps_per_block, self.gpu.n_sched)
            self._solo[id(p)] = homogeneous_ipc(p, w, self.gpu, self.three_state) * self.gpu.n_sched
        return self._solo[id(p)]


@dataclass
class CoSchedule:
    A: int
    B: int | None
    bA: int
    bB: int
    cp: float
    cipcA: float
    cipcB: float


def find_coschedule(R, tenants, model: PairModel, alpha_p=None, alpha_m=None) -> CoSchedule:
    R = sorted(R)
    if len(R) == 1:
        a = R[0]
        return CoSchedule(a, None, model.slots, 0, 0.0, model.solo_ipc(tenants[a].prof), 0.0)
    pairs = [(R[x], R[y]) for x in range(len(R)) for y in range(x + 1, len(R))]
    cand = prune_pairs(pairs, tenants, alpha_p, alpha_m)
    best = None
    for (i, j) in cand:          # ascending (i, j): a CP tie keeps the earlier pair
        ev, _, _ = model.pair(tenants[i].prof, tenants[j].prof)
        if best is None or ev.cp > best.cp + CP_TIE:
            best = CoSchedule(i, j, ev.bA, ev.bB, ev.cp, ev.cipcA, ev.cipcB)
    return best


def _rate(cipc, prof, gpu):
    return cipc * gpu.n_sm / prof.I_block      # blocks per cycle


def simulate(tenants, chooser, model: PairModel):
    """Run the greedy loop with `chooser(R, rem) -> CoSchedule`; returns
    (phases, makespan_cycles); each phase is (cs, duration_cycles)."""
    gpu = model.gpu
    rem = [float(t.blocks) for t in tenants]
    R = [i for i, t in enumerate(tenants) if t.blocks > 0]
    phases = []
    total = 0.0
    while R:
        cs = chooser(R, rem)
        if cs.B is None:
            dur = rem[cs.A] / _rate(cs.cipcA, tenants[cs.A].prof, gpu)
            rem[cs.A] = 0.0
            R.remove(cs.A)
        else:
            rA = _rate(cs.cipcA, tenants[cs.A].prof, gpu)
            rB = _rate(cs.cipcB, tenants[cs.B].prof, gpu)
            tA, tB = rem[cs.A] / rA, rem[cs.B] / rB
            dur = min(tA, tB)
            rem[cs.A] -= dur * rA
            rem[cs.B] -= dur * rB
            if tA <= tB:
                rem[cs.A] = 0.0
                R.remove(cs.A)
            if tB <= tA:
                rem[cs.B] = 0.0
                R.remove(cs.B)
        phases.append((cs, dur))
        total += dur
    return phases, total


def greedy_plan(tenants, model: PairModel, alpha_p=None, alpha_m=None):
    return simulate(tenants, lambda R, rem: find_coschedule(R, tenants, model, alpha_p, alpha_m), model)


def brute_force(tenants, model: PairModel):
    """Minimum makespan over every sequence of pairs and slot splits
    (solo only when one kernel is left). Tiny queues only."""
    gpu = model.gpu
    n = len(tenants)
    best = [np.inf]

    def rec(R, rem, acc):
        if acc >= best[0]:
            return
        if not R:
            best[0] = acc
            return
        if len(R) == 1:
            a = R[0]
            d = rem[a] / _rate(model.solo_ipc(tenants[a].prof), tenants[a].prof, gpu)
            rec([], rem, acc + d)
            return
        for x in range(len(R)):
            for y in range(x + 1, len(R)):
                i, j = R[x], R[y]
                _, evals, _ = model.pair(tenants[i].prof, tenants[j].prof)
                for ev in evals:
                    rA = _rate(ev.cipcA, tenants[i].prof, gpu)
                    rB = _rate(ev.cipcB, tenants[j].prof, gpu)
                    tA, tB = rem[i] / rA, rem[j] / rB
                    d = min(tA, tB)
                    nrem = list(rem)
                    nrem[i] -= d * rA
                    nrem[j] -= d * rB
                    nR = list(R)
                    if tA <= tB:
                        nrem[i] = 0.0
                        nR.remove(i)
                    if tB <= tA:
                        nrem[j] = 0.0
                        nR.remove(j)
                    rec(nR, nrem, acc + d)

    rec([i for i in range(n) if tenants[i].blocks > 0], [float(t.blocks) for t in tenants], 0.0)
    return best[0]


def monte_carlo(tenants, model: PairModel, s: int, seed: int = 0):
    """MC(s): makespans of s schedules with random pairs and random splits."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(s):
        def chooser(R, rem):
            R = sorted(R)
            if len(R) == 1:
                a = R[0]
                return CoSchedule(a, None, model.slots, 0, 0.0, model.solo_ipc(tenants[a].prof), 0.0)
            x, y = rng.choice(len(R), size=2, replace=False)
            i, j = sorted((R[x], R[y]))
            _, evals, _ = model.pair(tenants[i].prof, tenants[j].prof)
            ev = evals[rng.integers(len(evals))]
            return CoSchedule(i, j, ev.bA, ev.bB, ev.cp, ev.cipcA, ev.cipcB)
        out.append(simulate(tenants, chooser, model)[1])
    return np.array(out)
