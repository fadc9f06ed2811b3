"""Warp-level Monte Carlo simulation of the model's stochastic process: ORACLE.

An independent check of the Markov chain construction (Section 4.4): instead
of building transition probabilities and solving for the steady state, it
draws every warp's transition at random each round, under the same rules
(round = every ready warp issues once; duration = ready warps or 1; ready ->
idle with R_m, split coalesced/uncoalesced by f_u; idle -> ready with
min(1, d/L); latency read as in markov.py), and counts issued instructions
and cycles. Many independent replicas are simulated side by side.
"""
from __future__ import annotations

import numpy as np

from .markov import GPUParams


def simulate_ipc(profiles, warps, gpu: GPUParams, rounds: int = 4000, replicas: int = 512,
                 burn_in: int = 500, seed: int = 1, three_state: bool = False):
    """Returns (ipc_per_kernel, stderr_per_kernel) per virtual SM."""
    rng = np.random.default_rng(seed)
    kid = np.concatenate([np.full(w, k) for k, w in enumerate(warps)]).astype(np.int64)
    W = len(kid)
    Rm = np.array([p.R_m for p in profiles])[kid]
    fu = np.array([(p.f_u if three_state else 0.0) for p in profiles])[kid]
    L0 = np.array([p.L0 for p in profiles])[kid]
    mc = np.array([p.m_c for p in profiles])[kid]
    mu = np.array([p.m_u for p in profiles])[kid]
    state = np.zeros((replicas, W), dtype=np.int8)      # 0 ready, 1 idle-c, 2 idle-u
    K = len(warps)
    issued = np.zeros((replicas, K))
    cycles = np.zeros(replicas)
    onehot = np.zeros((W, K))
    onehot[np.arange(W), kid] = 1.0
    for t in range(rounds + burn_in):
        ready = state == 0
        nready = ready.sum(axis=1)
        d = np.maximum(nready, 1).astype(np.float64)
        I = (W - nready).astype(np.float64)
        m = np.where(state == 2, mu[None, :], mc[None, :])
        L = L0[None, :] + gpu.b0 + gpu.a0 * m * I[:, None] / gpu.B_v
        q = np.minimum(1.0, d[:, None] / L)
        u = rng.random((replicas, W))
        new = state.copy()
        to_c = ready & (u < Rm * (1.0 - fu))
        to_u = ready & (u >= Rm * (1.0 - fu)) & (u < Rm)
        wake = (~ready) & (u < q)
        new[to_c] = 1
        new[to_u] = 2
        new[wake] = 0
        if t >= burn_in:
            issued += ready.astype(np.float64) @ onehot
            cycles += d
        state = new
    per = issued / cycles[:, None]
    return per.mean(axis=0), per.std(axis=0, ddof=1) / np.sqrt(replicas)
