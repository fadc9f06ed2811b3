"""CPU oracle for the Kernelet hot path: TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package. The product path (paper_1303_5164_gb300) never
imports it, and it never imports the product path: the two share no code.

Contents
  tenants.c / tenants.py  plain CPU definitions of every tenant kernel
  markov.py               Markov-chain performance model (Section 4.4)
  schedule.py             pruning (Section 4.3), FindCoSchedule and the greedy
                          loop (Algorithm 1), plan simulation, brute force,
                          Monte Carlo co-schedules (Section 5.1, MC(s))
  mcsim.py                warp-level Monte Carlo simulation of the model's
                          stochastic process (an independent check of the chain)
"""
