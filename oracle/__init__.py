"""Oracle: plain, slow, obviously correct CPU implementations of what the engine computes.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` /
`--impl reference` legs of `bench.py` may import, call or link anything in this package.  The
engine (`paper_2507_20667_gb300`) never imports it, and it never imports the engine: the two share
no code.  Inputs reach both sides from `paper_2507_20667_gb300.inputs`, which holds no contraction,
cost or planning arithmetic.

Modules and the passages they follow:
  contract.c / contract.py  complex128 pairwise contraction along a tree (Eq. 2.4)
  costs.py                  legs (Eq. 2.6), mem (Eq. 3.1), con_serial (Eq. 3.2-3.3),
                            con_par (Eq. 3.4), con_dist (Eq. 3.5), tree acceptance (Eq. 2.7)
  greedy.py                 the Greedy contraction-order rule (Section 2.3, Eq. 4.5)
  statevector.py            brute-force state-vector simulation (textbook; pins the contractor)
  perm.py                   permutation index maps (numpy.transpose on an iota payload)
"""
