"""Program compiler (host only, no GPU): how the pairwise steps of a plan are split between warp
programs (subtrees of small steps, one warp each), block programs (subtrees that fit a block's
shared memory) and global dataflow steps.

Every pairwise step of the tree (n - 1 of them, Section 2.2) must be executed exactly once: the
steps inside warp programs, inside block programs, and the global steps (a DOTP + DOTF pair is one
pairwise step; a program's pseudo-step is not a pairwise step) add up to n - 1, at every budget.
The algorithmic flop count is the plan's con_serial times 8 (Eq. 3.2), whatever the split.
"""
import numpy as np
import pytest

from oracle import costs as ocost
from paper_2507_20667_gb300 import inputs as tni
from paper_2507_20667_gb300 import tnsa

KIND_LOCAL, KIND_DOTF = 5, 3


def _cfg2_like(n_qubits=16, depth=10, k=4):
    circ = tni.brickwork_1d(n_qubits, depth, seed=2)
    net = tni.amplitude_tn(circ, tni.random_bitstring(n_qubits, 1002))
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=k, iterations=200, seed=7,
                               position=net.qubit)
    return net, h, plan


@pytest.mark.parametrize("budget", [0, 4096, 32768, 100000])
@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_every_step_runs_once(budget, precision):
    net, h, plan = _cfg2_like()
    n = len(net.degrees)
    st = tnsa.tn_plan_compile_stats(h, plan, precision, budget)
    steps = tnsa.tn_plan_compile_steps(h, plan, precision, budget)
    kinds = steps[:, 0]
    global_pairwise = int(np.sum((kinds != KIND_LOCAL) & (kinds != KIND_DOTF)))
    assert global_pairwise + st["n_local_steps"] + st["n_warp_steps"] == n - 1
    assert int(np.sum(kinds == KIND_LOCAL)) == st["n_local"] + st["n_warp_progs"]
    total, _, _ = tnsa.tn_plan_counts(plan)
    assert st["flops"] == pytest.approx(8.0 * total, rel=1e-12)
    if budget == 0:
        assert st["n_local"] == 0 and st["n_warp_progs"] == 0


def test_small_step_subtrees_become_warp_programs():
    """With a budget, gate absorption (tiny steps near the leaves) runs in warp programs and the
    programs' shared-memory needs respect their limits."""
    net, h, plan = _cfg2_like()
    st = tnsa.tn_plan_compile_stats(h, plan, "c64", 100000)
    assert st["n_warp_progs"] > 0 and st["n_warp_steps"] > 0
    steps = tnsa.tn_plan_compile_steps(h, plan, "c64", 100000)
    progs = steps[steps[:, 0] == KIND_LOCAL]
    assert (progs[:, 7] <= 100000).all() and (progs[:, 6] >= 1).all()


@pytest.mark.parametrize("budget", [0, 4096])
def test_rows_chains_link_producer_to_consumer(budget):
    """A chain link s -> t (t continues s in the same block, s's output kept in shared memory) goes
    forward in the step list, joins ROWS steps only, is taken at most once per step, and stays
    within the 32-step chain limit; the stats count the continuations."""
    net, h, plan = _cfg2_like()
    st = tnsa.tn_plan_compile_stats(h, plan, "c64", budget)
    steps = tnsa.tn_plan_compile_steps(h, plan, "c64", budget)
    rows = np.flatnonzero(steps[:, 0] == 0)
    nxt = {int(i): int(steps[i, 6]) for i in rows if steps[i, 6] >= 0}
    assert len(nxt) == st["n_chained"] > 0
    assert len(set(nxt.values())) == len(nxt)
    for s, t in nxt.items():
        assert t > s and steps[t, 0] == 0
        assert steps[s, 1] * steps[s, 2] == steps[t, 1] * steps[t, 3]   # C of s is A of t
        assert steps[t, 5] > steps[s, 5]
    heads = set(nxt) - set(nxt.values())
    for hd in heads:
        n, s = 1, hd
        while s in nxt:
            s, n = nxt[s], n + 1
        assert n <= 32
    # complex128 storage never stages A in shared memory, so it has no chains
    assert tnsa.tn_plan_compile_stats(h, plan, "c128", budget)["n_chained"] == 0


def _grid():
    circ = tni.grid_2d(3, 4, 6, seed=4)
    net = tni.amplitude_tn(circ, tni.random_bitstring(12, 7))
    h = tnsa.tn_build(net)
    return net, h, tnsa.tn_plan_create(h, k=3, iterations=100, seed=5)


def _mixed(seed):
    net = tni.random_network(14, 10, (1, 2, 3, 5, 6), seed=seed)
    h = tnsa.tn_build(net)
    return net, h, tnsa.tn_plan_create(h, k=2, iterations=50, seed=seed)


@pytest.mark.parametrize("make", [_cfg2_like, _grid, lambda: _mixed(0), lambda: _mixed(3)],
                         ids=["brickwork16", "grid3x4", "mixed0", "mixed3"])
def test_step_geometry_matches_leg_sets(make):
    """Leg analysis (Eq. 2.6, Eq. 3.3): for every pairwise step of the plan's tree, the compiled
    M, N and K are the sizes of the two operands' free legs and of their shared legs, as the
    oracle's leg sets give them along the exported tree.  The compiler makes the larger operand A,
    so M and N are compared as an unordered pair; the DOTF entry of the root's DOTP + DOTF pair is
    not a pairwise step of its own."""
    net, h, plan = make()
    _, psteps, _ = tnsa.tn_plan_export(plan, net.n_tensors)
    dims = ocost.edge_dims(net)
    legs = dict(enumerate(ocost.leaf_legs(net)))
    want = []
    for l, r, o in psteps:
        a, b = legs[int(l)], legs[int(r)]
        shared = a & b
        legs[int(o)] = a ^ b
        m, n = ocost.prod(dims, a - shared), ocost.prod(dims, b - shared)
        want.append((min(m, n), max(m, n), ocost.prod(dims, shared)))
    got = [(int(min(M, N)), int(max(M, N)), int(K))
           for kind, M, N, K, *_ in tnsa.tn_plan_compile_steps(h, plan, "c64", 0) if kind != KIND_DOTF]
    assert len(want) == net.n_tensors - 1
    assert sorted(got) == sorted(want)
