"""Host planner (C++ library, no GPU) against the oracle.

  * k = 1: the library's Greedy tree equals the oracle Greedy tree step for step, and its counts
    (con_serial Eq. 3.2, con_dist Eq. 3.5, mem Eq. 3.1) equal the big-int oracle's bit for bit;
  * SA plans (Algorithms 1-2) are checked by postconditions: a valid partition with no empty part
    (Section 2.4), a tree that accepts it (Eq. 2.7), a cost no worse than the initial partition's
    (best tracking of Algorithm 1), per-partition trees equal to the oracle Greedy on the same
    members, and counts re-derived by the oracle from the exported tree;
  * imported trees: counts equal the oracle's for arbitrary trees;
  * tn_build rejects malformed networks.
"""
import numpy as np
import pytest

from oracle import costs as ocost
from oracle import greedy as og
from paper_2507_20667_gb300 import inputs as tni
from paper_2507_20667_gb300 import tnsa


def block_partition(net, n_qubits, k):
    """k contiguous blocks of qubits; each tensor goes to the block of the qubit it sits on."""
    return ((np.asarray(net.qubit, dtype=np.int64) * k) // n_qubits).astype(np.int32)


def oracle_partition_steps(net, part, k):
    legs = ocost.leaf_legs(net)
    dims = ocost.edge_dims(net)
    n = net.n_tensors
    steps = []
    for p in range(k):
        members = [t for t in range(n) if part[t] == p]
        ids = list(members)
        for i, j in og.greedy_steps([legs[t] for t in members], dims):
            steps.append((ids[i], ids[j]))
            ids.append(n + len(steps) - 1)
    return steps


def check_plan_against_oracle(net, plan, k):
    n = net.n_tensors
    part, steps, step_part = tnsa.tn_plan_export(plan, n)
    total, crit, mem = tnsa.tn_plan_counts(plan)
    # partition validity (cover, disjoint by construction, non-empty)
    assert part.min() >= 0 and part.max() < k
    assert all(np.sum(part == p) > 0 for p in range(k))
    # oracle counts from the exported tree (raises if the tree does not accept K)
    c = ocost.counts(net, [(int(l), int(r)) for l, r, o in steps], part=part)
    assert (total, crit, mem) == (c["con_serial"], c["con_dist"], c["mem"])
    info = tnsa.tn_plan_get_info(plan)
    assert info["con_par"] == c["con_par"]
    assert c["con_par"] <= c["con_dist"] <= c["con_serial"]
    # per-partition trees are the oracle Greedy trees on the same members
    inner = [(int(l), int(r)) for (l, r, o), sp in zip(steps, step_part) if sp >= 0]
    assert inner == oracle_partition_steps(net, part, k)
    assert list(steps[:, 2]) == list(range(n, 2 * n - 1))
    return part, steps, c, info


@pytest.mark.parametrize("maker", [
    lambda: tni.amplitude_tn(*tni.cfg1()),
    lambda: tni.amplitude_tn(tni.grid_2d(3, 4, 6, seed=4), tni.random_bitstring(12, 5)),
    lambda: tni.zz_tn(tni.brickwork_1d(7, 5, seed=8), 2, 5),
    lambda: tni.random_network(30, 20, (2, 3, 5), seed=3),
])
def test_greedy_k1_bit_exact(maker):
    net = maker()
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=1)
    part, steps, c, info = check_plan_against_oracle(net, plan, 1)
    ref = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    assert [(int(l), int(r)) for l, r, o in steps] == ref
    assert c["con_dist"] == c["con_serial"]          # k = 1: no fan-in path


@pytest.mark.parametrize("k,mode,threads", [(2, "directed", 1), (4, "directed", 1), (4, "naive", 1),
                                            (3, "directed", 3), (6, "directed", 2), (8, "naive", 1)])
def test_sa_postconditions(k, mode, threads):
    circ = tni.brickwork_1d(12, 8, seed=12)
    net = tni.amplitude_tn(circ, tni.random_bitstring(12, 3))
    h = tnsa.tn_build(net)
    init = block_partition(net, 12, k)
    plan = tnsa.tn_plan_create(h, k=k, mode=mode, iterations=40, steps_per_temp=8, threads=threads,
                               seed=7, initial_part=init)
    part, steps, c, info = check_plan_against_oracle(net, plan, k)
    assert info["sa_iterations"] == 40
    assert c["con_dist"] <= info["initial_con_dist"]
    # the initial partition's cost, re-derived by the oracle with Greedy trees and the best fan-in
    # tree the planner could pick, bounds the result from above as well
    init_steps = oracle_partition_steps(net, init, k)
    assert len(init_steps) == net.n_tensors - k


def test_sa_deterministic_and_seed_sensitive():
    circ = tni.brickwork_1d(10, 8, seed=21)
    net = tni.amplitude_tn(circ, tni.random_bitstring(10, 4))
    h = tnsa.tn_build(net)
    init = block_partition(net, 10, 4)
    runs = []
    for seed in (1, 1, 2):
        plan = tnsa.tn_plan_create(h, k=4, iterations=30, steps_per_temp=4, threads=2, seed=seed,
                                   initial_part=init)
        runs.append(tnsa.tn_plan_export(plan, net.n_tensors))
    assert all(np.array_equal(a, b) for a, b in zip(runs[0], runs[1]))


def test_sa_bfs_initial_partition():
    net = tni.amplitude_tn(tni.grid_2d(3, 3, 5, seed=2), tni.random_bitstring(9, 2))
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=5, iterations=20, seed=3)
    check_plan_against_oracle(net, plan, 5)


def test_fanin_exhaustive_k3_is_optimal():
    """For k <= 4 every fan-in tree is tried, so con_dist is minimal over fan-in trees for the
    given partition trees: compare against all three fan-in trees of k = 3 in the oracle."""
    net = tni.amplitude_tn(tni.brickwork_1d(6, 4, seed=5), tni.random_bitstring(6, 6))
    h = tnsa.tn_build(net)
    init = block_partition(net, 6, 3)
    plan = tnsa.tn_plan_create(h, k=3, iterations=0, initial_part=init)
    part, steps, c, info = check_plan_against_oracle(net, plan, 3)
    n = net.n_tensors
    inner = oracle_partition_steps(net, part, 3)
    # roots of the partition subtrees in export numbering
    roots = []
    cnt = 0
    for p in range(3):
        members = [v for v in range(n) if part[v] == p]
        cnt += len(members) - 1
        roots.append(n + cnt - 1 if len(members) > 1 else members[0])
    best = None
    for a, b, cc in ((0, 1, 2), (0, 2, 1), (1, 2, 0)):
        x, y = sorted((roots[a], roots[b]))
        first = n + len(inner)
        fan = [(x, y), tuple(sorted((first, roots[cc])))]
        cd = ocost.counts(net, inner + fan, part=part)["con_dist"]
        best = cd if best is None else min(best, cd)
    assert c["con_dist"] == best


@pytest.mark.parametrize("seed", range(4))
def test_import_arbitrary_tree(seed):
    net = tni.random_network(12, 8, (2, 3, 4), seed=seed)
    h = tnsa.tn_build(net)
    rng = np.random.default_rng(seed)
    n = net.n_tensors
    alive, steps, nxt = list(range(n)), [], n
    while len(alive) > 1:
        i, j = sorted(rng.choice(len(alive), 2, replace=False))
        a, b = alive[i], alive[j]
        steps.append((min(a, b), max(a, b)))
        alive = [t for t in alive if t not in (a, b)] + [nxt]
        nxt += 1
    plan = tnsa.tn_plan_import(h, steps)
    total, crit, mem = tnsa.tn_plan_counts(plan)
    c = ocost.counts(net, steps, part=[0] * n)
    assert (total, crit, mem) == (c["con_serial"], c["con_dist"], c["mem"])
    # a partition the tree does not accept is rejected (Eq. 2.7)
    bad = np.zeros(n, np.int32)
    bad[steps[0][0]] = 1
    bad[[t for t in range(n) if t not in steps[0]][0]] = 1
    with pytest.raises(tnsa.TnError):
        tnsa.tn_plan_import(h, steps, part=bad)


def test_counts_above_2_64():
    """Counts are exact 128-bit integers: a left-deep tree in tensor order over a 70-qubit circuit
    carries every wire as an open leg (a 2^70-element intermediate), so con_serial > 2^64."""
    net = tni.amplitude_tn(tni.brickwork_1d(70, 2, seed=1), tni.random_bitstring(70, 1))
    n = net.n_tensors
    steps = [(0, 1)] + [(s + 2, n + s) for s in range(n - 2)]
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, steps)
    total, crit, mem = tnsa.tn_plan_counts(plan)
    c = ocost.counts(net, steps, part=[0] * n)
    assert total > 2 ** 64 and mem > 2 ** 64
    assert (total, crit, mem) == (c["con_serial"], c["con_dist"], c["mem"])


def test_build_rejects_malformed():
    ok = tni.amplitude_tn(tni.brickwork_1d(3, 2, seed=1), [0, 1, 0])
    tnsa.tn_build(ok)

    class Bad:
        pass

    def variant(edges=None, dims=None):
        b = Bad()
        b.degrees = ok.degrees
        b.dims = ok.dims if dims is None else dims
        b.data = ok.data
        b.edges = ok.edges if edges is None else edges
        return b

    e = ok.edges.copy()
    e[0, 2] = e[0, 0]                      # self-loop
    with pytest.raises(tnsa.TnError):
        tnsa.tn_build(variant(edges=e))
    with pytest.raises(tnsa.TnError):      # an axis left unnamed
        tnsa.tn_build(variant(edges=ok.edges[:-1]))
    e = ok.edges.copy()
    e[1] = e[0]                            # an axis named twice
    with pytest.raises(tnsa.TnError):
        tnsa.tn_build(variant(edges=e))
    dims = ok.dims.copy()
    dims[0] = 3                            # n_{u,a} != n_{v,b}
    b = variant(dims=dims)
    b.data = np.zeros(2 * int(sum(np.prod(dims[o:o + d]) for o, d in
                                   zip(np.concatenate([[0], np.cumsum(ok.degrees)[:-1]]), ok.degrees))))
    with pytest.raises(tnsa.TnError):
        tnsa.tn_build(b)
    h = tnsa.tn_build(ok)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_plan_create(h, k=0)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_plan_create(h, k=ok.n_tensors + 1)


def test_entries_out_of_range_are_rejected():
    """Tensor entries must be finite with |Re|, |Im| below 2^127 (the max-abs of every tensor is
    tracked in FP32): tn_build and tn_net_set_tensor reject NaN, infinities and 2^127, and accept
    the largest double below it."""
    ok = tni.amplitude_tn(tni.brickwork_1d(3, 2, seed=1), [0, 1, 0])
    h = tnsa.tn_build(ok)
    n0 = ok.tensors[0].size

    class Net:
        pass

    for bad in (np.nan, np.inf, -np.inf, 2.0 ** 127, -(2.0 ** 127)):
        b = Net()
        b.degrees, b.dims, b.edges = ok.degrees, ok.dims, ok.edges
        d = np.array(ok.data, np.float64)
        d[1] = bad
        b.data = d
        with pytest.raises(tnsa.TnError):
            tnsa.tn_build(b)
        v = np.zeros(n0, np.complex128)
        v[0] = complex(bad, 0.0)
        with pytest.raises(tnsa.TnError):
            tnsa.tn_net_set_tensor(h, 0, v)
    v = np.zeros(n0, np.complex128)
    v[0] = np.nextafter(2.0 ** 127, 0.0)
    tnsa.tn_net_set_tensor(h, 0, v)


def _circuits_cfg1_to_cfg4():
    yield tni.cfg1()[0], 1
    yield tni.cfg2()[0], 4
    yield tni.cfg3(small=True)[0], 8
    yield tni.cfg3()[0], 8
    for circ, k, xs in tni.cfg4_circuits():
        yield circ, k


def test_qubit_block_initial_partition_in_library():
    """TN_INIT_QUBIT_BLOCK (the library's initial partition, Section 4.2's starting cut) equals the
    k contiguous qubit blocks on every workload circuit; with no annealing rounds it is the plan's
    partition."""
    for circ, k in _circuits_cfg1_to_cfg4():
        for kk in sorted({k, 2, 3}):
            net = tni.amplitude_tn(circ, np.zeros(circ.n_qubits, np.int32))
            h = tnsa.tn_build(net)
            plan = tnsa.tn_plan_create(h, k=kk, iterations=0, initial="qubit_block", position=net.qubit)
            part, _, _ = tnsa.tn_plan_export(plan, net.n_tensors)
            assert np.array_equal(part, block_partition(net, circ.n_qubits, kk)), (circ.n_qubits, kk)


def test_initial_partition_errors():
    net = tni.amplitude_tn(tni.brickwork_1d(6, 3, seed=1), np.zeros(6, np.int32))
    h = tnsa.tn_build(net)
    for kw in ({"initial": "given"}, {"initial": "qubit_block"},
               {"initial": "qubit_block", "position": -np.ones(net.n_tensors, np.int32)},
               {"initial": "given", "initial_part": np.full(net.n_tensors, 5, np.int32)},
               {"initial": 7}):
        with pytest.raises(tnsa.TnError) as ei:
            tnsa.tn_plan_create(h, k=3, iterations=0, **kw)
        assert ei.value.status == tnsa.TN_EINVAL
    # a block with no tensor in it: positions 0 and 5 only, k = 3
    pos = np.where(np.arange(net.n_tensors) % 2 == 0, 0, 5).astype(np.int32)
    with pytest.raises(tnsa.TnError):
        tnsa.tn_plan_create(h, k=3, iterations=0, position=pos)
