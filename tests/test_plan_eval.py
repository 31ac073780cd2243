"""Batched state evaluation (EvaluateState of Section 4.4, tn_plan_eval_states) on the host.

For random states -- qubit-block partitions perturbed by random moves of single tensors across
partition borders -- the counts of tn_plan_eval_states equal bit for bit the counts of the plan
tn_plan_create assembles from the same state (TN_INIT_GIVEN, no annealing rounds), and the big-int
oracle re-derives the same counts from that plan's exported tree (Eq. 3.1, 3.2, 3.5)."""
import numpy as np
import pytest

from oracle import costs as ocost
from paper_2507_20667_gb300 import inputs as tni
from paper_2507_20667_gb300 import tnsa


def random_states(net, n_qubits, k, count, moves, seed):
    """Initial partitions perturbed by `moves` random border moves each: qubit blocks when k does
    not exceed the qubits, else the planner's balanced breadth-first regions."""
    rng = np.random.default_rng(seed)
    if k <= n_qubits:
        base = ((np.asarray(net.qubit, np.int64) * k) // n_qubits).astype(np.int32)
    else:
        h = tnsa.tn_build(net)
        base = np.asarray(tnsa.tn_plan_export(tnsa.tn_plan_create(h, k=k, iterations=0, initial="bfs"),
                                              net.n_tensors)[0], np.int32)
    nbrs = [[] for _ in range(net.n_tensors)]
    for u, a, v, b in net.edges:
        if v >= 0:
            nbrs[u].append(int(v))
            nbrs[v].append(int(u))
    out = []
    for _ in range(count):
        p = base.copy()
        sizes = np.bincount(p, minlength=k)
        for _ in range(moves):
            t = int(rng.integers(0, net.n_tensors))
            u = nbrs[t][int(rng.integers(0, len(nbrs[t])))]
            if p[u] != p[t] and sizes[p[t]] > 1:
                sizes[p[t]] -= 1
                p[t] = p[u]
                sizes[p[t]] += 1
        out.append(p)
    return np.array(out, np.int32)


def plan_counts_of_state(h, k, part, samples=32):
    plan = tnsa.tn_plan_create(h, k=k, iterations=0, initial="given", initial_part=part, fanin_samples=samples)
    return tnsa.tn_plan_counts(plan), plan


@pytest.mark.parametrize("which,k", [("cfg1", 3), ("cfg1", 6), ("cfg3s", 4), ("cfg3s", 8)])
def test_eval_states_host_equals_planner_and_oracle(which, k):
    circ, x = tni.cfg1() if which == "cfg1" else tni.cfg3(small=True)
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    states = random_states(net, circ.n_qubits, k, 12, 25, seed=k)
    cs, cd, mm, sat = tnsa.tn_plan_eval_states(h, k, states, fanin_samples=8, device=-1)
    for q, part in enumerate(states):
        if sat[q]:
            continue
        (t, c, m), plan = plan_counts_of_state(h, k, part, samples=8)
        assert (cs[q], cd[q], mm[q]) == (t, c, m)
        p2, steps, _ = tnsa.tn_plan_export(plan, net.n_tensors)
        oc = ocost.counts(net, [(int(a), int(b)) for a, b, o in steps], part=p2)
        assert (oc["con_serial"], oc["con_dist"], oc["mem"]) == (t, c, m)


def test_eval_states_rejects_bad_states():
    net = tni.amplitude_tn(*tni.cfg1())
    h = tnsa.tn_build(net)
    bad = np.zeros((1, net.n_tensors), np.int32)   # partitions 1 and 2 empty
    with pytest.raises(tnsa.TnError) as ei:
        tnsa.tn_plan_eval_states(h, 3, bad)
    assert ei.value.status == tnsa.TN_EINVAL
    bad[0, 0] = 7
    with pytest.raises(tnsa.TnError):
        tnsa.tn_plan_eval_states(h, 3, bad)
