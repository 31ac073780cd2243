"""Batched EvaluateState on the GPU (Section 4.4; the RandomGreedy fan-in samples of Algorithm 1).

On 1200 random states (initial partitions perturbed by border moves) of the 24-qubit brickwork
network (cfg2) and of the 4x5 grid instance of cfg3 at k = 4, 16 and 64, the GPU evaluator's
counts equal bit for bit those of the host evaluation, of tn_plan_counts on the plan the planner
assembles from the state, and of the big-int oracle on that plan's tree (Eq. 3.1, 3.2, 3.5).
Simulated annealing with the fan-in trees evaluated on the GPU returns the same plan as with host
evaluation, and at k = 64 on cfg2 it finishes well within a minute."""
import time

import numpy as np
import pytest

from oracle import costs as ocost
from paper_2507_20667_gb300 import inputs as tni
from test_plan_eval import random_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tnsa():
    from paper_2507_20667_gb300 import tnsa as mod
    return mod


@pytest.mark.parametrize("which", ["cfg2", "cfg3s"])
@pytest.mark.parametrize("k", [4, 16, 64])
def test_gpu_state_counts_bit_exact(tnsa, which, k):
    circ, x = tni.cfg2() if which == "cfg2" else tni.cfg3(small=True)
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    states = random_states(net, circ.n_qubits, k, 200, 40, seed=100 + k)
    gpu = tnsa.tn_plan_eval_states(h, k, states, fanin_samples=32, device=0)
    host = tnsa.tn_plan_eval_states(h, k, states, fanin_samples=32, device=-1)
    assert gpu == host
    cs, cd, mm, sat = gpu
    checked = 0
    for q, part in enumerate(states):
        if sat[q]:
            continue
        plan = tnsa.tn_plan_create(h, k=k, iterations=0, initial="given", initial_part=part, fanin_samples=32)
        assert (cs[q], cd[q], mm[q]) == tnsa.tn_plan_counts(plan)
        p2, steps, _ = tnsa.tn_plan_export(plan, net.n_tensors)
        oc = ocost.counts(net, [(int(a), int(b)) for a, b, o in steps], part=p2)
        assert (oc["con_serial"], oc["con_dist"], oc["mem"]) == (cs[q], cd[q], mm[q])
        checked += 1
    assert checked >= 150


def test_annealing_with_gpu_fanin_equals_host(tnsa):
    circ, x = tni.cfg2()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plans = {}
    for dev in (-1, 0):
        t0 = time.perf_counter()
        p = tnsa.tn_plan_create(h, k=16, iterations=30, steps_per_temp=16, threads=8, seed=3, initial="bfs",
                                fanin_device=dev)
        plans[dev] = (tnsa.tn_plan_export(p, net.n_tensors), tnsa.tn_plan_counts(p), time.perf_counter() - t0)
    (a, ca, _), (b, cb, _) = plans[-1], plans[0]
    assert ca == cb and all(np.array_equal(u, v) for u, v in zip(a, b))


def test_annealing_k64_on_gpu_within_budget(tnsa):
    """Directed annealing of the 24-qubit brickwork network into k = 64 partitions, 64 chains of
    one move per round, 300 rounds, fan-in trees (32 RandomGreedy samples) on the GPU."""
    circ, x = tni.cfg2()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    t0 = time.perf_counter()
    p = tnsa.tn_plan_create(h, k=64, iterations=300, steps_per_temp=64, threads=64, seed=7, initial="bfs",
                            fanin_device=0)
    secs = time.perf_counter() - t0
    info = tnsa.tn_plan_get_info(p)
    assert info["con_dist"] <= info["initial_con_dist"]
    assert secs < 60.0, secs
    print(f"k=64 annealing: {secs:.1f} s, con_dist {info['initial_con_dist']} -> {info['con_dist']}")
