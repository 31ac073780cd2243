"""Slicing on top of partitioning (Section 4.1): the slice planner's counts against the big-int
oracle on the sliced network (the same tree with the sliced edges of dimension 1)."""
import numpy as np
import pytest

from oracle import costs as ocost
from paper_2507_20667_gb300 import inputs as tni
from paper_2507_20667_gb300 import tnsa


class _Sliced:
    """The network with the given edges of dimension 1 (entries: zeros of the reduced shapes)."""
    def __init__(self, net, edges):
        es = set(edges)
        off = np.concatenate([[0], np.cumsum(net.degrees)])
        dims = np.asarray(net.dims, np.int64).copy()
        for e, (u, a, v, b) in enumerate(net.edges):
            if e in es:
                dims[off[u] + a] = 1
                if v >= 0:
                    dims[off[v] + b] = 1
        self.degrees, self.dims, self.edges = net.degrees, dims, net.edges
        size = sum(int(np.prod(dims[off[t]:off[t + 1]])) for t in range(len(net.degrees)))
        self.data = np.zeros(2 * size)


@pytest.mark.parametrize("which,k,shrink", [("cfg3s", 8, 16), ("cfg3s", 4, 256), ("cfg2", 4, 64)])
def test_slice_counts_against_oracle(which, k, shrink):
    circ, x = tni.cfg3(small=True) if which == "cfg3s" else tni.cfg2()
    net = tni.amplitude_tn(circ, x)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_create(h, k=k, iterations=50, seed=7, position=net.qubit)
    total, crit, mem = tnsa.tn_plan_counts(plan)
    r = tnsa.tn_plan_slice(h, plan, mem // shrink)
    assert r["slice_mem"] <= mem // shrink and r["edges"] == sorted(r["edges"])
    dims = ocost.edge_dims(net)
    assert r["n_slices"] == int(np.prod([dims[e] for e in r["edges"]], dtype=object))
    part, steps, _ = tnsa.tn_plan_export(plan, net.n_tensors)
    tree = [(int(a), int(b)) for a, b, o in steps]
    oc = ocost.counts(_Sliced(net, r["edges"]), tree)
    assert (oc["con_serial"], oc["mem"]) == (r["slice_con"], r["slice_mem"])
    assert r["total_con"] == r["slice_con"] * r["n_slices"] >= total     # slicing repeats work
    # no slicing needed at the plan's own mem
    r0 = tnsa.tn_plan_slice(h, plan, mem)
    assert r0["edges"] == [] and r0["n_slices"] == 1 and r0["slice_con"] == total
