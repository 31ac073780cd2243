"""Pins for the oracle: each check compares it with something other than itself.

  * the state vector against a Kronecker-product unitary (a second route) and closed forms;
  * the contractor against the state vector, numpy.einsum on tiny networks (a library routine),
    closed forms (GHZ amplitude 1/sqrt 2, <0|C^-1 C|0> = 1, <psi|psi> = 1), and order
    independence of the result (the contraction result does not depend on the tree, Section 2.3);
  * the cost model against hand-derived numbers (tests/golden/costs_hand.txt) and the identities
    that follow from Eq. 3.4-3.5;
  * the greedy rule against a hand-derived sequence;
  * the permutation index map against index arithmetic written out with plain loops, and the
    matrix transpose.
"""
import math
import os

import numpy as np
import pytest

from oracle import contract as oc
from oracle import costs as ocost
from oracle import greedy as og
from oracle import perm as operm
from oracle import statevector as sv
from paper_2507_20667_gb300 import inputs as tni


def block_partition(net, n_qubits, k):
    """k contiguous blocks of qubits; each tensor goes to the block of the qubit it sits on."""
    return ((np.asarray(net.qubit, dtype=np.int64) * k) // n_qubits).astype(np.int32)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def greedy_full_tree(net):
    """Oracle Greedy over the whole network (one partition), in export node ids."""
    legs = ocost.leaf_legs(net)
    dims = ocost.edge_dims(net)
    return og.greedy_steps(list(legs), dims)  # local ids == global ids for k = 1


def random_tree(n, seed):
    """A uniformly random pairing order (any tree is a valid contraction tree). Only for
    networks small enough that every intermediate stays small."""
    rng = np.random.default_rng(seed)
    alive = list(range(n))
    steps, nxt = [], n
    while len(alive) > 1:
        i, j = sorted(rng.choice(len(alive), 2, replace=False))
        a, b = alive[i], alive[j]
        steps.append((min(a, b), max(a, b)))
        alive = [t for t in alive if t not in (a, b)] + [nxt]
        nxt += 1
    return steps


def relabelled_greedy_tree(net, seed):
    """A different but still cheap tree: Greedy run on a random relabelling of the tensors."""
    rng = np.random.default_rng(seed)
    n = net.n_tensors
    order = rng.permutation(n)
    legs = ocost.leaf_legs(net)
    local = og.greedy_steps([legs[t] for t in order], ocost.edge_dims(net))
    ids = [int(t) for t in order]
    steps = []
    for i, j in local:
        a, b = ids[i], ids[j]
        steps.append((min(a, b), max(a, b)))
        ids.append(n + len(steps) - 1)
    return steps


def einsum_network(net):
    letters = {}
    def sym(e):
        if e not in letters:
            letters[e] = chr(ord("a") + len(letters)) if len(letters) < 26 else chr(ord("A") + len(letters) - 26)
        return letters[e]
    ax = [[None] * t.ndim for t in net.tensors]
    opens = []
    for e, (u, a, v, b) in enumerate(net.edges):
        ax[u][a] = sym(e)
        if v >= 0:
            ax[v][b] = sym(e)
        else:
            opens.append(sym(e))
    spec = ",".join("".join(s) for s in ax) + "->" + "".join(opens)
    return np.einsum(spec, *net.tensors, optimize=True), opens


# ---------------------------------------------------------------- state vector
@pytest.mark.parametrize("maker", [lambda: tni.brickwork_1d(4, 3, seed=5), lambda: tni.grid_2d(2, 2, 4, seed=6),
                                   lambda: tni.ghz(3)])
def test_statevector_matches_kron_unitary(maker):
    circ = maker()
    u = sv.kron_unitary(circ)
    e0 = np.zeros(2 ** circ.n_qubits, np.complex128)
    e0[0] = 1
    np.testing.assert_allclose(sv.simulate(circ), u @ e0, atol=1e-13)
    np.testing.assert_allclose(u.conj().T @ u, np.eye(len(u)), atol=1e-12)


def test_statevector_closed_forms():
    n = 6
    psi = sv.simulate(tni.ghz(n))
    expect = np.zeros(2 ** n, np.complex128)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, expect, atol=1e-14)
    h_only = tni.Circuit(n)
    for q in range(n):
        h_only.add("H", (q,), tni.H_MAT)
    np.testing.assert_allclose(sv.simulate(h_only), np.full(2 ** n, 2 ** (-n / 2)), atol=1e-14)
    c = tni.brickwork_1d(8, 5, seed=9)
    assert abs(np.linalg.norm(sv.simulate(c)) - 1) < 1e-12
    # <Z_i Z_j> on |0..0> after identity-like circuit = 1; on GHZ = 1 for any pair
    assert abs(sv.zz_expectation(tni.ghz(5), 1, 3) - 1) < 1e-12
    # Haar U3 draw: the stated recipe gives a unitary with the stated form
    g = tni.u3(0.3, 0.2, 0.1)
    np.testing.assert_allclose(g.conj().T @ g, np.eye(2), atol=1e-15)


def test_statevector_qubit_order_msb():
    c = tni.Circuit(3)
    c.add("X", (0,), tni.X_MAT)       # flip qubit 0 -> |100> = index 4
    psi = sv.simulate(c)
    assert abs(psi[4] - 1) < 1e-15
    c2 = tni.Circuit(2)
    c2.add("X", (1,), tni.X_MAT)
    c2.add("CZ", (0, 1), tni.CZ_MAT)
    c2.add("X", (0,), tni.X_MAT)
    c2.add("CZ", (0, 1), tni.CZ_MAT)  # |11> picks up the -1
    assert abs(sv.simulate(c2)[3] + 1) < 1e-15


# ---------------------------------------------------------------- contractor
def test_contractor_cfg1_matches_statevector():
    circ, x = tni.cfg1()
    net = tni.amplitude_tn(circ, x)
    assert net.n_tensors == 146 and len(net.edges) == 172
    a = oc.contract_scalar(net, greedy_full_tree(net))
    ref = sv.amplitude(circ, x)
    assert abs(a - ref) <= 1e-12 * max(abs(ref), 1e-300) + 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_contractor_order_independent(seed):
    circ = tni.brickwork_1d(6, 4, seed=20 + seed)
    x = tni.random_bitstring(6, 30 + seed)
    net = tni.amplitude_tn(circ, x)
    ref = sv.amplitude(circ, x)
    for t in range(3):
        a = oc.contract_scalar(net, relabelled_greedy_tree(net, 100 * seed + t))
        assert abs(a - ref) < 1e-13


@pytest.mark.parametrize("seed", range(4))
def test_contractor_matches_einsum_mixed_dims(seed):
    net = tni.random_network(7, 4, (1, 2, 3, 5), seed=seed, n_open=2)
    ref, opens = einsum_network(net)
    val, legs = oc.contract(net, random_tree(net.n_tensors, seed))
    # the oracle returns the open legs in its own order; bring einsum's output to that order
    open_ids = [e for e, (u, a, v, b) in enumerate(net.edges) if v < 0]
    perm = [open_ids.index(e) for e in legs]
    np.testing.assert_allclose(val, np.transpose(ref, perm), rtol=1e-12, atol=1e-12)


def test_contractor_closed_forms():
    n = 7
    ghz = tni.ghz(n)
    for bits, want in (([0] * n, 1 / math.sqrt(2)), ([1] * n, 1 / math.sqrt(2)), ([0, 1] + [0] * (n - 2), 0.0)):
        net = tni.amplitude_tn(ghz, bits)
        assert abs(oc.contract_scalar(net, greedy_full_tree(net)) - want) < 1e-14
    circ = tni.brickwork_1d(6, 5, seed=11)
    for net in (tni.inverse_tn(circ), tni.norm_tn(circ)):
        assert abs(oc.contract_scalar(net, greedy_full_tree(net)) - 1) < 1e-12
    net = tni.zz_tn(circ, 1, 4)
    assert abs(oc.contract_scalar(net, greedy_full_tree(net)) - sv.zz_expectation(circ, 1, 4)) < 1e-12


def test_contractor_grid_small_instance():
    circ = tni.grid_2d(3, 3, 5, seed=3)
    x = tni.random_bitstring(9, 77)
    net = tni.amplitude_tn(circ, x)
    a = oc.contract_scalar(net, greedy_full_tree(net))
    assert abs(a - sv.amplitude(circ, x)) < 1e-13


# ---------------------------------------------------------------- cost model
class _Net:
    """A network with only structure (dims), for the cost model."""
    def __init__(self, shapes, edges):
        self.tensors = [np.zeros(s) for s in shapes]
        self.degrees = np.array([len(s) for s in shapes], np.int32)
        self.dims = np.array([d for s in shapes for d in s], np.int64)
        self.edges = np.array(edges, np.int32).reshape(-1, 4)


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = int(v)
    return out


def chain_net():
    # v1[2] -e0- M1[2,3] -e1- M2[3,5] -e2- v2[5]
    return _Net([(2,), (2, 3), (3, 5), (5,)], [(0, 0, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0)])


def test_costs_hand_chain():
    g = _read_golden("costs_hand.txt")
    net = chain_net()
    left = ocost.counts(net, [(0, 1), (2, 4), (3, 5)])
    assert left["con_serial"] == g["chain_left_con_serial"]
    assert left["mem"] == g["chain_left_mem"]
    assert left["con_par"] == g["chain_left_con_par"]
    split = ocost.counts(net, [(0, 1), (2, 3), (4, 5)], part=[0, 0, 1, 1])
    assert split["con_serial"] == g["chain_split_con_serial"]
    assert split["con_par"] == g["chain_split_con_par"]
    assert split["con_dist"] == g["chain_split_con_dist"]
    assert split["mem"] == g["chain_split_mem"]


def ring_net(m):
    shapes = [(2, 2)] * m
    edges = [(i, 1, (i + 1) % m, 0) for i in range(m)]
    return _Net(shapes, edges)


@pytest.mark.parametrize("m", [3, 4, 7, 12])
def test_costs_ring_closed_form(m):
    net = ring_net(m)
    steps = [(0, 1)] + [(m + s, s + 2) for s in range(m - 2)]
    c = ocost.counts(net, steps, part=[0] * m)
    assert c["con_serial"] == 8 * (m - 2) + 4
    assert c["mem"] == 12
    assert c["con_dist"] == c["con_serial"]      # k = 1: path_k is empty
    assert c["con_par"] == c["con_serial"]       # a left-deep chain is one path


@pytest.mark.parametrize("seed", range(5))
def test_costs_identities(seed):
    circ = tni.brickwork_1d(6, 4, seed=seed)
    net = tni.amplitude_tn(circ, tni.random_bitstring(6, seed))
    part = block_partition(net, 6, 3)
    # tree: greedy inside each partition, then a left-deep fan-in
    legs = ocost.leaf_legs(net)
    dims = ocost.edge_dims(net)
    n = net.n_tensors
    steps, roots = [], []
    for k in range(3):
        members = [t for t in range(n) if part[t] == k]
        local = og.greedy_steps([legs[t] for t in members], dims)
        ids = list(members)
        for i, j in local:
            steps.append((ids[i], ids[j]))
            ids.append(n + len(steps) - 1)
        roots.append(ids[-1])
    cur = roots[0]
    for r in roots[1:]:
        steps.append((min(cur, r), max(cur, r)))
        cur = n + len(steps) - 1
    c = ocost.counts(net, steps, part=part)
    assert c["con_par"] <= c["con_dist"] <= c["con_serial"]
    assert c["con_dist_par"] == c["con_par"]     # Eq. 3.5 with con = con_par and comm = 0
    assert c["mem"] >= 16                        # at least one 2q gate tensor and its partner


def test_costs_rejects_non_accepting_tree():
    net = chain_net()
    with pytest.raises(ValueError):
        ocost.counts(net, [(0, 1), (2, 4), (3, 5)], part=[0, 1, 0, 1])


# ---------------------------------------------------------------- greedy rule
def test_greedy_hand_star():
    # centre C[2,3,4] with vectors of dim 2, 3, 4: objectives 14, 19, 22 -> absorb dim 4 first,
    # then C'[2,3]: 5 (dim 2) vs 7 (dim 3) -> dim 3, then dim 2.
    net = _Net([(2, 3, 4), (2,), (3,), (4,)], [(0, 0, 1, 0), (0, 1, 2, 0), (0, 2, 3, 0)])
    steps = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    assert steps == [(0, 3), (2, 4), (1, 5)]


def test_greedy_ties_and_disconnected():
    # two disjoint 2x2 pairs: A0-A1 and B2-B3 (each pair shares two legs -> objective 4 + 4 - 1 = 7)
    net = _Net([(2, 2), (2, 2), (2, 2), (2, 2)],
               [(0, 0, 1, 0), (0, 1, 1, 1), (2, 0, 3, 0), (2, 1, 3, 1)])
    steps = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    # tie between (0,1) and (2,3) -> (0,1) first; then (2,3); then outer product of scalars 4, 5
    assert steps == [(0, 1), (2, 3), (4, 5)]


@pytest.mark.parametrize("dims,perm", [((2, 3, 4), (2, 0, 1)), ((3, 1, 5, 2), (3, 1, 0, 2)),
                                       ((2, 2, 2, 2, 2), (4, 3, 2, 1, 0)), ((5,), (0,)), ((), ())])
def test_permute_iota_brute_force(dims, perm):
    """Output element i (row-major over the permuted shape) is the input element whose index along
    axis perm[t] is the output's index along axis t: the map enumerated with plain loops."""
    out = operm.permute_iota(dims, perm)
    odims = [dims[p] for p in perm]
    expected = []
    for i in range(math.prod(dims)):
        idx, r = [], i
        for d in reversed(odims):
            idx.append(r % d)
            r //= d
        idx.reverse()
        src = [0] * len(dims)
        for t, p in enumerate(perm):
            src[p] = idx[t]
        lin = 0
        for a, d in enumerate(dims):
            lin = lin * d + src[a]
        expected.append(lin)
    assert out.tolist() == expected


def test_permute_iota_matrix_transpose():
    """Swapping the two axes of a rows x cols matrix: element (j, i) of the result is i cols + j."""
    rows, cols = 3, 5
    out = operm.permute_iota((rows, cols), (1, 0))
    assert out.tolist() == [i * cols + j for j in range(cols) for i in range(rows)]
