"""Seeded synthetic inputs: random quantum circuits and the closed tensor networks built from them.

This module only *produces* inputs (gate matrices, wiring, bitstrings). It holds none of the
contraction arithmetic, cost model or planner logic, so that both the CPU oracle (through the tests)
and the GPU engine can be fed from it without sharing any of the method's code.

Network model (Section 2.1, Eq. 2.1): a network is a list of tensors T_v with dims n_v and an edge
list ((u, a), (v, b)) pairing axis a of tensor u with axis b of tensor v; v = -1 stands for the
dummy vertex (an open leg). Axes are 0-based here.

Conventions (the paper is circuit-agnostic; these are the choices of this engine):
  * tensors are stored row-major (C order), leg 0 slowest;
  * gate tensors have legs (out..., in...): a 1-qubit gate is T[o, i] = U[o][i]; a 2-qubit gate on
    qubits a < b is T[oa, ob, ia, ib] = U[2*oa + ob][2*ia + ib];
  * |0> leaf is T[o] = delta(o, 0); <x| leaf on qubit q is T[i] = delta(i, x_q);
  * state-vector index: qubit 0 is the most significant bit;
  * depth counts U3 + CZ cycles after the Hadamard layer;
  * 1D brickwork cycle c uses CZ pairs (2j, 2j+1) if c is even, else (2j+1, 2j+2);
  * 2D grid (rows x cols, qubit q = r*cols + c) cycle c uses pattern c mod 4 in the order
    A: (r,c)-(r,c+1), c even; B: same, c odd; C: (r,c)-(r+1,c), r even; D: same, r odd;
  * Haar U3(theta, phi, lam) = [[cos t/2, -e^{i lam} sin t/2], [e^{i phi} sin t/2,
    e^{i(phi+lam)} cos t/2]] with theta = arccos(1 - 2u), u, phi/2pi, lam/2pi ~ U[0, 1), drawn in
    that order per gate, gates drawn qubit by qubit inside each cycle.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

H_MAT = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
Z_MAT = np.array([[1, 0], [0, -1]], dtype=np.complex128)
X_MAT = np.array([[0, 1], [1, 0]], dtype=np.complex128)
CZ_MAT = np.diag([1, 1, 1, -1]).astype(np.complex128)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def haar_u3(rng: np.random.Generator) -> np.ndarray:
    u = rng.random()
    phi = rng.random() * 2 * math.pi
    lam = rng.random() * 2 * math.pi
    return u3(math.acos(1 - 2 * u), phi, lam)


@dataclass
class Gate:
    name: str
    qubits: tuple
    matrix: np.ndarray  # 2x2 or 4x4, rows = out index, cols = in index


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)
    layout: tuple = ()  # (rows, cols) for 2D grids, () for 1D

    def add(self, name, qubits, matrix):
        self.gates.append(Gate(name, tuple(qubits), np.asarray(matrix, dtype=np.complex128)))

    def dagger(self) -> "Circuit":
        out = Circuit(self.n_qubits, layout=self.layout)
        for g in reversed(self.gates):
            out.add(g.name + "^dg", g.qubits, g.matrix.conj().T)
        return out


def brickwork_1d(n: int, depth: int, seed: int) -> Circuit:
    rng = np.random.default_rng(seed)
    c = Circuit(n)
    for q in range(n):
        c.add("H", (q,), H_MAT)
    for cyc in range(depth):
        for q in range(n):
            c.add("U3", (q,), haar_u3(rng))
        start = 0 if cyc % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            c.add("CZ", (a, a + 1), CZ_MAT)
    return c


def grid_pairs(rows: int, cols: int, pattern: int):
    pairs = []
    if pattern in (0, 1):
        for r in range(rows):
            for cc in range(pattern, cols - 1, 2):
                pairs.append((r * cols + cc, r * cols + cc + 1))
    else:
        for r in range(pattern - 2, rows - 1, 2):
            for cc in range(cols):
                pairs.append((r * cols + cc, (r + 1) * cols + cc))
    return pairs


def grid_2d(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    rng = np.random.default_rng(seed)
    n = rows * cols
    c = Circuit(n, layout=(rows, cols))
    for q in range(n):
        c.add("H", (q,), H_MAT)
    for cyc in range(depth):
        for q in range(n):
            c.add("U3", (q,), haar_u3(rng))
        for a, b in grid_pairs(rows, cols, cyc % 4):
            c.add("CZ", (a, b), CZ_MAT)
    return c


def ghz(n: int) -> Circuit:
    """H on qubit 0, then CNOT(q -> q+1) written as (I x H) CZ (I x H)."""
    c = Circuit(n)
    c.add("H", (0,), H_MAT)
    for q in range(n - 1):
        c.add("H", (q + 1,), H_MAT)
        c.add("CZ", (q, q + 1), CZ_MAT)
        c.add("H", (q + 1,), H_MAT)
    return c


def random_bitstring(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(0, 2, n).astype(np.int64)


@dataclass
class Network:
    """Flat tensor-network description in the form the C ABI takes (Eq. 2.1)."""
    tensors: list            # list of complex128 ndarrays, row-major
    edges: np.ndarray        # int32 [E, 4]: u, a, v, b (v = -1: open leg)
    qubit: np.ndarray        # int32 [n]: qubit each tensor sits on (2q gates: lower qubit); a hint
    kind: list               # tensor labels, for debugging

    @property
    def n_tensors(self) -> int:
        return len(self.tensors)

    @property
    def degrees(self) -> np.ndarray:
        return np.array([t.ndim for t in self.tensors], dtype=np.int32)

    @property
    def dims(self) -> np.ndarray:
        return np.array([d for t in self.tensors for d in t.shape], dtype=np.int64)

    @property
    def data(self) -> np.ndarray:
        """All tensors concatenated, complex128 interleaved (re, im) as float64."""
        flat = np.concatenate([np.ascontiguousarray(t).ravel() for t in self.tensors]) \
            if self.tensors else np.zeros(0, np.complex128)
        return np.ascontiguousarray(flat.astype(np.complex128)).view(np.float64)


class _Builder:
    def __init__(self, n_qubits):
        self.tensors, self.kind, self.qubit, self.edges = [], [], [], []
        self.front = [None] * n_qubits  # (tensor, axis) of the latest open output on each wire

    def add(self, t, kind, q):
        self.tensors.append(np.ascontiguousarray(t, dtype=np.complex128))
        self.kind.append(kind)
        self.qubit.append(q)
        return len(self.tensors) - 1

    def ket0(self, q):
        tid = self.add(np.array([1, 0]), "ket", q)
        self.front[q] = (tid, 0)

    def gate(self, g: Gate):
        if len(g.qubits) == 1:
            (q,) = g.qubits
            tid = self.add(g.matrix, g.name, q)
            u, a = self.front[q]
            self.edges.append((u, a, tid, 1))
            self.front[q] = (tid, 0)
        else:
            qa, qb = g.qubits
            if qa > qb:
                raise ValueError("2-qubit gates are stored with qubits in increasing order")
            tid = self.add(g.matrix.reshape(2, 2, 2, 2), g.name, qa)
            for q, ax_in, ax_out in ((qa, 2, 0), (qb, 3, 1)):
                u, a = self.front[q]
                self.edges.append((u, a, tid, ax_in))
                self.front[q] = (tid, ax_out)

    def bra(self, q, bit):
        t = np.zeros(2)
        t[int(bit)] = 1
        tid = self.add(t, "bra", q)
        u, a = self.front[q]
        self.edges.append((u, a, tid, 0))
        self.front[q] = None

    def network(self):
        return Network(self.tensors, np.array(self.edges, dtype=np.int32).reshape(-1, 4),
                       np.array(self.qubit, dtype=np.int32), self.kind)


def amplitude_tn(circ: Circuit, x) -> Network:
    """Closed network whose full contraction is <x| C |0^n>."""
    b = _Builder(circ.n_qubits)
    for q in range(circ.n_qubits):
        b.ket0(q)
    for g in circ.gates:
        b.gate(g)
    for q in range(circ.n_qubits):
        b.bra(q, x[q])
    return b.network()


def sandwich_tn(circ: Circuit, middle: list) -> Network:
    """Closed network <0^n| C^dagger M C |0^n> for a list of middle gates M."""
    b = _Builder(circ.n_qubits)
    for q in range(circ.n_qubits):
        b.ket0(q)
    for g in circ.gates:
        b.gate(g)
    for g in middle:
        b.gate(g)
    for g in circ.dagger().gates:
        b.gate(g)
    for q in range(circ.n_qubits):
        b.bra(q, 0)
    return b.network()


def inverse_tn(circ: Circuit) -> Network:
    """<0| C^-1 C |0>, which equals 1 for any unitary C."""
    return sandwich_tn(circ, [])


def zz_tn(circ: Circuit, i: int, j: int) -> Network:
    """<psi| Z_i Z_j |psi> with |psi> = C|0^n>."""
    return sandwich_tn(circ, [Gate("Z", (i,), Z_MAT), Gate("Z", (j,), Z_MAT)])


def zz_slots_tn(circ: Circuit):
    """<0^n| C^dagger D C |0^n> with D a layer of single-qubit identity slots, one per qubit.
    Replacing slots i and j by Z gives <psi| Z_i Z_j |psi>, so one network (and one plan) serves
    every pair.  Returns (network, slot tensor ids by qubit)."""
    n = circ.n_qubits
    net = sandwich_tn(circ, [Gate("slot", (q,), np.eye(2)) for q in range(n)])
    first = n + len(circ.gates)
    return net, [first + q for q in range(n)]


def bra_ids(net: Network, n_qubits: int):
    """Tensor ids of the bra leaves of an amplitude network, by qubit."""
    return [net.n_tensors - n_qubits + q for q in range(n_qubits)]


def norm_tn(circ: Circuit) -> Network:
    """<psi|psi>: C and its elementwise conjugate joined output wire to output wire (no bras)."""
    n = circ.n_qubits
    b = _Builder(n)
    for q in range(n):
        b.ket0(q)
    for g in circ.gates:
        b.gate(g)
    front_c = list(b.front)
    b.front = [None] * n
    for q in range(n):
        b.ket0(q)
    for g in circ.gates:
        b.gate(Gate(g.name + "*", g.qubits, g.matrix.conj()))
    for q in range(n):
        (u, a), (v, c) = front_c[q], b.front[q]
        b.edges.append((u, a, v, c))
    return b.network()


def random_network(n_tensors: int, n_extra_edges: int, dim_choices, seed: int,
                   n_open: int = 0) -> Network:
    """A connected random network: a random spanning tree plus extra (multi-)edges, each edge
    with a dimension drawn from dim_choices, plus n_open open legs; entries ~ CN(0, 1)."""
    rng = np.random.default_rng(seed)
    ends = []  # (u, v, dim)
    for v in range(1, n_tensors):
        ends.append((int(rng.integers(0, v)), v, int(rng.choice(dim_choices))))
    for _ in range(n_extra_edges):
        u, v = rng.choice(n_tensors, 2, replace=False)
        ends.append((int(u), int(v), int(rng.choice(dim_choices))))
    opens = [(int(rng.integers(0, n_tensors)), -1, int(rng.choice(dim_choices)))
             for _ in range(n_open)]
    axes = [[] for _ in range(n_tensors)]
    edges = []
    for u, v, d in ends + opens:
        a = len(axes[u])
        axes[u].append(d)
        if v >= 0:
            b = len(axes[v])
            axes[v].append(d)
        else:
            b = 0
        edges.append((u, a, v, b))
    tensors = []
    for t in range(n_tensors):
        shape = tuple(axes[t])
        z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        tensors.append(np.asarray(z / math.sqrt(2), dtype=np.complex128))
    return Network(tensors, np.array(edges, dtype=np.int32).reshape(-1, 4),
                   np.zeros(n_tensors, np.int32), ["rand"] * n_tensors)


# The five workloads (sizes, seeds, partition counts) used by the tests and the benchmark.
def cfg1():
    circ = brickwork_1d(10, 8, seed=1)
    return circ, random_bitstring(10, 1001)


def cfg2():
    circ = brickwork_1d(24, 14, seed=2)
    return circ, random_bitstring(24, 1002)


def cfg3(small: bool = False):
    circ = grid_2d(4, 5, 8, seed=3) if small else grid_2d(5, 8, 12, seed=3)
    return circ, random_bitstring(circ.n_qubits, 1003)


def cfg4_circuits():
    """32 circuits, seeds 100..131: n ~ U{16..36}, depth ~ U{8..16}; even seed 1D, odd seed 2D on
    a near-square grid (n rounded to rows*cols); k cycles 2, 4, 8; 16 bitstrings each."""
    out = []
    for i, s in enumerate(range(100, 132)):
        rng = np.random.default_rng(s)
        n = int(rng.integers(16, 37))
        depth = int(rng.integers(8, 17))
        k = (2, 4, 8)[i % 3]
        if s % 2 == 0:
            circ = brickwork_1d(n, depth, seed=s)
        else:
            rows = int(math.floor(math.sqrt(n)))
            cols = int(round(n / rows))
            circ = grid_2d(rows, cols, depth, seed=s)
        xs = [random_bitstring(circ.n_qubits, 10_000 * s + j) for j in range(16)]
        out.append((circ, k, xs))
    return out
