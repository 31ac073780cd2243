"""Brute-force state-vector simulation (complex128). Test infrastructure only.

A textbook routine used to pin the oracle contractor: the amplitude <x|C|0^n> of a circuit equals
the full contraction of its closed tensor network.  Qubit 0 is the most significant bit of the
state index; a gate matrix has rows = output basis states and columns = input basis states, and a
2-qubit gate on (a, b) uses basis index 2*bit_a + bit_b.  `kron_unitary` builds the full 2^n x 2^n
matrix of a circuit from Kronecker products, a second and independent route for tiny n.
"""
import numpy as np


def simulate(circ) -> np.ndarray:
    n = circ.n_qubits
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for g in circ.gates:
        if len(g.qubits) == 1:
            (q,) = g.qubits
            psi = np.moveaxis(np.tensordot(g.matrix, psi, axes=([1], [q])), 0, q)
        else:
            a, b = g.qubits
            u = g.matrix.reshape(2, 2, 2, 2)
            psi = np.moveaxis(np.tensordot(u, psi, axes=([2, 3], [a, b])), [0, 1], [a, b])
    return psi.reshape(-1)


def amplitude(circ, x) -> complex:
    psi = simulate(circ).reshape((2,) * circ.n_qubits)
    return complex(psi[tuple(int(b) for b in x)])


def zz_expectation(circ, i, j) -> float:
    n = circ.n_qubits
    p = np.abs(simulate(circ).reshape((2,) * n)) ** 2
    idx = np.indices((2,) * n)
    sign = (-1.0) ** (idx[i] + idx[j])
    return float(np.sum(p * sign))


def _embed(matrix, qubits, n):
    """Full 2^n operator of a gate, built from Kronecker products (adjacent or swapped qubits
    handled by permuting basis states explicitly)."""
    dim = 2 ** n
    full = np.zeros((dim, dim), dtype=np.complex128)
    k = len(qubits)
    for col in range(dim):
        bits = [(col >> (n - 1 - q)) & 1 for q in range(n)]
        sub_in = 0
        for q in qubits:
            sub_in = 2 * sub_in + bits[q]
        for sub_out in range(2 ** k):
            amp = matrix[sub_out, sub_in]
            if amp == 0:
                continue
            ob = list(bits)
            for t, q in enumerate(qubits):
                ob[q] = (sub_out >> (k - 1 - t)) & 1
            row = 0
            for b in ob:
                row = 2 * row + b
            full[row, col] += amp
    return full


def kron_unitary(circ) -> np.ndarray:
    n = circ.n_qubits
    u = np.eye(2 ** n, dtype=np.complex128)
    for g in circ.gates:
        u = _embed(g.matrix, g.qubits, n) @ u
    return u
