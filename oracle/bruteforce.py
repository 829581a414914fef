"""Brute-force definitions for tiny inputs (oracle, test infrastructure only).

* ``network_sum``: the contraction of a tensor network as the sum, over every
  assignment of the internal labels, of the product of the tensor entries
  (the definition behind Fig. 1 and Fig. 3), for each assignment of the open
  labels.  Exponential in the number of labels; use with at most ~16 labels.
* ``full_unitary`` / ``apply_full``: each gate as an explicit 2^n x 2^n matrix
  built entry by entry from bit extraction, then multiplied.  Used on <= 10
  qubits to pin the state-vector route.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def network_sum(labels: Sequence[Sequence[int]], tensors: Sequence[np.ndarray],
                open_labels: Sequence[int]) -> np.ndarray:
    all_labels = sorted({lab for l in labels for lab in l})
    internal = [lab for lab in all_labels if lab not in open_labels]
    k = len(open_labels)
    out = np.zeros(1 << k, dtype=np.complex128)
    flat = [np.asarray(t, dtype=np.complex128).reshape(-1) for t in tensors]
    for o in range(1 << k):
        val = {}
        for j, lab in enumerate(open_labels):
            val[lab] = (o >> (k - 1 - j)) & 1
        total = 0j
        for a in range(1 << len(internal)):
            for j, lab in enumerate(internal):
                val[lab] = (a >> j) & 1
            prod = 1 + 0j
            for labs, t in zip(labels, flat):
                idx = 0
                for lab in labs:  # first label = most significant axis
                    idx = (idx << 1) | val[lab]
                prod *= t[idx]
                if prod == 0:
                    break
            total += prod
        out[o] = total
    return out


def full_gate(n: int, matrix: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """2^n x 2^n matrix of a gate; qubit 0 = most significant bit."""
    dim = 1 << n
    k = len(qubits)
    m = np.zeros((dim, dim), dtype=np.complex128)
    g = np.asarray(matrix, dtype=np.complex128)
    for col in range(dim):
        sub_in = 0
        for q in qubits:
            sub_in = (sub_in << 1) | ((col >> (n - 1 - q)) & 1)
        base = col
        for q in qubits:
            base &= ~(1 << (n - 1 - q))
        for sub_out in range(1 << k):
            row = base
            for j, q in enumerate(qubits):
                bit = (sub_out >> (k - 1 - j)) & 1
                row |= bit << (n - 1 - q)
            m[row, col] += g[sub_out, sub_in]
    return m


def apply_full(circuit) -> np.ndarray:
    """U|0...0> as a flat vector, by explicit full-matrix products."""
    n = circuit.n_qubits
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = 1.0
    for gate in circuit.gates:
        v = full_gate(n, gate.matrix, gate.qubits) @ v
    return v


def full_unitary(circuit) -> np.ndarray:
    n = circuit.n_qubits
    u = np.eye(1 << n, dtype=np.complex128)
    for gate in circuit.gates:
        u = full_gate(n, gate.matrix, gate.qubits) @ u
    return u
