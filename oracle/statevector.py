"""Schroedinger state-vector simulation in complex128 (oracle, test
infrastructure only).

The amplitude the big-head method computes for a bitstring s = (s1; s2) is
<s|U|0...0> ("Big-head simulation" section; the Schroedinger method is the
first kind of simulator in the introduction).  This module computes it by
definition: apply every gate in circuit order to the full 2^n vector.

Axis q of the (2,)*n array is qubit q; qubit 0 is the most significant bit of
a flat index.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def apply_gate(psi: np.ndarray, matrix: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """psi'[.., o, ..] = sum_i G[o, i] psi[.., i, ..] on the gate's qubits."""
    k = len(qubits)
    g = np.asarray(matrix, dtype=np.complex128).reshape((2,) * (2 * k))
    out = np.tensordot(g, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    return np.moveaxis(out, list(range(k)), list(qubits))


def final_state(circuit) -> np.ndarray:
    """U|0...0> as an (2,)*n complex128 array."""
    n = circuit.n_qubits
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for gate in circuit.gates:
        psi = apply_gate(psi, gate.matrix, gate.qubits)
    return psi


def amplitudes(circuit, fixed_bits: Sequence[int], open_qubits: Sequence[int],
               psi: np.ndarray = None) -> np.ndarray:
    """A[s2] = <s1; s2|U|0> for every assignment s2 of the open qubits.

    ``fixed_bits`` has one entry per qubit (entries at open positions are
    ignored); the result is flat, index = sum_j s2_j 2^(k-1-j) in the order of
    ``open_qubits``."""
    n = circuit.n_qubits
    if psi is None:
        psi = final_state(circuit)
    idx = []
    for q in range(n):
        idx.append(slice(None) if q in open_qubits else int(fixed_bits[q]))
    sub = psi[tuple(idx)]
    # remaining axes are the open qubits in increasing qubit order
    remaining = sorted(open_qubits)
    perm = [remaining.index(q) for q in open_qubits]
    sub = np.transpose(sub, perm) if len(perm) > 1 else sub
    return np.ascontiguousarray(sub).reshape(-1)
