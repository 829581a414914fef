"""Circuit -> tensor network, one tensor per gate (oracle, test
infrastructure only).

Follows the circuit-as-tensor-network picture of Fig. 1: the initial |0>
vectors, one tensor per gate, and at the end either a closed qubit's bit
vector e_{s_q} or an open leg.  No gate absorption or other simplification is
done here, so the network is the circuit written out.

Bond labels follow the wire-segment convention (tn_inputs.networks): segment t
of qubit q is the wire after the t-th gate on q; label = offset_q + t.
A gate tensor's axes are (outputs..., inputs...) in the gate's qubit order,
matching its matrix reshaped to (2,)*(2k).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def wire_offsets(circuit) -> Tuple[List[int], List[int]]:
    n = circuit.n_qubits
    count = [0] * n
    for g in circuit.gates:
        for q in g.qubits:
            count[q] += 1
    offs, acc = [], 0
    for q in range(n):
        offs.append(acc)
        acc += count[q] + 1
    return offs, count


def circuit_network(circuit, fixed_bits: Sequence[int], open_qubits: Sequence[int]):
    """Return (labels, tensors, open_labels): lists of per-tensor label lists
    and complex128 arrays, and the open labels in amplitude-axis order."""
    n = circuit.n_qubits
    offs, count = wire_offsets(circuit)
    seen = [0] * n
    labels: List[List[int]] = []
    tensors: List[np.ndarray] = []
    zero = np.array([1.0, 0.0], dtype=np.complex128)
    for q in range(n):
        labels.append([offs[q]])
        tensors.append(zero.copy())
    for g in circuit.gates:
        k = len(g.qubits)
        ins = [offs[q] + seen[q] for q in g.qubits]
        for q in g.qubits:
            seen[q] += 1
        outs = [offs[q] + seen[q] for q in g.qubits]
        labels.append(outs + ins)
        tensors.append(np.asarray(g.matrix, dtype=np.complex128).reshape((2,) * (2 * k)))
    open_set = set(open_qubits)
    for q in range(n):
        if q in open_set:
            continue
        e = np.zeros(2, dtype=np.complex128)
        e[int(fixed_bits[q])] = 1.0
        labels.append([offs[q] + count[q]])
        tensors.append(e)
    open_labels = [offs[q] + count[q] for q in open_qubits]
    return labels, tensors, open_labels
