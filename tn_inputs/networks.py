"""Seeded random tensor networks and contraction trees (bond dimension 2), plus
the wire-segment naming convention for circuit networks.

Wire-segment convention: on qubit q the wire is cut into segments by the gates
acting on q; segment t (t = 0 .. g_q, g_q = gates on q) lies after the t-th
gate on q in circuit order (segment 0 carries the initial |0>, segment g_q is
the output leg).  Its integer label is offset_q + t with
offset_q = sum_{q' < q} (g_{q'} + 1).  Both the CUDA path's circuit builder and
the oracle name bonds this way, so a sliced or open label means the same wire
on both sides.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from .rng import SplitMix64


def segment_labels(circuit) -> Tuple[List[int], List[int]]:
    """Return (offset_q, gates_per_qubit) of the wire-segment convention."""
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


@dataclass
class RandomNetwork:
    """A tensor network: tensor i has labels[i] (axis 0 = most significant) and
    data[i] of shape (2,)*len(labels[i]), complex128."""
    labels: List[List[int]]
    data: List[np.ndarray]
    open_labels: List[int]
    n_labels: int


def random_network(seed: int, n_tensors: int, n_bonds: int, n_open: int,
                   max_rank: int = 8, scale_to_unit: bool = True) -> RandomNetwork:
    """Random connected network: a random spanning chain first, then extra
    bonds between random tensor pairs (repeats give multi-bonds), then open legs.
    Values are complex normal (variance 1/2 per real part), divided by
    2^(rank/4) so that contraction results stay of order one."""
    rng = SplitMix64(seed)
    labels: List[List[int]] = [[] for _ in range(n_tensors)]
    next_label = 0
    order = rng.permutation(n_tensors)
    for i in range(1, n_tensors):  # spanning tree keeps it connected
        a = order[i]
        b = order[rng.below(i)]
        if len(labels[a]) >= max_rank or len(labels[b]) >= max_rank:
            continue
        labels[a].append(next_label)
        labels[b].append(next_label)
        next_label += 1
    tries = 0
    while next_label < n_bonds and tries < 100 * (n_bonds + 1):
        tries += 1
        a, b = rng.below(n_tensors), rng.below(n_tensors)
        if a == b or len(labels[a]) >= max_rank or len(labels[b]) >= max_rank:
            continue
        labels[a].append(next_label)
        labels[b].append(next_label)
        next_label += 1
    open_labels = []
    tries = 0
    while len(open_labels) < n_open and tries < 1000:
        tries += 1
        a = rng.below(n_tensors)
        if len(labels[a]) >= max_rank:
            continue
        labels[a].append(next_label)
        open_labels.append(next_label)
        next_label += 1
    # shuffle each tensor's axis order
    for i in range(n_tensors):
        p = rng.permutation(len(labels[i]))
        labels[i] = [labels[i][j] for j in p]
    data = []
    for i in range(n_tensors):
        r = len(labels[i])
        size = 1 << r
        vals = np.empty(size, dtype=np.complex128)
        for j in range(size):
            x, y = rng.normal_pair()
            vals[j] = complex(x, y) * np.sqrt(0.5)
        if scale_to_unit:
            vals /= np.sqrt(2.0) ** (r / 2.0)
        data.append(vals.reshape((2,) * r) if r else vals.reshape(()))
    return RandomNetwork(labels, data, open_labels, next_label)


def random_tree(seed: int, n_tensors: int) -> List[Tuple[int, int]]:
    """Random full binary contraction tree in SSA form: leaves are 0..n-1 and
    step i creates node n+i from the listed pair."""
    rng = SplitMix64(seed)
    live = list(range(n_tensors))
    steps = []
    nid = n_tensors
    while len(live) > 1:
        i = rng.below(len(live))
        a = live.pop(i)
        j = rng.below(len(live))
        b = live.pop(j)
        steps.append((a, b))
        live.append(nid)
        nid += 1
    return steps
