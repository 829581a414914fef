"""Sycamore-style random circuits (the circuit model of the paper's
"Simulation of the Sycamore circuits" section), generated from a seed.

The paper names the single-qubit gate set {sqrt(X), sqrt(Y), sqrt(W)}, fSim
two-qubit gates and the coupler sequence ABCDCDAB, but gives neither the gate
matrices nor the coupler patterns for a generic grid.  The readings used here:

* sqrt(X) = (1/sqrt2)[[1,-i],[-i,1]], sqrt(Y) = (1/sqrt2)[[1,-1],[1,1]],
  sqrt(W) = (1/sqrt2)[[1,-sqrt(i)],[sqrt(-i),1]] with W = (X+Y)/sqrt2.
* fSim(theta, phi) = [[1,0,0,0],[0,cos t,-i sin t,0],[0,-i sin t,cos t,0],
  [0,0,0,exp(-i phi)]] on the basis index 2*b(q0) + b(q1), q0 = first qubit
  of the coupler; theta = pi/2, phi = pi/6 throughout.
* Each cycle is a single-qubit layer, then one coupler pattern of fSim gates;
  cycle t uses pattern "ABCDCDAB"[t mod 8]; a last single-qubit layer follows
  the final cycle; the initial state is |0...0>.
* Single-qubit gates are drawn uniformly from the three, excluding the gate the
  same qubit had in the previous layer (first layer: uniform over three).
* Rectangular R x C grid, qubit q = r*C + c: A = horizontal (r,c)-(r,c+1) with
  c even, B = horizontal with c odd, C = vertical (r,c)-(r+1,c) with r even,
  D = vertical with r odd.
* Rotated lattice (rows x cols sites, some removed; odd rows sit half a site to
  the right): site (r,c) couples down-right to (r+1,c) for even r and to
  (r+1,c+1) for odd r, and down-left to (r+1,c-1) for even r and to (r+1,c)
  for odd r.  A / B = down-right couplers from even / odd rows, C / D =
  down-left couplers from even / odd rows, so A and B (and C and D) are the
  two parities of one coupler orientation, as A/B and C/D are on the
  rectangular grid, and each AB (CD) pair of layers sweeps a whole diagonal.
  Qubits are the kept sites numbered row-major.
* Bit order: qubit 0 is the most significant bit of a state-vector index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .rng import SplitMix64

PATTERN_SEQUENCE = "ABCDCDAB"
SINGLE_QUBIT_KINDS = ("sqrtX", "sqrtY", "sqrtW")
FSIM_THETA = math.pi / 2
FSIM_PHI = math.pi / 6


def gate_matrix(kind: str, params: Tuple[float, ...] = ()) -> np.ndarray:
    """Complex128 matrix of a gate kind (row = output basis state)."""
    s = 1.0 / math.sqrt(2.0)
    if kind == "sqrtX":
        return s * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)
    if kind == "sqrtY":
        return s * np.array([[1, -1], [1, 1]], dtype=np.complex128)
    if kind == "sqrtW":
        sqrt_i = np.exp(1j * math.pi / 4)
        sqrt_mi = np.exp(-1j * math.pi / 4)
        return s * np.array([[1, -sqrt_i], [sqrt_mi, 1]], dtype=np.complex128)
    if kind == "fsim":
        theta, phi = params
        c, sn = math.cos(theta), math.sin(theta)
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0, 0] = 1
        m[1, 1] = c
        m[1, 2] = -1j * sn
        m[2, 1] = -1j * sn
        m[2, 2] = c
        m[3, 3] = np.exp(-1j * phi)
        return m
    raise ValueError(f"unknown gate kind {kind!r}")


@dataclass
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    matrix: np.ndarray  # (2^len(qubits), 2^len(qubits)) complex128
    params: Tuple[float, ...] = ()


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    name: str = ""
    sites: List[Tuple[int, int]] = field(default_factory=list)

    def n_two_qubit(self) -> int:
        return sum(1 for g in self.gates if len(g.qubits) == 2)


def rect_grid(rows: int, cols: int):
    """Sites and the four coupler patterns of a rows x cols rectangular grid."""
    sites = [(r, c) for r in range(rows) for c in range(cols)]
    idx = {s: i for i, s in enumerate(sites)}
    pats: Dict[str, List[Tuple[int, int]]] = {k: [] for k in "ABCD"}
    for r in range(rows):
        for c in range(cols - 1):
            pats["A" if c % 2 == 0 else "B"].append((idx[(r, c)], idx[(r, c + 1)]))
    for r in range(rows - 1):
        for c in range(cols):
            pats["C" if r % 2 == 0 else "D"].append((idx[(r, c)], idx[(r + 1, c)]))
    return sites, pats


def rotated_lattice(rows: int = 6, cols: int = 9, removed: Sequence[Tuple[int, int]] = ((0, 0),)):
    """Sites and coupler patterns of the rotated (Sycamore-like) lattice."""
    removed = set(tuple(x) for x in removed)
    sites = [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in removed]
    idx = {s: i for i, s in enumerate(sites)}
    pats: Dict[str, List[Tuple[int, int]]] = {k: [] for k in "ABCD"}
    for (r, c) in sites:
        even = r % 2 == 0
        down_right = (r + 1, c) if even else (r + 1, c + 1)
        down_left = (r + 1, c - 1) if even else (r + 1, c)
        if down_right in idx:
            pats["A" if even else "B"].append((idx[(r, c)], idx[down_right]))
        if down_left in idx:
            pats["C" if even else "D"].append((idx[(r, c)], idx[down_left]))
    return sites, pats


def coupler_patterns(layout: str, rows: int, cols: int, removed=((0, 0),)):
    if layout == "rect":
        return rect_grid(rows, cols)
    if layout == "rotated":
        return rotated_lattice(rows, cols, removed)
    raise ValueError(layout)


def _single_qubit_layer(rng: SplitMix64, n: int, prev: List[int]) -> List[int]:
    out = []
    for q in range(n):
        if prev[q] < 0:
            k = rng.below(3)
        else:
            others = [x for x in range(3) if x != prev[q]]
            k = others[rng.below(2)]
        out.append(k)
    return out


def sycamore_circuit(layout: str, rows: int, cols: int, cycles: int, seed: int,
                     removed=((0, 0),), theta: float = FSIM_THETA, phi: float = FSIM_PHI) -> Circuit:
    """Seeded Sycamore-style circuit: per cycle a 1q layer then an fSim pattern,
    plus a final 1q layer."""
    sites, pats = coupler_patterns(layout, rows, cols, removed)
    n = len(sites)
    rng = SplitMix64(seed)
    one_q = [gate_matrix(k) for k in SINGLE_QUBIT_KINDS]
    two_q = gate_matrix("fsim", (theta, phi))
    gates: List[Gate] = []
    prev = [-1] * n

    def add_layer():
        nonlocal prev
        ks = _single_qubit_layer(rng, n, prev)
        for q, k in enumerate(ks):
            gates.append(Gate(SINGLE_QUBIT_KINDS[k], (q,), one_q[k].copy()))
        prev = ks

    for t in range(cycles):
        add_layer()
        for (a, b) in pats[PATTERN_SEQUENCE[t % len(PATTERN_SEQUENCE)]]:
            gates.append(Gate("fsim", (a, b), two_q.copy(), (theta, phi)))
    add_layer()
    name = f"{layout}{rows}x{cols}_m{cycles}_s{seed}"
    return Circuit(n, gates, name, sites)


def random_bits(n: int, seed: int) -> List[int]:
    rng = SplitMix64(seed)
    return [rng.below(2) for _ in range(n)]
