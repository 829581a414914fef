"""Pins of the seeded inputs: gate matrices, coupler patterns, the generator.

The paper names the gate set and the ABCDCDAB sequence (Sycamore section);
the matrices and the patterns follow the readings stated in tn_inputs/circuits.
Each check below fails if a plausible mistake is made there (a sign, a swapped
off-diagonal, a wrong phase, a pattern that is not a matching).
"""
import math

import numpy as np
import pytest

from tn_inputs import SplitMix64, gate_matrix, rect_grid, rotated_lattice, sycamore_circuit
from tn_inputs.configs import make_config

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)


def test_splitmix64_reference_vector():
    # SplitMix64 with state 0: first outputs as published with the algorithm.
    r = SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_below_is_in_range_and_covers():
    r = SplitMix64(123)
    seen = [r.below(3) for _ in range(3000)]
    assert set(seen) == {0, 1, 2}
    counts = np.bincount(seen)
    assert np.all(np.abs(counts - 1000) < 150)


@pytest.mark.parametrize("kind", ["sqrtX", "sqrtY", "sqrtW"])
def test_single_qubit_unitary(kind):
    g = gate_matrix(kind)
    assert np.abs(g.conj().T @ g - np.eye(2)).max() < 1e-14


def test_square_roots_square_to_paulis():
    # With the stated matrices each square root squares to its Pauli times
    # the global phase -i: sqrtX^2 = -iX, sqrtY^2 = -iY, sqrtW^2 = -iW,
    # W = (X + Y)/sqrt2.  A sign or phase slip in any entry breaks this.
    W = (X + Y) / math.sqrt(2)
    for kind, P in (("sqrtX", X), ("sqrtY", Y), ("sqrtW", W)):
        g = gate_matrix(kind)
        assert np.abs(g @ g - (-1j) * P).max() < 1e-14, kind


def test_sqrt_x_closed_form_action():
    g = gate_matrix("sqrtX")
    v = g @ np.array([1, 0], dtype=complex)
    assert np.allclose(v, np.array([1, -1j]) / math.sqrt(2), atol=1e-15)


def test_fsim_unitary_and_closed_forms():
    g = gate_matrix("fsim", (math.pi / 2, math.pi / 6))
    assert np.abs(g.conj().T @ g - np.eye(4)).max() < 1e-14
    iswap_like = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    assert np.abs(gate_matrix("fsim", (math.pi / 2, 0.0)) - iswap_like).max() < 1e-15
    assert np.abs(gate_matrix("fsim", (0.0, 0.0)) - np.eye(4)).max() < 1e-15
    assert abs(g[3, 3] - np.exp(-1j * math.pi / 6)) < 1e-15


def _is_matching(pairs):
    qs = [q for p in pairs for q in p]
    return len(qs) == len(set(qs))


def test_rect_patterns_counts_and_matchings():
    for (r, c), expect in (((3, 4), (6, 3, 4, 4)), ((5, 6), (15, 10, 12, 12))):
        _, pats = rect_grid(r, c)
        assert tuple(len(pats[k]) for k in "ABCD") == expect
        assert all(_is_matching(pats[k]) for k in "ABCD")
        # every nearest-neighbour edge appears in exactly one pattern
        all_pairs = sorted(p for k in "ABCD" for p in pats[k])
        assert len(all_pairs) == len(set(all_pairs)) == r * (c - 1) + (r - 1) * c


def test_rotated_lattice_counts_and_orientation():
    sites, pats = rotated_lattice(6, 9, ((0, 0),))
    assert len(sites) == 53
    assert tuple(len(pats[k]) for k in "ABCD") == (26, 16, 24, 18)
    assert all(_is_matching(pats[k]) for k in "ABCD")
    # x position of a site: odd rows sit half a site to the right
    x = lambda s: s[1] + 0.5 * (s[0] % 2)
    for k, dx in (("A", 0.5), ("B", 0.5), ("C", -0.5), ("D", -0.5)):
        for a, b in pats[k]:
            assert sites[b][0] == sites[a][0] + 1          # adjacent rows
            assert x(sites[b]) - x(sites[a]) == dx, k      # one orientation per A/B and per C/D
    # every nearest-neighbour coupler of the lattice appears exactly once
    all_pairs = sorted(tuple(sorted(p)) for k in "ABCD" for p in pats[k])
    assert len(all_pairs) == len(set(all_pairs)) == 84


@pytest.mark.parametrize("idx,n2", [(1, 34), (2, 147), (4, 294), (5, 420)])
def test_config_gate_counts(idx, n2):
    cfg = make_config(idx)
    assert cfg["circuit"].n_two_qubit() == n2


def test_single_qubit_layers_never_repeat():
    circ = sycamore_circuit("rect", 3, 4, 8, 5)
    last = {}
    for g in circ.gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            assert last.get(q) != g.kind
            last[q] = g.kind
