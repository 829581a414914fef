"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds input generation only: a counter-based random generator,
Sycamore-style circuit descriptions (gate kinds, qubits, matrices), random
bitstrings, random tensor networks and random contraction trees.  It contains
none of the contraction method's arithmetic, and it imports neither the CUDA
package nor the oracle.
"""
from .rng import SplitMix64
from .circuits import (
    Gate, Circuit, gate_matrix, rect_grid, rotated_lattice, coupler_patterns,
    sycamore_circuit, random_bits, PATTERN_SEQUENCE,
)
from .networks import RandomNetwork, random_network, random_tree, segment_labels
from .configs import CONFIGS, make_config

__all__ = [
    "SplitMix64", "Gate", "Circuit", "gate_matrix", "rect_grid", "rotated_lattice",
    "coupler_patterns", "sycamore_circuit", "random_bits", "PATTERN_SEQUENCE",
    "RandomNetwork", "random_network", "random_tree", "segment_labels",
    "CONFIGS", "make_config",
]
