"""The five workload recipes (seeded circuits, open sets, fixed bits, caps).

Open qubits: a contiguous block of the highest-numbered qubits (the last grid
rows), listed in increasing qubit order, which is also the amplitude tensor's
axis order (first listed = most significant bit).  Fixed bits: a seeded random
bitstring over all qubits (entries at open positions are ignored).
"""
from __future__ import annotations

from typing import Dict, List

from .circuits import sycamore_circuit, random_bits
from .rng import SplitMix64

CONFIGS: Dict[int, dict] = {
    1: dict(name="rect3x4_m8_allopen", layout="rect", rows=3, cols=4, cycles=8, seed=20210305,
            n_open=12, n_sliced=0, log2_cap=None, slice_subset=None),
    2: dict(name="rect5x6_m12_open8_sliced8", layout="rect", rows=5, cols=6, cycles=12, seed=20210306,
            n_open=8, n_sliced=8, log2_cap=None, slice_subset=None),
    4: dict(name="rotated6x9m1_m14_open16_cap30", layout="rotated", rows=6, cols=9, cycles=14,
            seed=20210308, n_open=16, n_sliced=None, log2_cap=30, slice_subset=1024),
    5: dict(name="rotated6x9m1_m20_open21_cap31", layout="rotated", rows=6, cols=9, cycles=20,
            seed=20210309, n_open=21, n_sliced=None, log2_cap=31, slice_subset=64),
}

BATCH_GRIDS = [(3, 6), (3, 7), (3, 8), (3, 9), (3, 10), (4, 4), (4, 5), (4, 6), (4, 7), (5, 5), (5, 6)]
BATCH_SEED = 20210307


def make_config(idx: int) -> dict:
    """Materialise recipe ``idx`` (1, 2, 4 or 5): circuit, open qubits, fixed bits."""
    cfg = dict(CONFIGS[idx])
    circ = sycamore_circuit(cfg["layout"], cfg["rows"], cfg["cols"], cfg["cycles"], cfg["seed"])
    n = circ.n_qubits
    cfg["circuit"] = circ
    cfg["open_qubits"] = list(range(n - cfg["n_open"], n))
    cfg["fixed_bits"] = random_bits(n, cfg["seed"] ^ 0x5A5A5A5A)
    return cfg


def batch_recipes(n_circuits: int = 256, seed: int = BATCH_SEED) -> List[dict]:
    """Recipes of the batched workload: uneven rectangular grids of 16-30 qubits,
    8-14 cycles, 6-10 open qubits and 2^0-2^6 slices each."""
    rng = SplitMix64(seed)
    out = []
    for i in range(n_circuits):
        rows, cols = BATCH_GRIDS[rng.below(len(BATCH_GRIDS))]
        cycles = 8 + rng.below(7)
        n_open = 6 + rng.below(5)
        log2_slices = rng.below(7)
        cseed = seed * 1000 + i
        out.append(dict(layout="rect", rows=rows, cols=cols, cycles=cycles, seed=cseed,
                        n_open=n_open, n_sliced=log2_slices))
    return out


def make_batch_member(recipe: dict) -> dict:
    cfg = dict(recipe)
    circ = sycamore_circuit("rect", cfg["rows"], cfg["cols"], cfg["cycles"], cfg["seed"])
    n = circ.n_qubits
    cfg["circuit"] = circ
    cfg["open_qubits"] = list(range(n - cfg["n_open"], n))
    cfg["fixed_bits"] = random_bits(n, cfg["seed"] ^ 0x5A5A5A5A)
    return cfg
