"""Host-side parts of bench.py (no GPU): the whole-step roofline entry of
the bench line, computed from the host-compiled plan of the 30-qubit
workload's tree."""
import os
import sys

import pytest

from tn_inputs.configs import make_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    return tn


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_step_roofline_matches_the_estimate(tn, bench):
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sl, _ = tn.find_order(L, O, tn.search_opts(trials=32, n_sliced=8))
    e = tn.estimate_tree_ms(L, O, sl, tree, form="bf16x3", batch_log2=6)
    # a step of all 256 slices in blocks of 64: the prologue once, 4 blocks
    r = bench.step_roofline(tn, L, O, sl, tree, "bf16x3", 64, 256, 10.0)
    assert r["estimate_ms"] == pytest.approx(e.prologue_ms + 4 * e.block_ms, rel=1e-12)
    assert r["estimate_ms"] == pytest.approx(e.ms, rel=1e-12)
    assert r["frac"] == pytest.approx(r["estimate_ms"] / 10.0)
    # a step over part of the slices (the 20-cycle line's 64 of 2^17)
    part = bench.step_roofline(tn, L, O, sl, tree, "bf16x3", 64, 128, 10.0)
    assert part["estimate_ms"] == pytest.approx(e.prologue_ms + 2 * e.block_ms, rel=1e-12)


def test_step_roofline_never_raises(tn, bench):
    r = bench.step_roofline(tn, [[0, 1], [1, 2]], [0, 2], [], [(0, 0)], "bf16x3", 1, 1, 1.0)
    assert set(r) == {"error"}
