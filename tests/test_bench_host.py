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


@pytest.mark.parametrize("name,cfg_idx", [("rect5x6", 2), ("syc53_m14", 4), ("syc53_m20", 5)])
def test_stored_trees_fit_their_networks(tn, name, cfg_idx):
    """The trees bench.py runs by default are stored (their search's float
    tie-breaks could differ on another CPU); each must be a full binary tree
    over its workload's network whose slices keep every intermediate under
    the workload's cap, with the statistics the search reported."""
    from paper_2103_03074_gb300.trees import make_trees
    cfg = make_config(cfg_idx)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, st = make_trees.load(name, L, O)
    assert len(tree) == len(L) - 1
    seen = sorted(x for p in tree for x in p)
    assert seen == list(range(2 * len(L) - 2))  # every leaf and step but the root used once
    assert not set(sliced) & set(O)
    if cfg.get("log2_cap"):
        assert st["log2_width"] <= cfg["log2_cap"]
    # re-slicing the stored tree to the same cap finds a slice set no larger
    if cfg.get("log2_cap"):
        sl2, st2 = tn.slice_tree(L, O, tree, log2_cap=cfg["log2_cap"])
        assert st2["log2_width"] <= cfg["log2_cap"]
    # another network (other fixed bits give the same labels; other open
    # qubits do not) is refused
    L2, _, O2 = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"][1:])
    assert make_trees.load(name, L2, O2) is None


def test_reference_arm_loads_no_product_code():
    """bench.py --impl reference times the CPU oracle and must not load the
    CUDA library (its slice set comes from the stored tree's JSON)."""
    import subprocess
    code = ("import sys; sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'rect3x4', '--steps', '1', "
            "'--warmup', '1']; import bench; bench.main(); "
            "maps = open('/proc/self/maps').read(); "
            "print('LOADED' if ('libtn.so' in maps or 'paper_2103_03074_gb300' in sys.modules) else 'CLEAN')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert lines[-1] == "CLEAN"
    import json
    line = json.loads(lines[-2])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "slices/s"


def test_profile_summary_arithmetic(bench):
    """The bench line's roofline entry from step-timing rows, against numbers
    worked out by hand: over 2 recorded steps, a tensor-core GEMM class (two
    launches per step of 2^40 complex MACs and 2^33 bytes, 2 ms each) and a
    small step (one launch per step, 2^32 bytes, 1 ms).  Peaks: HBM 8192 GB/s,
    bf16 2000 TFLOP/s, FP32 ALU from 2070 MHz."""
    pk = dict(hbm_gbs=8192.0, bf16_tflops=2000.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
              source="test")
    rows = [dict(kind="gemm", ms=8.0, launches=4, macs=2.0 ** 40, bytes=2.0 ** 33),
            dict(kind="small", ms=2.0, launches=2, macs=2.0 ** 26, bytes=2.0 ** 32)]
    roof, share = bench.summarise_profile(rows, "fp16x3", pk, steps=2)
    # the GEMM class dominates: 8 of 10 ms
    assert share == {"gemm": 0.8, "small": 0.2}
    assert roof["bound"] == "tensor" and roof["peak"] == 2000.0
    # 24 flops per complex MAC, 2^40 MACs per launch, 2 ms per launch
    achieved = 24.0 * 2.0 ** 40 / 2e-3 / 1e12
    assert abs(roof["achieved"] - achieved) < 1e-9 * achieved
    assert abs(roof["frac"] - achieved / 2000.0) < 1e-12
    assert roof["launches_per_step"] == 2.0 and roof["share_of_step"] == 0.8
    # per launch: tensor time 24 * 2^40 / 2e15 s = 13.19 ms > HBM time
    # 2^33 / 8.192e12 s = 1.05 ms, so the class's roofline time is 4 x 13.19 ms
    t_gemm = 24.0 * 2.0 ** 40 / 2e15 * 1e3
    assert abs(roof["roofline_time_frac"] - 4 * t_gemm / 8.0) < 1e-9
    # the small step: HBM 2^32 / 8.192e12 s = 0.524 ms against FP32 ALU
    # 8 * 2^26 / (152 * 128 * 2 * 2.07e9) s = 0.0068 ms
    t_small = 2.0 ** 32 / 8.192e12 * 1e3
    assert abs(roof["step_roofline_time_frac"] - (4 * t_gemm + 2 * t_small) / 10.0) < 1e-9


@pytest.mark.parametrize("form,flops_per_mac,peak_ratio", [("tf32x3", 24.0, 0.5), ("fp16x3_3m", 18.0, 1.0),
                                                           ("fp16s", 8.0, 1.0)])
def test_profile_summary_per_form(bench, form, flops_per_mac, peak_ratio):
    """The tensor-core class is priced per form: 24 tensor flops per complex
    MAC for the four-product hi/lo forms, 18 for Gauss's 3M product, 8 for
    the single-piece FP16S; TF32 against half the bf16 peak.  The FP32 form's
    GEMM class is priced against the derived FP32 ALU peak (8 flops per
    complex MAC)."""
    pk = dict(hbm_gbs=8192.0, bf16_tflops=2000.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
              source="test")
    rows = [dict(kind="gemm", ms=4.0, launches=2, macs=2.0 ** 38, bytes=2.0 ** 30)]
    roof, _ = bench.summarise_profile(rows, form, pk, steps=1)
    achieved = flops_per_mac * 2.0 ** 38 / 2e-3 / 1e12
    assert roof["bound"] == "tensor" and abs(roof["peak"] - 2000.0 * peak_ratio) < 1e-9
    assert abs(roof["achieved"] - achieved) < 1e-9 * achieved
    roof, _ = bench.summarise_profile(rows, "fp32", pk, steps=1)
    alu = 152 * 128 * 2 * 2.07e9 / 1e12
    assert roof["bound"] == "alu" and abs(roof["peak"] - alu) < 1e-9 * alu
    assert abs(roof["achieved"] - 8.0 * 2.0 ** 38 / 2e-3 / 1e12) < 1e-6
