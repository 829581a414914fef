"""Batched execution of many independent circuits (tn_batch_*) and the GEMM
autotuner (tn_plan_autotune), against the CPU FP64 oracle.

The batch follows the batched workload's recipe (tn_inputs.configs.batch_recipes:
uneven rectangular grids, 8-14 cycles, 6-10 open qubits, 2^0-2^6 slices each),
restricted to circuits of at most 24 qubits so that every circuit is checked
against its own FP64 state vector (plain C oracle) within 1e-5.  The full
recipe (256 circuits of 16-30 qubits) checks every member against the same
plan run alone, those of at most 20 qubits against a live FP64 state vector,
and the larger ones whose FP64 state-vector amplitudes are stored
(tests/golden/cfg3_amplitudes.txt: every member of up to 28 qubits and a
seeded sample of the 30-qubit ones) against those, all within 1e-5.
"""
import os

import numpy as np
import pytest

from tn_inputs.configs import batch_recipes, make_batch_member, make_config
from oracle import sv_native

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def tn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    return tn


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stored_member_amplitudes():
    """{member index: FP64 amplitudes} from tests/golden/cfg3_amplitudes.txt
    (the FP64 state vectors of the batch members of more than 20 qubits that
    tests/golden/make_golden.py has written; members appear whole)."""
    path = os.path.join(HERE, "golden", "cfg3_amplitudes.txt")
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        if line.startswith("#"):
            continue
        i, j, re_, im_ = line.split()
        out.setdefault(int(i), []).append((int(j), complex(float(re_), float(im_))))
    return {i: np.array([v for _, v in sorted(vals)]) for i, vals in out.items()}


def to_complex(t):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a[0::2] + 1j * a[1::2]


@pytest.mark.parametrize("form", ["fp32", "tf32x3"])
def test_batch_of_uneven_circuits(tn, form):
    import torch
    recipes = [r for r in batch_recipes() if r["rows"] * r["cols"] <= 24][:24]
    members = [make_batch_member(r) for r in recipes]
    plans, amps = [], []
    for m in members:
        L, T, O = tn.circuit_network(m["circuit"], m["fixed_bits"], m["open_qubits"])
        tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=64, n_sliced=m["n_sliced"]))
        assert len(sliced) == m["n_sliced"]
        plans.append(tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(batch_log2=2)))
        amps.append(torch.full((2 << len(O),), float("nan"), dtype=torch.float64, device="cuda"))
    batch = tn.Batch(plans, amps, n_streams=4)
    refs = [sv_native.amplitudes(m["circuit"], m["fixed_bits"], m["open_qubits"]) for m in members]
    for run in range(2):  # eager run, then graph replay (overwrites)
        batch.run()
        for i, (a, ref) in enumerate(zip(amps, refs)):
            assert rel(to_complex(a), ref) < 1e-5, (run, i, members[i]["rows"], members[i]["cols"])
    batch.close()
    for p in plans:
        p.close()


def test_autotune_keeps_results(tn):
    import torch
    cfg = make_config(2)
    path = os.path.join(HERE, "golden", "cfg2_amplitudes.txt")
    ref = np.array([complex(float(l.split()[1]), float(l.split()[2])) for l in open(path) if not l.startswith("#")])
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    plan = tn.Plan(L, T, O, sliced, tree, form="tf32x3", opts=tn.plan_opts(use_graph=1))
    amp = torch.zeros(2 << 8, dtype=torch.float64, device="cuda")
    plan.contract(0, 256, amp)
    plan.autotune(reps=2)
    for _ in range(2):  # eager (recapture) then replay with the tuned configuration
        amp.zero_()
        plan.contract(0, 256, amp)
        assert rel(to_complex(amp), ref) < 1e-5
    plan.close()


def test_full_batched_recipe(tn):
    """All 256 circuits of the batched workload (16-30 qubits) in one batch,
    TF32x3.  Circuits of at most 20 qubits against their FP64 state vectors,
    larger ones against their stored FP64 state-vector amplitudes where
    present; every circuit against its own plan contracted alone (eager
    path)."""
    import time
    import torch
    members = [make_batch_member(r) for r in batch_recipes()]
    plans, amps, n_slices = [], [], 0
    for m in members:
        L, T, O = tn.circuit_network(m["circuit"], m["fixed_bits"], m["open_qubits"])
        tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=32, n_sliced=m["n_sliced"]))
        plans.append(tn.Plan(L, T, O, sliced, tree, form="tf32x3", opts=tn.plan_opts(batch_log2=3)))
        amps.append(torch.zeros(2 << len(O), dtype=torch.float64, device="cuda"))
        n_slices += 1 << len(sliced)
    batch = tn.Batch(plans, amps, n_streams=8)
    batch.run()
    batch.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        batch.run()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    print(f"batched recipe: {len(members)} circuits, {n_slices} slices, {dt * 1e3:.2f} ms per batch, "
          f"{n_slices / dt:.0f} slices/s")
    stored = stored_member_amplitudes()
    checked = from_store = 0
    for mi, (m, p, a) in enumerate(zip(members, plans, amps)):
        got = to_complex(a)
        single = torch.zeros_like(a)
        p.contract(0, 1 << p.n_sliced, single)
        # same kernels and data; split-K GEMMs add FP32 partial tiles with
        # atomics in a launch-dependent order, so the two runs differ by
        # rounding noise (amplified where partial tiles cancel), far below
        # the form's 1e-5 bound, while any executor fault shows as O(1)
        assert rel(got, to_complex(single)) < 5e-6
        if m["circuit"].n_qubits <= 20:
            assert rel(got, sv_native.amplitudes(m["circuit"], m["fixed_bits"], m["open_qubits"])) < 1e-5
            checked += 1
        elif mi in stored:
            assert len(stored[mi]) == len(got)
            assert rel(got, stored[mi]) < 1e-5, (mi, m["circuit"].n_qubits)
            from_store += 1
    print(f"batched recipe: {checked} members against a live FP64 state vector, {from_store} against stored "
          f"FP64 state-vector amplitudes, all {len(members)} against the same plan run alone")
    assert checked >= 40
    assert from_store == sum(1 for i in stored if i < len(members))
    batch.close()
    for p in plans:
        p.close()
