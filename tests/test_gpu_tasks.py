"""GPU: small steps run as the tasks of one persistent launch.

The plan compiler gathers the tiny small steps (T and C of at most 2^17
elements) whose inputs are leaves or each other's outputs into one launch
that orders them by device-side completion counters ("Dynamic slicing" and
the appendix's computation details: every subtask runs the same sequence of
pairwise steps).  A task computes its items exactly as the one-thread-per-row
kernel does (k ascending, the same fused multiply-adds), so where the
per-step launches use that kernel or the tiled one (the same order), tasks
on (the default) and off (small_tasks -1) agree bit for bit in FP32.  A step
with a long K and few rows runs, as its own launch, on the K-split kernel,
which adds its K terms in another order (lanes, then a warp reduction); there
the two runs agree to FP32 rounding (1e-6).  Every run also meets the form's
bound against the FP64 oracle.
"""
import os

import numpy as np
import pytest

from tn_inputs import random_network, random_tree, SplitMix64
from tn_inputs.configs import make_config
from oracle import contract as oc

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-5


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
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_complex(t):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a[0::2] + 1j * a[1::2]


def load_golden(name):
    vals = []
    for line in open(os.path.join(HERE, "golden", name)):
        if line.startswith("#"):
            continue
        _, re_, im_ = line.split()
        vals.append(complex(float(re_), float(im_)))
    return np.array(vals)


def cfg2_inputs(tn):
    from paper_2103_03074_gb300.trees import make_trees
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    stored = make_trees.load("rect5x6", L, O)
    if stored is None:
        tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    else:
        tree, sliced, _ = stored
    return L, T, O, tree, sliced


def run(tn, L, T, O, sliced, tree, form, reps=1, **opts):
    import torch
    plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(**opts))
    desc = plan.describe()
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    for _ in range(reps):  # with use_graph: eager, then graph replay
        amp.zero_()
        plan.contract(0, 1 << len(sliced), amp)
    got = to_complex(amp)
    plan.close()
    return got, desc


def n_tasks(desc, phase=None):
    return sum(1 for l in desc.splitlines() if " tasks n=" in l and (phase is None or l.startswith(phase)))


@pytest.mark.parametrize("form", ["fp32", "fp16x3", "tf32x3"])
def test_tasks_match_per_step_launches(tn, form):
    """The 30-qubit workload on its stored tree, all 2^8 slices in one block:
    the tiny steps run as tasks; eager call and graph replay."""
    L, T, O, tree, sliced = cfg2_inputs(tn)
    ref = load_golden("cfg2_amplitudes.txt")
    on, d_on = run(tn, L, T, O, sliced, tree, form, reps=2, use_graph=1)
    off, d_off = run(tn, L, T, O, sliced, tree, form, reps=2, use_graph=1, small_tasks=-1)
    assert n_tasks(d_on) >= 1 and n_tasks(d_off) == 0
    print(f"{form}: {len(d_on.splitlines())} ops with tasks, {len(d_off.splitlines())} without; "
          f"vs oracle {rel(on, ref):.2e}")
    if form == "fp32":
        assert np.array_equal(on, off)
    else:
        assert rel(on, off) < 1e-6
    assert rel(on, ref) < TOL


@pytest.mark.parametrize("batch_log2", [0, 3])
def test_tasks_in_the_block_body(tn, batch_log2):
    """One or eight slices per block: the slice-dependent tiny steps (fed by
    the block's extracted leaves) form task launches inside the per-block
    body, replayed once per block."""
    L, T, O, tree, sliced = cfg2_inputs(tn)
    ref = load_golden("cfg2_amplitudes.txt")
    on, d_on = run(tn, L, T, O, sliced, tree, "fp32", reps=2, use_graph=1, batch_log2=batch_log2)
    off, _ = run(tn, L, T, O, sliced, tree, "fp32", reps=1, batch_log2=batch_log2, small_tasks=-1)
    assert n_tasks(d_on, "batch") >= 1
    # blocks of few slices run some long-K steps on the K-split kernel when
    # launched one by one (module docstring)
    assert rel(on, off) < 1e-6
    assert rel(on, ref) < TOL


@pytest.mark.parametrize("seed,bits", [(41, 0), (42, 6), (43, 9), (44, 0), (45, 8)])
def test_tasks_random_networks(tn, seed, bits):
    """Random networks and random trees (deep and uneven dependency chains,
    rank-0 and rank-1 intermediates), sliced: against the FP64 oracle's
    pairwise contraction summed over slices; small_tasks = bits bounds the
    size of a task (0 = the default 2^17 elements), so groups split where a
    larger step sits between them."""
    net = random_network(seed, n_tensors=16, n_bonds=30, n_open=4, max_rank=8)
    cnt = {}
    for l in net.labels:
        for x in l:
            cnt[x] = cnt.get(x, 0) + 1
    internal = sorted(x for x, c in cnt.items() if c == 2)
    rng = SplitMix64(seed)
    sliced = [internal[i] for i in rng.permutation(len(internal))[:3]]
    tree = random_tree(seed + 1, len(net.labels))
    ref = oc.sliced_sum(net.labels, net.data, net.open_labels, sliced)
    on, d_on = run(tn, net.labels, net.data, net.open_labels, sliced, tree, "fp32", small_tasks=bits, batch_log2=1)
    off, _ = run(tn, net.labels, net.data, net.open_labels, sliced, tree, "fp32", small_tasks=-1, batch_log2=1)
    assert n_tasks(d_on) >= 1
    assert rel(on, off) < 1e-6
    assert rel(on, ref) < TOL
