"""GPU parity of the two-stage big-head contraction (tn_head_tail_amplitudes,
with trees from tn_find_order_head_tail) against the FP64 oracle.

Stage 1 contracts the head (closed qubits) into v_head over the first cut,
summed over the head's slices; stage 2 contracts the tail with v_head into
all open amplitudes.  The result is the same amplitude tensor as the
single-tree contraction: relative L2 <= 1e-5 for the complex64 forms.
"""
import os
import time

import numpy as np
import pytest

from tn_inputs import sycamore_circuit, random_bits
from tn_inputs.configs import make_config
from oracle import statevector as osv

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def to_complex(t):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a[0::2] + 1j * a[1::2]


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "fp16x3"])
def test_head_tail_matches_statevector(tn, form):
    import torch
    circ = sycamore_circuit("rect", 4, 5, 10, 77)
    fixed, open_q = random_bits(20, 77), list(range(15, 20))
    L, T, O = tn.circuit_network(circ, fixed, open_q)
    tree, sl_head, st = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=64, n_sliced=2))
    ref = osv.amplitudes(circ, fixed, open_q)
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    n_cut = tn.head_tail_amplitudes(L, T, O, tree, sl_head, [], amp, form=form)
    assert n_cut == st["n_cut"]
    assert rel(to_complex(amp), ref) < TOL
    # stage 2 sliced over two cut bonds: the same amplitudes
    head_labels = set()
    n = len(L)

    def leaves(x):
        return [x] if x < n else leaves(tree[x - n][0]) + leaves(tree[x - n][1])
    sides = [set(x for i in leaves(r) for x in L[i]) for r in tree[-1]]
    cut = sorted(sides[0] & sides[1])
    amp2 = torch.zeros_like(amp)
    tn.head_tail_amplitudes(L, T, O, tree, sl_head, cut[:2], amp2, form=form)
    assert rel(to_complex(amp2), ref) < TOL


def test_head_tail_on_the_30_qubit_workload(tn):
    """The 30-qubit workload: head sliced over 8 bonds, against the stored
    FP64 oracle amplitudes; the v_head output has the cut's size."""
    import torch
    cfg = make_config(2)
    ref = np.array([complex(float(l.split()[1]), float(l.split()[2]))
                    for l in open(os.path.join(HERE, "golden", "cfg2_amplitudes.txt")) if not l.startswith("#")])
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sl_head, st = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=1024, n_sliced=8))
    vhead = torch.zeros(2 << int(st["n_cut"]), dtype=torch.float64, device="cuda")
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    opts = tn.plan_opts(use_graph=1)
    tn.head_tail_amplitudes(L, T, O, tree, sl_head, [], amp, form="tf32x3", opts=opts, d_vhead=vhead)
    assert rel(to_complex(amp), ref) < TOL
    assert np.linalg.norm(to_complex(vhead)) > 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        tn.head_tail_amplitudes(L, T, O, tree, sl_head, [], amp, form="tf32x3", opts=opts)
    dt = (time.perf_counter() - t0) / 3
    print(f"head/tail on the 30-qubit workload: cut {int(st['n_cut'])} bonds, head 2^{st['log2_head_slice']:.1f} "
          f"MACs x 2^{int(st['n_sliced_head'])} slices, tail 2^{st['log2_tail']:.1f} MACs, total "
          f"2^{st['log2_total']:.1f}; {dt * 1e3:.1f} ms per call including plan builds")


def test_head_tail_rejects_a_tree_without_the_cut(tn):
    import torch
    circ = sycamore_circuit("rect", 3, 4, 6, 5)
    L, T, O = tn.circuit_network(circ, random_bits(12, 5), list(range(8, 12)))
    tree, _, _ = tn.find_order(L, O, tn.search_opts(trials=16, n_sliced=0))
    n = len(L)

    def leaves(x):
        return [x] if x < n else leaves(tree[x - n][0]) + leaves(tree[x - n][1])
    opens = [len(set(x for i in leaves(r) for x in L[i]) & set(O)) for r in tree[-1]]
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    if min(opens) > 0:
        with pytest.raises(tn.TNError):
            tn.head_tail_amplitudes(L, T, O, tree, [], [], amp)
    else:
        tn.head_tail_amplitudes(L, T, O, tree, [], [], amp)
        ref = osv.amplitudes(circ, random_bits(12, 5), list(range(8, 12)))
        assert rel(to_complex(amp), ref) < TOL
