"""GPU parity: the CUDA path (through the C-ABI) against the CPU FP64 oracle.

Tolerance: relative L2 error <= 1e-5 for the complex64 forms (the bound the
workload states for FP32 and split-precision forms: FP32, TF32x3 and FP16X3
keep 22+ significant bits per operand); XEB within 1e-4 absolute.  FP16S is
held to the 2e-3 bound stated for the scaled-FP16 form.  BF16x3 is NOT held
to 1e-5 and its checks here are not parity claims at that bound: two bf16
pieces keep 16 significant bits, so a single GEMM step already carries a
relative error near 2^-16 (1.5e-5), and over a tree the steps' errors add
(8.8e-6 to 2.0e-5 measured on the 30- and 53-qubit workloads).  It is
checked against BF16X3_BOUND = 1e-4 (2^-16 times a margin of ~6.5 for the
steps along the tree) so that a broken BF16x3 kernel (a dropped or misplaced
product term is off by ~4e-3) still fails.
Expected values come from oracle/ or from stored oracle output
(tests/golden/, written by tests/golden/make_golden.py).
"""
import os

import numpy as np
import pytest

from tn_inputs import random_network, random_tree, sycamore_circuit, random_bits, segment_labels, SplitMix64
from tn_inputs.configs import make_config
from oracle import contract as oc, network as onet, statevector as osv, xeb as oxeb

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-5
BF16X3_BOUND = 1e-4
BOUND = {"bf16x3": BF16X3_BOUND, "fp16s": 2e-3}


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


def dev_zeros(k):
    import torch
    return torch.zeros(2 << k, dtype=torch.float64, device="cuda:0")


def to_complex(t):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a[0::2] + 1j * a[1::2]


def internal_labels(labels):
    cnt = {}
    for l in labels:
        for x in l:
            cnt[x] = cnt.get(x, 0) + 1
    return sorted(x for x, c in cnt.items() if c == 2)


def pick(seed, items, k):
    rng = SplitMix64(seed)
    p = rng.permutation(len(items))
    return [items[i] for i in p[:k]]


@pytest.mark.parametrize("seed,batch_log2,tree_kind", [
    (1, 0, "random"), (2, 2, "random"), (3, 4, "search"), (4, -1, "search"), (5, 1, "random")])
def test_random_network_sliced(tn, seed, batch_log2, tree_kind):
    net = random_network(seed, n_tensors=12, n_bonds=22, n_open=3, max_rank=7)
    sliced = pick(seed + 7, internal_labels(net.labels), 4)
    if tree_kind == "random":
        tree = random_tree(seed + 11, len(net.labels))
    else:
        tree, _, _ = tn.find_order(net.labels, net.open_labels, tn.search_opts(trials=16, n_sliced=0))
    plan = tn.Plan(net.labels, net.data, net.open_labels, sliced, tree,
                   opts=tn.plan_opts(batch_log2=batch_log2))
    k = len(net.open_labels)
    full = dev_zeros(k)
    plan.contract(0, 16, full)
    ref = oc.sliced_sum(net.labels, net.data, net.open_labels, sliced)
    assert rel(to_complex(full), ref) < TOL
    # ragged range and single slices
    part = dev_zeros(k)
    plan.contract(3, 11, part)
    assert rel(to_complex(part), oc.sliced_sum(net.labels, net.data, net.open_labels, sliced, 3, 11)) < TOL
    for s in (0, 5, 15):
        one = dev_zeros(k)
        plan.contract(s, s + 1, one)
        assert rel(to_complex(one), oc.slice_partial(net.labels, net.data, net.open_labels, sliced, s)) < TOL
    plan.close()


@pytest.mark.parametrize("seed", [21, 22])
def test_gemm_path_large_operands(tn, seed):
    # ranks large enough that both operands of late steps exceed the small-step
    # limit, so the strided batched GEMM (and permutes) run
    net = random_network(seed, n_tensors=16, n_bonds=44, n_open=4, max_rank=10)
    tree, _, st = tn.find_order(net.labels, net.open_labels, tn.search_opts(trials=8, n_sliced=0))
    sliced = pick(seed, internal_labels(net.labels), 3)
    for bl in (0, 3):
        plan = tn.Plan(net.labels, net.data, net.open_labels, sliced, tree, opts=tn.plan_opts(batch_log2=bl))
        amp = dev_zeros(4)
        plan.contract(0, 8, amp)
        ref = oc.contract(net.labels, net.data, net.open_labels)
        assert rel(to_complex(amp), ref) < TOL
        plan.close()


def test_range_composition_and_empty(tn):
    net = random_network(9, n_tensors=10, n_bonds=18, n_open=2, max_rank=7)
    sliced = pick(3, internal_labels(net.labels), 5)
    tree = random_tree(4, len(net.labels))
    plan = tn.Plan(net.labels, net.data, net.open_labels, sliced, tree, opts=tn.plan_opts(batch_log2=2))
    a = dev_zeros(2)
    plan.contract(0, 13, a)
    plan.contract(13, 32, a)
    plan.contract(7, 7, a)  # empty: adds nothing
    b = dev_zeros(2)
    plan.contract(0, 32, b)
    assert rel(to_complex(a), to_complex(b)) < 1e-6
    assert rel(to_complex(b), oc.contract(net.labels, net.data, net.open_labels)) < TOL
    with pytest.raises(tn.TNError):
        plan.contract(0, 33, a)
    with pytest.raises(tn.TNError):
        plan.contract(5, 4, a)
    plan.close()


@pytest.mark.parametrize("n_sliced", [0, 3])
def test_cfg1_amplitudes(tn, n_sliced):
    cfg = make_config(1)
    amp = dev_zeros(12)
    tn.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"], amp,
                  search=tn.search_opts(trials=64, n_sliced=n_sliced))
    ref = osv.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    assert rel(to_complex(amp), ref) < TOL


def test_partial_open_circuit_per_slice(tn):
    # 20 qubits, 10 cycles, 6 open; 4 sliced bonds picked by the test from the
    # circuit's own wire segments; each slice against the oracle's own network
    circ = sycamore_circuit("rect", 4, 5, 10, 31)
    bits = random_bits(20, 32)
    open_q = [14, 15, 16, 17, 18, 19]
    offs, count = segment_labels(circ)
    seg = [0] * 20
    after2 = {q: [] for q in range(20)}
    for g in circ.gates:
        for q in g.qubits:
            seg[q] += 1
        if len(g.qubits) == 2:
            for q in g.qubits:
                after2[q].append(offs[q] + seg[q])
    bonds = sorted(x for q in range(20) for x in after2[q][:-1])
    sliced = pick(77, bonds, 4)
    L, T, O = tn.circuit_network(circ, bits, open_q)
    assert set(sliced) <= set(internal_labels(L))
    tree, _, _ = tn.find_order(L, O, tn.search_opts(trials=64, n_sliced=0))
    plan = tn.Plan(L, T, O, sliced, tree, opts=tn.plan_opts(batch_log2=2))
    oL, oT, oO = onet.circuit_network(circ, bits, open_q)
    for s in (0, 9, 15):
        one = dev_zeros(6)
        plan.contract(s, s + 1, one)
        ref = oc.slice_partial(oL, oT, oO, sliced, s)
        assert rel(to_complex(one), ref) < TOL
    full = dev_zeros(6)
    plan.contract(0, 16, full)
    assert rel(to_complex(full), osv.amplitudes(circ, bits, open_q)) < TOL
    plan.close()


def load_golden(name):
    path = os.path.join(HERE, "golden", name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    vals = []
    for line in open(path):
        if line.startswith("#"):
            continue
        i, re_, im_ = line.split()
        vals.append(complex(float(re_), float(im_)))
    return np.array(vals)


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "fp16x3", "bf16x3", "fp16s"])
def test_cfg2_amplitudes_vs_golden(tn, form):
    """The 30-qubit workload exactly as the benchmark plans it: 8 sliced bonds
    from the order search (16384 trials), all 2^8 slices in one batch."""
    cfg = make_config(2)
    ref = load_golden("cfg2_amplitudes.txt")
    amp = dev_zeros(8)
    tn.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"], amp, form=form,
                  search=tn.search_opts(trials=16384, n_sliced=8))
    got = to_complex(amp)
    print(f"cfg2 {form}: relative L2 error {rel(got, ref):.3e}")
    # FP32, TF32x3 and FP16X3 meet the 1e-5 bound; BF16x3 and FP16S get
    # their forms' own bounds (module docstring)
    bound = BOUND.get(form, TOL)
    assert rel(got, ref) < bound
    # XEB from the GPU probabilities against the oracle's, 1e-4 absolute; the
    # marginal sum |a|^2 moves by at most (2 e + e^2) of itself when the
    # amplitudes move by a relative L2 error e
    p_s1, f, pmax = tn.probabilities_xeb(amp, 8, 30)
    if form != "fp16s":
        assert abs(f - oxeb.linear_xeb(ref, 30)) < 1e-4
        assert abs(p_s1 - oxeb.marginal(ref)) < (2 * bound + bound ** 2) * oxeb.marginal(ref)


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "fp16x3"])
def test_tiled_small_steps_match_row_kernel(tn, form):
    """Small steps on the tiled kernel (the default) against the
    one-thread-per-row kernel (small_tiled -1): both sum over k in ascending
    order with the same fused multiply-adds, so the amplitudes agree bit for
    bit; both meet the form's bound against the FP64 golden amplitudes."""
    import torch
    cfg = make_config(2)
    ref = load_golden("cfg2_amplitudes.txt")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    got = {}
    for tiled in (0, -1):
        plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(small_tiled=tiled, use_graph=1))
        amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
        for _ in range(2):  # eager, then graph replay
            amp.zero_()
            plan.contract(0, 1 << len(sliced), amp)
        torch.cuda.synchronize()
        got[tiled] = to_complex(amp)
        plan.close()
    assert np.array_equal(got[0], got[-1])
    bound = BOUND.get(form, TOL)
    assert rel(got[0], ref) < bound


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_tiled_small_steps_random_layouts(tn, seed):
    """Circuits on uneven grids with open qubits spread over the lattice put
    the K and N labels of the small steps at varied bit positions (low,
    high, interleaved with the row bits); tiled and row kernels agree bit for
    bit, and both match the FP64 state vector."""
    import torch
    rows, cols = [(4, 5), (3, 7), (5, 4)][seed - 31]
    circ = sycamore_circuit("rect", rows, cols, 10, seed)
    n = circ.n_qubits
    open_q = sorted(pick(seed, list(range(n)), 6))
    fixed = random_bits(n, seed)
    L, T, O = tn.circuit_network(circ, fixed, open_q)
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=64, seed=seed, n_sliced=4))
    got = {}
    for tiled in (0, -1):
        plan = tn.Plan(L, T, O, sliced, tree, form="fp32", opts=tn.plan_opts(small_tiled=tiled))
        amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
        plan.contract(0, 1 << len(sliced), amp)
        torch.cuda.synchronize()
        got[tiled] = to_complex(amp)
        plan.close()
    assert np.array_equal(got[0], got[-1])
    ref = osv.amplitudes(circ, fixed, open_q)
    assert rel(got[0], ref) < TOL


@pytest.mark.parametrize("form", ["tf32x3", "bf16x3", "fp16x3", "fp16s"])
def test_planar_epilogue_matches_split_pass(tn, form):
    """GEMMs that write the next step's hi/lo planes from their epilogue
    (tc_planar on, the default) against complex64 output plus a separate
    split pass (tc_planar -1).  BF16x3 / TF32x3: the same pieces and
    products, so they agree to FP32 rounding of the split-K atomics elsewhere
    in the plan (1e-6).  Both meet the form's bound against the FP64 golden
    amplitudes."""
    import torch
    cfg = make_config(2)
    ref = load_golden("cfg2_amplitudes.txt")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    got = {}
    for planar in (0, -1):
        plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(tc_planar=planar))
        amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
        plan.contract(0, 1 << len(sliced), amp)
        torch.cuda.synchronize()
        got[planar] = to_complex(amp)
        plan.close()
    # the scaled forms' planar outputs take their exponent from a bound
    # (eA + eB + 15 + log2 K) instead of the output's max, which moves the
    # fp16 pieces' rounding: the two runs then agree to the forms' own
    # accuracy rather than to 1e-6
    agree = {"fp16x3": 5e-6, "fp16s": 2e-3}.get(form, 1e-6)
    print(f"planar vs split pass, {form}: {rel(got[0], got[-1]):.2e}; vs oracle {rel(got[0], ref):.2e} / "
          f"{rel(got[-1], ref):.2e}")
    assert rel(got[0], got[-1]) < agree
    bound = BOUND.get(form, TOL)
    assert rel(got[0], ref) < bound and rel(got[-1], ref) < bound


def test_sharded_contract_single_rank(tn):
    """The multi-rank helper at world size 1: the rank's range is every slice
    and the host sum is the identity, so it reproduces the golden amplitudes."""
    import torch
    from paper_2103_03074_gb300.shard import sharded_contract
    cfg = make_config(2)
    ref = load_golden("cfg2_amplitudes.txt")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    plan = tn.Plan(L, T, O, sliced, tree, form="fp32")
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    got = sharded_contract(plan, amp, 0, 1)
    plan.close()
    assert rel(got.reshape(-1), ref) < TOL


def _prologue_feeds_block_network():
    """A slice-invariant tensor-core GEMM (X Y, in the prologue) feeding a
    slice-dependent one (Z W, W holds the sliced label s): in the scaled forms
    Z's scale comes from the prologue GEMM's epilogue and W's from a max-abs
    pass inside each block, into one pair of slots."""
    m, k, n = list(range(0, 8)), list(range(10, 15)), list(range(20, 28))
    o, s = list(range(30, 38)), 40
    labels = [m + k, k + n, m[:5] + [s] + o, [s] + o + m[5:] + n[3:]]
    rng = np.random.default_rng(20210308)
    data = [(rng.standard_normal((2,) * len(l)) + 1j * rng.standard_normal((2,) * len(l))).astype(np.complex64)
            * np.float32(2.0 ** (-len(l) / 4)) for l in labels]
    return labels, data, n[:3], [s], [(0, 1), (4, 2), (5, 3)]


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "fp16x3", "bf16x3", "fp16s"])
def test_prologue_gemm_feeds_every_block(tn, form):
    """Two blocks of one slice each (batch_log2 0): values and scales the
    prologue writes once must survive both blocks."""
    labels, data, open_l, sliced, tree = _prologue_feeds_block_network()
    ref = oc.sliced_sum(labels, data, open_l, sliced)
    for use_graph in (0, 1):
        plan = tn.Plan(labels, data, open_l, sliced, tree, form=form,
                       opts=tn.plan_opts(batch_log2=0, use_graph=use_graph))
        for rep in range(2):
            amp = dev_zeros(len(open_l))
            plan.contract(0, 2, amp)
            assert rel(to_complex(amp), ref) < BOUND.get(form, TOL), (use_graph, rep)
        plan.close()


def test_probabilities_xeb_on_oracle_amplitudes(tn):
    import torch
    cfg = make_config(1)
    ref = osv.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"][:8])
    inter = np.stack([ref.real, ref.imag], axis=1).reshape(-1)
    d = torch.tensor(inter, dtype=torch.float64, device="cuda:0")
    prob = torch.zeros(256, dtype=torch.float64, device="cuda:0")
    p_s1, f, pmax = tn.probabilities_xeb(d, 8, 12, d_prob=prob)
    p = oxeb.probabilities(ref)
    assert np.abs(prob.cpu().numpy() - p).max() < 1e-15
    assert abs(p_s1 - p.sum()) < 1e-14
    assert abs(f - oxeb.linear_xeb(ref, 12)) < 1e-12
    assert abs(pmax - p.max()) < 1e-18


@pytest.mark.parametrize("form", ["fp32", "tf32x3"])
def test_graph_replay_matches_oracle(tn, form):
    """use_graph: the first call runs eagerly and captures the prologue and the
    per-block body; later calls replay the graphs.  Full and ragged ranges,
    several blocks per call."""
    net = random_network(31, n_tensors=16, n_bonds=40, n_open=3, max_rank=10)
    sliced = pick(5, internal_labels(net.labels), 4)
    tree, _, _ = tn.find_order(net.labels, net.open_labels, tn.search_opts(trials=8, n_sliced=0))
    plan = tn.Plan(net.labels, net.data, net.open_labels, sliced, tree, form=form,
                   opts=tn.plan_opts(batch_log2=2, use_graph=1))
    ref = oc.sliced_sum(net.labels, net.data, net.open_labels, sliced)
    for rep in range(3):
        amp = dev_zeros(3)
        plan.contract(0, 16, amp)
        assert rel(to_complex(amp), ref) < TOL, rep
    part = dev_zeros(3)
    plan.contract(3, 13, part)
    assert rel(to_complex(part), oc.sliced_sum(net.labels, net.data, net.open_labels, sliced, 3, 13)) < TOL
    assert plan.stats()["graph_replays"] >= 3
    plan.close()


@pytest.mark.parametrize("form", ["tf32x3", "fp16x3", "bf16x3"])
def test_cfg2_amplitudes_3m(tn, form):
    """The 30-qubit workload with Gauss's 3M complex product on the tensor
    cores (tc_products 3): against the FP64 golden amplitudes at the form's
    bound (1e-5 for TF32x3 and FP16X3; BF16x3 its own), with the GEMMs
    writing the next step's six planes from their epilogue and, separately,
    through split passes (tc_planar -1): the two runs agree to the forms' own
    accuracy."""
    import torch
    cfg = make_config(2)
    ref = load_golden("cfg2_amplitudes.txt")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = tn.find_order(L, O, tn.search_opts(trials=16384, n_sliced=8))
    got = {}
    for planar in (0, -1):
        plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(tc_planar=planar, tc_products=3,
                                                                            use_graph=1))
        desc = plan.describe()
        assert "tensor-core 3M" in desc and "tensor-core ksplit" not in desc
        amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
        for _ in range(2):  # eager, then graph replay
            amp.zero_()
            plan.contract(0, 1 << len(sliced), amp)
        got[planar] = to_complex(amp)
        plan.close()
    bound = BOUND.get(form, TOL)
    print(f"cfg2 3M {form}: relative L2 error {rel(got[0], ref):.3e} (split passes: {rel(got[-1], ref):.3e})")
    assert rel(got[0], ref) < bound and rel(got[-1], ref) < bound
    assert rel(got[0], got[-1]) < {"fp16x3": 5e-6, "bf16x3": 2e-5}.get(form, 2e-6)


@pytest.mark.parametrize("n_new,form", [(4, "fp32"), (4, "fp16x3"), (5, "fp32"), (5, "fp16x3")])
def test_intermediate_beyond_2_32_elements(tn, n_new, form):
    """Offsets past 32 bits: the explicit tree's first step is the outer
    product of A (17 labels) and B (16 labels), a 2^33-element intermediate
    in layout [a][b] whose a labels sit at bit positions 16..32.  The second
    step contracts 8 of those a labels with W: a small step (W of 12 labels,
    n_new = 4: its K bits at positions up to 32 of T) or a GEMM (W of 13
    labels, n_new = 5: the intermediate is first permuted / split into the
    GEMM's layout, a rank-33 bit permutation).  Vectors then close every
    label but four.  The FP64 oracle contracts the same network in its own
    order (the vectors first), so its intermediates stay small.  Bound: 1e-5
    (plain sums of a few hundred products per output)."""
    import torch
    rng = np.random.default_rng(33 + n_new)

    def rnd(rank):
        return ((rng.standard_normal((2,) * rank) + 1j * rng.standard_normal((2,) * rank)) /
                np.sqrt(2.0 ** rank)).astype(np.complex64)
    a = list(range(100, 117))
    b = list(range(200, 216))
    w = list(range(300, 300 + n_new))
    labels = [a, b, a[:8] + w]
    tensors = [rnd(17), rnd(16), rnd(8 + n_new)]
    open_l = [w[0], w[1], b[0], b[1]]
    closed = a[8:] + b[2:] + w[2:]
    for lab in closed:
        labels.append([lab])
        tensors.append(rnd(1) * np.float32(np.sqrt(2.0)))
    n = len(labels)
    tree = [(0, 1), (n, 2)]  # A x B (2^33 elements), then with W
    cur = n + 1
    for j in range(3, n):
        tree.append((cur, j))
        cur += 1
    ref = oc.contract(labels, tensors, open_l)
    plan = tn.Plan(labels, tensors, open_l, [], tree, form=form)
    desc = plan.describe()
    amp = dev_zeros(len(open_l))
    plan.contract(0, 1, amp)
    got = to_complex(amp)
    plan.close()
    torch.cuda.empty_cache()
    print(f"2^33-element intermediate, {form}, W with {8 + n_new} labels: relative L2 error {rel(got, ref):.2e}")
    # the steps this test is for: a small step reading the 2^33-element T with
    # K bits up to position 32, or (FP16X3) a rank-33 split pass before the GEMM
    if n_new == 4:
        assert "step 1 small rows=33554432 K=256" in desc
    elif form == "fp16x3":
        assert "step 1 split rank=33" in desc
    assert rel(got, ref.reshape(-1)) < TOL
