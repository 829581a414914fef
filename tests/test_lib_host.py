"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
symbol include/tn.h declares, builds the circuit network the oracle agrees
with, finds valid orders, and rejects malformed input before touching CUDA."""
import os
import re

import numpy as np
import pytest

from tn_inputs import random_network, sycamore_circuit, random_bits
from tn_inputs.configs import make_config
from oracle import contract as oc, statevector as osv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    return tn


def test_exports_every_declared_symbol(tn):
    header = open(os.path.join(ROOT, "include", "tn.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char \*)\s*(tn_\w+)\s*\(", header, re.M))
    assert {"tn_plan_create", "tn_contract_slices", "tn_amplitudes", "tn_plan_destroy", "tn_last_error"} <= declared
    for name in declared:
        assert hasattr(tn._lib, name), name
    assert declared == set(tn.EXPORTED)


@pytest.mark.parametrize("cfg_idx", [1])
def test_circuit_network_matches_statevector(tn, cfg_idx):
    cfg = make_config(cfg_idx)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    got = oc.contract(L, [np.asarray(t, np.complex128) for t in T], O).reshape(-1)
    ref = osv.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    # complex64 leaves: error of order 1e-7 relative
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6


def test_circuit_network_partial_open_and_labels(tn):
    circ = sycamore_circuit("rect", 3, 3, 6, 4)
    bits = random_bits(9, 1)
    open_q = [7, 2, 5]
    L, T, O = tn.circuit_network(circ, bits, open_q)
    # every leaf is a two-qubit gate of rank <= 4; labels held at most twice
    assert all(len(l) <= 4 for l in L)
    cnt = {}
    for l in L:
        for x in l:
            cnt[x] = cnt.get(x, 0) + 1
    assert all(c in (1, 2) for c in cnt.values())
    assert {x for x, c in cnt.items() if c == 1} == set(O)
    # open labels are the final wire segments (wire-segment convention)
    from tn_inputs import segment_labels
    offs, count = segment_labels(circ)
    assert O == [offs[q] + count[q] for q in open_q]
    got = oc.contract(L, [np.asarray(t, np.complex128) for t in T], O).reshape(-1)
    ref = osv.amplitudes(circ, bits, open_q)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6


def test_find_order_valid_tree_and_slices(tn):
    net = random_network(5, n_tensors=14, n_bonds=22, n_open=3, max_rank=6)
    tree, sliced, st = tn.find_order(net.labels, net.open_labels, tn.search_opts(trials=32, n_sliced=3))
    n = len(net.labels)
    used = set()
    for t, (a, b) in enumerate(tree):
        assert 0 <= a < n + t and 0 <= b < n + t and a != b
        assert a not in used and b not in used
        used |= {a, b}
    assert len(tree) == n - 1
    assert len(sliced) == 3 and not set(sliced) & set(net.open_labels)
    # the result of the tree does not depend on it: oracle contraction with
    # this tree equals its own greedy contraction
    ref = oc.contract(net.labels, net.data, net.open_labels)
    got = oc.contract(net.labels, net.data, net.open_labels, tree=tree)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_find_order_cap_reduces_width(tn):
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    _, _, st0 = tn.find_order(L, O, tn.search_opts(trials=16, n_sliced=0))
    _, sl, st1 = tn.find_order(L, O, tn.search_opts(trials=16, log2_cap=int(st0["log2_width"]) - 4))
    # the capped search may also pick a narrower tree, so the number of
    # sliced labels is not fixed by the cap; the width bound and the count are
    assert st1["log2_width"] <= st0["log2_width"] - 4
    assert len(sl) == st1["n_sliced"] >= 1


def test_search_is_deterministic(tn):
    cfg = make_config(1)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    a = tn.find_order(L, O, tn.search_opts(trials=64, threads=1, n_sliced=2))
    b = tn.find_order(L, O, tn.search_opts(trials=64, threads=4, n_sliced=2))
    assert a[0] == b[0] and a[1] == b[1]


def _plan_args_error(tn, **kw):
    net = random_network(3, n_tensors=5, n_bonds=7, n_open=2, max_rank=5)
    labels = kw.get("labels", net.labels)
    open_l = kw.get("open", net.open_labels)
    sliced = kw.get("sliced", [])
    tree = kw.get("tree", [(0, 1), (5, 2), (6, 3), (7, 4)])
    with pytest.raises(tn.TNError) as ei:
        tn.Plan(labels, net.data, open_l, sliced, tree)
    return ei.value


def test_plan_rejects_sliced_open_label(tn):
    net = random_network(3, n_tensors=5, n_bonds=7, n_open=2, max_rank=5)
    err = _plan_args_error(tn, sliced=[net.open_labels[0]])
    assert err.code == -1 and "open" in str(err)


def test_plan_rejects_bad_tree(tn):
    err = _plan_args_error(tn, tree=[(0, 1), (0, 2), (6, 3), (7, 4)])
    assert err.code == -1
    err = _plan_args_error(tn, tree=[(0, 1)])
    assert err.code == -1


def test_plan_rejects_dangling_label(tn):
    net = random_network(3, n_tensors=5, n_bonds=7, n_open=2, max_rank=5)
    err = _plan_args_error(tn, open=net.open_labels[:1])
    assert err.code == -1


@pytest.mark.parametrize("method", ["greedy", "bipartition"])
def test_head_tail_order_has_the_cut_at_its_root(tn, method):
    """tn_find_order_head_tail: a valid SSA tree whose last step joins a side
    without open labels (the head) and a side holding all of them; the head
    is sliced as asked; the reported cut equals the labels the sides share.
    The bipartition method refines the first cut, which never grows it, and
    its tree contracts (FP64 oracle) to the state vector's amplitudes."""
    from tn_inputs import sycamore_circuit, random_bits
    circ = sycamore_circuit("rect", 4, 5, 10, 77)
    bits = random_bits(20, 77)
    L, T, O = tn.circuit_network(circ, bits, list(range(15, 20)))
    tree, sliced, st = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=64, n_sliced=2, method=method))
    if method != "greedy":
        st0 = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=64, n_sliced=2))[2]
        assert st["n_cut"] <= st0["n_cut"]
        amp = oc.contract(L, [np.asarray(t, np.complex128) for t in T], O, tree=tree).reshape(-1)
        sv = osv.amplitudes(circ, bits, list(range(15, 20)))
        assert np.linalg.norm(amp - sv) / np.linalg.norm(sv) < 1e-6
    n = len(L)
    assert len(tree) == n - 1 and len(sliced) == 2
    used = set()
    for t, (a, b) in enumerate(tree):
        assert 0 <= a < n + t and 0 <= b < n + t and a != b and a not in used and b not in used
        used.update((a, b))

    def leaves(x):
        return [x] if x < n else leaves(tree[x - n][0]) + leaves(tree[x - n][1])
    sides = [set(), set()]
    for k, root in enumerate(tree[-1]):
        for i in leaves(root):
            sides[k].update(L[i])
    opens = [len(s & set(O)) for s in sides]
    assert sorted(opens) == [0, len(O)]
    head = sides[0] if opens[0] == 0 else sides[1]
    tail = sides[1] if opens[0] == 0 else sides[0]
    assert st["n_cut"] == len(head & tail)
    assert all(x in head and x not in tail for x in sliced)


def _sides(tree, labels, n):
    def leaves(x):
        return [x] if x < n else leaves(tree[x - n][0]) + leaves(tree[x - n][1])
    return [set(l for i in leaves(r) for l in labels[i]) for r in tree[-1]]


def test_head_tail_rejects_bad_cuts_and_slices(tn):
    """tn_head_tail_amplitudes checks its tree and sliced labels on the host,
    before any CUDA call: a root step with open legs on both sides, a head
    sliced label outside the head, an open label sliced in the tail."""
    import torch
    from tn_inputs import random_tree
    amp = torch.zeros(64, dtype=torch.float64)  # never touched: the call fails first
    # a random tree whose root has open legs on both sides
    for seed in range(1, 50):
        net = random_network(seed, n_tensors=8, n_bonds=12, n_open=4, max_rank=6)
        tree = random_tree(seed, len(net.labels))
        s = _sides(tree, net.labels, len(net.labels))
        if all(x & set(net.open_labels) for x in s):
            break
    with pytest.raises(tn.TNError) as e:
        tn.head_tail_amplitudes(net.labels, net.data, net.open_labels, tree, [], [], amp)
    assert e.value.code == -1 and "both sides" in str(e.value)
    # a proper head/tail tree with misplaced sliced labels
    circ = sycamore_circuit("rect", 3, 4, 6, 5)
    L, T, O = tn.circuit_network(circ, random_bits(12, 5), list(range(8, 12)))
    tree, sl_head, st = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=16, n_sliced=0))
    head, tail = _sides(tree, L, len(L))
    if head & set(O):
        head, tail = tail, head
    with pytest.raises(tn.TNError) as e:
        tn.head_tail_amplitudes(L, T, O, tree, [sorted(tail - head)[0]], [], amp)
    assert "head sliced label" in str(e.value)
    with pytest.raises(tn.TNError) as e:
        tn.head_tail_amplitudes(L, T, O, tree, [], [O[0]], amp)
    assert "tail sliced label" in str(e.value)


def test_postselect_and_histogram_reject_bad_arguments(tn):
    """Count and size checks of tn_postselect_xeb, tn_conditional_sample and
    tn_probability_histogram run before any CUDA call."""
    import torch
    amp = torch.zeros(32, dtype=torch.float64)
    for counts in ([0], [17], [1, 2, 100]):
        with pytest.raises(tn.TNError) as e:
            tn.postselect_xeb(amp, 4, 10, counts)
        assert e.value.code == -1
    cnt = torch.zeros(5, dtype=torch.int64)
    for n_bins, x_max, scale in ((0, 1.0, 1.0), (5000, 1.0, 1.0), (4, 0.0, 1.0), (4, 1.0, -1.0)):
        with pytest.raises(tn.TNError):
            tn.probability_histogram(amp, 4, scale, n_bins, x_max, cnt)
    with pytest.raises(tn.TNError):
        tn.conditional_sample(amp, 41, torch.zeros(3, dtype=torch.float64), torch.zeros(3, dtype=torch.int64))


def test_find_order_head_tail_rejects_networks_without_open_legs(tn):
    net = random_network(4, n_tensors=6, n_bonds=9, n_open=0, max_rank=5)
    with pytest.raises(tn.TNError):
        tn.find_order_head_tail(net.labels, [])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_branch_merging_keeps_the_contraction(tn, seed):
    """tn_merge_branches rewrites ((X a) b) into (X (a b)): a valid SSA tree
    over the same leaves whose contraction (by the FP64 oracle, following
    each tree) equals the original's, on random and circuit networks."""
    from tn_inputs import random_tree
    net = random_network(seed, n_tensors=14, n_bonds=24, n_open=3, max_rank=6)
    tree = random_tree(seed, len(net.labels))
    sliced = internal_labels_of(net.labels)[:2]
    merged, st = tn.merge_branches(net.labels, net.open_labels, sliced, tree, max_small_rank=6)
    n = len(net.labels)
    used = set()
    for t, (a, b) in enumerate(merged):
        assert 0 <= a < n + t and 0 <= b < n + t and a != b and a not in used and b not in used
        used.update((a, b))
    ref = oc.contract(net.labels, net.data, net.open_labels, tree=tree)
    got = oc.contract(net.labels, net.data, net.open_labels, tree=merged)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    circ = sycamore_circuit("rect", 3, 4, 8, seed)
    L, T, O = tn.circuit_network(circ, random_bits(12, seed), list(range(8, 12)))
    ctree, csl, _ = tn.find_order(L, O, tn.search_opts(trials=16, n_sliced=2))
    cm, cst = tn.merge_branches(L, O, csl, ctree)
    a0 = oc.contract(L, T, O, tree=ctree)
    a1 = oc.contract(L, T, O, tree=cm)
    assert np.allclose(a1, a0, rtol=1e-12, atol=1e-12 * np.abs(a0).max())


def internal_labels_of(labels):
    cnt = {}
    for l in labels:
        for x in l:
            cnt[x] = cnt.get(x, 0) + 1
    return sorted(x for x, c in cnt.items() if c == 2)


@pytest.mark.parametrize("method", ["bipartition", "mixed"])
@pytest.mark.parametrize("seed", [1, 2])
def test_bipartition_search_gives_valid_exact_trees(tn, method, seed):
    """Hierarchical-bipartition trials (appendix, "Finding contraction order
    using hierarchical partitioning"): a valid SSA tree over every leaf, whose
    FP64 oracle contraction equals the plain one on a random network and the
    state vector on a circuit network (3x4 grid, parts of a few tensors, so
    the splits, not only the greedy inside a part, decide the tree)."""
    net = random_network(seed, n_tensors=18, n_bonds=30, n_open=3, max_rank=6)
    tree, sliced, st = tn.find_order(net.labels, net.open_labels,
                                     tn.search_opts(trials=24, n_sliced=2, method=method))
    n = len(net.labels)
    used = set()
    for t, (a, b) in enumerate(tree):
        assert 0 <= a < n + t and 0 <= b < n + t and a != b and a not in used and b not in used
        used.update((a, b))
    assert len(tree) == n - 1 and len(sliced) == 2
    ref = oc.contract(net.labels, net.data, net.open_labels)
    got = oc.contract(net.labels, net.data, net.open_labels, tree=tree)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    circ = sycamore_circuit("rect", 3, 4, 8, seed)
    bits = random_bits(12, seed)
    L, T, O = tn.circuit_network(circ, bits, [9, 10, 11])
    ctree, _, _ = tn.find_order(L, O, tn.search_opts(trials=24, n_sliced=0, method=method))
    amp = oc.contract(L, [np.asarray(t, np.complex128) for t in T], O, tree=ctree).reshape(-1)
    sv = osv.amplitudes(circ, bits, [9, 10, 11])
    assert np.linalg.norm(amp - sv) / np.linalg.norm(sv) < 1e-6


def test_bipartition_search_is_deterministic_and_checks_its_method(tn):
    cfg = make_config(1)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    a = tn.find_order(L, O, tn.search_opts(trials=64, threads=1, n_sliced=2, method="bipartition"))
    b = tn.find_order(L, O, tn.search_opts(trials=64, threads=4, n_sliced=2, method="bipartition"))
    assert a[0] == b[0] and a[1] == b[1]
    with pytest.raises(tn.TNError):
        tn.find_order(L, O, tn.search_opts(trials=4, method=3))


def test_bipartition_finds_cheaper_trees_on_the_53_qubit_network(tn):
    """On the 53-qubit 14-cycle network (294 tensors, intermediates capped at
    2^30), hierarchical bipartition ends below randomised greedy in total
    complex MACs at the same number of trials (the appendix's reason for
    partitioning: the split structure keeps every pairwise step small)."""
    cfg = make_config(4)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    _, _, g = tn.find_order(L, O, tn.search_opts(trials=256, log2_cap=30))
    _, _, b = tn.find_order(L, O, tn.search_opts(trials=256, log2_cap=30, method="bipartition"))
    assert b["log2_width"] <= 30 and g["log2_width"] <= 30
    assert b["log2_total"] < g["log2_total"] - 0.5, (b, g)


@pytest.mark.parametrize("labels,open_labels,why", [
    ([[1, 2], [1, 3], [1, 4], [2, 3, 4, 5]], [5], "more than two tensors"),
    ([[1, 1], [2]], [2], "repeated within a tensor"),
    ([[1, 2], [2, 3]], [1], "must be open"),
    ([[1, 2], [2, 1, 3]], [1, 3], "open label held by two tensors"),
    ([[1, 2], [2, 3]], [1, 3, 1], "open label repeated"),
    ([[1, 2], [2, 3]], [1, 3, 9], "held by no tensor"),
])
def test_order_search_rejects_malformed_networks(tn, labels, open_labels, why):
    """The order searches apply tn_plan_create's network rules on the host
    (a label is a bond between at most two tensors, held once by each; the
    labels held once are the open ones) and return TN_ERR_ARG, whatever the
    method; a label held twice by one tensor used to leave the greedy search
    without any valid tree."""
    for method in ("greedy", "bipartition"):
        with pytest.raises(tn.TNError, match=why):
            tn.find_order(labels, open_labels, tn.search_opts(trials=4, method=method))
    with pytest.raises(tn.TNError):
        tn.find_order_head_tail(labels, open_labels, opts=tn.search_opts(trials=4))


def test_estimate_tree_ms_prices_each_op_at_its_roofline(tn):
    """tn_estimate_tree_ms compiles the plan on the host and prices each op
    at max(bytes / 7 TB/s, flops / unit peak) + 2 us.  One small step (a
    rank-4 tensor met by a rank-20 one over 2 bonds): 8 B x (|T| + |S| + |C|)
    against 8 flops per MAC on the 80 TFLOP/s CUDA cores.  One GEMM-shaped
    step (2^14 x 2^10 x 2^14) in FP32: 8 flops per MAC on the CUDA cores; in
    the tensor-core forms between 24 (8 for FP16S) tensor flops per MAC at
    2.25 PFLOP/s and the FP32 time."""
    T, S = list(range(20)), [18, 19, 20, 21]
    ms, nb, arena, pro, blk = tn.estimate_tree_ms([T, S], list(range(18)) + [20, 21], [], [(0, 1)], form="fp32")
    byts, macs = 8.0 * (2 ** 20 + 2 ** 4 + 2 ** 20), 2.0 ** 22
    assert ms == pytest.approx(max(byts / 7e12, 8 * macs / 80e12) * 1e3 + 2e-3, rel=1e-12)
    assert nb == 0 and arena >= 8 * 2 ** 20 and pro + blk == pytest.approx(ms, rel=1e-12)
    A, B = list(range(24)), list(range(14, 38))
    O = list(range(14)) + list(range(24, 38))
    macs = 2.0 ** 38
    f32 = tn.estimate_tree_ms([A, B], O, [], [(0, 1)], form="fp32").ms
    assert f32 == pytest.approx(8 * macs / 80e12 * 1e3 + 2e-3, rel=1e-9)
    for form, fl in (("bf16x3", 24), ("fp16x3", 24), ("fp16s", 8)):
        t = tn.estimate_tree_ms([A, B], O, [], [(0, 1)], form=form).ms
        assert fl * macs / 2.25e15 * 1e3 < t < f32, form
    with pytest.raises(tn.TNError):
        tn.estimate_tree_ms([A, B], O, [], [(0, 0)], form="bf16x3")  # malformed tree


def test_estimate_tree_ms_counts_blocks_and_the_prologue(tn):
    """Slicing: the per-block body counts once per block and a slice-
    invariant subtree once in all.  On the 30-qubit network with its 8
    sliced bonds, a block of 2^8 slices prices below 2^8 blocks of one
    slice (launch floors, narrower steps), and every block width gives a
    time at least the sum of the roofline floors of one launch per step."""
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sl, st = tn.find_order(L, O, tn.search_opts(trials=64, n_sliced=8))
    t8, nb8, a8, p8, b8 = tn.estimate_tree_ms(L, O, sl, tree, form="bf16x3", batch_log2=8)
    t0, nb0, a0, p0, b0 = tn.estimate_tree_ms(L, O, sl, tree, form="bf16x3", batch_log2=0)
    assert (nb8, nb0) == (8, 0) and a8 > a0
    assert t8 < t0
    assert t8 == pytest.approx(p8 + b8, rel=1e-12) and t0 == pytest.approx(p0 + 256 * b0, rel=1e-12)
    # the budget picks the block: a budget between the two arenas gives fewer bits
    tb, nbb, ab, _, _ = tn.estimate_tree_ms(L, O, sl, tree, form="bf16x3", arena_budget=(a0 + a8) // 2)
    assert 0 <= nbb < 8 and ab <= (a0 + a8) // 2


def test_roofline_objective_ranks_trees_by_estimated_time(tn):
    """objective="roofline" keeps the trials with the smallest estimated time
    (and, as candidates for reconfiguration, the smallest MAC counts) and
    returns the tree with the smallest estimate: on the 53-qubit 14-cycle
    network it is no slower, by tn_estimate_tree_ms, than the MAC-ranked
    tree of the same trials."""
    cfg = make_config(4)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    est = {}
    for ob in ("macs", "roofline"):
        tree, sl, st = tn.find_order(L, O, tn.search_opts(trials=128, log2_cap=30, method="bipartition",
                                                            objective=ob, rank_form="fp16x3"))
        assert st["log2_width"] <= 30
        est[ob] = tn.estimate_tree_ms(L, O, sl, tree, form="fp16x3")[0]
    assert est["roofline"] <= est["macs"] * 1.0001, est
    with pytest.raises(tn.TNError):
        tn.find_order(L, O, tn.search_opts(trials=2, objective=3))


def _best_connected_tail(L, O, nq, k):
    """Brute force: the smallest cut over connected tensor sets of at most
    half the network holding exactly k qubit ends (None if there is none)."""
    h = {}
    for i, l in enumerate(L):
        for x in l:
            h.setdefault(x, []).append(i)
    ends = {q: h[O[q]][0] for q in range(nq)}
    n, best = len(L), None
    for mask in range(1, 1 << n):
        S = {i for i in range(n) if mask >> i & 1}
        if len(S) > n // 2 or sum(1 for q in range(nq) if ends[q] in S) != k:
            continue
        start = next(iter(S))
        seen, stack = {start}, [start]
        while stack:
            u = stack.pop()
            for x in L[u]:
                for w in h[x]:
                    if w in S and w not in seen:
                        seen.add(w)
                        stack.append(w)
        if seen != S:
            continue
        cut = sum(1 for hh in h.values() if len(hh) == 2 and ((hh[0] in S) != (hh[1] in S)))
        best = cut if best is None else min(best, cut)
    return best, h, ends


@pytest.mark.parametrize("r,c,cyc,seed,k", [(2, 2, 3, 2, 2), (2, 3, 2, 3, 2), (3, 2, 2, 5, 2), (2, 3, 3, 9, 2),
                                            (3, 3, 3, 10, 3), (2, 4, 2, 11, 4), (3, 3, 2, 12, 2), (2, 5, 2, 15, 4),
                                            (2, 3, 2, 7, 4)])
def test_choose_open_qubits_finds_the_best_connected_tail(tn, r, c, cyc, seed, k):
    """tn_choose_open_qubits ("Big-head simulation": the open qubits are
    those whose last tensors lie behind the first cut): on circuits small
    enough to enumerate every tensor set, its tail has the smallest cut of
    all connected sets with exactly k qubit ends, and what it returns is
    consistent: the tail is connected, holds the ends of exactly the returned
    qubits, and cuts the reported number of bonds."""
    circ = sycamore_circuit("rect", r, c, cyc, seed)
    nq = circ.n_qubits
    L, T, O = tn.circuit_network(circ, np.zeros(nq, np.uint8), list(range(nq)))
    best, h, ends = _best_connected_tail(L, O, nq, k)
    if best is None:
        with pytest.raises(tn.TNError):
            tn.choose_open_qubits(circ, k)
        return
    oq, tail, cut, cost = tn.choose_open_qubits(circ, k)
    assert cut == best and cost == -1
    S = set(tail)
    assert oq == sorted(oq) and len(set(oq)) == k
    assert sorted(q for q in range(nq) if ends[q] in S) == oq
    assert cut == sum(1 for hh in h.values() if len(hh) == 2 and ((hh[0] in S) != (hh[1] in S)))


def test_choose_open_qubits_prices_the_candidates(tn):
    """With search options the smallest-cut candidates are priced by the
    order search: the returned cost is that search's cost on the network with
    the returned open qubits, and no higher than the smallest-cut set's."""
    cfg = make_config(2)
    circ = cfg["circuit"]
    opts = tn.search_opts(trials=16, n_sliced=4)
    oq0, _, cut0, c0 = tn.choose_open_qubits(circ, 8)
    oq, tail, cut, cost = tn.choose_open_qubits(circ, 8, opts)
    assert c0 == -1 and cut >= cut0
    L, T, O = tn.circuit_network(circ, cfg["fixed_bits"], oq)
    assert cost == pytest.approx(tn.find_order(L, O, opts)[2]["log2_total"], abs=1e-12)
    L0, T0, O0 = tn.circuit_network(circ, cfg["fixed_bits"], oq0)
    assert cost <= tn.find_order(L0, O0, opts)[2]["log2_total"] + 1e-12
    for bad in (0, circ.n_qubits):
        with pytest.raises(tn.TNError):
            tn.choose_open_qubits(circ, bad)


def test_describe_tree_lists_the_priced_ops(tn):
    """tn_describe_tree (host only) lists the ops of the plan that
    tn_estimate_tree_ms prices: the prologue lines' roofline times add up to
    its prologue time and the batch lines' to its block time; a tensor-core
    form lists tensor-core GEMMs, the FP32 form CUDA-core ones."""
    import re as _re
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sl, _ = tn.find_order(L, O, tn.search_opts(trials=64, n_sliced=8))
    for form in ("bf16x3", "fp32"):
        txt = tn.describe_tree(L, O, sl, tree, form=form, batch_log2=8)
        e = tn.estimate_tree_ms(L, O, sl, tree, form=form, batch_log2=8)
        pro = sum(float(m) for m in _re.findall(r"^prologue .*roofline_ms=([0-9.e+-]+)", txt, _re.M))
        body = sum(float(m) for m in _re.findall(r"^batch .*roofline_ms=([0-9.e+-]+)", txt, _re.M))
        assert pro == pytest.approx(e.prologue_ms, rel=1e-4) and body == pytest.approx(e.block_ms, rel=1e-4)
        gemms = [l for l in txt.splitlines() if " gemm " in l]
        assert gemms and all(("tensor-core" in l) == (form != "fp32") for l in gemms)


def _one_step(tn, row_bits, k_bits, n_bits, form="bf16x3", k_low=False):
    """The compiled op list of one step C[rows, N] = sum_K T[., .] S[K, N]
    (first label = most significant: K above or below T's row labels)."""
    rows = list(range(row_bits))
    K = list(range(100, 100 + k_bits))
    N = list(range(200, 200 + n_bits))
    T = rows + K if k_low else K + rows
    return tn.describe_tree([T, K + N], rows + N, [], [(0, 1)], form=form).strip().splitlines()


def test_plan_compiler_kernel_selection(tn):
    """The plan compiler's kernel choices (host logic, seen through
    tn_describe_tree): a step whose small operand has <= 2^12 values streams
    the big one once on the CUDA cores, one thread per row where N <= 8, in
    row tiles staged through shared memory where K and N are 16..32 (stores
    straight from registers when T's lowest bits are row bits, staged
    otherwise), one thread per row again past K = 32; in the split forms a
    step of at least 2^16 rows with K of 16 or 32 and N of 8, 16 or 32 whose
    rows' 7 lowest bits are T's and C's lowest runs on the tensor cores, T
    split in shared memory; a larger step is a GEMM, on the tensor cores
    after a split pass per operand in the split forms, on the CUDA cores in
    FP32."""
    (op,) = _one_step(tn, 22, 3, 3)
    assert " small rows=4194304 K=8 N=8 " in op and "kernel=row" in op
    (op,) = _one_step(tn, 21, 5, 3)
    assert "K=32 N=8" in op and "kernel=tensor cores, split in shared memory" in op
    (op,) = _one_step(tn, 21, 5, 2)
    assert "K=32 N=4" in op and "kernel=row" in op
    (op,) = _one_step(tn, 21, 5, 3, form="fp32")
    assert "K=32 N=8" in op and "kernel=row" in op
    (op,) = _one_step(tn, 21, 4, 5)
    assert "K=16 N=32" in op and "kernel=tensor cores, split in shared memory" in op
    (op,) = _one_step(tn, 21, 4, 5, form="fp32")
    assert "K=16 N=32" in op and "kernel=tiled, direct C" in op
    (op,) = _one_step(tn, 21, 4, 5, k_low=True)
    assert "kernel=tiled, staged C" in op
    (op,) = _one_step(tn, 21, 5, 5)
    assert "K=32 N=32" in op and "kernel=tensor cores" in op
    (op,) = _one_step(tn, 15, 5, 5)  # fewer than 2^16 rows
    assert "K=32 N=32" in op and "kernel=tiled" in op
    (op,) = _one_step(tn, 21, 5, 5, form="fp32")
    assert "K=32 N=32" in op and "kernel=tiled" in op
    (op,) = _one_step(tn, 12, 6, 3)
    assert "K=64 N=8" in op and "kernel=row" in op
    ops = _one_step(tn, 16, 10, 10)
    assert [o.split()[3] for o in ops] == ["split", "split", "gemm"]
    assert "M=65536 N=1024 K=1024 tensor-core" in ops[-1]
    (op,) = _one_step(tn, 16, 10, 10, form="fp32")
    assert "gemm H=1 M=65536 N=1024 K=1024 fp32" in op


@pytest.mark.parametrize("form", ["bf16x3", "tf32x3", "fp16x3"])
def test_plan_compiler_fuses_the_split_into_the_producing_gemm(tn, form):
    """Two GEMM steps in a chain, (A B) D: the first GEMM's epilogue writes
    the second GEMM's hi/lo planes (out=planes), so step 1 splits only D; in
    the scaled form the max-abs passes are for the leaves only (the producing
    epilogue publishes its output's maximum)."""
    rows, K1, N1, N2 = list(range(16)), list(range(100, 110)), list(range(200, 210)), list(range(300, 310))
    ops = tn.describe_tree([K1 + rows, K1 + N1, N1 + N2], rows + N2, [], [(0, 1), (3, 2)], form=form)
    ops = ops.strip().splitlines()
    gemms = [o for o in ops if " gemm " in o]
    assert len(gemms) == 2 and "out=planes" in gemms[0] and "out=complex64" in gemms[1]
    step1_splits = [o for o in ops if o.startswith("prologue step 1 split")]
    assert len(step1_splits) == 1 and "rank=20" in step1_splits[0]
    maxabs = [int(o.split("n=")[1].split()[0]) for o in ops if " maxabs " in o]
    assert sorted(maxabs) == ([2 ** 20, 2 ** 20, 2 ** 26] if form == "fp16x3" else [])


def test_plan_compiler_runs_slice_invariant_steps_once(tn):
    """Slicing ("Dynamic slicing"): a step whose operands hold no sliced
    label is the same for every slice and runs once per call (prologue); a
    step that depends on a sliced label runs once per block of slices.  With
    the block holding every slice, the sliced label is a batch label and the
    whole tree runs once."""
    rows, K, N, X, s = list(range(14)), list(range(100, 110)), list(range(200, 210)), list(range(300, 306)), 500
    L = [K + rows, K + N, N[:5] + [s] + X, [s] + N[5:]]
    tree = [(0, 1), (2, 3), (4, 5)]
    ops = tn.describe_tree(L, rows + X, [s], tree, form="fp32", batch_log2=0).strip().splitlines()
    phase = {int(o.split()[2]): o.split()[0] for o in ops}
    assert phase == {0: "prologue", 1: "batch", 2: "batch"}
    e = tn.estimate_tree_ms(L, rows + X, [s], tree, form="fp32", batch_log2=0)
    assert e.ms == pytest.approx(e.prologue_ms + 2 * e.block_ms, rel=1e-12)
    ops1 = tn.describe_tree(L, rows + X, [s], tree, form="fp32", batch_log2=1).strip().splitlines()
    assert all(o.startswith("prologue") for o in ops1)


def _fig3_costs(labels, open_labels, tree, sliced):
    """Fig. 3: a step joining A and B costs 2^(n_A + n_B + n_AB) complex MACs
    (the labels of A and B together; sliced labels are fixed, so they do not
    count); a node's size is 2^(its labels minus the sliced ones)."""
    keep, cut = set(open_labels), set(sliced)
    nodes = [set(l) for l in labels]
    per_slice, width = 0, max(len(s - cut) for s in nodes)
    for a, b in tree:
        A, B = nodes[a], nodes[b]
        per_slice += 2 ** len((A | B) - cut)
        C = (A | B) - ((A & B) - keep)
        nodes.append(C)
        width = max(width, len(C - cut))
    return np.log2(per_slice), width


@pytest.mark.parametrize("method", ["greedy", "bipartition"])
def test_search_costs_follow_fig3(tn, method):
    """The search's reported costs are Fig. 3's: per-slice MACs summed over
    the steps of the returned tree, the total that times 2^n_sliced, and the
    width the largest node, recomputed here from the tree alone."""
    cases = [random_network(41, n_tensors=16, n_bonds=30, n_open=3, max_rank=8), None]
    for net in cases:
        if net is None:
            cfg = make_config(2)
            L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
        else:
            L, O = net.labels, net.open_labels
        tree, sl, st = tn.find_order(L, O, tn.search_opts(trials=32, n_sliced=3, method=method))
        log2_slice, width = _fig3_costs(L, O, tree, sl)
        assert st["log2_slice"] == pytest.approx(log2_slice, abs=1e-9)
        assert st["log2_total"] == pytest.approx(log2_slice + len(sl), abs=1e-9)
        assert st["log2_width"] == width


def test_slice_tree_meets_the_cap_on_a_given_tree(tn):
    """tn_slice_tree slices a caller's tree: every intermediate then fits the
    cap, the sliced labels are internal bonds, the reported costs are Fig. 3's
    for that tree, and summing the FP64 oracle's slices gives the unsliced
    contraction (the slicing invariant)."""
    net = random_network(43, n_tensors=14, n_bonds=26, n_open=3, max_rank=8)
    tree, _, st0 = tn.find_order(net.labels, net.open_labels, tn.search_opts(trials=16, n_sliced=0))
    cap = int(st0["log2_width"]) - 3
    sl, st = tn.slice_tree(net.labels, net.open_labels, tree, log2_cap=cap)
    assert st["log2_width"] <= cap and len(sl) == st["n_sliced"] == len(set(sl)) >= 1
    assert not set(sl) & set(net.open_labels)
    log2_slice, width = _fig3_costs(net.labels, net.open_labels, tree, sl)
    assert st["log2_slice"] == pytest.approx(log2_slice, abs=1e-9) and st["log2_width"] == width
    full = oc.contract(net.labels, net.data, net.open_labels, tree=tree)
    parts = sum(oc.slice_partial(net.labels, net.data, net.open_labels, sl, s) for s in range(1 << len(sl)))
    assert np.abs(parts - full).max() < 1e-12 * max(1.0, np.abs(full).max())
    sl2, st2 = tn.slice_tree(net.labels, net.open_labels, tree, n_sliced=2)
    assert len(sl2) == 2
    with pytest.raises(tn.TNError):
        tn.slice_tree(net.labels, net.open_labels, tree)  # neither a cap nor a count
    with pytest.raises(tn.TNError):
        tn.slice_tree(net.labels, net.open_labels, [(0, 0)] * len(tree), log2_cap=cap)


def _leaves_of(tree, n, x):
    return [x] if x < n else _leaves_of(tree, n, tree[x - n][0]) + _leaves_of(tree, n, tree[x - n][1])


def test_slice_stage2_bounds_the_second_stage(tn):
    """The two-stage form with its second stage sliced, end to end on the
    FP64 oracle ("Big-head simulation": psi = v_head . v_tail): v_head is the
    head contracted over the cut, stage 2 is the tail with v_head as one more
    leaf, and tn_slice_stage2's labels (tail or cut bonds, never open) bound
    its intermediates; summing the oracle's slices of stage 2 gives the state
    vector's amplitudes."""
    circ = sycamore_circuit("rect", 3, 4, 8, 5)
    bits, open_q = random_bits(12, 5), [8, 9, 10, 11]
    L, T, O = tn.circuit_network(circ, bits, open_q)
    T = [np.asarray(t, np.complex128) for t in T]
    n = len(L)
    tree, _, st = tn.find_order_head_tail(L, O, opts=tn.search_opts(trials=32, n_sliced=0))
    a, b = (_leaves_of(tree, n, r) for r in tree[-1])
    head, tail = (a, b) if not {x for i in a for x in L[i]} & set(O) else (b, a)
    lh, lt = {x for i in head for x in L[i]}, {x for i in tail for x in L[i]}
    cut = sorted(lh & lt)
    v_head = oc.contract([L[i] for i in head], [T[i] for i in head], cut)
    L2, T2 = [L[i] for i in tail] + [cut], [T[i] for i in tail] + [v_head]
    full = tn.slice_tree(L2, O, _stage2_tree(tree, n, tail), n_sliced=0)[1]["log2_width"]
    cap = int(full) - 3
    sl, st2 = tn.slice_stage2(L, O, tree, log2_cap=cap)
    assert st2["log2_width"] <= cap and sl and not set(sl) & set(O) and set(sl) <= lt
    amp = sum(oc.slice_partial(L2, T2, O, sl, s) for s in range(1 << len(sl))).reshape(-1)
    ref = osv.amplitudes(circ, bits, open_q)
    assert np.linalg.norm(amp - ref) / np.linalg.norm(ref) < 1e-6
    with pytest.raises(tn.TNError):
        tn.slice_stage2(L, O, tn.find_order(L, O, tn.search_opts(trials=4, n_sliced=0))[0], log2_cap=cap)


def _stage2_tree(tree, n, tail):
    """The stage-2 tree as tn_head_tail_amplitudes builds it: the tail's
    subtree renumbered over the tail's leaves, then v_head (the next leaf)
    joined at its root."""
    idx = {x: i for i, x in enumerate(tail)}
    m, out = len(tail), []
    for t, (a, b) in enumerate(tree[:-1]):
        if a in idx and b in idx:
            out.append((idx[a] + (idx[a] >= m), idx[b] + (idx[b] >= m)))
            idx[n + t] = m + len(out) - 1
    root = max(idx.values())
    out.append((root + 1 if root >= m else root, m))
    return out


def test_choose_open_qubits_prices_by_the_search_objective(tn):
    """With the roofline objective the candidates are compared by their
    plans' roofline time, and the cost returned is log2 of the winner's."""
    cfg = make_config(2)
    opts = tn.search_opts(trials=8, n_sliced=4, objective="roofline", rank_form="bf16x3")
    oq, _, _, cost = tn.choose_open_qubits(cfg["circuit"], 8, opts)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], oq)
    tree, sl, _ = tn.find_order(L, O, opts)
    assert cost == pytest.approx(np.log2(tn.estimate_tree_ms(L, O, sl, tree, form="bf16x3").ms), abs=1e-9)
    oq0, _, _, _ = tn.choose_open_qubits(cfg["circuit"], 8)
    L0, T0, O0 = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], oq0)
    t0, s0, _ = tn.find_order(L0, O0, opts)
    assert cost <= np.log2(tn.estimate_tree_ms(L0, O0, s0, t0, form="bf16x3").ms) + 1e-9


def test_choose_open_qubits_takes_the_cheapest_candidate_below_1ms(tn):
    """With the roofline objective every candidate's cost is log2 of a plan
    time in ms, negative for plans under 1 ms.  The chooser must return the
    smallest of the 8 smallest-cut candidates' costs, whatever their sign
    (a negative 'nothing chosen yet' sentinel would keep the last candidate
    instead)."""
    from tn_inputs import sycamore_circuit, random_bits
    circ = sycamore_circuit("rect", 3, 5, 8, 77)
    n_open = 5
    opts = tn.search_opts(trials=8, n_sliced=2, objective="roofline", rank_form="tf32x3")
    cands = tn.open_qubit_candidates(circ, n_open)
    assert cands and [c[1] for c in cands] == sorted(c[1] for c in cands)
    costs = []
    for oq, _ in cands[:8]:
        L, T, O = tn.circuit_network(circ, [0] * circ.n_qubits, oq)
        tree, sl, _ = tn.find_order(L, O, opts)
        costs.append(np.log2(tn.estimate_tree_ms(L, O, sl, tree, form="tf32x3").ms))
    assert max(costs) < 0, "the case needs every candidate below 1 ms"
    oq, _, _, cost = tn.choose_open_qubits(circ, n_open, opts)
    i = int(np.argmin(costs))
    assert cost == pytest.approx(costs[i], abs=1e-9)
    assert cost <= min(costs) + 1e-9
    assert oq in [c[0] for c in cands[:8]]


def test_expected_time_objective(tn):
    """objective 'expected' (2): the roofline time with each tensor-core GEMM
    priced at no less than its epilogue's output rate.  It searches like the
    other objectives (a valid, sliced tree, deterministic), the open-qubit
    chooser takes it too, and an unknown objective is refused."""
    cfg = make_config(2)
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    o2 = tn.search_opts(trials=64, n_sliced=4, objective="expected", rank_form="fp16x3")
    tree, sl, st = tn.find_order(L, O, o2)
    assert len(tree) == len(L) - 1 and len(sl) == 4
    assert tn.find_order(L, O, o2)[0] == tree
    oq, _, _, cost = tn.choose_open_qubits(cfg["circuit"], 8, o2)
    assert len(oq) == 8 and np.isfinite(cost)
    with pytest.raises(tn.TNError):
        tn.find_order(L, O, tn.search_opts(trials=8, n_sliced=4, objective=3))


def test_plan_compiler_tma_store_box_views(tn):
    """The box view that a TMA-stored planar epilogue writes through (host
    side of tc_tma_store, shown in the plan line as start@log2-box per
    dimension): a GEMM whose half tile is the destination's 4,096 lowest
    elements (c0..c5, then r0..r5) gets two dimensions; the bench tree's
    largest GEMM (c0..c4 r0 at bits 0..5, c5 at 7, r1..r5 at 16..20) gets
    five, gaps as boxes of one.  TF32 planes, single read-out tiles (the
    sixteen-warp kernel) and tc_tma_store -1 keep the staged store."""
    m, n, p = 14, 9, 4
    ml, nl, pl = list(range(m)), list(range(200, 200 + n)), list(range(400, 400 + p))
    for k, form, opts, want in [(9, "fp16x3", None, "tma box=0@6,6@6"), (9, "bf16x3", None, "tma box=0@6,6@6"),
                                (9, "fp16s", None, "tma box=0@6,6@6"), (7, "fp16x3", None, "staged"),
                                (9, "tf32x3", None, "staged"), (9, "fp16x3", tn.plan_opts(tc_tma_store=-1), "staged")]:
        kl = list(range(100, 100 + k))
        ops = tn.describe_tree([ml + kl, kl + nl, nl + pl], ml + pl, [], [(0, 1), (3, 2)], form=form, opts=opts)
        first = [o for o in ops.splitlines() if " gemm " in o][0]
        assert "out=planes" in first and f" {want} " in first, (form, k, first)
    import bench
    from paper_2103_03074_gb300.trees import make_trees
    cfg = bench.workload("syc53_m14")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    tree, sliced, _ = make_trees.load("syc53_m14", L, O)
    ops = tn.describe_tree(L, O, sliced, tree, form="fp16x3")
    big = [o for o in ops.splitlines() if " gemm " in o and "M=4194304 N=256 K=256" in o]
    assert len(big) == 1 and "tma box=0@6,6@0,7@1,8@0,16@5 " in big[0], big
