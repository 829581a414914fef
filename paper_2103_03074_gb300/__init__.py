"""Python binding of libtn (include/tn.h): argument marshalling only.

Every step of the contraction runs in the library's CUDA kernels; PyTorch is
used by callers only for device memory and streams.  Importing this package
loads ``libtn.so`` built in place by ``build.py``; a missing library is an
ImportError, never a silent fallback.
"""
from __future__ import annotations

import collections
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtn.so is not built ({LIB_PATH}); run `python -m paper_2103_03074_gb300.build` "
                      "or __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

TN_FP32, TN_BF16X3, TN_TF32X3, TN_FP16S, TN_FP16X3 = 0, 1, 2, 3, 4
FORMS = {"fp32": TN_FP32, "bf16x3": TN_BF16X3, "tf32x3": TN_TF32X3, "fp16s": TN_FP16S, "fp16x3": TN_FP16X3}
ERRORS = {-1: "TN_ERR_ARG", -2: "TN_ERR_OOM", -3: "TN_ERR_CUDA", -4: "TN_ERR_TIMEOUT", -5: "TN_ERR_STATE"}

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class PlanOpts(ctypes.Structure):
    _fields_ = [("batch_log2", _i32), ("mem_budget", _i64), ("profile", _i32), ("use_graph", _i32),
                ("tc_chunk_bytes", _i32), ("tc_flush_bytes", _i32), ("tc_planar", _i32),
                ("graph_branches", _i32),
                ("small_tc_bits", _i32), ("small_tiled", _i32), ("tc_products", _i32), ("small_tasks", _i32),
                ("small_tc", _i32), ("tc_tma_store", _i32)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("trials", _i32), ("seed", ctypes.c_uint64), ("log2_cap", _i32), ("n_sliced", _i32),
                ("threads", _i32), ("candidates", _i32), ("rank_batch_log2", _i32), ("rank_form", _i32),
                ("cost_model", _vp), ("method", _i32), ("objective", _i32)]


class Circuit(ctypes.Structure):
    _fields_ = [("n_qubits", _i32), ("n_gates", _i32), ("gate_nq", _vp), ("gate_q", _vp), ("gate_m", _vp)]


_lib.tn_last_error.restype = ctypes.c_char_p
_lib.tn_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(PlanOpts)]
_lib.tn_contract_slices.argtypes = [_vp, _i64, _i64, _vp, _vp]
_lib.tn_contract_slices_host.argtypes = [_vp, _i64, _i64, _vp, ctypes.c_int, _vp, _vp, _vp]
_lib.tn_amplitudes.argtypes = [ctypes.POINTER(Circuit), _vp, ctypes.c_int, _vp, ctypes.c_int,
                               ctypes.POINTER(SearchOpts), ctypes.POINTER(PlanOpts), _vp, _vp]
_lib.tn_probabilities_xeb.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.tn_plan_update_data.argtypes = [_vp, _vp, _vp]
_lib.tn_plan_profile.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int]
_lib.tn_plan_destroy.argtypes = [_vp]
_lib.tn_plan_destroy.restype = None
_lib.tn_find_order.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(SearchOpts), _vp,
                               ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int), _vp]
_lib.tn_circuit_network.argtypes = [ctypes.POINTER(Circuit), _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64), _vp, _vp, _vp, _vp]
_lib.tn_plan_stats.argtypes = [_vp, _vp]
_lib.tn_gemm_split_noalloc.argtypes = [_vp, _vp, _vp, _i64, _i64, _i64, ctypes.c_int, _vp]
_lib.tn_costmodel_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_uint64]
_lib.tn_costmodel_destroy.argtypes = [_vp]
_lib.tn_costmodel_destroy.restype = None
_lib.tn_costmodel_params.argtypes = [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int)]
_lib.tn_costmodel_grad.argtypes = [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), _vp]
_lib.tn_costmodel_train.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_double), _vp]
_lib.tn_costmodel_predict.argtypes = [_vp, _vp, _vp, _i64, _vp]
_lib.tn_plan_op_features.argtypes = [_vp, _vp, ctypes.c_int]
_lib.tn_plan_autotune.argtypes = [_vp, ctypes.c_int, _vp]
_lib.tn_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, _vp, ctypes.c_int]
_lib.tn_batch_run.argtypes = [_vp, _vp]
_lib.tn_batch_destroy.argtypes = [_vp]
_lib.tn_batch_destroy.restype = None
_lib.tn_plan_describe.argtypes = [_vp, _vp, ctypes.c_int]
_lib.tn_merge_branches.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                   ctypes.c_int, _vp, _vp]
_lib.tn_find_order_head_tail.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                         ctypes.POINTER(SearchOpts), _vp, ctypes.c_int, _vp,
                                         ctypes.POINTER(ctypes.c_int), _vp]
_lib.tn_head_tail_amplitudes.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                         ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                         ctypes.POINTER(PlanOpts), _vp, _vp, ctypes.POINTER(ctypes.c_int), _vp]
_lib.tn_postselect_xeb.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.tn_conditional_sample.argtypes = [_vp, ctypes.c_int, _i64, _vp, _vp, _vp]
_lib.tn_probability_histogram.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _vp,
                                          _vp]
COST_FEATURES = 16

EXPORTED = ["tn_plan_create", "tn_contract_slices", "tn_amplitudes", "tn_probabilities_xeb", "tn_plan_destroy",
            "tn_last_error", "tn_find_order", "tn_circuit_network", "tn_plan_stats", "tn_plan_update_data",
            "tn_plan_profile", "tn_gemm_split_noalloc", "tn_costmodel_create", "tn_costmodel_destroy",
            "tn_costmodel_params", "tn_costmodel_grad", "tn_costmodel_train", "tn_costmodel_predict",
            "tn_plan_op_features", "tn_plan_autotune", "tn_batch_create", "tn_batch_run", "tn_batch_destroy",
            "tn_postselect_xeb", "tn_conditional_sample", "tn_probability_histogram", "tn_plan_describe",
            "tn_find_order_head_tail", "tn_head_tail_amplitudes", "tn_merge_branches", "tn_estimate_tree_ms", "tn_choose_open_qubits",
            "tn_open_qubit_candidates", "tn_contract_slices_host", "tn_describe_tree", "tn_slice_tree", "tn_slice_stage2"]
PROFILE_KINDS = {0: "small", 1: "permute", 2: "gemm", 3: "extract", 4: "accumulate", 5: "split", 6: "maxabs",
                 7: "tasks"}


class TNError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.tn_last_error().decode()
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, where):
    if rc != 0:
        raise TNError(rc, where)


def _ptr(a):
    return a.ctypes.data_as(_vp) if a is not None else None


def _host_ptr(a):
    """Host address of a numpy array or a CPU torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(_vp)
    if getattr(a, "is_cuda", False):
        raise ValueError("expected a host buffer")
    return ctypes.c_void_p(a.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return _vp(stream.cuda_stream)
    return _vp(int(stream))


def _dev_ptr(t):
    return _vp(t.data_ptr())


SEARCH_METHODS = {"greedy": 0, "bipartition": 1, "mixed": 2}
SEARCH_OBJECTIVES = {"macs": 0, "roofline": 1, "expected": 2}


def search_opts(trials=256, seed=0x2103030740, log2_cap=-1, n_sliced=-1, threads=0, candidates=0,
                rank_batch_log2=-1, rank_form="fp32", cost_model=None, method="greedy", objective="macs"):
    """Order-search options (tn_search_opts).  method: "greedy" (randomised
    greedy trials), "bipartition" (hierarchical min-cut bipartition, greedy
    inside parts of a few dozen tensors) or "mixed" (alternating).
    objective: "macs" (total complex MACs), "roofline" (the tree's plan for
    rank_form priced at its roofline time, as estimate_tree_ms does) or
    "expected" (that time with each tensor-core GEMM priced at no less than
    its epilogue's measured output rate)."""
    f = FORMS[rank_form] if isinstance(rank_form, str) else int(rank_form)
    m = SEARCH_METHODS[method] if isinstance(method, str) else int(method)
    ob = SEARCH_OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    cm = cost_model._h if cost_model is not None else None
    return SearchOpts(trials, seed, log2_cap, n_sliced, threads, candidates, rank_batch_log2, f, cm, m, ob)


def plan_opts(batch_log2=-1, mem_budget=0, profile=0, use_graph=0, tc_chunk_bytes=0, tc_flush_bytes=0,
              tc_planar=0, graph_branches=0, small_tc_bits=0, small_tiled=0, tc_products=0, small_tasks=0,
              small_tc=0, tc_tma_store=0):
    """Plan options (tn_plan_opts).  tc_products: 4 (default) or 3, the real
    products per complex product of the split forms' tensor-core GEMMs (3:
    Gauss's 3M product).  small_tasks: 0 (default) runs tiny small steps as
    tasks of persistent launches, -1 one launch per step, > 0 the size bound
    (log2 elements) of a task.  small_tc: 0 (default) large small steps of
    the split forms on the tensor cores (T split in shared memory), -1 on the
    CUDA cores.  tc_tma_store: 0 (default) GEMMs store a staged planar output
    by TMA where its layout allows, -1 from the epilogue warps."""
    return PlanOpts(batch_log2, mem_budget, profile, use_graph, tc_chunk_bytes, tc_flush_bytes, tc_planar,
                    graph_branches, small_tc_bits, small_tiled, tc_products, small_tasks, small_tc, tc_tma_store)


def marshal_circuit(circuit):
    """tn_inputs.Circuit -> (ctypes Circuit, keep-alive arrays)."""
    gates = circuit.gates
    ng = len(gates)
    nq = np.array([len(g.qubits) for g in gates], dtype=np.int32)
    qs = np.zeros(2 * ng, dtype=np.int32)
    ms = np.zeros(32 * ng, dtype=np.float64)
    for i, g in enumerate(gates):
        for j, q in enumerate(g.qubits):
            qs[2 * i + j] = q
        m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
        ms[32 * i:32 * i + 2 * m.size:2] = m.real
        ms[32 * i + 1:32 * i + 2 * m.size:2] = m.imag
    keep = (nq, qs, ms)
    return Circuit(circuit.n_qubits, ng, _ptr(nq), _ptr(qs), _ptr(ms)), keep


def circuit_network(circuit, fixed_bits, open_qubits):
    """The network tn_amplitudes contracts: (labels list, complex64 tensors, open labels)."""
    c, keep = marshal_circuit(circuit)
    fb = np.asarray(fixed_bits, dtype=np.uint8)
    oq = np.asarray(open_qubits, dtype=np.int32)
    nt, tr, te = ctypes.c_int(), ctypes.c_int(), _i64()
    _check(_lib.tn_circuit_network(ctypes.byref(c), _ptr(fb), len(oq), _ptr(oq), ctypes.byref(nt), ctypes.byref(tr),
                                   ctypes.byref(te), None, None, None, None), "tn_circuit_network")
    ranks = np.zeros(nt.value, np.int32)
    labs = np.zeros(max(tr.value, 1), np.int32)
    data = np.zeros(2 * te.value, np.float32)
    ol = np.zeros(max(len(oq), 1), np.int32)
    _check(_lib.tn_circuit_network(ctypes.byref(c), _ptr(fb), len(oq), _ptr(oq), ctypes.byref(nt), ctypes.byref(tr),
                                   ctypes.byref(te), _ptr(ranks), _ptr(labs), _ptr(data), _ptr(ol)),
           "tn_circuit_network")
    labels, tensors = [], []
    lo = do = 0
    for r in ranks:
        labels.append([int(x) for x in labs[lo:lo + r]])
        lo += r
        size = 1 << int(r)
        v = data[do:do + 2 * size]
        do += 2 * size
        tensors.append((v[0::2] + 1j * v[1::2]).astype(np.complex64).reshape((2,) * int(r)))
    return labels, tensors, [int(x) for x in ol[:len(oq)]]


def _flatten(labels, tensors):
    ranks = np.array([len(l) for l in labels], dtype=np.int32)
    flat = np.array([x for l in labels for x in l] or [0], dtype=np.int32)
    parts = []
    for t in tensors:
        c = np.asarray(t, dtype=np.complex64).reshape(-1)
        parts.append(np.stack([c.real, c.imag], axis=1).reshape(-1))
    data = np.ascontiguousarray(np.concatenate(parts).astype(np.float32))
    return ranks, flat, data


def find_order(labels, open_labels, opts=None, max_sliced=64):
    """(tree [(a, b), ...], sliced labels, stats dict) from the library's order search."""
    ranks, flat, _ = _flatten(labels, [np.zeros((2,) * len(l), np.complex64) for l in labels])
    ol = np.asarray(open_labels or [0], dtype=np.int32)
    n = len(labels)
    tree = np.zeros(max(2 * (n - 1), 1), np.int32)
    sl = np.zeros(max_sliced, np.int32)
    nsl = ctypes.c_int()
    st = np.zeros(4)
    o = opts if opts is not None else search_opts()
    _check(_lib.tn_find_order(n, _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol), ctypes.byref(o), _ptr(tree),
                              max_sliced, _ptr(sl), ctypes.byref(nsl), _ptr(st)), "tn_find_order")
    steps = [(int(tree[2 * i]), int(tree[2 * i + 1])) for i in range(n - 1)]
    stats = dict(log2_total=st[0], log2_width=st[1], n_sliced=int(st[2]), log2_slice=st[3])
    return steps, [int(x) for x in sl[:nsl.value]], stats


TreeEstimate = collections.namedtuple("TreeEstimate", "ms batch_log2 arena prologue_ms block_ms")


def estimate_tree_ms(labels, open_labels, sliced_labels, tree, form="fp32", batch_log2=-1, arena_budget=0,
                     opts=None):
    """tn_estimate_tree_ms: TreeEstimate(ms for all slices, block width in
    sliced bits, arena bytes, prologue ms, ms per block) of the plan the tree
    compiles to, every op at its roofline time (host only, no GPU needed)."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    sl = np.asarray(list(sliced_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    f = FORMS[form] if isinstance(form, str) else int(form)
    ms, pro, blk = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    nb = ctypes.c_int(0)
    arena = ctypes.c_int64(0)
    _check(_lib.tn_estimate_tree_ms(len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol),
                                    len(sliced_labels), _ptr(sl), len(tree), _ptr(tr), f,
                                    ctypes.byref(opts) if opts is not None else None, int(batch_log2),
                                    ctypes.c_int64(int(arena_budget)), ctypes.byref(ms), ctypes.byref(nb),
                                    ctypes.byref(arena), ctypes.byref(pro), ctypes.byref(blk)), "tn_estimate_tree_ms")
    return TreeEstimate(ms.value, nb.value, arena.value, pro.value, blk.value)


def describe_tree(labels, open_labels, sliced_labels, tree, form="fp32", batch_log2=-1, arena_budget=0,
                  opts=None):
    """tn_describe_tree: the ops the tree's plan compiles to (host only), one
    line each with its roofline_ms."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    sl = np.asarray(list(sliced_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    f = FORMS[form] if isinstance(form, str) else int(form)
    args = (len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol), len(sliced_labels), _ptr(sl),
            len(tree), _ptr(tr), f, ctypes.byref(opts) if opts is not None else None, int(batch_log2),
            ctypes.c_int64(int(arena_budget)))
    n = _lib.tn_describe_tree(*args, None, 0)
    if n < 0:
        _check(n, "tn_describe_tree")
    buf = ctypes.create_string_buffer(n + 1)
    _check(min(0, _lib.tn_describe_tree(*args, buf, n + 1)), "tn_describe_tree")
    return buf.value.decode()


def slice_tree(labels, open_labels, tree, log2_cap=-1, n_sliced=-1, max_sliced=64):
    """tn_slice_tree: (sliced labels, stats dict) for a given tree, sliced
    until every intermediate fits 2^log2_cap (or exactly n_sliced labels)."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    sl = np.zeros(max(max_sliced, 1), dtype=np.int32)
    nsl = ctypes.c_int(0)
    st = np.zeros(4)
    _check(_lib.tn_slice_tree(len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol), len(tree), _ptr(tr),
                              int(log2_cap), int(n_sliced), int(max_sliced), _ptr(sl), ctypes.byref(nsl), _ptr(st)),
           "tn_slice_tree")
    stats = dict(log2_total=st[0], log2_width=st[1], n_sliced=int(st[2]), log2_slice=st[3])
    return [int(x) for x in sl[:nsl.value]], stats


def slice_stage2(labels, open_labels, tree, log2_cap, max_sliced=64):
    """tn_slice_stage2: (sliced_tail labels, stats dict) bounding the
    intermediates of head_tail_amplitudes' stage 2 by 2^log2_cap."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    sl = np.zeros(max(max_sliced, 1), dtype=np.int32)
    nsl = ctypes.c_int(0)
    st = np.zeros(4)
    _check(_lib.tn_slice_stage2(len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol), len(tree),
                                _ptr(tr), int(log2_cap), int(max_sliced), _ptr(sl), ctypes.byref(nsl), _ptr(st)),
           "tn_slice_stage2")
    stats = dict(log2_total=st[0], log2_width=st[1], n_sliced=int(st[2]), log2_slice=st[3])
    return [int(x) for x in sl[:nsl.value]], stats


def merge_branches(labels, open_labels, sliced_labels, tree, max_small_rank=0):
    """tn_merge_branches: (rewritten tree, stats dict) with ((X a) b) turned
    into (X (a b)) where that lowers the estimated step time."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    sl = np.asarray(list(sliced_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    out = np.zeros(max(2 * len(tree), 1), dtype=np.int32)
    st = np.zeros(3)
    _check(_lib.tn_merge_branches(len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol),
                                  len(sliced_labels), _ptr(sl), len(tree), _ptr(tr), int(max_small_rank), _ptr(out),
                                  _ptr(st)), "tn_merge_branches")
    steps = [(int(out[2 * t]), int(out[2 * t + 1])) for t in range(len(tree))]
    return steps, dict(rewrites=int(st[0]), log2_macs_before=float(st[1]), log2_macs_after=float(st[2]))


def choose_open_qubits(circuit, n_open, opts=None):
    """tn_choose_open_qubits: (open qubits, tail tensor ids in the all-open
    network, cut, log2 cost or -1) for the open set behind a small first cut
    (with opts: the cheapest to contract of the 8 smallest cuts)."""
    c, keep = marshal_circuit(circuit)
    n_max = len(circuit.gates) + 2 * circuit.n_qubits + 1
    oq = np.zeros(n_open, dtype=np.int32)
    tail = np.zeros(n_max, dtype=np.int32)
    nt = ctypes.c_int(0)
    cut = ctypes.c_int(0)
    cost = ctypes.c_double(0)
    _check(_lib.tn_choose_open_qubits(ctypes.byref(c), int(n_open), ctypes.byref(opts) if opts is not None else None,
                                      _ptr(oq), _ptr(tail), ctypes.byref(nt), ctypes.byref(cut),
                                      ctypes.byref(cost)), "tn_choose_open_qubits")
    return [int(x) for x in oq], [int(x) for x in tail[:nt.value]], cut.value, cost.value


def open_qubit_candidates(circuit, n_open, max_out=64):
    """tn_open_qubit_candidates: [(open qubits, cut)] in the order
    tn_choose_open_qubits takes them (smallest cut first)."""
    c, keep = marshal_circuit(circuit)
    oq = np.zeros(max(1, max_out * n_open), dtype=np.int32)
    cuts = np.zeros(max(1, max_out), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(_lib.tn_open_qubit_candidates(ctypes.byref(c), int(n_open), int(max_out), _ptr(oq), _ptr(cuts),
                                         ctypes.byref(n)), "tn_open_qubit_candidates")
    m = min(max_out, n.value)
    return [([int(x) for x in oq[i * n_open:(i + 1) * n_open]], int(cuts[i])) for i in range(m)]


def find_order_head_tail(labels, open_labels, tail_max=0, opts=None, max_sliced=64):
    """tn_find_order_head_tail: (tree whose last step is the first cut, head
    sliced labels, stats dict)."""
    ranks = np.asarray([len(l) for l in labels], dtype=np.int32)
    flat = np.asarray([x for l in labels for x in l] or [0], dtype=np.int32)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    tree = np.zeros(2 * (len(labels) - 1), dtype=np.int32)
    sl = np.zeros(max_sliced, dtype=np.int32)
    nsl = ctypes.c_int(0)
    st = np.zeros(7)
    o = opts if opts is not None else search_opts()
    _check(_lib.tn_find_order_head_tail(len(labels), _ptr(ranks), _ptr(flat), len(open_labels), _ptr(ol),
                                        int(tail_max), ctypes.byref(o), _ptr(tree), max_sliced, _ptr(sl),
                                        ctypes.byref(nsl), _ptr(st)), "tn_find_order_head_tail")
    steps = [(int(tree[2 * t]), int(tree[2 * t + 1])) for t in range(len(labels) - 1)]
    keys = ["log2_head_slice", "log2_head_width", "n_sliced_head", "log2_tail", "log2_tail_width", "n_cut",
            "log2_total"]
    return steps, [int(x) for x in sl[:nsl.value]], dict(zip(keys, (float(x) for x in st)))


def head_tail_amplitudes(labels, tensors, open_labels, tree, sliced_head, sliced_tail, d_amp, form="fp32",
                         opts=None, d_vhead=None, stream=None):
    """tn_head_tail_amplitudes: two-stage contraction into d_amp (device
    complex128); returns the number of cut bonds."""
    ranks, flat, data = _flatten(labels, tensors)
    ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
    tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
    sh = np.asarray(list(sliced_head) or [0], dtype=np.int32)
    st = np.asarray(list(sliced_tail) or [0], dtype=np.int32)
    f = FORMS[form] if isinstance(form, str) else int(form)
    o = opts if opts is not None else plan_opts()
    nc = ctypes.c_int(0)
    _check(_lib.tn_head_tail_amplitudes(len(labels), _ptr(ranks), _ptr(flat), _ptr(data), len(open_labels),
                                        _ptr(ol), len(tree), _ptr(tr), len(sliced_head), _ptr(sh),
                                        len(sliced_tail), _ptr(st), f, ctypes.byref(o), _dev_ptr(d_amp),
                                        _dev_ptr(d_vhead) if d_vhead is not None else None, ctypes.byref(nc),
                                        _stream_ptr(stream)), "tn_head_tail_amplitudes")
    return nc.value


class Plan:
    """A compiled sliced contraction (tn_plan_create); owns its device memory."""

    def __init__(self, labels, tensors, open_labels, sliced_labels, tree, form="fp32", opts=None):
        ranks, flat, data = _flatten(labels, tensors)
        ol = np.asarray(list(open_labels) or [0], dtype=np.int32)
        sl = np.asarray(list(sliced_labels) or [0], dtype=np.int32)
        tr = np.asarray([x for p in tree for x in p] or [0], dtype=np.int32)
        self.n_open = len(open_labels)
        self.n_sliced = len(sliced_labels)
        self.form = FORMS[form] if isinstance(form, str) else int(form)
        h = _vp()
        o = opts if opts is not None else plan_opts()
        _check(_lib.tn_plan_create(ctypes.byref(h), len(labels), _ptr(ranks), _ptr(flat), _ptr(data), 0, None,
                                   len(open_labels), _ptr(ol), len(sliced_labels), _ptr(sl), len(tree), _ptr(tr),
                                   self.form, ctypes.byref(o)), "tn_plan_create")
        self._h = h

    def contract(self, begin, end, d_amp, stream=None):
        """Add the sum of slices [begin, end) into d_amp (device complex128 tensor)."""
        _check(_lib.tn_contract_slices(self._h, int(begin), int(end), _dev_ptr(d_amp), _stream_ptr(stream)),
               "tn_contract_slices")

    def contract_ptr(self, begin, end, d_amp_ptr, stream_ptr=None):
        _check(_lib.tn_contract_slices(self._h, int(begin), int(end), _vp(d_amp_ptr),
                                       _vp(stream_ptr) if stream_ptr else None), "tn_contract_slices")

    def contract_host(self, begin, end, h_data=None, n_qubits=0, h_amp=None, h_stats=None, stream=None):
        """tn_contract_slices_host: host buffers in and out (numpy arrays or
        pinned CPU tensors): optional new leaf values (float32), amplitudes
        (float64, 2 << n_open) and {P(s1), XEB, max p} (float64, 3).
        Synchronises the stream."""
        _check(_lib.tn_contract_slices_host(self._h, ctypes.c_int64(int(begin)), ctypes.c_int64(int(end)),
                                            _host_ptr(h_data), int(n_qubits), _host_ptr(h_amp),
                                            _host_ptr(h_stats), _stream_ptr(stream)), "tn_contract_slices_host")

    def update_data(self, data_f32, stream=None):
        """Async H2D copy of new leaf values (flat interleaved complex64, host)."""
        if hasattr(data_f32, "data_ptr"):
            ptr = _vp(data_f32.data_ptr())
        else:
            ptr = data_f32.ctypes.data_as(_vp)
        _check(_lib.tn_plan_update_data(self._h, ptr, _stream_ptr(stream)), "tn_plan_update_data")

    def profile(self, reset=False, max_rows=4096):
        """Per-op timing rows of the step-timing recorder (profile mode)."""
        rows = np.zeros(12 * max_rows)
        n = _lib.tn_plan_profile(self._h, max_rows, _ptr(rows), 1 if reset else 0)
        if n < 0:
            raise TNError(n, "tn_plan_profile")
        out = []
        for i in range(n):
            r = rows[12 * i:12 * i + 12]
            out.append(dict(phase=int(r[0]), index=int(r[1]), kind=PROFILE_KINDS[int(r[2])], step=int(r[3]),
                            ms=float(r[4]), launches=int(r[5]), macs=float(r[6]), bytes=float(r[7]),
                            shape=[float(x) for x in r[8:12]]))
        return out

    def autotune(self, reps=3, stream=None):
        """tn_plan_autotune: pick each tensor-core GEMM's (chunk, read-out) by timing."""
        _check(_lib.tn_plan_autotune(self._h, int(reps), _stream_ptr(stream)), "tn_plan_autotune")

    def op_features(self, max_ops=4096):
        """Step features (rows of 16) in the order of profile() rows without
        the extraction and FP64-sum rows."""
        out = np.zeros(COST_FEATURES * max_ops, dtype=np.float32)
        n = _lib.tn_plan_op_features(self._h, _ptr(out), max_ops)
        if n < 0:
            raise TNError(n, "tn_plan_op_features")
        return out[:COST_FEATURES * n].reshape(n, COST_FEATURES)

    def describe(self):
        """tn_plan_describe: one line per compiled op (kind, shape, kernel variant)."""
        n = _lib.tn_plan_describe(self._h, None, 0)
        if n < 0:
            raise TNError(n, "tn_plan_describe")
        buf = ctypes.create_string_buffer(n + 1)
        _lib.tn_plan_describe(self._h, buf, n + 1)
        return buf.value.decode()

    def stats(self):
        out = np.zeros(16)
        _check(_lib.tn_plan_stats(self._h, _ptr(out)), "tn_plan_stats")
        keys = ["macs_batch", "slices_per_batch", "arena_bytes", "n_steps", "launches_batch", "bytes_batch",
                "macs_prologue", "bytes_prologue", "launches_prologue", "batch_log2", "graph_replays"]
        return {k: float(out[i]) for i, k in enumerate(keys)}

    def close(self):
        if getattr(self, "_h", None):
            _lib.tn_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def amplitudes(circuit, fixed_bits, open_qubits, d_amp, form="fp32", search=None, opts=None, stream=None):
    """tn_amplitudes: overwrite d_amp (device complex128, 2^k) with the circuit's amplitudes."""
    c, keep = marshal_circuit(circuit)
    fb = np.asarray(fixed_bits, dtype=np.uint8)
    oq = np.asarray(list(open_qubits) or [0], dtype=np.int32)
    f = FORMS[form] if isinstance(form, str) else int(form)
    so = search if search is not None else search_opts()
    po = opts if opts is not None else plan_opts()
    _check(_lib.tn_amplitudes(ctypes.byref(c), _ptr(fb), len(open_qubits), _ptr(oq), f, ctypes.byref(so),
                              ctypes.byref(po), _dev_ptr(d_amp), _stream_ptr(stream)), "tn_amplitudes")


def probabilities_xeb(d_amp, n_open, n_qubits, d_prob=None, d_out=None, stream=None, sync=True):
    """(marginal P(s1), linear XEB, max p) of a device amplitude tensor; fills d_prob if given.
    With sync=False only enqueues the work and returns None (results in d_out)."""
    import torch
    if d_out is None:
        d_out = torch.zeros(3, dtype=torch.float64, device=d_amp.device)
    out = np.zeros(3) if sync else None
    _check(_lib.tn_probabilities_xeb(_dev_ptr(d_amp), n_open, n_qubits,
                                     _dev_ptr(d_prob) if d_prob is not None else None, _dev_ptr(d_out),
                                     _ptr(out), _stream_ptr(stream)), "tn_probabilities_xeb")
    if not sync:
        return None
    return float(out[0]), float(out[1]), float(out[2])


def postselect_xeb(d_amp, n_open, n_qubits, counts, d_order=None, stream=None):
    """tn_postselect_xeb: XEB of the N most probable bitstrings for each N in
    counts (sorted on the device); fills d_order (device int64) if given."""
    cnt = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    out = np.zeros(max(len(cnt), 1))
    _check(_lib.tn_postselect_xeb(_dev_ptr(d_amp), int(n_open), int(n_qubits), len(cnt),
                                  _ptr(cnt) if len(cnt) else None, _ptr(out),
                                  _dev_ptr(d_order) if d_order is not None else None, _stream_ptr(stream)),
           "tn_postselect_xeb")
    return out[:len(cnt)]


def conditional_sample(d_amp, n_open, d_u, d_out, stream=None):
    """tn_conditional_sample: d_out[j] = amplitude index drawn from P(s2|s1)
    by inverse transform of the uniform d_u[j] (device arrays)."""
    _check(_lib.tn_conditional_sample(_dev_ptr(d_amp), int(n_open), int(d_u.numel()), _dev_ptr(d_u),
                                      _dev_ptr(d_out), _stream_ptr(stream)), "tn_conditional_sample")


def probability_histogram(d_amp, n_open, scale, n_bins, x_max, d_counts, stream=None):
    """tn_probability_histogram: counts of p * scale in n_bins bins of [0, x_max)
    plus an overflow bin (device int64 d_counts[n_bins + 1])."""
    _check(_lib.tn_probability_histogram(_dev_ptr(d_amp), int(n_open), float(scale), int(n_bins), float(x_max),
                                         _dev_ptr(d_counts), _stream_ptr(stream)), "tn_probability_histogram")


def gemm_split_noalloc(d_a, d_b, d_c, m, n, k, form="tf32x3", stream=None):
    """tn_gemm_split_noalloc: C = A B (complex64, row-major device buffers) on the
    tensor cores with the library's fixed scratch array, no device allocation.
    For callers that may not allocate (an allocator owned elsewhere, real-time
    loops); calls that overlap on the GPU share the scratch and race."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    _check(_lib.tn_gemm_split_noalloc(_dev_ptr(d_a), _dev_ptr(d_b), _dev_ptr(d_c), int(m), int(n), int(k), f,
                                      _stream_ptr(stream)), "tn_gemm_split_noalloc")


class CostModel:
    """Learned step-cost model (tn_costmodel_*): predicts log2 of a step's
    device time in ms from its 16 features; trained on the GPU by the
    library's own forward/backward/Adam kernels."""

    def __init__(self, seed=1):
        h = _vp()
        _check(_lib.tn_costmodel_create(ctypes.byref(h), seed), "tn_costmodel_create")
        self._h = h
        n = ctypes.c_int()
        _check(_lib.tn_costmodel_params(self._h, None, None, ctypes.byref(n)), "tn_costmodel_params")
        self.n_params = n.value

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib.tn_costmodel_params(self._h, _ptr(out), None, None), "tn_costmodel_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.tn_costmodel_params(self._h, None, _ptr(p), None), "tn_costmodel_params")

    def grad(self, d_x, d_t, d_grad=None, stream=None):
        """(loss, device gradient) of the mean squared error on device data."""
        loss = ctypes.c_double()
        n = d_t.numel()
        _check(_lib.tn_costmodel_grad(self._h, _dev_ptr(d_x), _dev_ptr(d_t), n,
                                      _dev_ptr(d_grad) if d_grad is not None else None, ctypes.byref(loss),
                                      _stream_ptr(stream)), "tn_costmodel_grad")
        return loss.value

    def train(self, d_x, d_t, epochs=500, lr=1e-3, stream=None):
        loss = ctypes.c_double()
        _check(_lib.tn_costmodel_train(self._h, _dev_ptr(d_x), _dev_ptr(d_t), d_t.numel(), int(epochs), float(lr),
                                       ctypes.byref(loss), _stream_ptr(stream)), "tn_costmodel_train")
        return loss.value

    def predict(self, d_x, d_y, stream=None):
        _check(_lib.tn_costmodel_predict(self._h, _dev_ptr(d_x), _dev_ptr(d_y), d_y.numel(), _stream_ptr(stream)),
               "tn_costmodel_predict")

    def close(self):
        if getattr(self, "_h", None):
            _lib.tn_costmodel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """tn_batch_*: many independent plans run together (one CUDA graph after the
    first run); run() overwrites each plan's amplitude tensor."""

    def __init__(self, plans, amps, n_streams=4):
        self._plans = list(plans)  # keep alive
        self._amps = list(amps)
        hp = (_vp * len(plans))(*[p._h for p in plans])
        ha = (_vp * len(amps))(*[a.data_ptr() for a in amps])
        h = _vp()
        _check(_lib.tn_batch_create(ctypes.byref(h), len(plans), ctypes.cast(hp, _vp), ctypes.cast(ha, _vp),
                                    int(n_streams)), "tn_batch_create")
        self._h = h

    def run(self, stream=None):
        _check(_lib.tn_batch_run(self._h, _stream_ptr(stream)), "tn_batch_run")

    def close(self):
        if getattr(self, "_h", None):
            _lib.tn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
