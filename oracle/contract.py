"""Plain pairwise tensor-network contraction with slicing (oracle, test
infrastructure only).

* A contraction sums, over every internal label, the product of the tensor
  entries (the tensor-network picture of Fig. 1).  Here it is done pair by pair
  with numpy.tensordot as the library step (Fig. 3: a pair A, B shares n_AB
  labels; the result keeps the n_A + n_B outer labels).
* Slicing ("Dynamic slicing" paragraph of the appendix): a set of n_e labels is
  fixed; slice id s gives sliced label j the value bit j of s; the full
  contraction equals the sum of the 2^{n_e} sliced contractions.  A sliced
  label is fixed at the leaves (each tensor holding it is indexed at the value).

Labels are ints; every label appears in at most two tensors.  A label held by
one tensor and not open is summed over.  The pair order is the oracle's own
(greedy on result size, or a caller-given SSA tree); the order changes
rounding only.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def fix_labels(labels: Sequence[Sequence[int]], tensors: Sequence[np.ndarray],
               fixed: Dict[int, int]):
    """Index every tensor at the fixed labels; returns new (labels, tensors)."""
    out_l, out_t = [], []
    for labs, t in zip(labels, tensors):
        t = np.asarray(t, dtype=np.complex128)
        labs = list(labs)
        idx = []
        keep = []
        for a, lab in enumerate(labs):
            if lab in fixed:
                idx.append(int(fixed[lab]))
            else:
                idx.append(slice(None))
                keep.append(lab)
        out_t.append(t[tuple(idx)] if idx else t)
        out_l.append(keep)
    return out_l, out_t


def greedy_order(label_lists: Sequence[Sequence[int]], open_labels: Sequence[int]) -> List[Tuple[int, int]]:
    """SSA pair list: repeatedly merge the connected pair whose result grows
    the stored size least (2^|out| - 2^|a| - 2^|b|); ties by smallest ids.
    Disconnected parts are joined smallest-first at the end."""
    open_set = set(open_labels)
    live: Dict[int, frozenset] = {i: frozenset(l) for i, l in enumerate(label_lists)}
    holders: Dict[int, set] = {}
    for i, l in live.items():
        for lab in l:
            holders.setdefault(lab, set()).add(i)
    nxt = len(label_lists)
    steps = []

    def result_labels(a, b):
        la, lb = live[a], live[b]
        out = set()
        for lab in la | lb:
            h = holders[lab]
            inside = (lab in la) + (lab in lb)
            if lab in open_set or len(h) > inside:
                out.add(lab)
        return frozenset(out)

    while len(live) > 1:
        best = None
        seen_pairs = set()
        for lab, h in holders.items():
            if len(h) != 2:
                continue
            a, b = sorted(h)
            if (a, b) in seen_pairs:
                continue
            seen_pairs.add((a, b))
            out = result_labels(a, b)
            cost = (1 << len(out)) - (1 << len(live[a])) - (1 << len(live[b]))
            key = (cost, a, b)
            if best is None or key < best[0]:
                best = (key, a, b, out)
        if best is None:  # nothing shares a label: outer product of the two smallest
            ids = sorted(live, key=lambda i: (len(live[i]), i))
            a, b = sorted(ids[:2])
            out = result_labels(a, b)
        else:
            _, a, b, out = best
        steps.append((a, b))
        for lab in live[a] | live[b]:
            holders[lab].discard(a)
            holders[lab].discard(b)
        del live[a]
        del live[b]
        live[nxt] = out
        for lab in out:
            holders.setdefault(lab, set()).add(nxt)
        for lab in [l for l, h in holders.items() if not h]:
            del holders[lab]
        nxt += 1
    return steps


def contract(labels: Sequence[Sequence[int]], tensors: Sequence[np.ndarray],
             open_labels: Sequence[int], fixed: Optional[Dict[int, int]] = None,
             tree: Optional[Sequence[Tuple[int, int]]] = None) -> np.ndarray:
    """Contract the network (with ``fixed`` labels held at their values) and
    return a complex128 array of shape (2,)*len(open_labels), axes in the order
    of ``open_labels``."""
    it = contract_iter(labels, tensors, open_labels, fixed, tree)
    while True:
        try:
            next(it)
        except StopIteration as done:
            return done.value


def contract_iter(labels, tensors, open_labels, fixed=None, tree=None):
    """contract() as a generator: after pairwise step t it yields
    (t, per-step complex MACs of the whole tree), where a pair holding the
    labels U in total costs 2^|U| MACs (Fig. 3); its return value
    (StopIteration.value) is contract()'s result.  Lets a caller time a
    bounded part of a long contraction."""
    fixed = fixed or {}
    for lab in open_labels:
        if lab in fixed:
            raise ValueError("an open label cannot be fixed")
    labs, ts = fix_labels(labels, tensors, fixed)
    if tree is None:
        tree = greedy_order(labs, open_labels)
    open_set = set(open_labels)
    count: Dict[int, int] = {}
    for l in labs:
        for lab in l:
            count[lab] = count.get(lab, 0) + 1
    nodes: Dict[int, Tuple[List[int], np.ndarray]] = {i: (list(l), t) for i, (l, t) in enumerate(zip(labs, ts))}
    # sum dangling (held once, not open) labels right away
    for i, (l, t) in list(nodes.items()):
        dang = [a for a, lab in enumerate(l) if count[lab] == 1 and lab not in open_set]
        if dang:
            t = t.sum(axis=tuple(dang))
            l = [lab for a, lab in enumerate(l) if a not in dang]
            nodes[i] = (l, t)
    # complex MACs of every step: 2^|labels of the pair|
    sets = {i: set(l) for i, (l, _) in nodes.items()}
    step_macs = []
    nxt = len(labs)
    for (a, b) in tree:
        u = sets.pop(a) | sets.pop(b)
        step_macs.append(2.0 ** len(u))
        sets[nxt] = {lab for lab in u if lab in open_set or sum(lab in s2 for s2 in sets.values()) > 0}
        nxt += 1
    nxt = len(labs)
    for t, (a, b) in enumerate(tree):
        la, ta = nodes.pop(a)
        lb, tb = nodes.pop(b)
        shared = [lab for lab in la if lab in lb and lab not in open_set]
        ax_a = [la.index(lab) for lab in shared]
        ax_b = [lb.index(lab) for lab in shared]
        tc = np.tensordot(ta, tb, axes=(ax_a, ax_b))
        lc = [lab for lab in la if lab not in shared] + [lab for lab in lb if lab not in shared]
        nodes[nxt] = (lc, tc)
        nxt += 1
        yield t, step_macs
    # any disconnected leftovers: outer products
    items = list(nodes.values())
    lc, tc = items[0]
    for l2, t2 in items[1:]:
        tc = np.tensordot(tc, t2, axes=0)
        lc = lc + l2
    if sorted(lc) != sorted(open_labels):
        raise ValueError(f"result labels {sorted(lc)} != open labels {sorted(open_labels)}")
    perm = [lc.index(lab) for lab in open_labels]
    return np.transpose(tc, perm) if perm else tc


def slice_values(sliced_labels: Sequence[int], s: int) -> Dict[int, int]:
    """Slice id s -> {label_j: bit j of s}."""
    return {lab: (s >> j) & 1 for j, lab in enumerate(sliced_labels)}


def slice_partial(labels, tensors, open_labels, sliced_labels, s: int, tree=None) -> np.ndarray:
    """The contraction of slice s (one subtask of the sliced contraction)."""
    return contract(labels, tensors, open_labels, slice_values(sliced_labels, s), tree)


def sliced_sum(labels, tensors, open_labels, sliced_labels, begin: int = 0,
               end: Optional[int] = None, tree=None) -> np.ndarray:
    """Sum of the slice contractions for slice ids in [begin, end)."""
    if end is None:
        end = 1 << len(sliced_labels)
    acc = None
    for s in range(begin, end):
        part = slice_partial(labels, tensors, open_labels, sliced_labels, s, tree)
        acc = part if acc is None else acc + part
    if acc is None:
        acc = np.zeros((2,) * len(open_labels), dtype=np.complex128)
    return acc
