"""Sharding of the sliced contraction over ranks (one process per GPU).

Slices are independent subtasks ("Dynamic slicing" appendix paragraph), so a
circuit's slice ids split into contiguous ranges, one per rank, and a batch
of circuits splits by whole circuits.  The only exchange is one sum of the
per-rank partial amplitude tensors (complex128, 2^n_open entries), done on
the host over a CPU process group (gloo): no GPU collective on the data path.
"""
from __future__ import annotations

import numpy as np


def slice_range(n_slices: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice ids [begin, end) of `rank`; the first n_slices % world
    ranks take one more slice, so the ranges tile [0, n_slices) in order."""
    if world < 1 or not 0 <= rank < world or n_slices < 0:
        raise ValueError("need 0 <= rank < world and n_slices >= 0")
    q, r = divmod(n_slices, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def assign_circuits(costs, world: int) -> list[list[int]]:
    """Whole circuits per rank, longest first onto the least loaded rank
    (ties to the lower rank); returns each rank's circuit indices, ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-float(costs[j]), j)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(x) for x in out]


def host_sum(partial, group=None) -> np.ndarray:
    """Sum of every rank's partial amplitude tensor (complex128 numpy array of
    the same shape on every rank), on the host over the CPU process group
    `group` (default: the default group, which must use the gloo backend)."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(np.asarray(partial, dtype=np.complex128))
    t = torch.from_numpy(a.view(np.float64).copy())
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy().view(np.complex128).reshape(a.shape)


def sharded_contract(plan, d_amp, rank: int, world: int, group=None, stream=None) -> np.ndarray:
    """Contract this rank's slice range of `plan` into the device complex128
    buffer d_amp (zeroed first), then sum the partials of all ranks on the
    host.  Returns the full amplitude tensor (complex128, host) on every rank."""
    import torch
    b, e = slice_range(1 << plan.n_sliced, rank, world)
    d_amp.zero_()
    plan.contract(b, e, d_amp, stream)
    torch.cuda.synchronize()
    a = d_amp.cpu().numpy()
    return host_sum(a[0::2] + 1j * a[1::2], group)
