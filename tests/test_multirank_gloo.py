"""The N > 1 path on CPU: slice ranges per rank, circuits per rank, and the
host-side sum of partial amplitude tensors over a 2-rank gloo group.  The
partials are the FP64 oracle's own slice contractions, so the check is that
sharding plus the host sum reproduces the unsliced amplitudes; bench's
max-over-ranks timing is checked the same way."""
import os
import socket

import numpy as np
import pytest

from paper_2103_03074_gb300.shard import assign_circuits, host_sum, slice_range


def test_slice_ranges_tile_in_order():
    for n in (0, 1, 5, 256, 1000):
        for world in (1, 2, 3, 8):
            got = [slice_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (b0, e0), (b1, e1) in zip(got, got[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_range(4, 2, 2)


def test_assign_circuits_longest_first():
    costs = [5, 1, 4, 3, 3, 2]
    parts = assign_circuits(costs, 2)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert loads == [9, 9]                       # 5+3+1 | 4+3+2
    assert assign_circuits([], 3) == [[], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import contract as oc, network as onet
        from tn_inputs.configs import make_config
        import bench
        cfg = make_config(1)
        L, T, O = onet.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"][:6])
        count = {}
        for lab in L:
            for x in lab:
                count[x] = count.get(x, 0) + 1
        internal = sorted(x for x, c in count.items() if c == 2)
        sliced = internal[5:8]                    # three internal bonds: 8 slices
        b, e = slice_range(1 << len(sliced), rank, world)
        part = oc.sliced_sum(L, T, O, sliced, b, e)
        total = host_sum(part)
        np.save(os.path.join(outdir, f"total{rank}.npy"), total)
        np.save(os.path.join(outdir, f"part{rank}.npy"), part)
        m = bench.max_over_ranks(float(10 + rank), world)
        np.save(os.path.join(outdir, f"max{rank}.npy"), np.array([m]))
    finally:
        dist.destroy_process_group()


def test_two_rank_host_sum_matches_unsliced(tmp_path):
    import torch.multiprocessing as mp
    from oracle import contract as oc, network as onet
    from tn_inputs.configs import make_config
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    cfg = make_config(1)
    L, T, O = onet.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"][:6])
    ref = oc.contract(L, T, O)
    t0, t1 = np.load(tmp_path / "total0.npy"), np.load(tmp_path / "total1.npy")
    p0, p1 = np.load(tmp_path / "part0.npy"), np.load(tmp_path / "part1.npy")
    assert np.array_equal(t0, t1)                 # every rank holds the same sum
    assert np.allclose(t0, p0 + p1, rtol=0, atol=1e-15)
    assert np.linalg.norm(t0 - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(p0) > 0 and np.linalg.norm(p1) > 0
    assert float(np.load(tmp_path / "max0.npy")[0]) == 11.0
    assert float(np.load(tmp_path / "max1.npy")[0]) == 11.0
