"""GPU: small steps on the tensor cores with T split in shared memory.

A small step C[r, n] = sum_k T[r, k] S[k, n] of a split form (K and N of 16
or 32 values, at least 2^16 rows, the rows' 7 lowest bits lowest in T and C)
runs on the tensor cores: T is split into hi/lo pieces tile by tile in shared
memory (FP16X3: every 128-row tile scaled by its own power of two), S once
per CTA, with the form's three piece products and FP32 read-out.  Expected
values are the FP64 oracle's pairwise contraction of the same two tensors.
Tolerances: relative L2 <= 1e-5 for FP16X3 and TF32x3 (22 significant bits
per operand piece pair, the bound the workload states), 1e-4 for BF16x3 (16
bits; see test_gpu_parity.py); the CUDA-core path (small_tc -1) of the same
step in the same form meets the same bounds.
"""
import numpy as np
import pytest

from oracle import contract as oc
from tn_inputs import SplitMix64

pytestmark = pytest.mark.gpu
BOUND = {"fp16x3": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-4}


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
    return float(np.linalg.norm(np.asarray(a).ravel() - np.asarray(b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def rows_of(r, kpos):
    """Row index of every element of a rank-r T: the element index with the
    K bits (positions kpos) removed."""
    e = np.arange(2 ** r, dtype=np.int64)
    row = np.zeros_like(e)
    out_bit = 0
    for p in range(r):
        if p in kpos:
            continue
        row |= ((e >> p) & 1) << out_bit
        out_bit += 1
    return row


def step_network(row_bits, kpos, n_bits, seed, tile_scales=False, lead_scalar=False):
    """Labels and complex64 data of T (rank row_bits + len(kpos), its K labels
    at the bit positions kpos, counted from the lowest) and S [K][N]; with
    tile_scales every 128-row tile of T is multiplied by its own power of two
    in [2^-24, 2^24]; with lead_scalar a rank-0 leaf comes first, so that T
    starts at an odd element offset of the leaf buffer."""
    nk = len(kpos)
    r = row_bits + nk
    pos_label = list(range(1000, 1000 + r))
    klab = list(range(2000, 2000 + nk))
    for j, p in enumerate(kpos):
        pos_label[p] = klab[j]
    T_labels = list(reversed(pos_label))  # first label = most significant
    nlab = list(range(3000, 3000 + n_bits))
    rng = np.random.default_rng(seed)
    T = (rng.standard_normal(2 ** r) + 1j * rng.standard_normal(2 ** r)).astype(np.complex64)
    if tile_scales:
        row = rows_of(r, kpos)
        sm = SplitMix64(seed)
        n_tiles = 2 ** row_bits // 128
        exps = np.array([sm.below(49) - 24 for _ in range(n_tiles)], dtype=np.float64)
        T = (T * np.exp2(exps[row >> 7])).astype(np.complex64)
    S = (rng.standard_normal(2 ** (nk + n_bits)) + 1j * rng.standard_normal(2 ** (nk + n_bits))).astype(np.complex64)
    labels = [T_labels, klab + nlab]
    data = [T.reshape((2,) * r), S.reshape((2,) * (nk + n_bits))]
    out = [x for x in T_labels if x not in klab] + nlab
    if lead_scalar:
        labels = [[]] + labels
        data = [np.array(1.0 + 0.0j, dtype=np.complex64).reshape(())] + data
    return labels, data, out


def run(tn, labels, data, out, tree, form, **opts):
    import torch
    plan = tn.Plan(labels, data, out, [], tree, form=form, opts=tn.plan_opts(**opts))
    desc = plan.describe()
    amp = torch.zeros(2 << len(out), dtype=torch.float64, device="cuda")
    plan.contract(0, 1, amp)
    torch.cuda.synchronize()
    a = amp.cpu().numpy()
    plan.close()
    return a[0::2] + 1j * a[1::2], desc


@pytest.mark.parametrize("form", ["fp16x3", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("kpos,n_bits", [((7, 9, 12, 15), 5), ((8, 15, 17, 19, 20), 5), ((10, 11, 12, 13), 4),
                                         ((7, 8, 9, 10, 16), 4), ((8, 15, 17, 19, 20), 3), ((9, 10, 14, 16), 3)])
def test_small_step_on_tensor_cores(tn, form, kpos, n_bits):
    row_bits = 17
    labels, data, out = step_network(row_bits, kpos, n_bits, seed=len(kpos) * 10 + n_bits)
    ref = oc.contract(labels, data, out, tree=[(0, 1)])
    got, desc = run(tn, labels, data, out, [(0, 1)], form)
    assert "tensor cores, split in shared memory" in desc
    cc, desc_cc = run(tn, labels, data, out, [(0, 1)], form, small_tc=-1)
    assert "tensor cores" not in desc_cc
    e, e_cc = rel(got, ref), rel(cc, ref)
    print(f"{form} K bits {kpos} N 2^{n_bits}: tensor cores {e:.2e}, CUDA cores {e_cc:.2e}")
    assert e < BOUND[form] and e_cc < BOUND[form]


@pytest.mark.parametrize("form", ["fp16x3", "tf32x3"])
def test_small_step_tile_scales(tn, form):
    """Tiles of T spanning 2^-24 .. 2^24 (FP16X3 scales each tile by its own
    power of two; a single scale for all of T would push the small tiles'
    pieces below fp16's range): element-wise against the FP64 oracle."""
    labels, data, out = step_network(18, (8, 10, 14, 16, 19), 5, seed=7, tile_scales=True)
    ref = oc.contract(labels, data, out, tree=[(0, 1)])
    got, desc = run(tn, labels, data, out, [(0, 1)], form)
    assert "tensor cores" in desc
    # relative to each element's own row scale: compare row by row
    ref2 = ref.reshape(-1, 32)
    got2 = got.reshape(-1, 32)
    err = np.linalg.norm(got2 - ref2, axis=1) / np.maximum(np.linalg.norm(ref2, axis=1), 1e-300)
    print(f"{form} per-tile scales: worst row {err.max():.2e}")
    assert err.max() < 1e-5


def test_small_step_zero_tiles_and_misaligned_leaf(tn):
    """A T whose first tiles are all zero (the tile scale of a zero tile) and
    a T that starts at an odd element offset (16-byte copies need alignment:
    the step then runs on the CUDA cores, same result)."""
    kpos = (7, 9, 12, 15)
    labels, data, out = step_network(17, kpos, 5, seed=3)
    T = data[0].reshape(-1).copy()
    T[rows_of(21, kpos) < 8 * 128] = 0  # the first eight 128-row tiles, every k
    data = [T.reshape(data[0].shape), data[1]]
    ref = oc.contract(labels, data, out, tree=[(0, 1)])
    got, desc = run(tn, labels, data, out, [(0, 1)], "fp16x3")
    assert "tensor cores" in desc and rel(got, ref) < 1e-5
    labels2, data2, out2 = step_network(17, kpos, 5, seed=3, lead_scalar=True)
    data2[1] = data[0]
    tree = [(1, 2), (0, 3)]
    ref2 = oc.contract(labels2, data2, out2, tree=tree)
    got2, _ = run(tn, labels2, data2, out2, tree, "fp16x3")
    assert rel(got2, ref2) < 1e-5
