"""GPU parity of post-selection, conditional sampling and the probability
histogram (tn_postselect_xeb, tn_conditional_sample,
tn_probability_histogram) against the FP64 oracle on the same amplitudes.

* Probabilities are re^2 + im^2 with separately rounded products on both
  sides, so sorted probabilities and histogram bins are compared exactly.
* XEB of the top-N bitstrings: the prefix sums are taken in a different
  order, so F + 1 agrees to 1e-12 relative.
* Samples: the cumulative sums are taken in a different order too, so a
  sample may move to the neighbouring index only where its threshold lies
  within 1e-12 of a cumulative probability; every other sample is compared
  exactly (and the excluded ones are counted).
Inputs: seeded complex normal amplitudes (Porter-Thomas probabilities) of
sizes around the shared-memory sort chunk (2^11) and the paper's 2^21 head,
plus the 30-qubit workload's amplitudes computed by the contraction itself.
"""
import os
import time

import numpy as np
import pytest

from tn_inputs.configs import make_config
from oracle import xeb as ox

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


def amplitudes(k, n_qubits, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(1 << k) + 1j * rng.standard_normal(1 << k)
    return a / np.sqrt(2.0 * 2.0 ** n_qubits)


def to_device(a):
    import torch
    v = np.empty(2 * a.size)
    v[0::2], v[1::2] = a.real, a.imag
    return torch.from_numpy(v).cuda()


def counts_for(k):
    L = 1 << k
    return sorted(c for c in {1, 2, 3, 10, 1000, L // 3, L // 2, L - 1, L} if 1 <= c <= L)


def check_postselect(tn, a, k, n_qubits):
    import torch
    d = to_device(a)
    order = torch.empty(1 << k, dtype=torch.int64, device="cuda")
    cnt = counts_for(k)
    got = tn.postselect_xeb(d, k, n_qubits, cnt, d_order=order)
    want = ox.postselect_xeb(a, n_qubits, cnt)
    assert np.all(np.abs((got + 1) - (want + 1)) <= 1e-12 * np.abs(want + 1))
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(1 << k))  # a permutation
    p = ox.probabilities(a)
    # probabilities along the order are exactly the oracle's sorted ones
    assert np.array_equal(p[o], np.sort(p)[::-1])
    return got


@pytest.mark.parametrize("k", [0, 1, 5, 10, 11, 12, 15])
def test_postselect_sizes(tn, k):
    check_postselect(tn, amplitudes(k, k + 7, 100 + k), k, k + 7)


def test_postselect_head_of_2_21(tn):
    """The paper's head size: 2^21 amplitudes of a 53-qubit circuit."""
    import torch
    k, n = 21, 53
    a = amplitudes(k, n, 7)
    got = check_postselect(tn, a, k, n)
    d = to_device(a)
    cnt = [10 ** 6]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        tn.postselect_xeb(d, k, n, cnt)
    dt = (time.perf_counter() - t0) / 5
    print(f"post-selection of 2^21 probabilities (sort + XEB of the top 10^6): {dt * 1e3:.2f} ms per call; "
          f"XEB all {got[-1]:+.4f}, top 10^6 {tn.postselect_xeb(d, k, n, cnt)[0]:+.4f}")


def test_postselect_on_contracted_amplitudes(tn):
    """The 30-qubit workload's 256 amplitudes from the contraction itself."""
    import torch
    cfg = make_config(2)
    amp = torch.zeros(2 << 8, dtype=torch.float64, device="cuda")
    tn.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"], amp, form="tf32x3",
                  search=tn.search_opts(trials=1024, n_sliced=8))
    torch.cuda.synchronize()
    v = amp.cpu().numpy()
    a = v[0::2] + 1j * v[1::2]
    got = check_postselect(tn, a, 8, 30)
    # the full set is Eq. 1 over the head, as tn_probabilities_xeb gives it
    _, f, _ = tn.probabilities_xeb(amp, 8, 30)
    assert abs(got[-1] - f) < 1e-12 * abs(f + 1)


@pytest.mark.parametrize("k", [0, 3, 11, 12, 21])
def test_conditional_sample(tn, k):
    import torch
    a = amplitudes(k, k + 10, 200 + k)
    d = to_device(a)
    u = np.random.default_rng(300 + k).random(100000)
    du = torch.from_numpy(u).cuda()
    out = torch.empty(u.size, dtype=torch.int64, device="cuda")
    tn.conditional_sample(d, k, du, out)
    got = out.cpu().numpy()
    want = ox.conditional_sample(a, u)
    safe = ox.sample_margins(a, u) > 1e-12
    assert np.array_equal(got[safe], want[safe])
    assert np.all(np.abs(got[~safe] - want[~safe]) <= 1)
    assert safe.sum() >= u.size - 10


@pytest.mark.parametrize("k,n_bins,x_max", [(0, 4, 2.0), (12, 50, 10.0), (21, 200, 12.0)])
def test_histogram(tn, k, n_bins, x_max):
    import torch
    n = k + 32
    a = amplitudes(k, n, 400 + k)
    d = to_device(a)
    cnt = torch.empty(n_bins + 1, dtype=torch.int64, device="cuda")
    tn.probability_histogram(d, k, 2.0 ** n, n_bins, x_max, cnt)  # Fig. 2 (left): 2^n p
    assert np.array_equal(cnt.cpu().numpy(), ox.histogram(a, 2.0 ** n, n_bins, x_max))
    # Fig. 5: the conditional probabilities times L, which sum to L
    ps1 = ox.marginal(a)
    tn.probability_histogram(d, k, (1 << k) / ps1, n_bins, x_max, cnt)
    assert np.array_equal(cnt.cpu().numpy(), ox.histogram(a, (1 << k) / ps1, n_bins, x_max))


def test_rejects_bad_arguments(tn):
    import torch
    d = to_device(amplitudes(4, 10, 1))
    with pytest.raises(tn.TNError):
        tn.postselect_xeb(d, 4, 10, [0])
    with pytest.raises(tn.TNError):
        tn.postselect_xeb(d, 4, 10, [17])
    cnt = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(tn.TNError):
        tn.probability_histogram(d, 4, 1.0, 0, 1.0, cnt)
