"""Pins of the oracle's post-selection, conditional sampling and histogram
(no GPU): hand-computed cases with exactly representable probabilities, the
identities that tie them to Eq. 1, and a Porter-Thomas sanity check."""
import math

import numpy as np

from oracle import xeb as ox

# probabilities 1/16, 1/4, 1/16, 9/16 (exact in FP64), total 15/16
AMP = np.array([0.25, 0.5, 0.25j, 0.75])


def test_postselect_hand_computed():
    # sorted: 9/16, 1/4, 1/16, 1/16; n = 2 qubits -> 2^n = 4
    f = ox.postselect_xeb(AMP, 2, [1, 2, 3, 4])
    want = [4 * 9 / 16 - 1, 4 * (9 / 16 + 1 / 4) / 2 - 1, 4 * (14 / 16) / 3 - 1, 4 * (15 / 16) / 4 - 1]
    assert np.allclose(f, want, rtol=0, atol=1e-15)


def test_postselect_identities():
    rng = np.random.default_rng(5)
    a = (rng.standard_normal(4096) + 1j * rng.standard_normal(4096)) / math.sqrt(2 * 2 ** 20)
    n = 20
    f = ox.postselect_xeb(a, n, [1, 7, 100, 4096])
    # all bitstrings: Eq. 1 itself; one bitstring: 2^n p_max - 1
    assert abs(f[-1] - ox.linear_xeb(a, n)) < 1e-12
    assert abs(f[0] - (2.0 ** n * ox.probabilities(a).max() - 1)) < 1e-12
    # more bitstrings can only lower the mean probability
    assert np.all(np.diff(f) <= 1e-12)


def test_postselect_porter_thomas_sanity():
    # p = e / 2^n with e ~ Exp(1): the top fraction q has mean 1 + ln(1/q),
    # so its XEB is close to ln(1/q) (a sanity check of the sort direction)
    rng = np.random.default_rng(6)
    L, n = 1 << 16, 30
    e = rng.exponential(size=L)
    a = np.sqrt(e / 2.0 ** n).astype(np.complex128)
    for q in (0.5, 0.1, 0.01):
        f = ox.postselect_xeb(a, n, [int(q * L)])[0]
        # the tail above the q-quantile is Exp(1)-shaped: its mean has a
        # standard error of about 1 / sqrt(q L); allow four of them
        assert abs(f - math.log(1 / q)) < 4 / math.sqrt(q * L) + 0.01


def test_conditional_sample_hand_computed():
    # cumulative 1/16, 5/16, 6/16, 15/16; thresholds u * 15/16
    u = [0.05, 0.2, 0.32, 0.35, 0.5, 1 / 15, 0.9999]
    assert list(ox.conditional_sample(AMP, u)) == [0, 1, 1, 2, 3, 1, 3]


def test_conditional_sample_frequencies():
    rng = np.random.default_rng(7)
    u = rng.random(200000)
    s = ox.conditional_sample(AMP, u)
    freq = np.bincount(s, minlength=4) / s.size
    assert np.allclose(freq, ox.conditional(AMP), atol=0.005)


def test_histogram_hand_computed():
    # x = 4 p = 1/4, 1, 1/4, 9/4 in 4 bins of width 1/2 below 2
    assert list(ox.histogram(AMP, 4.0, 4, 2.0)) == [2, 0, 1, 0, 1]
