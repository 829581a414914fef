"""Probabilities, linear XEB, marginal and conditional probabilities in FP64
(oracle, test infrastructure only).

* P(s) = |psi(s)|^2.
* Linear XEB (Eq. 1): F = (2^n / L) * sum_i P(s_i) - 1 over L bitstrings.
* Marginal and conditional (appendix "Distribution of conditional
  probabilities"): P(s1) = sum_{s2} P(s1; s2), P(s2|s1) = P(s1; s2) / P(s1).
  With the L = 2^k strings of one s1, F = 2^(n-k) P(s1) - 1 (the appendix's
  "P(s1) is XEB + 1", read with the 2^{n1} factor it leaves out).
"""
from __future__ import annotations

import numpy as np


def probabilities(amp: np.ndarray) -> np.ndarray:
    a = np.asarray(amp, dtype=np.complex128).reshape(-1)
    return a.real * a.real + a.imag * a.imag


def linear_xeb(amp: np.ndarray, n_qubits: int) -> float:
    p = probabilities(amp)
    return float((2.0 ** n_qubits) / p.size * p.sum() - 1.0)


def marginal(amp: np.ndarray) -> float:
    return float(probabilities(amp).sum())


def conditional(amp: np.ndarray) -> np.ndarray:
    p = probabilities(amp)
    return p / p.sum()


def postselect_xeb(amp: np.ndarray, n_qubits: int, counts) -> np.ndarray:
    """Post-selection ("Fidelity" paragraph and Fig. 2, right): sort the
    probabilities in decreasing order and, for each N in counts, apply Eq. 1
    to the N most probable bitstrings: F = 2^n / N * (sum of the N largest
    p) - 1."""
    p = np.sort(probabilities(amp))[::-1]
    c = np.cumsum(p)
    return np.array([(2.0 ** n_qubits) / N * c[N - 1] - 1.0 for N in counts])


def conditional_sample(amp: np.ndarray, u) -> np.ndarray:
    """Draws from P(s2|s1) = P(s1; s2) / P(s1) by inverse transform: with the
    cumulative probabilities c_i in index order and P(s1) = c_last, sample j
    is the smallest i with c_i > u_j * P(s1)."""
    c = np.cumsum(probabilities(amp))
    total = c[-1]
    out = np.searchsorted(c, np.asarray(u, dtype=np.float64) * total, side="right")
    return np.minimum(out, c.size - 1).astype(np.int64)


def sample_margins(amp: np.ndarray, u) -> np.ndarray:
    """Distance of each threshold u_j * P(s1) to the nearest cumulative
    probability, relative to P(s1): where it is tiny, summation order alone
    may move a sample to the neighbouring index."""
    c = np.cumsum(probabilities(amp))
    t = np.asarray(u, dtype=np.float64) * c[-1]
    i = np.clip(np.searchsorted(c, t), 0, c.size - 1)
    d = np.abs(c[i] - t)
    d = np.minimum(d, np.abs(c[np.maximum(i - 1, 0)] - t))
    return d / c[-1]


def histogram(amp: np.ndarray, scale: float, n_bins: int, x_max: float) -> np.ndarray:
    """Counts of x = p * scale in n_bins equal bins of [0, x_max) plus an
    overflow bin (the histograms of Fig. 2, left, and Fig. 5): bin
    floor(x / (x_max / n_bins)), clamped to n_bins - 1 below x_max."""
    x = probabilities(amp) * scale
    width = x_max / n_bins
    b = np.where(x < x_max, np.minimum(np.floor(x / width), n_bins - 1), n_bins).astype(np.int64)
    return np.bincount(b, minlength=n_bins + 1)
