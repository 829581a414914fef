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
