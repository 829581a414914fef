"""CPU FP64 oracle for the sliced big-head contraction (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA path
(the ``paper_2103_03074_gb300`` package) and imports nothing from it; both
sides take their seeded inputs from ``tn_inputs``.

Routes (each function cites the passage of the paper it follows):

* ``statevector``  - Schroedinger simulation: apply the gates in circuit order
  to |0...0> and read amplitudes <s1; s2|U|0> (the definition of the
  amplitudes the method computes, "Big-head simulation" section).
* ``network``      - circuit -> tensor network with one tensor per gate plus
  boundary vectors, bonds named by the wire-segment convention of
  ``tn_inputs.networks`` (the circuit-as-tensor-network picture of Fig. 1).
* ``contract``     - plain pairwise contraction (numpy tensordot per pair) with
  sliced labels fixed at the leaves, and the sum over all slices ("Dynamic
  slicing" appendix paragraph).
* ``bruteforce``   - the contraction as an explicit sum over every label
  assignment, and the circuit as a product of full 2^n x 2^n matrices; used
  only on tiny inputs to pin the routes above.
* ``xeb``          - probabilities, linear XEB (Eq. 1), marginal and
  conditional probabilities (appendix on conditional probabilities).
* ``mlp``          - float64 forward/backward of the learned step-cost MLP
  (not a step of the paper's method; checks the GPU training kernels).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from . import statevector, network, contract, bruteforce, xeb, mlp  # noqa: F401
