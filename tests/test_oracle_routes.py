"""Pins of the oracle's routes against closed forms, brute force and
invariants (no GPU).

* State vector: a hand-computed two-qubit circuit; the qubit-0-is-MSB bit
  order; normalisation; explicit 2^n x 2^n matrix products on <= 9 qubits;
  unitarity of the whole circuit.
* Pairwise contraction: the explicit sum over all label assignments on small
  random networks (every label order, every tree); the state vector on whole
  circuits; the slicing identity sum over slices = unsliced contraction
  ("Dynamic slicing" paragraph); slice values taken from the slice id bits.
* XEB (Eq. 1): zero over the whole space; equal to 2^(n-k) P(s1) - 1 with
  P(s1) summed independently from the full state vector.
"""
import math

import numpy as np
import pytest

from tn_inputs import Circuit, Gate, gate_matrix, random_bits, random_network, random_tree, sycamore_circuit
from tn_inputs.configs import make_config
from oracle import bruteforce, contract, network, statevector, sv_native, xeb


def test_two_qubit_closed_form():
    # sqrtX (x) sqrtX on |00> = (|00> - i|01> - i|10> - |11>)/2; then
    # fSim(pi/2, pi/6): |01> -> -i|10>, |10> -> -i|01>, |11> -> e^{-i pi/6}|11>
    # giving (|00> - |01> - |10> - e^{-i pi/6}|11>)/2.
    sx = gate_matrix("sqrtX")
    fs = gate_matrix("fsim", (math.pi / 2, math.pi / 6))
    circ = Circuit(2, [Gate("sqrtX", (0,), sx), Gate("sqrtX", (1,), sx), Gate("fsim", (0, 1), fs)])
    psi = statevector.final_state(circ).reshape(-1)
    expect = np.array([1, -1, -1, -np.exp(-1j * math.pi / 6)]) / 2
    assert np.abs(psi - expect).max() < 1e-15
    assert np.abs(bruteforce.apply_full(circ) - expect).max() < 1e-15
    assert np.abs(sv_native.amplitudes(circ, [0, 0], [0, 1]) - expect).max() < 1e-15


def test_bit_order_qubit0_is_msb():
    sx = gate_matrix("sqrtX")
    circ = Circuit(3, [Gate("sqrtX", (0,), sx), Gate("sqrtX", (0,), sx)])  # = -iX on qubit 0
    psi = statevector.final_state(circ).reshape(-1)
    assert abs(psi[4] - (-1j)) < 1e-15 and np.abs(np.delete(psi, 4)).max() < 1e-15
    # amplitudes with qubit 0 open, listed first, others fixed to 0
    a = statevector.amplitudes(circ, [0, 0, 0], [0])
    assert abs(a[1] - (-1j)) < 1e-15 and abs(a[0]) < 1e-15


def test_normalisation_all_open():
    cfg = make_config(1)
    a = statevector.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12


@pytest.mark.parametrize("rows,cols,cycles,seed", [(2, 4, 6, 1), (3, 3, 5, 2), (2, 3, 8, 3)])
def test_statevector_vs_full_matrices(rows, cols, cycles, seed):
    circ = sycamore_circuit("rect", rows, cols, cycles, seed)
    v = bruteforce.apply_full(circ)
    psi = statevector.final_state(circ).reshape(-1)
    assert np.abs(v - psi).max() < 1e-12
    n = circ.n_qubits
    c = sv_native.amplitudes(circ, [0] * n, list(range(n)))
    assert np.abs(c - psi).max() < 1e-12


def test_whole_circuit_unitary():
    circ = sycamore_circuit("rect", 2, 3, 4, 9)
    u = bruteforce.full_unitary(circ)
    assert np.abs(u.conj().T @ u - np.eye(u.shape[0])).max() < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_pairwise_contraction_vs_explicit_sum(seed):
    net = random_network(seed, n_tensors=6, n_bonds=9, n_open=3, max_rank=5)
    ref = bruteforce.network_sum(net.labels, net.data, net.open_labels)
    got = contract.contract(net.labels, net.data, net.open_labels).reshape(-1)
    assert np.abs(got - ref).max() < 1e-12 * max(1, np.abs(ref).max())
    tree = random_tree(seed + 100, len(net.labels))
    got2 = contract.contract(net.labels, net.data, net.open_labels, tree=tree).reshape(-1)
    assert np.abs(got2 - ref).max() < 1e-12 * max(1, np.abs(ref).max())
    # a permuted open order permutes the result axes
    perm = list(reversed(net.open_labels))
    got3 = contract.contract(net.labels, net.data, perm)
    assert np.abs(np.transpose(got3, (2, 1, 0)).reshape(-1) - ref).max() < 1e-12 * max(1, np.abs(ref).max())


def test_fixed_label_is_an_index():
    net = random_network(42, n_tensors=5, n_bonds=7, n_open=2, max_rank=5)
    lab = next(l for l in range(net.n_labels) if l not in net.open_labels)
    for v in (0, 1):
        got = contract.contract(net.labels, net.data, net.open_labels, fixed={lab: v}).reshape(-1)
        # explicit sum with the label held at v: replace the label by a
        # one-hot vector tensor on a fresh label pair
        labs = [list(l) for l in net.labels]
        data = list(net.data)
        e = np.zeros(2, dtype=complex)
        e[v] = 1
        fresh = net.n_labels + 10
        holders = [i for i, l in enumerate(labs) if lab in l]
        # split the bond: each holder gets its own fresh label with a one-hot vector
        for j, i in enumerate(holders):
            labs[i] = [fresh + j if x == lab else x for x in labs[i]]
            labs.append([fresh + j])
            data.append(e)
        ref = bruteforce.network_sum(labs, data, net.open_labels)
        assert np.abs(got - ref).max() < 1e-12 * max(1, np.abs(ref).max())


@pytest.mark.parametrize("idx_open", [[0, 5, 11], [11, 2, 7, 4]])
def test_network_route_vs_statevector(idx_open):
    cfg = make_config(1)
    circ = cfg["circuit"]
    bits = cfg["fixed_bits"]
    a = statevector.amplitudes(circ, bits, idx_open)
    L, T, O = network.circuit_network(circ, bits, idx_open)
    b = contract.contract(L, T, O).reshape(-1)
    assert np.abs(a - b).max() < 1e-12


def test_network_route_vs_statevector_deeper():
    circ = sycamore_circuit("rect", 4, 4, 10, 77)
    bits = random_bits(16, 5)
    open_q = [10, 11, 14, 15, 3, 6]
    a = statevector.amplitudes(circ, bits, open_q)
    L, T, O = network.circuit_network(circ, bits, open_q)
    b = contract.contract(L, T, O).reshape(-1)
    assert np.abs(a - b).max() < 1e-12


def test_slice_sum_equals_unsliced():
    cfg = make_config(1)
    circ = cfg["circuit"]
    L, T, O = network.circuit_network(circ, cfg["fixed_bits"], cfg["open_qubits"][:6])
    full = contract.contract(L, T, O)
    internal = sorted({x for l in L for x in l} - set(O))
    sliced = [internal[7], internal[40], internal[90]]
    total = contract.sliced_sum(L, T, O, sliced)
    assert np.abs(total - full).max() < 1e-12
    # each slice holds label j at bit j of the slice id
    parts = [contract.slice_partial(L, T, O, sliced, s) for s in range(8)]
    manual = contract.contract(L, T, O, fixed={sliced[0]: 1, sliced[1]: 0, sliced[2]: 1})
    assert np.abs(parts[0b101] - manual).max() < 1e-15
    # a partial range sums its slices only
    assert np.abs(contract.sliced_sum(L, T, O, sliced, 2, 5) - (parts[2] + parts[3] + parts[4])).max() < 1e-14


def test_slice_sum_random_network():
    net = random_network(7, n_tensors=10, n_bonds=16, n_open=3, max_rank=6)
    full = contract.contract(net.labels, net.data, net.open_labels)
    internal = [l for l in range(net.n_labels) if l not in net.open_labels]
    sliced = internal[1:5]
    total = contract.sliced_sum(net.labels, net.data, net.open_labels, sliced)
    assert np.abs(total - full).max() < 1e-12 * max(1, np.abs(full).max())


def test_open_label_cannot_be_sliced():
    net = random_network(3, n_tensors=4, n_bonds=5, n_open=2, max_rank=5)
    with pytest.raises(ValueError):
        contract.contract(net.labels, net.data, net.open_labels, fixed={net.open_labels[0]: 0})


def test_xeb_whole_space_is_zero():
    cfg = make_config(1)
    a = statevector.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    assert abs(xeb.linear_xeb(a, 12)) < 1e-12


def test_xeb_equals_scaled_marginal():
    circ = sycamore_circuit("rect", 3, 4, 8, 11)
    bits = random_bits(12, 12)
    open_q = [8, 9, 10, 11]
    psi = statevector.final_state(circ)
    a = statevector.amplitudes(circ, bits, open_q, psi=psi)
    # marginal P(s1) summed straight from |psi|^2 over the open axes
    p = np.abs(psi) ** 2
    idx = tuple(slice(None) if q in open_q else bits[q] for q in range(12))
    p_s1 = p[idx].sum()
    assert abs(xeb.linear_xeb(a, 12) - (2 ** (12 - 4) * p_s1 - 1)) < 1e-12
    assert abs(xeb.marginal(a) - p_s1) < 1e-15
    cond = xeb.conditional(a)
    assert abs(cond.sum() - 1) < 1e-12


def test_porter_thomas_sanity():
    # Deep random circuits: N p is close to Exp(1) (Eq. 2): mean exactly 1 by
    # normalisation, second moment close to 2 (statistical, not a parity pin).
    circ = sycamore_circuit("rect", 4, 4, 14, 3)
    p = np.abs(statevector.final_state(circ).reshape(-1)) ** 2 * 2 ** 16
    assert abs(p.mean() - 1) < 1e-12
    assert abs((p ** 2).mean() - 2) < 0.1
