"""Write the stored oracle values under tests/golden/.

Calls only ``oracle/`` (and the seeded inputs of ``tn_inputs``).  Each file
holds one value per line: index, real part, imaginary part (repr of FP64),
after a header that names the workload recipe.

    python tests/golden/make_golden.py [cfg2] [cfg4] [cfg3]

cfg2: the 30-qubit 5x6 grid, 12 cycles, 8 open qubits, 22 fixed bits; FP64
Schroedinger state vector (16 GiB of host memory, several minutes on 8 cores).

cfg4: the 53-qubit rotated lattice, 14 cycles, 16 open qubits.  No state
vector fits, so a seeded sample of entries of the 2^16 amplitude tensor is
computed one at a time: each entry is the fully closed network (open qubits
set to that entry's bits) contracted by the oracle's own pairwise route in
FP64 with its own greedy order (no slicing; about 25 GiB of host memory and
several minutes per entry on 8 cores).  Lines are appended as they finish.

cfg3: the batched workload's members of more than 20 qubits (those of 20 or
fewer are checked against a live state vector in the tests).  Every member of
up to 28 qubits, then the 30-qubit ones in a seeded order (CFG3_SAMPLES_30 of
them: all), get their full 2^k open-qubit amplitude tensor from the FP64
state vector (oracle.sv_native; about ten minutes per 30-qubit member on 8
cores).  Lines: member index, amplitude index, real, imaginary; members are
appended as they finish, cheapest first, so a partly written file holds a
prefix of that order.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from tn_inputs.configs import make_config  # noqa: E402
from tn_inputs import SplitMix64  # noqa: E402
from oracle import sv_native  # noqa: E402
from oracle import network as onet, contract as oc  # noqa: E402


def write_amplitudes(path, header, amp):
    with open(path, "w") as f:
        f.write(f"# {header}\n")
        for i, a in enumerate(amp):
            f.write(f"{i} {float(a.real)!r} {float(a.imag)!r}\n")


def cfg2():
    cfg = make_config(2)
    amp = sv_native.amplitudes(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    header = (f"{cfg['name']} circuit={cfg['circuit'].name} open={cfg['open_qubits']} "
              f"fixed_bits={''.join(map(str, cfg['fixed_bits']))} route=oracle.sv_native (FP64 state vector)")
    write_amplitudes(os.path.join(HERE, "cfg2_amplitudes.txt"), header, amp)


CFG4_SAMPLES = 8
CFG4_SAMPLE_SEED = 0x2103C4


def cfg4_sample_indices():
    """Seeded amplitude indices of the cfg4 sample (distinct, drawn uniformly)."""
    cfg = make_config(4)
    k = len(cfg["open_qubits"])
    rng = SplitMix64(CFG4_SAMPLE_SEED)
    out = []
    while len(out) < CFG4_SAMPLES:
        i = rng.below(1 << k)
        if i not in out:
            out.append(i)
    return out


def cfg4():
    import time
    cfg = make_config(4)
    circ, openq = cfg["circuit"], cfg["open_qubits"]
    k = len(openq)
    path = os.path.join(HERE, "cfg4_amplitudes_sampled.txt")
    done = set()
    if os.path.exists(path):
        done = {int(l.split()[0]) for l in open(path) if not l.startswith("#")}
    else:
        header = (f"{cfg['name']} circuit={circ.name} open={openq} "
                  f"fixed_bits={''.join(map(str, cfg['fixed_bits']))} "
                  f"samples={CFG4_SAMPLES} sample_seed={CFG4_SAMPLE_SEED:#x} "
                  "route=oracle.contract (closed network per entry, FP64, greedy order)")
        with open(path, "w") as f:
            f.write(f"# {header}\n")
    for idx in cfg4_sample_indices():
        if idx in done:
            continue
        bits = list(cfg["fixed_bits"])
        for j, q in enumerate(openq):
            bits[q] = (idx >> (k - 1 - j)) & 1
        t0 = time.time()
        L, T, O = onet.circuit_network(circ, bits, [])
        a = complex(oc.contract(L, T, O))
        with open(path, "a") as f:
            f.write(f"{idx} {a.real!r} {a.imag!r}\n")
        print(f"cfg4 entry {idx}: {a} ({time.time() - t0:.0f} s)", flush=True)


CFG3_SAMPLES_30 = 42  # every 30-qubit member (the first 8 of the seeded order were written first)
CFG3_SAMPLE_SEED = 0x2103C3


def cfg3_members():
    """Indices of the batch members that get stored amplitudes: all of more
    than 20 and at most 28 qubits, then a seeded sample of the 30-qubit
    ones; ordered by qubit count (cheapest first)."""
    from tn_inputs.configs import batch_recipes
    rs = batch_recipes()
    nq = [r["rows"] * r["cols"] for r in rs]
    small = [i for i in range(len(rs)) if 20 < nq[i] <= 28]
    big = [i for i in range(len(rs)) if nq[i] > 28]
    rng = SplitMix64(CFG3_SAMPLE_SEED)
    pick = []
    while len(pick) < min(CFG3_SAMPLES_30, len(big)):
        i = big[rng.below(len(big))]
        if i not in pick:
            pick.append(i)
    return sorted(small, key=lambda i: (nq[i], i)) + pick


def cfg3():
    import time
    from tn_inputs.configs import batch_recipes, make_batch_member
    path = os.path.join(HERE, "cfg3_amplitudes.txt")
    header = (f"# batch256 members of more than 20 qubits: all up to 28 qubits, then up to {CFG3_SAMPLES_30} "
              f"30-qubit ones in a seeded order (sample_seed={CFG3_SAMPLE_SEED:#x}; a prefix while being written); "
              "member index, amplitude index, re, im; route=oracle.sv_native (FP64 state vector)\n")
    done = set()
    if os.path.exists(path):
        lines = open(path).readlines()
        done = {int(l.split()[0]) for l in lines if not l.startswith("#")}
        if lines and lines[0] != header:  # the recipe's description changed, not its values
            lines[0] = header
            with open(path, "w") as f:
                f.writelines(lines)
    else:
        with open(path, "w") as f:
            f.write(header)
    rs = batch_recipes()
    for i in cfg3_members():
        if i in done:
            continue
        m = make_batch_member(rs[i])
        t0 = time.time()
        amp = sv_native.amplitudes(m["circuit"], m["fixed_bits"], m["open_qubits"])
        # the whole file is rewritten and renamed into place, so a reader
        # never sees a member that is only partly written
        with open(path) as f:
            text = f.read()
        text += "".join(f"{i} {j} {float(a.real)!r} {float(a.imag)!r}\n" for j, a in enumerate(amp))
        with open(path + ".tmp", "w") as f:
            f.write(text)
        os.replace(path + ".tmp", path)
        print(f"cfg3 member {i}: {m['circuit'].n_qubits} qubits ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["cfg2"]
    for w in which:
        globals()[w]()
