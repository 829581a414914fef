"""Write the stored oracle values under tests/golden/.

Calls only ``oracle/`` (and the seeded inputs of ``tn_inputs``).  Each file
holds one value per line: index, real part, imaginary part (repr of FP64),
after a header that names the workload recipe.

    python tests/golden/make_golden.py [cfg2]

cfg2: the 30-qubit 5x6 grid, 12 cycles, 8 open qubits, 22 fixed bits; FP64
Schroedinger state vector (16 GiB of host memory, several minutes on 8 cores).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from tn_inputs.configs import make_config  # noqa: E402
from oracle import sv_native  # noqa: E402


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


if __name__ == "__main__":
    which = sys.argv[1:] or ["cfg2"]
    for w in which:
        globals()[w]()
