"""The stored oracle values under tests/golden/ are the ones the committed
generator defines: the right workload header and, for sampled files, the
seeded sample indices (no recomputation; the values themselves come from
oracle/ only)."""
import importlib.util
import os

from tn_inputs.configs import make_config

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _read(name):
    header, rows = None, []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#"):
            header = line[1:].strip()
            continue
        i, re, im = line.split()
        rows.append((int(i), float(re), float(im)))
    return header, rows


def test_cfg2_file_covers_every_amplitude():
    cfg = make_config(2)
    header, rows = _read("cfg2_amplitudes.txt")
    assert header.startswith(cfg["name"]) and cfg["circuit"].name in header
    assert [r[0] for r in rows] == list(range(1 << len(cfg["open_qubits"])))


def test_cfg4_file_holds_the_seeded_sample():
    mg = _make_golden()
    cfg = make_config(4)
    header, rows = _read("cfg4_amplitudes_sampled.txt")
    assert header.startswith(cfg["name"]) and cfg["circuit"].name in header
    assert "".join(map(str, cfg["fixed_bits"])) in header
    assert sorted(r[0] for r in rows) == sorted(mg.cfg4_sample_indices())
    # Porter-Thomas scale of a 53-qubit amplitude: |a|^2 averages 2^-53
    mean_p = sum(re * re + im * im for _, re, im in rows) / len(rows)
    assert 0.1 < mean_p * 2.0 ** 53 < 10
