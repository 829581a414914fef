"""ctypes wrapper of the plain-C state-vector oracle (oracle/sv.c); test
infrastructure only.  ``build()`` compiles it with gcc + OpenMP in place."""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv.c")
_LIB = os.path.join(_HERE, "liboracle_sv.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle_sv.so unless a digest of the source, the command
    and the machine matches the one stored beside it (a library built from
    another source or on another machine is never reused)."""
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"]
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update("\0".join(cmd).encode())
    with open(_SRC, "rb") as f:
        h.update(f.read())
    digest = h.hexdigest()
    stamp = _LIB + ".digest"
    fresh = os.path.exists(_LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest
    if force or not fresh:
        subprocess.check_call(cmd)
        with open(stamp, "w") as f:
            f.write(digest + "\n")
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.oracle_sv_amplitudes.restype = ctypes.c_int
    return _lib


def amplitudes(circuit, fixed_bits, open_qubits) -> np.ndarray:
    """Complex128 amplitudes over the open qubits (first listed = MSB)."""
    lib = _load()
    gates = circuit.gates
    ng = len(gates)
    nq = np.array([len(g.qubits) for g in gates], dtype=np.int32)
    qs = np.zeros(2 * ng, dtype=np.int32)
    ms = np.zeros(32 * ng, dtype=np.float64)
    for i, g in enumerate(gates):
        for j, q in enumerate(g.qubits):
            qs[2 * i + j] = q
        m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
        ms[32 * i:32 * i + 2 * m.size:2] = m.real
        ms[32 * i + 1:32 * i + 2 * m.size:2] = m.imag
    fb = np.array(fixed_bits, dtype=np.int32)
    oq = np.array(open_qubits, dtype=np.int32)
    out = np.zeros(2 << len(open_qubits), dtype=np.float64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.oracle_sv_amplitudes(circuit.n_qubits, ng, p(nq), p(qs), p(ms), p(fb),
                                  len(open_qubits), p(oq), p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_sv_amplitudes failed: {rc}")
    return out[0::2] + 1j * out[1::2]
