"""CPU oracle: plain, slow, obviously correct complex128 state-vector simulator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_2604_12256_gb300``) and never
imports it; the only shared module is the seeded circuit generator, which
holds none of the simulation arithmetic.

Pieces (each pinned by ``tests/test_oracle_pins.py``):

* :func:`run` -- the gate-by-gate scheme of Algorithm 1 (Section 2.4): each
  gate sweeps the whole 2^n vector (Eq. 1) with its 2^k x 2^k matrix (Eqs. 2-3,
  qubit j = bit j of the index).  Implemented in ``oracle.c`` (C, OpenMP).
* :func:`probabilities`, :func:`norm`, :func:`top_k`, :func:`expectation_z`,
  :func:`fidelity` -- plain numpy definitions of the read-out quantities:
  p_x = |a_x|^2; top-k by probability with ties to the lower index;
  <Z-string m> = sum_x p_x (-1)^popcount(x & m); |<psi|phi>|^2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# oracle-local gate codes; must match the enum in oracle.c
KIND = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5, "rx": 6, "ry": 7, "rz": 8,
        "p": 9, "cx": 10, "cz": 11, "cp": 12, "rzz": 13, "swap": 14, "u1q": 15,
        "unitary": 16, "diag": 17}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.orc_run.restype = ctypes.c_int64
            lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int]
            lib.orc_gate_matrix.restype = ctypes.c_int
            lib.orc_gate_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _marshal(gates):
    ng = len(gates)
    kind = np.zeros(ng, np.int32)
    nq = np.zeros(ng, np.int32)
    qubits = np.zeros((ng, 6), np.int32)
    params = np.zeros((ng, 3), np.float64)
    ext_off = np.full(ng, -1, np.int64)
    ext_parts = []
    off = 0
    for i, g in enumerate(gates):
        kind[i] = KIND[g.kind]
        nq[i] = len(g.qubits)
        qubits[i, :len(g.qubits)] = g.qubits
        params[i, :len(g.params)] = g.params
        if g.matrix is not None:
            flat = np.ascontiguousarray(g.matrix, np.complex128).reshape(-1).view(np.float64)
            ext_off[i] = off
            ext_parts.append(flat)
            off += flat.size
    ext = np.concatenate(ext_parts) if ext_parts else np.zeros(1, np.float64)
    return kind, nq, qubits, params, ext, ext_off


def basis_state(n: int, basis: int = 0) -> np.ndarray:
    a = np.zeros(1 << n, np.complex128)
    a[basis] = 1.0
    return a


def run(circuit, state: Optional[np.ndarray] = None, n_threads: int = 0,
        gates: Optional[Sequence] = None) -> np.ndarray:
    """Apply ``circuit``'s gates (or ``gates``) one at a time, Algorithm 1.

    Starts from ``state`` (copied) or from ``|circuit.basis>``; returns the
    final complex128 state vector."""
    n = circuit.n
    gl = circuit.gates if gates is None else gates
    a = basis_state(n, circuit.basis) if state is None else np.array(state, np.complex128, copy=True)
    if a.shape != (1 << n,):
        raise ValueError("state has the wrong size")
    run_inplace(n, a, gl, n_threads)
    return a


def run_inplace(n: int, a: np.ndarray, gates: Sequence, n_threads: int = 0) -> None:
    if not (a.dtype == np.complex128 and a.flags.c_contiguous):
        raise ValueError("state must be a contiguous complex128 array")
    if len(gates) == 0:
        return
    kind, nq, qubits, params, ext, ext_off = _marshal(gates)
    lib = _load()
    bad = lib.orc_run(n, a.ctypes.data, len(gates), kind.ctypes.data, nq.ctypes.data,
                      qubits.ctypes.data, params.ctypes.data, ext.ctypes.data,
                      ext_off.ctypes.data, int(n_threads))
    if bad >= 0:
        raise ValueError(f"oracle: invalid gate #{bad}: {gates[bad]}")


def gate_matrix(g) -> np.ndarray:
    """The oracle's matrix for one gate (2^k x 2^k complex128)."""
    kind, nq, qubits, params, ext, ext_off = _marshal([g])
    out = np.zeros(64 * 64, np.complex128)
    e = ext.ctypes.data if ext_off[0] >= 0 else None
    dim = _load().orc_gate_matrix(int(kind[0]), int(nq[0]), params.ctypes.data, e, out.ctypes.data)
    if dim <= 0:
        raise ValueError(g)
    return out[:dim * dim].reshape(dim, dim).copy()


# ------------------------------------------------------------ read-out
def probabilities(a: np.ndarray) -> np.ndarray:
    """p_x = |a_x|^2 (float64)."""
    return a.real * a.real + a.imag * a.imag


def norm(a: np.ndarray) -> float:
    """Sum of probabilities (the squared 2-norm)."""
    return float(np.sum(probabilities(a)))


def top_k(a: np.ndarray, k: int):
    """The k largest probabilities, ties broken towards the lower index.
    Returns (indices uint64, probabilities float64), largest first."""
    p = probabilities(a)
    k = min(k, p.size)
    idx = np.arange(p.size, dtype=np.int64)
    order = np.lexsort((idx, -p))[:k]
    return order.astype(np.uint64), p[order]


def _popcount_parity(x: np.ndarray) -> np.ndarray:
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(x) & 1
    v = x.copy()
    par = np.zeros_like(v)
    while np.any(v):
        par ^= v & 1
        v >>= 1
    return par


def expectation_z(a: np.ndarray, masks: Iterable[int]) -> np.ndarray:
    """<Z-string m> = sum_x |a_x|^2 (-1)^popcount(x & m) for each mask m."""
    p = probabilities(a)
    x = np.arange(p.size, dtype=np.uint64)
    out = []
    for m in masks:
        sign = 1.0 - 2.0 * _popcount_parity(x & np.uint64(m)).astype(np.float64)
        out.append(float(np.sum(p * sign)))
    return np.array(out)


def fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """|<a|b>|^2 for normalised states."""
    return float(abs(np.vdot(a, b)) ** 2)
