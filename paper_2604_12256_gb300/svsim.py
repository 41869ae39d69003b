"""Thin ctypes binding of the C ABI in ``include/svsim.h`` (same names).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``libsvsim.so``.  Loading fails loudly when the library is missing
or was not built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import itertools
import json
import os
from typing import Iterable, Optional, Sequence

import numpy as np

from . import circuits as _circ

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsvsim.so")

SIM_C64, SIM_C128 = 0, 1
SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ETIMEOUT, SIM_EBUSY, SIM_EUNSUPPORTED = range(7)
SIM_F_DIAG, SIM_F_BOOST, SIM_F_BLOCK, SIM_F_FUSE, SIM_F_TC, SIM_F_REMAP, SIM_F_JIT = 1, 2, 4, 8, 16, 32, 64
SIM_F_ALL = 0x7F
SIM_DENSE_SPLIT_TF32, SIM_DENSE_FP32, SIM_DENSE_FP64, SIM_DENSE_DOUBLE_FLOAT = 0, 1, 2, 3

KIND = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5, "rx": 6, "ry": 7, "rz": 8, "p": 9,
        "cx": 10, "cz": 11, "cp": 12, "rzz": 13, "swap": 14, "u1q": 15, "unitary": 16, "diag": 17}
STATUS = {0: "SIM_OK", 1: "SIM_EINVAL", 2: "SIM_ENOMEM", 3: "SIM_ECUDA", 4: "SIM_ETIMEOUT",
          5: "SIM_EBUSY", 6: "SIM_EUNSUPPORTED"}


class sim_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("nq", ctypes.c_uint32), ("q", ctypes.c_uint32 * 6),
                ("param", ctypes.c_double * 3), ("matrix", ctypes.POINTER(ctypes.c_double))]


class sim_options(ctypes.Structure):
    _fields_ = [("max_fuse_qubits", ctypes.c_int), ("max_diag_qubits", ctypes.c_int),
                ("chunk_qubits", ctypes.c_int), ("booster_div", ctypes.c_int),
                ("flags", ctypes.c_uint32), ("dense_precision", ctypes.c_int),
                ("max_stages", ctypes.c_int), ("register_bits", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class sim_plan_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in
                ("gates_in", "ops", "sweeps", "chunk_ops", "diag_ops", "gate_ops", "dense_ops",
                 "tensor_ops", "permute_ops", "diag_fused", "boosted_gates", "state_updates", "bytes")] + \
               [("flops", ctypes.c_double), ("plan_ms", ctypes.c_double), ("tensor_fused", ctypes.c_uint64)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sim_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 16), ("ms", ctypes.c_double * 16), ("bytes", ctypes.c_double * 16),
                ("h2d_bytes", ctypes.c_uint64)]

    KINDS = ("init", "gate", "gate_diag", "diag", "chunk", "tensor", "dense", "phase_small")

    def asdict(self):
        d = {}
        for i, k in enumerate(self.KINDS):
            d[k] = {"launches": int(self.launches[i]), "ms": float(self.ms[i]), "bytes": float(self.bytes[i])}
            d["sub_" + k] = {"launches": int(self.launches[8 + i]), "ms": float(self.ms[8 + i]),
                             "bytes": float(self.bytes[8 + i])}
        d["h2d_bytes"] = int(self.h2d_bytes)
        return d


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, restype, argtypes) of every exported function of include/svsim.h
_P = ctypes.c_void_p
_SIGS = [
    ("sim_default_options", ctypes.c_int, [ctypes.POINTER(sim_options)]),
    ("sim_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    ("sim_create_on", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("sim_destroy", ctypes.c_int, [_P]),
    ("sim_reset", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("sim_apply_circuit", ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(sim_options)]),
    ("sim_sync", ctypes.c_int, [_P]),
    ("sim_probabilities", ctypes.c_int, [_P, _P]),
    ("sim_top_k", ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    ("sim_expectation", ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    ("sim_norm", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("sim_get_state", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("sim_set_state", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("sim_state_device", ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    ("sim_last_plan_stats", ctypes.c_int, [_P, ctypes.POINTER(sim_plan_stats)]),
    ("sim_profile_enable", ctypes.c_int, [_P, ctypes.c_int]),
    ("sim_profile_read", ctypes.c_int, [_P, ctypes.POINTER(sim_profile)]),
    ("sim_kernel_launches", ctypes.c_uint64, []),
    ("sim_selftest_wait_timeout", ctypes.c_int, []),
    ("sim_expectation_noalloc", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, _P, _P]),
    ("srv_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_P)]),
    ("srv_submit", ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    ("srv_poll", ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_int]),
    ("srv_get_stats", ctypes.c_int, [_P, _P]),
    ("srv_destroy", ctypes.c_int, [_P]),
    ("sim_noalloc_error", ctypes.c_char_p, []),
    ("sim_last_error", ctypes.c_char_p, [_P]),
    ("sim_global_error", ctypes.c_char_p, []),
    ("sim_plan_json", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _P, ctypes.c_size_t,
                                     ctypes.POINTER(sim_options), ctypes.c_char_p, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_size_t)]),
    ("sim_jit_info", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
    ("sim_jit_check", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _P, ctypes.c_size_t,
                                     ctypes.POINTER(sim_options), ctypes.POINTER(ctypes.c_int)]),
    ("sim_fault_inject", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("sim_top_k_expectation", ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_size_t, _P]),
    ("sim_jit_cache", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    ("sim_jit_sources", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _P, ctypes.c_size_t,
                                       ctypes.POINTER(sim_options), ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
]


def load(path: Optional[str] = None):
    """Load libsvsim.so (built by ``paper_2604_12256_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsvsim.so not built ({p}); run paper_2604_12256_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, res, args in _SIGS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc, h=None):
    if rc != SIM_OK:
        lib = load()
        msg = lib.sim_last_error(h) if h else lib.sim_global_error()
        raise SimError(rc, (msg or b"").decode(errors="replace"))


def default_options(**kw) -> sim_options:
    o = sim_options()
    _check(load().sim_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# sim_gate as a numpy record (same layout: 64 bytes)
_GATE_DTYPE = np.dtype([("kind", "<u4"), ("nq", "<u4"), ("q", "<u4", (6,)), ("param", "<f8", (3,)),
                        ("matrix", "<u8")])
assert _GATE_DTYPE.itemsize == ctypes.sizeof(sim_gate)


class GateArray:
    """A circuit marshalled into a contiguous sim_gate array (keeps the
    matrix buffers alive).  Built column by column as a numpy record array:
    no per-field ctypes writes."""

    def __init__(self, gates: Sequence[_circ.Gate]):
        self.n = n = len(gates)
        self.arr = np.zeros(max(1, n), dtype=_GATE_DTYPE)
        self._keep = []
        if n == 0:
            return
        z6, z3 = (0,) * 6, (0.0,) * 3
        chain = itertools.chain.from_iterable
        self.arr["kind"][:n] = np.fromiter((KIND[g.kind] for g in gates), np.uint32, n)
        self.arr["nq"][:n] = np.fromiter((len(g.qubits) for g in gates), np.uint32, n)
        self.arr["q"][:n] = np.fromiter(chain((tuple(g.qubits) + z6)[:6] for g in gates), np.uint32,
                                        6 * n).reshape(n, 6)
        self.arr["param"][:n] = np.fromiter(chain((tuple(g.params) + z3)[:3] for g in gates), np.float64,
                                            3 * n).reshape(n, 3)
        for i, g in enumerate(gates):
            if g.matrix is not None:
                buf = np.ascontiguousarray(g.matrix, np.complex128).reshape(-1).view(np.float64).copy()
                self._keep.append(buf)
                self.arr["matrix"][i] = buf.ctypes.data

    @property
    def ptr(self):
        return ctypes.c_void_p(self.arr.ctypes.data)


def plan_json(n: int, gates, dtype: int = SIM_C64, basis: Optional[int] = 0,
              opt: Optional[sim_options] = None) -> dict:
    """The optimizer's plan for a circuit (no GPU needed)."""
    lib = load()
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    b = (1 << 64) - 1 if basis is None else basis
    need = ctypes.c_size_t(0)
    optp = ctypes.byref(opt) if opt is not None else None
    lib.sim_plan_json(n, dtype, b, ga.ptr, ga.n, optp, None, 0, ctypes.byref(need))
    if need.value == 0:
        _check(lib.sim_plan_json(n, dtype, b, ga.ptr, ga.n, optp, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.sim_plan_json(n, dtype, b, ga.ptr, ga.n, optp, buf, need.value, ctypes.byref(need)))
    return json.loads(buf.value.decode())


def jit_check(n: int, gates, dtype: int = SIM_C64, basis: Optional[int] = 0,
              opt: Optional[sim_options] = None) -> int:
    """Generate and compile (no GPU needed) the specialised kernels that
    SIM_F_JIT would run for this circuit; returns how many there are."""
    lib = load()
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    b = (1 << 64) - 1 if basis is None else basis
    cnt = ctypes.c_int(0)
    optp = ctypes.byref(opt) if opt is not None else None
    _check(lib.sim_jit_check(n, dtype, b, ga.ptr, ga.n, optp, ctypes.byref(cnt)))
    return cnt.value


def jit_info() -> dict:
    """Specialised kernels cached in this process now, NVRTC compiles so far
    and their total compile time."""
    lib = load()
    n, ms = ctypes.c_uint64(0), ctypes.c_double(0)
    _check(lib.sim_jit_info(ctypes.byref(n), ctypes.byref(ms)))
    k, c = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib.sim_jit_cache(0, ctypes.byref(k), ctypes.byref(c)))
    return {"programs": n.value, "compiles": c.value, "compile_ms": ms.value}


SIM_FAULT_ALLOC = 1
SIM_FAULT_LAUNCH = 2


def fault_inject(kind: int, count: int, skip: int = 0) -> None:
    """Arm host-side fault injection: after ``skip`` successful ones, the next
    ``count`` device allocations (SIM_FAULT_ALLOC) or kernel launches
    (SIM_FAULT_LAUNCH) fail; count 0 disarms."""
    _check(load().sim_fault_inject(int(kind), int(skip), int(count)))


def jit_cache_limit(max_kernels: int) -> None:
    """At most max_kernels specialised kernels stay loaded (LRU)."""
    _check(load().sim_jit_cache(int(max_kernels), None, None))


def jit_sources(n: int, gates, dtype: int = SIM_C64, basis: Optional[int] = 0,
                opt: Optional[sim_options] = None) -> str:
    """The generated sources of the plan's specialised sweeps (no GPU needed)."""
    lib = load()
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    b = (1 << 64) - 1 if basis is None else basis
    optp = ctypes.byref(opt) if opt is not None else None
    need = ctypes.c_size_t(0)
    rc = lib.sim_jit_sources(n, dtype, b, ga.ptr, ga.n, optp, None, 0, ctypes.byref(need))
    if rc not in (SIM_OK, SIM_ENOMEM):
        _check(rc)
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.sim_jit_sources(n, dtype, b, ga.ptr, ga.n, optp, buf, need.value, ctypes.byref(need)))
    return buf.value.decode()


class Sim:
    """Owner of one sim_t handle."""

    def __init__(self, n: int, dtype: int = SIM_C64, dev_buf: Optional[int] = None, nbytes: int = 0,
                 stream: Optional[int] = None):
        self.lib = load()
        self.n = n
        self.dtype = dtype
        h = ctypes.c_void_p()
        if dev_buf is None:
            _check(self.lib.sim_create(n, dtype, ctypes.byref(h)))
        else:
            _check(self.lib.sim_create_on(n, dtype, ctypes.c_void_p(dev_buf), nbytes,
                                          ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h

    @property
    def amp_bytes(self):
        return 8 if self.dtype == SIM_C64 else 16

    def close(self):
        if self.h:
            self.lib.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self, basis: int = 0):
        _check(self.lib.sim_reset(self.h, basis), self.h)

    def apply(self, gates, opt: Optional[sim_options] = None):
        ga = gates if isinstance(gates, GateArray) else GateArray(gates)
        _check(self.lib.sim_apply_circuit(self.h, ga.ptr, ga.n, ctypes.byref(opt) if opt is not None else None),
               self.h)

    def sync(self):
        _check(self.lib.sim_sync(self.h), self.h)

    def stats(self) -> dict:
        st = sim_plan_stats()
        _check(self.lib.sim_last_plan_stats(self.h, ctypes.byref(st)), self.h)
        return st.asdict()

    def profile_enable(self, on: bool = True, state_only: bool = False):
        """sim_profile_enable: state_only records only the launches on this
        handle's state (not on the merge booster's sub-states)."""
        _check(self.lib.sim_profile_enable(self.h, (2 if state_only else 1) if on else 0), self.h)

    def profile_read(self) -> dict:
        p = sim_profile()
        _check(self.lib.sim_profile_read(self.h, ctypes.byref(p)), self.h)
        return p.asdict()

    def norm(self) -> float:
        v = ctypes.c_double()
        _check(self.lib.sim_norm(self.h, ctypes.byref(v)), self.h)
        return v.value

    def probabilities(self) -> np.ndarray:
        out = np.empty(1 << self.n, np.float64)
        _check(self.lib.sim_probabilities(self.h, out.ctypes.data), self.h)
        return out

    def top_k(self, k: int):
        idx = np.empty(k, np.uint64)
        p = np.empty(k, np.float64)
        _check(self.lib.sim_top_k(self.h, k, idx.ctypes.data, p.ctypes.data), self.h)
        return idx, p

    def expectation(self, masks: Iterable[int]) -> np.ndarray:
        m = np.ascontiguousarray(np.array(list(masks), dtype=np.uint64))
        out = np.empty(len(m), np.float64)
        _check(self.lib.sim_expectation(self.h, m.ctypes.data, len(m), out.ctypes.data), self.h)
        return out

    def top_k_expectation(self, k: int, masks: Iterable[int]):
        """(top-k indices, probabilities, <Z-string> values) in one call: the
        two read-outs run concurrently (sim_top_k_expectation)."""
        idx = np.empty(k, np.uint64)
        p = np.empty(k, np.float64)
        m = np.ascontiguousarray(np.array(list(masks), dtype=np.uint64))
        out = np.empty(max(1, len(m)), np.float64)
        _check(self.lib.sim_top_k_expectation(self.h, k, idx.ctypes.data, p.ctypes.data, m.ctypes.data if len(m) else None,
                                              len(m), out.ctypes.data), self.h)
        return idx, p, out[:len(m)]

    def get_state(self) -> np.ndarray:
        dt = np.complex64 if self.dtype == SIM_C64 else np.complex128
        out = np.empty(1 << self.n, dt)
        _check(self.lib.sim_get_state(self.h, out.ctypes.data, out.nbytes), self.h)
        return out

    def set_state(self, a: np.ndarray):
        dt = np.complex64 if self.dtype == SIM_C64 else np.complex128
        a = np.ascontiguousarray(a, dt)
        _check(self.lib.sim_set_state(self.h, a.ctypes.data, a.nbytes), self.h)

    def device(self):
        p, s = ctypes.c_void_p(), ctypes.c_void_p()
        _check(self.lib.sim_state_device(self.h, ctypes.byref(p), ctypes.byref(s)), self.h)
        return p.value, s.value


class srv_request(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("dtype", ctypes.c_int), ("gates", ctypes.c_void_p),
                ("n_gates", ctypes.c_size_t), ("basis", ctypes.c_uint64), ("top_k", ctypes.c_int),
                ("z_masks", ctypes.c_void_p), ("n_masks", ctypes.c_size_t)]


class srv_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("top_k", ctypes.c_int), ("n_masks", ctypes.c_int), ("path", ctypes.c_int),
                ("top_idx", ctypes.c_uint64 * 1024), ("top_p", ctypes.c_double * 1024),
                ("expect", ctypes.c_double * 64), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class srv_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "failed", "batched", "batches")] + \
               [(f, ctypes.c_double) for f in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "elapsed_s",
                                              "circuits_per_s")] + \
               [("hbm_budget", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """srv_* binding: a continuous-batching request loop on the GPU."""

    def __init__(self, hbm_budget: int, n_streams: int = 2):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.srv_create(ctypes.c_size_t(hbm_budget), n_streams, ctypes.byref(h)))
        self.h = h

    def submit(self, circuit: _circ.Circuit, top_k: int = 64, masks: Sequence[int] = (),
               dtype: int = SIM_C64) -> int:
        return self.submit_array(GateArray(circuit.gates), circuit.n, circuit.basis, top_k, masks, dtype)

    def submit_array(self, ga: "GateArray", n: int, basis: int = 0, top_k: int = 64, masks: Sequence[int] = (),
                     dtype: int = SIM_C64) -> int:
        """Queue an already marshalled gate list (the server copies it)."""
        m = np.ascontiguousarray(np.array(list(masks), dtype=np.uint64)) if len(masks) else None
        req = srv_request(n, dtype, ga.ptr, ga.n, basis, top_k,
                          m.ctypes.data if m is not None else None, 0 if m is None else len(m))
        t = ctypes.c_uint64()
        _check(self.lib.srv_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = srv_result()
        rc = self.lib.srv_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r), timeout_ms)
        if rc != SIM_OK:
            raise SimError(rc, "srv_poll")
        return {"status": r.status, "path": r.path, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms,
                "top_idx": np.array(r.top_idx[:r.top_k], dtype=np.uint64),
                "top_p": np.array(r.top_p[:r.top_k]), "expect": np.array(r.expect[:r.n_masks])}

    def stats(self) -> dict:
        st = srv_stats()
        _check(self.lib.srv_get_stats(self.h, ctypes.byref(st)))
        return st.asdict()

    def close(self):
        if self.h:
            self.lib.srv_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def kernel_launches() -> int:
    """sim_kernel_launches: kernels this library has launched in this process."""
    return int(load().sim_kernel_launches())


def expectation_noalloc(dev_state: int, n: int, dtype: int, dev_masks: int, n_terms: int, dev_out: int,
                        stream: Optional[int] = None) -> None:
    """sim_expectation_noalloc: <Z-string> values for callers that cannot
    allocate device memory; all pointers are device addresses owned by the
    caller, the results land in dev_out when the stream reaches the kernels."""
    lib = load()
    rc = lib.sim_expectation_noalloc(ctypes.c_void_p(dev_state), n, dtype, ctypes.c_void_p(dev_masks), n_terms,
                                     ctypes.c_void_p(dev_out), ctypes.c_void_p(stream or 0))
    if rc != SIM_OK:
        raise SimError(rc, (lib.sim_noalloc_error() or b"").decode(errors="replace"))


def run(circuit: _circ.Circuit, dtype: int = SIM_C64, opt: Optional[sim_options] = None) -> np.ndarray:
    """Convenience: simulate a circuit from its basis state, return the state."""
    with Sim(circuit.n, dtype) as s:
        s.reset(circuit.basis)
        s.apply(circuit.gates, opt)
        return s.get_state()
