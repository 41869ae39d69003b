"""Seeded synthetic circuit generators.

This module only draws random circuits; it holds none of the simulation
arithmetic. Both the CUDA path and the CPU oracle consume the gate lists it
produces, so both see bit-identical inputs (angles and Haar matrices are drawn
once here, in float64, and stored in the gates).

Gate convention (Section 2.2 of the paper): qubit ``j`` is bit ``j`` of the
amplitude index.  For a gate listed on qubits ``q[0..k-1]`` bit ``i`` of the
local matrix index belongs to ``q[i]``; so for ``cx`` ``q[0]`` is the control
and ``q[1]`` the target.

Workload shapes follow the paper's evaluation (Section 5): a diagonal-heavy
gate-level stream (its RZZ benchmark), the QFT and QAOA circuit-level
benchmarks, and depth-``d`` random layered circuits; plus a Poisson request
stream for the serving loop.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate names understood by both sides.  Arity is fixed except for
# "unitary" and "diag", whose arity is the number of listed qubits.
GATE_ARITY = {
    "h": 1, "x": 1, "y": 1, "z": 1, "s": 1, "t": 1,
    "rx": 1, "ry": 1, "rz": 1, "p": 1,
    "cx": 2, "cz": 2, "cp": 2, "rzz": 2, "swap": 2,
    "u1q": 1, "unitary": None, "diag": None,
}
GATE_NPARAMS = {"rx": 1, "ry": 1, "rz": 1, "p": 1, "cp": 1, "rzz": 1}


@dataclass
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    # row-major complex matrix (u1q: 2x2, unitary: 2^k x 2^k) or
    # the 2^k diagonal entries (diag); None for named gates
    matrix: Optional[np.ndarray] = None

    def __post_init__(self):
        self.qubits = tuple(int(q) for q in self.qubits)
        self.params = tuple(float(p) for p in self.params)
        if self.matrix is not None:
            self.matrix = np.ascontiguousarray(self.matrix, dtype=np.complex128)


@dataclass
class Circuit:
    n: int
    gates: List[Gate] = field(default_factory=list)
    basis: int = 0           # initial computational basis state |basis>
    name: str = ""

    def __len__(self):
        return len(self.gates)


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random 2x2 unitary by QR of a complex Ginibre matrix with the
    phase correction of Mezzadri, "How to generate random matrices from the
    classical compact groups" (2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def haar_unitary(rng: np.random.Generator, dim: int) -> np.ndarray:
    """Haar-random dim x dim unitary (same method as :func:`haar_u2`)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def haar_u2_batch(rng: np.random.Generator, count: int) -> np.ndarray:
    """``count`` Haar-random 2x2 unitaries, shape (count, 2, 2): the QR
    factorisation of complex Ginibre matrices whose R has a positive real
    diagonal, the unique one that Mezzadri's phase correction selects, so Q is
    Haar distributed as in :func:`haar_u2`.  In two dimensions it is closed
    form: q0 = z0 / |z0|, and q1 is the unit vector orthogonal to q0,
    (-conj(q0[1]), conj(q0[0])), times the phase that makes r11 = q1^H z1 real
    and positive."""
    z = (rng.standard_normal((count, 2, 2)) + 1j * rng.standard_normal((count, 2, 2))) / math.sqrt(2.0)
    c0, c1 = z[:, :, 0], z[:, :, 1]
    q0 = c0 / np.linalg.norm(c0, axis=1)[:, None]
    a, b = q0[:, 0], q0[:, 1]
    w = a * c1[:, 1] - b * c1[:, 0]          # (-conj b, conj a)^H z1
    q1 = (w / np.abs(w))[:, None] * np.stack([-b.conj(), a.conj()], axis=1)
    return np.stack([q0, q1], axis=2)


def layered(n: int, depth: int, seed: int = 0) -> Circuit:
    """Random layered circuit: every layer puts a Haar U(2) on each qubit, then
    CZ on (0,1),(2,3),... in even layers and (1,2),(3,4),... in odd ones."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    for layer in range(depth):
        us = haar_u2_batch(rng, n)
        for q in range(n):
            gates.append(Gate("u1q", (q,), matrix=us[q]))
        start = 0 if layer % 2 == 0 else 1
        for q in range(start, n - 1, 2):
            gates.append(Gate("cz", (q, q + 1)))
    return Circuit(n, gates, 0, f"layered{n}x{depth}")


def _distinct(rng: np.random.Generator, n: int, k: int) -> Tuple[int, ...]:
    return tuple(int(v) for v in rng.choice(n, size=k, replace=False))


def diag_heavy(n: int, n_gates: int = 500, seed: int = 1, p_diag: float = 0.8,
               prefix_h: bool = True) -> Circuit:
    """Diagonal-heavy gate-level stream: each gate is diagonal with probability
    ``p_diag`` (uniform over RZ, CP, RZZ) else uniform over H, RX; qubits
    uniform and distinct; angles uniform in [0, 2pi).  Prefixed by H on every
    qubit so that it starts from the uniform superposition."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    if prefix_h:
        gates += [Gate("h", (q,)) for q in range(n)]
    for _ in range(n_gates):
        if rng.random() < p_diag:
            kind = ("rz", "cp", "rzz")[int(rng.integers(3))]
        else:
            kind = ("h", "rx")[int(rng.integers(2))]
        k = GATE_ARITY[kind]
        qs = _distinct(rng, n, k)
        params = (float(rng.uniform(0.0, 2.0 * math.pi)),) if kind in GATE_NPARAMS else ()
        gates.append(Gate(kind, qs, params))
    return Circuit(n, gates, 0, f"diagheavy{n}x{n_gates}")


def qft(n: int, seed: int = 2, random_basis: bool = True, swaps: bool = True) -> Circuit:
    """QFT: for j = n-1 .. 0, H(j) then CP(pi/2^(j-k)) on (k, j) for
    k = j-1 .. 0; then SWAP(i, n-1-i).  Starts on a random basis state."""
    rng = np.random.default_rng(seed)
    basis = int(rng.integers(0, 1 << n)) if random_basis else 0
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("h", (j,)))
        for k in range(j - 1, -1, -1):
            gates.append(Gate("cp", (k, j), (math.pi / (1 << (j - k)),)))
    if swaps:
        for i in range(n // 2):
            gates.append(Gate("swap", (i, n - 1 - i)))
    return Circuit(n, gates, basis, f"qft{n}")


def random_regular3(n: int, rng: np.random.Generator, max_tries: int = 10000) -> List[Tuple[int, int]]:
    """Random 3-regular simple graph on n nodes (n even) by the pairing
    (configuration) model with rejection of loops and multi-edges."""
    if n % 2:
        raise ValueError("3-regular graph needs an even node count")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in seen:
                ok = False
                break
            seen.add(e)
        if ok:
            return sorted(seen)
    raise RuntimeError("could not draw a simple 3-regular graph")


def qaoa(n: int, p: int = 4, seed: int = 3) -> Circuit:
    """QAOA-style ansatz: H on every qubit, then p layers of RZZ(gamma_l) on
    each edge of a random 3-regular graph followed by RX(beta_l) on every
    qubit; gamma_l, beta_l uniform in [0, pi).  For odd n the graph spans the
    first n-1 qubits and the last qubit only gets the mixer."""
    rng = np.random.default_rng(seed)
    m = n if n % 2 == 0 else n - 1
    edges = random_regular3(m, rng) if m >= 4 else []
    gates: List[Gate] = [Gate("h", (q,)) for q in range(n)]
    for _ in range(p):
        gamma = float(rng.uniform(0.0, math.pi))
        beta = float(rng.uniform(0.0, math.pi))
        for a, b in edges:
            gates.append(Gate("rzz", (a, b), (gamma,)))
        for q in range(n):
            gates.append(Gate("rx", (q,), (beta,)))
    return Circuit(n, gates, 0, f"qaoa{n}p{p}")


def rzz_full(n: int, seed: int = 5) -> Circuit:
    """The paper's gate-level benchmark shape: RZZ on every qubit pair
    (full connectivity), angles uniform in [0, 2pi), from |+...+>."""
    rng = np.random.default_rng(seed)
    gates = [Gate("h", (q,)) for q in range(n)]
    for a in range(n):
        for b in range(a + 1, n):
            gates.append(Gate("rzz", (a, b), (float(rng.uniform(0.0, 2.0 * math.pi)),)))
    return Circuit(n, gates, 0, f"rzzfull{n}")


# ---------------------------------------------------------------- circuit
# families of the per-gate comparison (Table 2): written from each family's
# textbook definition, seeded, any qubit count.

def bernstein_vazirani(n: int, seed: int = 6) -> Circuit:
    """Bernstein-Vazirani on n - 1 data qubits (0..n-2) and an ancilla (n-1):
    X and H on the ancilla, H on the data, CX(i -> ancilla) for each bit i
    of a random secret s, H on the data.  The data register ends in |s>, the
    ancilla in |->.  ``Circuit.name`` carries the secret."""
    rng = np.random.default_rng(seed)
    secret = [int(b) for b in rng.integers(0, 2, n - 1)]
    anc = n - 1
    g = [Gate("x", (anc,)), Gate("h", (anc,))] + [Gate("h", (q,)) for q in range(n - 1)]
    g += [Gate("cx", (q, anc)) for q in range(n - 1) if secret[q]]
    g += [Gate("h", (q,)) for q in range(n - 1)]
    s = sum(b << q for q, b in enumerate(secret))
    return Circuit(n, g, 0, f"bv{n}:secret={s}")


def hidden_shift(n: int, seed: int = 7) -> Circuit:
    """Hidden shift for the bent function f(x, y) = x . y on n = 2m qubits
    (x = qubits 0..m-1, y = m..2m-1), whose dual is itself: H on all, X on
    the shift bits, the f phase (CZ(i, m + i)), X on the shift bits, H on
    all, the dual's phase (CZ(i, m + i)), H on all.  Ends in |s>.
    ``Circuit.name`` carries the shift s."""
    if n % 2:
        raise ValueError("hidden shift needs an even qubit count")
    m = n // 2
    rng = np.random.default_rng(seed)
    shift = [int(b) for b in rng.integers(0, 2, n)]
    xs = [Gate("x", (q,)) for q in range(n) if shift[q]]
    phase = [Gate("cz", (i, m + i)) for i in range(m)]
    hs = [Gate("h", (q,)) for q in range(n)]
    g = hs + xs + phase + xs + hs + phase + hs
    s = sum(b << q for q, b in enumerate(shift))
    return Circuit(n, g, 0, f"hs{n}:shift={s}")


def quantum_volume(n: int, depth: int = 0, seed: int = 8) -> Circuit:
    """Quantum-volume model circuit: ``depth`` (default n) layers, each a
    random permutation of the qubits followed by a Haar-random SU(4)-class
    unitary (U(4), Mezzadri's method) on each consecutive pair."""
    rng = np.random.default_rng(seed)
    g: List[Gate] = []
    for _ in range(depth or n):
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            g.append(Gate("unitary", (int(perm[i]), int(perm[i + 1])), matrix=haar_unitary(rng, 4)))
    return Circuit(n, g, 0, f"qv{n}x{depth or n}")


_SQRT_X = np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]) / 2.0
_SQRT_Y = np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]]) / 2.0
_W = (np.array([[0, 1], [1, 0]]) + np.array([[0, -1j], [1j, 0]])) / math.sqrt(2.0)
_SQRT_W = (np.eye(2) - 1j * _W) / math.sqrt(2.0) * np.exp(1j * math.pi / 4)   # (W ** 0.5: eigenvalues 1, i)


def supremacy(n: int, cycles: int = 20, seed: int = 9) -> Circuit:
    """Random-circuit-sampling style circuit on a line: H on every qubit, then
    ``cycles`` cycles of a random gate from {sqrt(X), sqrt(Y), sqrt(W)} on
    every qubit (never the same twice in a row on a qubit) followed by CZ on
    (0,1),(2,3),... in even cycles and (1,2),(3,4),... in odd ones."""
    rng = np.random.default_rng(seed)
    mats = [_SQRT_X, _SQRT_Y, _SQRT_W]
    last = [-1] * n
    g = [Gate("h", (q,)) for q in range(n)]
    for c in range(cycles):
        for q in range(n):
            k = int(rng.integers(3))
            while k == last[q]:
                k = int(rng.integers(3))
            last[q] = k
            g.append(Gate("u1q", (q,), matrix=mats[k]))
        for q in range(c % 2, n - 1, 2):
            g.append(Gate("cz", (q, q + 1)))
    return Circuit(n, g, 0, f"sc{n}x{cycles}")


def variational(n: int, layers: int = 10, seed: int = 10) -> Circuit:
    """Hardware-efficient variational ansatz: ``layers`` layers of RY(a) and
    RZ(b) on every qubit (angles uniform in [0, 2pi)) followed by a CZ chain
    (0,1),(1,2),...,(n-2,n-1)."""
    rng = np.random.default_rng(seed)
    g: List[Gate] = []
    for _ in range(layers):
        for q in range(n):
            g.append(Gate("ry", (q,), (float(rng.uniform(0, 2 * math.pi)),)))
            g.append(Gate("rz", (q,), (float(rng.uniform(0, 2 * math.pi)),)))
        for q in range(n - 1):
            g.append(Gate("cz", (q, q + 1)))
    return Circuit(n, g, 0, f"vc{n}x{layers}")


FAMILIES = {"bv": bernstein_vazirani, "hs": hidden_shift, "qv": quantum_volume, "sc": supremacy,
            "vc": variational}


def random_mixed(n: int, n_gates: int, seed: int, max_k: int = 3) -> Circuit:
    """Random test circuit over the whole gate set (named gates, u1q, small
    dense unitaries and diagonals) for parity tests."""
    rng = np.random.default_rng(seed)
    named = ["h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p", "cx", "cz", "cp", "rzz", "swap", "u1q"]
    gates: List[Gate] = []
    for _ in range(n_gates):
        r = rng.random()
        if r < 0.08 and n >= 2:
            k = int(rng.integers(2, min(max_k, n) + 1))
            gates.append(Gate("unitary", _distinct(rng, n, k), matrix=haar_unitary(rng, 1 << k)))
        elif r < 0.14 and n >= 1:
            k = int(rng.integers(1, min(max_k, n) + 1))
            ph = rng.uniform(0.0, 2.0 * math.pi, size=1 << k)
            gates.append(Gate("diag", _distinct(rng, n, k), matrix=np.exp(1j * ph)))
        else:
            kind = named[int(rng.integers(len(named)))]
            k = GATE_ARITY[kind]
            if k > n:
                kind, k = "h", 1
            qs = _distinct(rng, n, k)
            params = (float(rng.uniform(0.0, 2.0 * math.pi)),) if kind in GATE_NPARAMS else ()
            mat = haar_u2(rng) if kind == "u1q" else None
            gates.append(Gate(kind, qs, params, mat))
    return Circuit(n, gates, int(rng.integers(0, 1 << n)), f"mixed{n}x{n_gates}")


def inverse(c: Circuit) -> Circuit:
    """The adjoint circuit C^dagger expressed in the same gate set (reversed
    order; rotation angles negated; fixed gates replaced by their adjoints)."""
    out: List[Gate] = []
    for g in reversed(c.gates):
        k = g.kind
        if k in ("h", "x", "y", "z", "cx", "cz", "swap"):
            out.append(Gate(k, g.qubits))
        elif k in ("rx", "ry", "rz", "p", "cp", "rzz"):
            out.append(Gate(k, g.qubits, (-g.params[0],)))
        elif k == "s":
            out.append(Gate("p", g.qubits, (-math.pi / 2,)))
        elif k == "t":
            out.append(Gate("p", g.qubits, (-math.pi / 4,)))
        elif k in ("u1q", "unitary"):
            out.append(Gate(k, g.qubits, matrix=np.conj(g.matrix).T))
        elif k == "diag":
            out.append(Gate(k, g.qubits, matrix=np.conj(g.matrix)))
        else:
            raise ValueError(k)
    return Circuit(c.n, out, c.basis, c.name + "_inv")


# ----------------------------------------------------------------- serving
@dataclass
class Request:
    arrival_s: float
    circuit: Circuit
    z_pairs: Tuple[Tuple[int, int], ...]
    top_k: int = 64


def serving_stream(n_requests: int, rate_hz: float, seed: int = 4,
                   n_lo: int = 10, n_hi: int = 26, d_lo: int = 10, d_hi: int = 200,
                   n_pairs: int = 16) -> List[Request]:
    """Poisson request stream: qubit count uniform in [n_lo, n_hi], depth
    uniform in [d_lo, d_hi], family uniform over layered / diagonal-heavy /
    QFT / QAOA with fresh seeds; each asks for the top-64 probabilities and
    <Z_i Z_j> on ``n_pairs`` random pairs.  Depth per family: layered -> d
    layers, diagonal-heavy -> d*ceil(n/2) gates, QFT -> fixed by n,
    QAOA -> p = max(1, d // 20)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out: List[Request] = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz)) if rate_hz > 0 else 0.0
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(d_lo, d_hi + 1))
        fam = int(rng.integers(4))
        s = int(rng.integers(1 << 30))
        if fam == 0:
            c = layered(n, d, s)
        elif fam == 1:
            c = diag_heavy(n, d * ((n + 1) // 2), s)
        elif fam == 2:
            c = qft(n, s)
        else:
            c = qaoa(n, max(1, d // 20), s)
        pairs = tuple(_distinct(rng, n, 2) for _ in range(n_pairs))
        out.append(Request(t, c, pairs))
    return out


def z_masks(pairs: Sequence[Tuple[int, int]]) -> np.ndarray:
    """Z-string masks for <Z_i Z_j> terms."""
    return np.array([(1 << a) | (1 << b) for a, b in pairs], dtype=np.uint64)
