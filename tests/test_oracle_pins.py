"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these retypes the oracle's formulas: gate matrices are checked
against exponentials of Pauli generators; whole circuits against the
Kronecker-product operator of Section 2.2 built from matrix units; and
circuits against closed forms (GHZ, uniform superposition, the discrete
Fourier transform), invariants (norm, C C^dagger = I, diagonal circuits keep
|a_x|) and brute force on tiny inputs.  ``test_planted_*`` compile mutated
copies of the oracle to show that plausible mistakes fail these pins.
"""
import math
import os
import shutil
import subprocess
import ctypes

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2604_12256_gb300 import circuits as C

X = np.array([[0, 1], [1, 0]], complex)
Y = np.array([[0, -1j], [1j, 0]], complex)
Z = np.array([[1, 0], [0, -1]], complex)
I2 = np.eye(2, dtype=complex)
P0 = np.array([[1, 0], [0, 0]], complex)
P1 = np.array([[0, 0], [0, 1]], complex)


def local2(a_hi, b_lo):
    """2-qubit local operator with local index m = b0 + 2 b1 (bit 0 = q[0])."""
    return np.kron(a_hi, b_lo)


def expected_matrix(g):
    """Independent definitions: Pauli exponentials and projector sums."""
    k, p = g.kind, g.params
    if k == "h":
        return (X + Z) / math.sqrt(2)
    if k == "x":
        return X
    if k == "y":
        return Y
    if k == "z":
        return Z
    if k == "s":
        return expm(1j * math.pi / 4 * I2) @ expm(-1j * math.pi / 4 * Z)
    if k == "t":
        return expm(1j * math.pi / 8 * I2) @ expm(-1j * math.pi / 8 * Z)
    if k == "rx":
        return expm(-1j * p[0] / 2 * X)
    if k == "ry":
        return expm(-1j * p[0] / 2 * Y)
    if k == "rz":
        return expm(-1j * p[0] / 2 * Z)
    if k == "p":
        return np.exp(1j * p[0] / 2) * expm(-1j * p[0] / 2 * Z)
    if k == "cx":   # q[0] = control = local bit 0
        return local2(I2, P0) + local2(X, P1)
    if k == "cz":
        return local2(I2, P0) + local2(Z, P1)
    if k == "cp":
        return local2(I2, P0) + local2(expm(1j * p[0] / 2 * I2) @ expm(-1j * p[0] / 2 * Z), P1)
    if k == "rzz":
        return expm(-1j * p[0] / 2 * np.kron(Z, Z))
    if k == "swap":
        return 0.5 * (np.kron(I2, I2) + np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z))
    if k in ("u1q", "unitary"):
        return g.matrix
    if k == "diag":
        return np.diag(g.matrix)
    raise ValueError(k)


@pytest.mark.parametrize("kind", ["h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p",
                                  "cx", "cz", "cp", "rzz", "swap"])
def test_gate_matrices_match_generators(kind):
    rng = np.random.default_rng(11)
    for _ in range(5):
        ar = C.GATE_ARITY[kind]
        params = (float(rng.uniform(-7, 7)),) if kind in C.GATE_NPARAMS else ()
        g = C.Gate(kind, tuple(range(ar)), params)
        np.testing.assert_allclose(oracle.gate_matrix(g), expected_matrix(g), atol=1e-14)


def full_operator(n, g):
    """The 2^n x 2^n operator of one gate as a sum over matrix units of
    Kronecker products, qubit j in the I^{n-j-1} (x) U (x) I^{j} position."""
    M = expected_matrix(g)
    k = len(g.qubits)
    dim = 1 << k
    U = np.zeros((1 << n, 1 << n), complex)
    for r in range(dim):
        for c in range(dim):
            if M[r, c] == 0:
                continue
            factors = []
            for j in range(n - 1, -1, -1):          # leftmost factor = qubit n-1
                if j in g.qubits:
                    i = g.qubits.index(j)
                    E = np.zeros((2, 2), complex)
                    E[(r >> i) & 1, (c >> i) & 1] = 1
                    factors.append(E)
                else:
                    factors.append(I2)
            op = factors[0]
            for f in factors[1:]:
                op = np.kron(op, f)
            U += M[r, c] * op
    return U


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (5, 4), (6, 5)])
def test_circuit_matches_kronecker_brute_force(n, seed):
    c = C.random_mixed(n, 30, seed, max_k=min(3, n))
    psi = oracle.basis_state(n, c.basis)
    for g in c.gates:
        psi = full_operator(n, g) @ psi
    np.testing.assert_allclose(oracle.run(c), psi, atol=1e-13)


def test_single_qubit_kron_position():
    # Section 2.2: U_j = I^{n-j-1} (x) U (x) I^{j}, checked on every j
    n = 4
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    for j in range(n):
        U = C.haar_u2(rng)
        op = np.kron(np.kron(np.eye(1 << (n - j - 1)), U), np.eye(1 << j))
        got = oracle.run(C.Circuit(n, [C.Gate("u1q", (j,), matrix=U)]), state=psi0)
        np.testing.assert_allclose(got, op @ psi0, atol=1e-14)


@pytest.mark.parametrize("n", [1, 3, 8, 13])
def test_ghz_closed_form(n):
    gates = [C.Gate("h", (0,))] + [C.Gate("cx", (0, i)) for i in range(1, n)]
    a = oracle.run(C.Circuit(n, gates))
    exp = np.zeros(1 << n, complex)
    exp[0] = exp[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(a, exp, atol=1e-15)


@pytest.mark.parametrize("n", [1, 5, 12])
def test_uniform_superposition_closed_form(n):
    a = oracle.run(C.Circuit(n, [C.Gate("h", (q,)) for q in range(n)]))
    np.testing.assert_allclose(a, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 9, 12])
def test_qft_closed_form(n):
    c = C.qft(n, seed=n)
    a = oracle.run(c)
    e = np.zeros(1 << n, complex)
    e[c.basis] = 1
    exp = np.fft.ifft(e) * math.sqrt(1 << n)     # 2^{-n/2} sum_y e^{2 pi i x y / 2^n} |y>
    np.testing.assert_allclose(a, exp, atol=1e-12)


@pytest.mark.parametrize("maker", [lambda: C.random_mixed(10, 200, 7),
                                   lambda: C.layered(9, 12, 1),
                                   lambda: C.diag_heavy(11, 150, 2),
                                   lambda: C.qaoa(10, 3, 4)])
def test_norm_and_inverse(maker):
    c = maker()
    a = oracle.run(c)
    assert abs(oracle.norm(a) - 1.0) < 1e-12
    back = oracle.run(C.inverse(c), state=a)
    exp = oracle.basis_state(c.n, c.basis)
    np.testing.assert_allclose(back, exp, atol=1e-12)


def test_diagonal_circuit_keeps_magnitudes():
    rng = np.random.default_rng(5)
    n = 9
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    c = C.diag_heavy(n, 300, 9, p_diag=1.0, prefix_h=False)
    got = oracle.run(c, state=psi)
    np.testing.assert_allclose(np.abs(got), np.abs(psi), atol=1e-14)


def test_readout_closed_forms():
    # product of RY rotations: <Z_j> = cos t_j, <Z_i Z_j> = cos t_i cos t_j
    n = 6
    th = np.linspace(0.3, 2.9, n)
    a = oracle.run(C.Circuit(n, [C.Gate("ry", (q,), (th[q],)) for q in range(n)]))
    masks = [1 << 0, 1 << 3, (1 << 1) | (1 << 4), (1 << 2) | (1 << 5), 0]
    exp = [math.cos(th[0]), math.cos(th[3]), math.cos(th[1]) * math.cos(th[4]),
           math.cos(th[2]) * math.cos(th[5]), 1.0]
    np.testing.assert_allclose(oracle.expectation_z(a, masks), exp, atol=1e-14)
    # basis state: <Z_m> = (-1)^popcount(x & m)
    x = 0b101101
    b = oracle.basis_state(n, x)
    for m in range(1 << n):
        assert oracle.expectation_z(b, [m])[0] == (-1) ** bin(x & m).count("1")


def test_fidelity_closed_forms():
    """|<a|b>|^2 for states whose overlap has a closed form: RY(t)|0> on
    every qubit against RY(u)|0> gives prod_q cos^2((t_q - u_q) / 2); a
    basis state against the uniform superposition gives 2^-n; a global
    phase changes nothing and the overlap is symmetric."""
    n = 5
    t = np.linspace(0.2, 2.6, n)
    u = np.linspace(1.9, -0.4, n)
    a = oracle.run(C.Circuit(n, [C.Gate("ry", (q,), (t[q],)) for q in range(n)]))
    b = oracle.run(C.Circuit(n, [C.Gate("ry", (q,), (u[q],)) for q in range(n)]))
    exp = float(np.prod(np.cos((t - u) / 2) ** 2))
    assert abs(oracle.fidelity(a, b) - exp) <= 1e-14
    assert abs(oracle.fidelity(b, a) - exp) <= 1e-14
    assert abs(oracle.fidelity(a, np.exp(0.83j) * a) - 1.0) <= 1e-14
    plus = oracle.run(C.Circuit(n, [C.Gate("h", (q,)) for q in range(n)]))
    assert abs(oracle.fidelity(oracle.basis_state(n, 19), plus) - 2.0 ** -n) <= 1e-15
    assert oracle.fidelity(oracle.basis_state(n, 3), oracle.basis_state(n, 4)) == 0.0


def test_top_k_brute_force_and_ties():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    a[[3, 9, 40]] = 2.0          # exact ties: must come out lowest index first
    idx, p = oracle.top_k(a, 10)
    pr = [(v.real * v.real + v.imag * v.imag, i) for i, v in enumerate(a)]
    exp = sorted(pr, key=lambda t: (-t[0], t[1]))[:10]
    assert list(idx) == [i for _, i in exp]
    np.testing.assert_allclose(p, [q for q, _ in exp], rtol=0, atol=0)
    u = np.full(32, 1 / math.sqrt(32), complex)
    idx, _ = oracle.top_k(u, 5)
    assert list(idx) == [0, 1, 2, 3, 4]


def test_invalid_gates_are_rejected():
    with pytest.raises(ValueError):
        oracle.run(C.Circuit(3, [C.Gate("cx", (1, 1))]))
    with pytest.raises(ValueError):
        oracle.run(C.Circuit(3, [C.Gate("h", (3,))]))


# ---------------------------------------------------------- planted mistakes
def _mutant(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src
    p = tmp_path / "mut.c"
    p.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(p), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_run.restype = ctypes.c_int64
    lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 6 + [ctypes.c_int]
    return lib


def _run_with(lib, c):
    a = oracle.basis_state(c.n, c.basis)
    kind, nq, qubits, params, ext, ext_off = oracle._marshal(c.gates)
    lib.orc_run(c.n, a.ctypes.data, len(c.gates), kind.ctypes.data, nq.ctypes.data, qubits.ctypes.data,
                params.ctypes.data, ext.ctypes.data, ext_off.ctypes.data, 1)
    return a


@pytest.mark.parametrize("old,new", [
    ("m[r * dim + c] * v[c]", "m[c * dim + r] * v[c]"),          # transposed operand
    ("m[0] = c; m[1] = -s; m[2] = s;", "m[0] = c; m[1] = s; m[2] = -s;"),   # RY sign
    ("m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1;", "m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;"),  # CX control/target
    ("o |= (int64_t)1 << q[i]", "o |= (int64_t)1 << sq[i]"),     # local bit order ignored
])
def test_planted_mistakes_fail_the_pins(tmp_path, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    lib = _mutant(tmp_path, old, new)
    failures = 0
    for n, seed in [(3, 2), (4, 3), (5, 4)]:
        c = C.random_mixed(n, 30, seed, max_k=3)
        rng = np.random.default_rng(seed)
        for kind in ("h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p", "cx", "cz", "cp", "rzz", "swap"):
            qs = tuple(int(v) for v in rng.choice(n, C.GATE_ARITY[kind], replace=False))
            c.gates.append(C.Gate(kind, qs, (0.7,) if kind in C.GATE_NPARAMS else ()))
        psi = oracle.basis_state(n, c.basis)
        for g in c.gates:
            psi = full_operator(n, g) @ psi
        if not np.allclose(_run_with(lib, c), psi, atol=1e-12):
            failures += 1
    assert failures > 0
