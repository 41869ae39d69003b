"""Circuit families of the per-gate comparison (Table 2): closed-form outputs
pin the generators through the oracle, and the optimizer's plans for every
family are exact (CPU plan interpreter vs the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S
from plan_interp import interpret

pytestmark = pytest.mark.usefixtures("built_lib")


@pytest.mark.parametrize("n", [5, 9, 12])
def test_bernstein_vazirani_returns_the_secret(n):
    c = C.bernstein_vazirani(n, seed=n)
    s = int(c.name.split("secret=")[1])
    p = oracle.probabilities(oracle.run(c))
    anc = 1 << (n - 1)
    np.testing.assert_allclose([p[s], p[s | anc]], [0.5, 0.5], atol=1e-12)
    assert abs(p.sum() - 1.0) < 1e-12 and p[s] + p[s | anc] > 1 - 1e-12
    # the ancilla is |->: the two amplitudes have opposite signs
    a = oracle.run(c)
    assert abs(a[s] + a[s | anc]) < 1e-12


@pytest.mark.parametrize("n", [4, 8, 12])
def test_hidden_shift_returns_the_shift(n):
    c = C.hidden_shift(n, seed=n + 1)
    s = int(c.name.split("shift=")[1])
    p = oracle.probabilities(oracle.run(c))
    assert abs(p[s] - 1.0) < 1e-12


def test_family_gates_are_unitary_and_shaped():
    for name, f in C.FAMILIES.items():
        c = f(8)
        for g in c.gates:
            if g.matrix is not None:
                m = np.asarray(g.matrix).reshape(1 << len(g.qubits), -1)
                assert np.abs(m @ m.conj().T - np.eye(len(m))).max() < 1e-12, name
        a = oracle.run(c)
        assert abs(np.vdot(a, a).real - 1.0) < 1e-12, name
    assert len(C.quantum_volume(6).gates) == 6 * 3
    assert sum(g.kind == "cz" for g in C.variational(6, 4).gates) == 4 * 5


@pytest.mark.parametrize("name", sorted(C.FAMILIES))
@pytest.mark.parametrize("flags", [S.SIM_F_DIAG | S.SIM_F_BOOST | S.SIM_F_BLOCK | S.SIM_F_FUSE,
                                   S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE])
def test_family_plans_are_exact(name, flags):
    c = C.FAMILIES[name](14)
    plan = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, S.default_options(flags=flags))
    np.testing.assert_allclose(interpret(plan, basis=c.basis), oracle.run(c), atol=1e-12, rtol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(C.FAMILIES))
def test_family_parity_on_gpu(name):
    c = C.FAMILIES[name](16)
    exp = oracle.run(c)
    for dt, tol in ((S.SIM_C128, 1e-12), (S.SIM_C64, 1e-5)):
        with S.Sim(c.n, dt) as s:
            s.reset(c.basis)
            s.apply(c.gates)
            got = s.get_state().astype(np.complex128)
        assert np.abs(got - exp).max() < tol, (name, dt)
        if dt == S.SIM_C64:
            fid = abs(np.vdot(exp, got)) ** 2 / np.vdot(got, got).real
            assert fid > 1 - 1e-6, name
