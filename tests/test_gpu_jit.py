"""Chunk sweeps specialised to their program (SIM_F_JIT) against the
interpreter kernel and the oracle.

The specialised kernel runs the same device templates as the interpreter
with the program's op sequence, register positions and one-qubit matrices
compiled in; the two states agree to within a few float ulps (max |d amp|
<= 1e-6 here); the oracle comparison uses the complex64 tolerances (max
|d amp| <= 1e-5, fidelity >= 1 - 1e-6)."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]

BASE = S.SIM_F_DIAG | S.SIM_F_BOOST | S.SIM_F_BLOCK | S.SIM_F_FUSE


def run(c, flags, **kw):
    opt = S.default_options(flags=flags, **kw)
    with S.Sim(c.n, S.SIM_C64) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        st = s.stats()
        return s.get_state(), st


# every op kind of a chunk program: one-qubit special forms (H, RX, RY) and
# general 2x2, fused two-qubit blocks, phase segments without and with the
# register-only table and with terms on several register bits (3-qubit
# diagonals), SWAP relabels, sweeps fed by the merge booster
CASES = {
    "diag_heavy16": lambda: C.diag_heavy(16, 300, 3),
    "layered16": lambda: C.layered(16, 12, 1),
    "qft16_swaps": lambda: C.qft(16, 5),
    "qaoa16": lambda: C.qaoa(16, 2, 3),
    "mixed16": lambda: C.random_mixed(16, 300, 11),
    "mixed14": lambda: C.random_mixed(14, 400, 12),
    "supremacy16": lambda: C.supremacy(16, 8, 13),
    "rzz_full16": lambda: C.rzz_full(16, 14),   # a fused diagonal sweep (K3) fed by the booster
}


@pytest.mark.parametrize("rb", [4, 5])
@pytest.mark.parametrize("name", sorted(CASES))
def test_jit_equals_interpreter(name, rb):
    """Same plan (explicit register bits), both kernels."""
    c = CASES[name]()
    ref, st_ref = run(c, BASE, register_bits=rb, chunk_qubits=12)
    got, st = run(c, BASE | S.SIM_F_JIT, register_bits=rb, chunk_qubits=12)
    assert st["chunk_ops"] + st["diag_ops"] > 0
    st.pop("plan_ms"), st_ref.pop("plan_ms")
    assert st == st_ref   # same plan
    assert np.max(np.abs(got - ref)) <= 1e-6


@pytest.mark.parametrize("rb", [0, 4])
def test_jit_against_oracle(rb):
    """The default shape of specialised kernels (32 amplitudes per thread)
    and the 16-amplitude one."""
    c = C.random_mixed(15, 250, 21)
    exp = oracle.run(c)
    got, _ = run(c, BASE | S.SIM_F_JIT, register_bits=rb)
    got = got.astype(np.complex128)
    assert np.max(np.abs(got - exp)) <= 1e-5
    assert abs(np.vdot(got, exp)) ** 2 / (np.vdot(got, got).real * np.vdot(exp, exp).real) >= 1 - 1e-6


def test_jit_cached_and_launch_count():
    """A second apply of the same circuit reuses the compiled kernels: same
    number of launches as the interpreter, same result."""
    c = C.diag_heavy(18, 200, 4)
    a, st = run(c, BASE | S.SIM_F_JIT)
    k0 = S.kernel_launches()
    b, _ = run(c, BASE | S.SIM_F_JIT)
    k1 = S.kernel_launches()
    d, _ = run(c, BASE, register_bits=5)
    k2 = S.kernel_launches()
    assert k1 - k0 == k2 - k1
    assert np.array_equal(a, b) and np.max(np.abs(a - d)) <= 1e-6


def _redraw(c, seed):
    import math
    rng = np.random.default_rng(seed)
    gs = []
    for g in c.gates:
        if g.kind == "u1q":
            gs.append(C.Gate("u1q", g.qubits, matrix=C.haar_u2(rng)))
        elif g.params:
            gs.append(C.Gate(g.kind, g.qubits, tuple(float(rng.uniform(0, 2 * math.pi)) for _ in g.params)))
        else:
            gs.append(g)
    return C.Circuit(c.n, gs, c.basis, c.name)


def test_fresh_angles_reuse_kernels():
    """After a warm run of the 28-qubit diagonal-heavy stream, the same
    stream with every angle drawn anew compiles nothing (its kernels hold
    the structure, its numbers go in the parameter block) and still agrees
    with the interpreter; a 22-qubit stream with fresh angles agrees with the
    oracle."""
    c = C.diag_heavy(28, 500, 1)
    opt = S.default_options(flags=BASE | S.SIM_F_JIT)
    with S.Sim(28, S.SIM_C64) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        s.sync()
        before = S.jit_info()["compiles"]
        for seed in (7, 8):
            f = _redraw(c, seed)
            s.reset(f.basis)
            s.apply(f.gates, opt)
            got = s.get_state()
            assert S.jit_info()["compiles"] == before
            s.reset(f.basis)
            s.apply(f.gates, S.default_options(flags=BASE, register_bits=5))
            assert np.max(np.abs(got - s.get_state())) <= 1e-6
    small = C.diag_heavy(22, 300, 3)
    run(small, BASE | S.SIM_F_JIT)
    before = S.jit_info()["compiles"]
    f = _redraw(small, 9)
    got, _ = run(f, BASE | S.SIM_F_JIT)
    assert S.jit_info()["compiles"] == before
    exp = oracle.run(f)
    got = got.astype(np.complex128)
    assert np.max(np.abs(got - exp)) <= 1e-5
    assert abs(np.vdot(got, exp)) ** 2 / (np.vdot(got, got).real * np.vdot(exp, exp).real) >= 1 - 1e-6


def test_cache_limit_evicts_and_recompiles():
    """With room for two kernels, a plan of more programs evicts (unloading
    the modules once the device is idle) and recompiles on its next apply;
    results stay exact to the interpreter.  The limit is restored after."""
    c = C.random_mixed(18, 300, 41)
    try:
        S.jit_cache_limit(2)
        a, _ = run(c, BASE | S.SIM_F_JIT)
        assert S.jit_info()["programs"] <= 2
        before = S.jit_info()["compiles"]
        b, _ = run(c, BASE | S.SIM_F_JIT)
        assert S.jit_info()["compiles"] > before
        assert np.array_equal(a, b)
        ref, _ = run(c, BASE, register_bits=5)
        assert np.max(np.abs(a - ref)) <= 1e-6
    finally:
        S.jit_cache_limit(256)
