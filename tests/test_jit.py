"""Specialised sweep kernels on the CPU: the generated source of every chunk
and fused diagonal sweep program of a plan compiles (NVRTC, no GPU needed)."""
import pytest

from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = pytest.mark.usefixtures("built_lib")


def test_generated_sources_compile():
    c = C.random_mixed(13, 120, 31)   # dense 1- and 2-qubit ops, phases, swaps
    opt = S.default_options(flags=S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_JIT)
    n = S.jit_check(c.n, c.gates, S.SIM_C64, c.basis, opt)
    plan = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, opt)
    assert n >= sum(1 for o in plan["ops"] if o["op"] == "chunk") >= 1   # + fused diagonal sweeps


def test_complex128_has_no_specialised_kernels():
    c = C.random_mixed(13, 40, 32)
    assert S.jit_check(c.n, c.gates, S.SIM_C128, c.basis, S.default_options(flags=S.SIM_F_BLOCK | S.SIM_F_JIT)) == 0


def test_diagonal_sweep_sources_compile():
    c = C.rzz_full(14, 3)
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    assert S.jit_check(c.n, c.gates, S.SIM_C64, c.basis, opt) >= 1


def _redraw(c, seed):
    """The same circuit with every angle and one-qubit matrix drawn anew."""
    import math
    import numpy as np
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


@pytest.mark.parametrize("maker", [lambda: C.diag_heavy(28, 500, 1), lambda: C.layered(26, 20, 0),
                                   lambda: C.qaoa(26, 4, 3), lambda: C.random_mixed(20, 300, 11)],
                         ids=["diag_heavy28", "layered26", "qaoa26", "mixed20"])
def test_sources_hold_structure_only(maker):
    """Kernels are keyed by their generated source, which holds the program's
    structure only: the same circuit with fresh angles (and fresh Haar
    one-qubit matrices) generates the same sources, so it reuses the cached
    kernels; the numbers travel in the parameter block."""
    c = maker()
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    a = S.jit_sources(c.n, c.gates, S.SIM_C64, c.basis, opt)
    assert "specialised sweep" in a and "P.w[" in a
    for seed in (101, 102):
        assert S.jit_sources(c.n, _redraw(c, seed).gates, S.SIM_C64, c.basis, opt) == a


@pytest.mark.parametrize("maker", [lambda: C.diag_heavy(28, 500, 1), lambda: C.layered(26, 20, 0),
                                   lambda: C.qft(24, 2), lambda: C.rzz_full(14, 3)],
                         ids=["diag_heavy28", "layered26", "qft24", "rzz14"])
def test_parameter_blocks_hold_aligned_packed_constants(maker):
    """A specialised kernel reads each constant phase factor as two 64-bit
    packed operands of its parameter block: every such read starts on an
    even word (8-byte aligned, the block being declared 8-byte aligned) and
    lies inside the block, and every block is a whole number of 8-byte units
    (the launch passes exactly its words)."""
    import re
    c = maker()
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    src = S.jit_sources(c.n, c.gates, S.SIM_C64, c.basis, opt)
    parts = [p for p in re.split(r"(?=// ---- specialised sweep)", src) if p.startswith("// ---- specialised")]
    assert parts
    packed = 0
    for p in parts:
        words = int(re.match(r"// ---- specialised sweep \d+: (\d+) parameter words", p).group(1))
        assert words % 2 == 0
        assert "struct __align__(8) JP { uint32_t w[%d]; };" % words in p
        for k in map(int, re.findall(r"\*\(const u64 \*\)&P\.w\[(\d+)\]", p)):
            assert k % 2 == 0 and k + 1 < words
            packed += 1
        # the amplitudes' phase products are packed (no scalar product of an amplitude)
        assert not re.search(r"v\[\d+\] = cmul\(v\[", p)
    assert packed > 0   # each of these circuits has constant phase factors
