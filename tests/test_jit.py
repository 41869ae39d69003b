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
