"""Dense 5-qubit fused blocks (tensor-core GEMM path) against the oracle:
split-TF32 on the tensor cores and FP32 CUDA cores for complex64 states,
double-float (about 48 bits) and true FP64 for complex128 states."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]

PRECISIONS = [(S.SIM_C64, S.SIM_DENSE_SPLIT_TF32, 1e-5), (S.SIM_C64, S.SIM_DENSE_FP32, 1e-5),
              (S.SIM_C128, S.SIM_DENSE_DOUBLE_FLOAT, 1e-12), (S.SIM_C128, S.SIM_DENSE_FP64, 1e-12)]


def fid(a, b):
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def run_tc(c, dtype, prec):
    opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG, dense_precision=prec)
    with S.Sim(c.n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        st = s.stats()
        return s.get_state().astype(np.complex128), st


@pytest.mark.parametrize("dtype,prec,tol", PRECISIONS, ids=["tf32x3", "fp32", "double-float", "fp64"])
@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4), (3, 7, 9, 11, 14), (10, 11, 12, 13, 14), (13, 1, 6, 12, 5)])
def test_single_block(dtype, prec, tol, targets):
    rng = np.random.default_rng(sum(targets))
    n = 15
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    g = C.Gate("unitary", targets, matrix=C.haar_unitary(rng, 32))
    c = C.Circuit(n, [g])
    exp = oracle.run(c, state=psi)
    opt = S.default_options(flags=S.SIM_F_TC, dense_precision=prec)
    with S.Sim(n, dtype) as s:
        s.set_state(psi)
        s.apply(c.gates, opt)
        assert s.stats()["dense_ops"] == 1
        got = s.get_state().astype(np.complex128)
    err = np.max(np.abs(got - exp))
    assert err <= tol * 0.1, err


@pytest.mark.parametrize("dtype,prec,tol", PRECISIONS, ids=["tf32x3", "fp32", "double-float", "fp64"])
@pytest.mark.parametrize("maker", [lambda: C.layered(14, 8, 3), lambda: C.random_mixed(13, 150, 9, max_k=3),
                                   lambda: C.qft(12, 5), lambda: C.layered(20, 6, 4)],
                         ids=["layered14", "mixed13", "qft12", "layered20"])
def test_circuits(dtype, prec, tol, maker):
    c = maker()
    exp = oracle.run(c)
    got, st = run_tc(c, dtype, prec)
    assert st["dense_ops"] > 0
    err = np.max(np.abs(got - exp))
    assert err <= tol, err
    if dtype == S.SIM_C64:
        assert fid(exp, got) >= 1 - 1e-6


def test_split_tf32_keeps_fp32_grade_accuracy():
    """Split-TF32 (three products, hi.hi apart from the hi.lo + lo.hi
    corrections) stays within a small factor of the FP32 CUDA-core path's
    error against the oracle (one TF32 product alone keeps ~11 bits, 2^13
    times coarser than FP32's 24); the omitted lo.lo term is 2^-22 relative."""
    c = C.layered(16, 10, 11)
    exp = oracle.run(c)
    e_tc = np.max(np.abs(run_tc(c, S.SIM_C64, S.SIM_DENSE_SPLIT_TF32)[0] - exp))
    e_32 = np.max(np.abs(run_tc(c, S.SIM_C64, S.SIM_DENSE_FP32)[0] - exp))
    assert e_tc <= 16 * e_32 + 1e-9, (e_tc, e_32)
    assert e_tc <= 1e-6


def test_bounded_wait_times_out_and_recovers():
    """The tensor-core kernel's mbarrier waits are bounded: with its MMA issue
    suppressed (self-test entry point) every wait gives up, the kernel sets its
    status word, leaves the state alone and frees its tensor memory, and a
    normal block launch afterwards is still exact; then the regular path
    reports no timeout."""
    lib = S.load()
    assert lib.sim_selftest_wait_timeout() == S.SIM_OK, (lib.sim_global_error() or b"").decode()
    c = C.layered(12, 2, 3)
    opt = S.default_options(flags=S.SIM_F_TC, dense_precision=S.SIM_DENSE_SPLIT_TF32)
    with S.Sim(12, S.SIM_C64) as s:
        s.reset(0)
        s.apply(c.gates, opt)
        got = s.get_state()
    exp = oracle.run(c)
    assert np.abs(got - exp).max() < 1e-5


def test_fp64_and_double_float_agree():
    """The two complex128 arms on a 20-qubit layered circuit: true FP64 (the
    reference of the precision study) and double-float agree far inside the
    complex128 tolerance."""
    c = C.layered(20, 8, 21)
    a, _ = run_tc(c, S.SIM_C128, S.SIM_DENSE_FP64)
    b, _ = run_tc(c, S.SIM_C128, S.SIM_DENSE_DOUBLE_FLOAT)
    assert np.max(np.abs(a - b)) <= 1e-13
