"""Full-size workloads, in the launch configuration the bench times, checked
through properties that hold at any size (the oracle cannot hold these
states): the norm, closed-form probability distributions and C C^dagger
returning |0...0>.  Read out with the device kernels (norm, top-k), without
copying the 128 GiB states to the host."""
import numpy as np
import pytest

from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]


def _uniform(s, n, rel):
    """Every basis state has probability 2^-n: the 64 largest do too."""
    idx, p = s.top_k(64)
    assert len(set(idx.tolist())) == 64
    np.testing.assert_allclose(p, 2.0 ** -n, rtol=rel, atol=0)


@pytest.mark.parametrize("n,dtype,rel,jit", [(30, S.SIM_C64, 1e-4, False), (30, S.SIM_C64, 1e-4, True),
                                            (33, S.SIM_C128, 1e-10, False)])
def test_qft_of_a_basis_state_is_uniform(n, dtype, rel, jit):
    """QFT|x> = 2^(-n/2) sum_y e^{2 pi i x y / 2^n} |y>: all magnitudes equal
    (the 30-qubit circuit-level workload, also on the kernels specialised to
    their programs as the bench runs it; 33 qubits in complex128)."""
    c = C.qft(n, 2)
    opt = S.default_options(flags=S.default_options().flags | (S.SIM_F_JIT if jit else 0))
    with S.Sim(n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        assert abs(s.norm() - 1.0) < 10 * rel
        _uniform(s, n, rel)


def test_rzz_full_34_keeps_uniform_magnitudes():
    """Diagonal gates after H on every qubit keep |a_x| = 2^-17 for all x:
    the 34-qubit gate-level workload, one fused write-only phase sweep."""
    c = C.rzz_full(34)
    with S.Sim(34, S.SIM_C64) as s:
        s.reset(0)
        s.apply(c.gates)
        assert s.stats()["sweeps"] == 1
        assert abs(s.norm() - 1.0) < 1e-4
        _uniform(s, 34, 1e-4)


def test_layered_34_dense_blocks_inverse_returns_zero():
    """The 34-qubit depth-20 layered circuit in split-TF32 dense 5-qubit
    blocks on the tensor cores, then its inverse: back to |0...0>."""
    c = C.layered(34, 20, 0)
    opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG, dense_precision=S.SIM_DENSE_SPLIT_TF32)
    with S.Sim(34, S.SIM_C64) as s:
        s.reset(0)
        s.apply(c.gates, opt)
        assert s.stats()["dense_ops"] > 0
        assert abs(s.norm() - 1.0) < 1e-3
        s.apply(C.inverse(c).gates, opt)
        idx, p = s.top_k(2)
    assert idx[0] == 0 and abs(p[0] - 1.0) < 1e-3 and p[1] < 1e-6


def test_diag_heavy_28_specialised_inverse_returns_basis():
    """The 28-qubit diagonal-heavy stream in the bench's configuration (merge
    booster, diagonal detector, chunk sweeps on the kernels specialised to
    their programs), then its inverse on the same path: back to the basis
    state, with the norm kept."""
    c = C.diag_heavy(28, 500, 1)
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    with S.Sim(28, S.SIM_C64) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        st = s.stats()
        assert st["sweeps"] == 7 and st["diag_fused"] > 0
        assert S.jit_info()["programs"] > 0
        assert abs(s.norm() - 1.0) < 1e-4
        s.apply(C.inverse(c).gates, opt)
        idx, p = s.top_k(2)
    assert idx[0] == c.basis and abs(p[0] - 1.0) < 1e-3 and p[1] < 1e-6
