"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: complex128 max |d amp| <= 1e-12; complex64 max |d amp| <= 1e-5
and fidelity >= 1 - 1e-6 (circuits of depth <= 200 and more)."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]

TOL128 = 1e-12
TOL64 = 1e-5
FID64 = 1 - 1e-6

FLAG_SETS = {
    "unfused": 0,
    "diag": S.SIM_F_DIAG,
    "block": S.SIM_F_BLOCK,
    "all": S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_BOOST,
}


def gpu_run(c, dtype, flags=None, **kw):
    opt = S.default_options(**({"flags": flags} if flags is not None else {}), **kw)
    with S.Sim(c.n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        return s.get_state().astype(np.complex128), s.stats()


def fidelity(a, b):
    """|<a|b>|^2 / (<a|a><b|b>): the overlap of the two states as quantum
    states.  complex64 gate matrices are not exactly unitary (H's 1/sqrt2
    rounds to 0.70710677, shrinking ||psi||^2 by ~3e-8 per gate), so the
    norm drift is checked separately (NORM64) from the state's direction."""
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


NORM64 = 2e-5


def check(c, dtype, got, exp):
    err = np.max(np.abs(got - exp))
    if dtype == S.SIM_C128:
        assert err <= TOL128, err
    else:
        assert err <= TOL64, err
        assert fidelity(exp, got) >= FID64
        assert abs(np.vdot(got, got).real - 1.0) <= NORM64


def test_config0_layered14_c128():
    """14-qubit random layered circuit, complex128, depth 20 (config 0)."""
    c = C.layered(14, 20, 0)
    exp = oracle.run(c)
    for flags in FLAG_SETS.values():
        got, st = gpu_run(c, S.SIM_C128, flags)
        check(c, S.SIM_C128, got, exp)
    with S.Sim(14, S.SIM_C128) as s:
        s.apply(c.gates)
        p = s.probabilities()
    np.testing.assert_allclose(p, oracle.probabilities(exp), atol=1e-13, rtol=0)


@pytest.mark.parametrize("dtype", [S.SIM_C64, S.SIM_C128])
@pytest.mark.parametrize("flags", list(FLAG_SETS))
@pytest.mark.parametrize("maker", [
    lambda: C.random_mixed(12, 200, 1, max_k=3),
    lambda: C.random_mixed(11, 200, 2, max_k=3),
    lambda: C.random_mixed(9, 150, 3, max_k=3),
    lambda: C.random_mixed(7, 100, 4, max_k=3),
    lambda: C.diag_heavy(16, 300, 5),
    lambda: C.qft(15, 6),
    lambda: C.qaoa(16, 3, 7),
    lambda: C.layered(13, 8, 8),
    lambda: C.rzz_full(14, 9),
], ids=["mixed12", "mixed11", "mixed9", "mixed7", "diag16", "qft15", "qaoa16", "layered13", "rzz14"])
def test_parity_small(maker, flags, dtype):
    c = maker()
    exp = oracle.run(c)
    got, _ = gpu_run(c, dtype, FLAG_SETS[flags])
    check(c, dtype, got, exp)


@pytest.mark.parametrize("dtype", [S.SIM_C64, S.SIM_C128])
@pytest.mark.parametrize("maker", [
    lambda: C.diag_heavy(21, 500, 11),
    lambda: C.qft(20, 12),
    lambda: C.qaoa(20, 4, 13),
    lambda: C.layered(19, 20, 14),
    lambda: C.random_mixed(20, 300, 15, max_k=3),
], ids=["diag21", "qft20", "qaoa20", "layered19", "mixed20"])
def test_parity_multi_tile(maker, dtype):
    """Sizes that span hundreds of chunks (2^12 amplitudes each)."""
    c = maker()
    exp = oracle.run(c)
    got, st = gpu_run(c, dtype)
    check(c, dtype, got, exp)
    assert st["sweeps"] < len(c.gates)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_tiny_registers(n):
    c = C.random_mixed(n, 60, 20 + n, max_k=min(3, n))
    exp = oracle.run(c)
    for dtype in (S.SIM_C64, S.SIM_C128):
        got, _ = gpu_run(c, dtype)
        check(c, dtype, got, exp)


def test_empty_circuit_and_reset():
    with S.Sim(13, S.SIM_C64) as s:
        s.reset(1234)
        s.apply([])
        a = s.get_state()
        assert a[1234] == 1 and np.count_nonzero(a) == 1
        with pytest.raises(S.SimError):
            s.reset(1 << 13)


@pytest.mark.parametrize("dtype", [S.SIM_C64, S.SIM_C128])
def test_readouts(dtype):
    c = C.random_mixed(14, 150, 30, max_k=2)
    exp = oracle.run(c)
    masks = [1 << 0, (1 << 3) | (1 << 9), (1 << 13) | (1 << 2), 0x3FFF, 0, 0b1010101]
    with S.Sim(14, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates)
        tol = 1e-12 if dtype == S.SIM_C128 else 2e-5
        assert abs(s.norm() - 1.0) <= tol
        np.testing.assert_allclose(s.expectation(masks), oracle.expectation_z(exp, masks), atol=tol)
        np.testing.assert_allclose(s.probabilities(), oracle.probabilities(exp), atol=tol)
        k = 64
        idx, p = s.top_k(k)
        eidx, ep = oracle.top_k(exp, k)
        np.testing.assert_allclose(p, ep, atol=tol)
        if dtype == S.SIM_C128:
            assert list(idx) == list(eidx)
        else:   # near-ties may swap in complex64: every index must be a valid top-k member
            pe = oracle.probabilities(exp)
            assert len(set(idx.tolist())) == k
            assert np.all(pe[idx.astype(np.int64)] >= ep[-1] - 2 * tol)


@pytest.mark.parametrize("dtype", [S.SIM_C64, S.SIM_C128])
@pytest.mark.parametrize("k", [1, 64, 1000])
def test_topk_large_random_state(dtype, k):
    """Top-k over 2^21 amplitudes (many blocks, the float pre-filter and the
    merge pass): the same probabilities as the oracle's definition, exactly,
    and the same indices (ties to the lower index)."""
    n = 21
    rng = np.random.default_rng(k)
    a = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) * (rng.random(1 << n) ** 3)
    a /= np.linalg.norm(a)
    a[[5, 77, 123456]] = a[999]          # exact ties
    with S.Sim(n, dtype) as s:
        s.set_state(a)
        ref = s.get_state().astype(np.complex128)   # the values the GPU holds
        idx, p = s.top_k(k)
    eidx, ep = oracle.top_k(ref, k)
    assert list(idx) == list(eidx)
    np.testing.assert_array_equal(p, ep)


def _topk_state(n, seed, peaks=()):
    """a random complex64-representable state; `peaks` = (start, count):
    that many large distinct amplitudes at consecutive indices"""
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) * 1e-3
    for start, count in peaks:
        a[start:start + count] = np.linspace(1.0, 2.0, count) * np.exp(1j * rng.uniform(0, 6.28, count))
    return a / np.linalg.norm(a)


@pytest.mark.parametrize("k,peaks,launches", [
    (64, (), 3),                        # spread: the warps' best 16 suffice, one pass
    (128, (), 3),
    (64, ((1024, 40),), 6),             # 40 of the top 64 in one warp's slice: exact rerun
    (64, ((1024, 15), (8192, 15)), None),   # 15 per slice: below the rerun bound, still exact
    (17, ((4096, 17),), 6),             # k just above the per-warp keep, all in one slice
])
def test_topk_warp_keep_and_rerun(k, peaks, launches):
    """complex64 top-k with k <= 128 first lets each warp keep only its best
    16 candidates; the result is exact unless some warp's whole kept list is
    in it, and then the call reruns the kernel that keeps k per warp (3
    kernel launches per pass).  Either way the result equals the oracle's."""
    n = 20
    a = _topk_state(n, k + len(peaks), peaks)
    with S.Sim(n, S.SIM_C64) as s:
        s.set_state(a)
        ref = s.get_state().astype(np.complex128)
        l0 = S.kernel_launches()
        idx, p = s.top_k(k)
        used = S.kernel_launches() - l0
    eidx, ep = oracle.top_k(ref, k)
    assert list(idx) == list(eidx)
    np.testing.assert_array_equal(p, ep)
    if launches is not None:
        assert used == launches
    else:
        assert used in (3, 6)


def test_topk_ties_uniform():
    with S.Sim(16, S.SIM_C64) as s:
        s.apply([C.Gate("h", (q,)) for q in range(16)])
        idx, p = s.top_k(100)
        assert list(idx) == list(range(100))
        np.testing.assert_allclose(p, 2.0 ** -16, rtol=1e-6)


def test_deterministic():
    c = C.diag_heavy(20, 300, 40)
    a1, _ = gpu_run(c, S.SIM_C64)
    a2, _ = gpu_run(c, S.SIM_C64)
    assert np.array_equal(a1, a2)


def test_set_get_state_roundtrip():
    rng = np.random.default_rng(0)
    a = (rng.standard_normal(1 << 12) + 1j * rng.standard_normal(1 << 12))
    a /= np.linalg.norm(a)
    c = C.random_mixed(12, 80, 41)
    exp = oracle.run(c, state=a)
    with S.Sim(12, S.SIM_C128) as s:
        s.set_state(a)
        s.apply(c.gates)
        np.testing.assert_allclose(s.get_state(), exp, atol=TOL128)


@pytest.mark.parametrize("dtype", [S.SIM_C64, S.SIM_C128])
def test_full_size_config1_properties(dtype):
    """28-qubit diagonal-heavy stream at full size (the bench workload):
    norm preserved and C C^dagger returns |0...0>."""
    c = C.diag_heavy(28, 500, 1)
    with S.Sim(28, dtype) as s:
        s.apply(c.gates)
        nrm = s.norm()
        s.apply(C.inverse(c).gates)
        idx, p = s.top_k(2)
    tol = 1e-12 if dtype == S.SIM_C128 else 1e-5
    assert abs(nrm - 1) < tol * 10
    assert idx[0] == 0 and abs(p[0] - 1) < (1e-11 if dtype == S.SIM_C128 else 1e-4)
    assert p[1] < 1e-10


def test_qubit_reversal_by_swaps():
    """A full qubit reversal as SWAP gates on a random state: the relabelling
    chunk stores give the permuted state exactly (a permutation moves
    amplitudes without arithmetic)."""
    n = 20
    rng = np.random.default_rng(11)
    a = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
    c = C.Circuit(n, [C.Gate("swap", (i, n - 1 - i)) for i in range(n // 2)])
    exp = oracle.run(c, state=a.astype(np.complex128))
    with S.Sim(n, S.SIM_C64) as s:
        s.set_state(a)
        s.apply(c.gates)
        got = s.get_state()
        assert s.stats()["sweeps"] <= 3
    assert np.array_equal(got, exp.astype(np.complex64))


@pytest.mark.parametrize("dtype,tol", [(S.SIM_C128, 1e-12), (S.SIM_C64, 1e-5)])
def test_remap_frames_on_gpu(dtype, tol):
    """Qubit reordering through the block stores (SIM_F_REMAP): the blocks
    run in moving frames and the state comes back in the identity frame."""
    c = C.layered(20, 12, 4)
    flags = S.SIM_F_DIAG | S.SIM_F_BOOST | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_REMAP
    exp = oracle.run(c)
    with S.Sim(c.n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates, S.default_options(flags=flags))
        got = s.get_state().astype(np.complex128)
    assert np.abs(got - exp).max() < tol


@pytest.mark.parametrize("dtype,tol", [(S.SIM_C128, 1e-12), (S.SIM_C64, 1e-5)])
def test_rzz_full_fed_phase_sweep(dtype, tol):
    """Full-connectivity RZZ at 24 qubits: the merge booster's last product
    (two 12-qubit halves) is computed by the loads of the single fused phase
    sweep, whose tiles share one hi factor."""
    c = C.rzz_full(24)
    exp = oracle.run(c)
    with S.Sim(c.n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates)
        st = s.stats()
        got = s.get_state().astype(np.complex128)
    assert st["tensor_fused"] == 1 and st["sweeps"] == 1
    assert np.abs(got - exp).max() < tol


@pytest.mark.parametrize("n", [22, 24])
def test_expectation_on_larger_states(n):
    """<Z-string> at sizes where every thread of the reduction grid walks
    several amplitudes (Gray-code parity updates across the grid stride),
    with masks on bits below and above the stride; the reference is the same
    sum in FP64 over the GPU's own state."""
    rng = np.random.default_rng(n)
    a = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
    a /= np.linalg.norm(a)
    masks = [1, (1 << 17) | (1 << 18), (1 << (n - 1)) | 1, (1 << 19) | (1 << 5) | (1 << 21), (1 << n) - 1, 0,
             (1 << 20) | (1 << 3)]
    with S.Sim(n, S.SIM_C64) as s:
        s.set_state(a)
        got = s.expectation(masks)
        back = s.get_state()
    exp = oracle.expectation_z(back.astype(np.complex128), masks)
    np.testing.assert_allclose(got, exp, atol=2e-6, rtol=0)


@pytest.mark.parametrize("nmask", [0, 5, 16, 21])
def test_combined_readout_equals_separate_calls(nmask):
    """sim_top_k_expectation runs the top-k and the <Z> sums concurrently
    on two streams: the results are bit-equal to the two separate calls,
    and equal the oracle's within the complex64 tolerance."""
    c = C.diag_heavy(20, 150, 17)
    rng = np.random.default_rng(nmask)
    masks = [int(rng.integers(1, 1 << 20)) for _ in range(nmask)]
    with S.Sim(20, S.SIM_C64) as s:
        s.reset(c.basis)
        s.apply(c.gates)
        i1, p1 = s.top_k(64)
        e1 = s.expectation(masks) if nmask else np.zeros(0)
        for _ in range(2):   # twice: the second stream and events are reused
            i2, p2, e2 = s.top_k_expectation(64, masks)
            assert np.array_equal(i1, i2) and np.array_equal(p1, p2) and np.array_equal(e1, e2)
    exp = oracle.run(c)
    if nmask:
        np.testing.assert_allclose(e2, oracle.expectation_z(exp, masks), atol=2e-5)
    np.testing.assert_allclose(p2, oracle.top_k(exp, 64)[1], atol=2e-5)
