"""Element-wise parity at the sizes where the benchmarked kernels take their
full-size code paths.

- The chunk sweep specialised to its program (svs_chunk_jit) runs a
  persistent grid of SMs x resident CTAs; only when a launch has more chunks
  of 2^12 amplitudes than CTAs does a CTA loop over chunks (the next chunk's
  phase sums, the rotation of its triple-buffered CTA tables).  The cases
  below run at 22-23 qubits (1024-2048 chunks on at most 456 CTAs) and at the
  28-qubit diagonal-heavy stream itself, in the bench's configuration.
- The dense 5-qubit block kernels loop over tiles of 128 columns from
  2^(n-5) > 128 x grid: 24 qubits puts about 13 tiles on every tensor-core
  CTA (grid 2 x SMs) and 3 column blocks on every CUDA-core CTA (grid 8 x SMs).
- The 30-qubit QFT is compared with its closed form (Eq. 1 state of
  QFT|x>) on every amplitude; the 33-qubit complex128 QFT and the 34-qubit
  full-connectivity RZZ stream on seeded samples of indices.

Tolerances are the stated ones: complex128 max |d amp| <= 1e-12; complex64
max |d amp| <= 1e-5 and fidelity >= 1 - 1e-6 against the complex128 oracle.
Where amplitudes are far below 1e-5 in magnitude (2^-15 and smaller) the
absolute bound says little, so those checks also bound the error relative
to the amplitude's magnitude."""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]

TOL128 = 1e-12
TOL64 = 1e-5
FID64 = 1 - 1e-6
BASE = S.SIM_F_DIAG | S.SIM_F_BOOST | S.SIM_F_BLOCK | S.SIM_F_FUSE


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _fid(a, b):
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def _check64(got, exp):
    got = got.astype(np.complex128)
    err = float(np.max(np.abs(got - exp)))
    assert err <= TOL64, err
    assert _fid(exp, got) >= FID64
    return err


def _run(c, dtype, opt):
    with S.Sim(c.n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates, opt)
        return s.get_state(), s.stats()


class DeviceState:
    """A simulator whose state lives in a torch-owned device buffer, so that a
    test can read slices and gathers of a state too large to copy whole."""

    def __init__(self, n, dtype):
        import torch
        self.torch = torch
        # 2^n interleaved (re, im) pairs of the dtype's real type
        fdt = torch.float64 if dtype == S.SIM_C128 else torch.float32
        self.buf = torch.empty(2 << n, dtype=fdt, device="cuda")
        self.cview = self.buf.view(torch.complex128 if dtype == S.SIM_C128 else torch.complex64)
        stream = torch.cuda.current_stream()
        self.sim = S.Sim(n, dtype, dev_buf=self.buf.data_ptr(), nbytes=self.buf.numel() * self.buf.element_size(),
                         stream=stream.cuda_stream)

    def sync(self):
        self.torch.cuda.synchronize()

    def slice(self, lo, hi):
        """Amplitudes lo..hi-1 (call sync() first)."""
        return self.cview[lo:hi].cpu().numpy().astype(np.complex128)

    def gather(self, idx):
        self.torch.cuda.synchronize()
        t = self.torch.as_tensor(np.asarray(idx, np.int64), device="cuda")
        return self.cview[t].cpu().numpy().astype(np.complex128)

    def close(self):
        self.sim.close()
        del self.cview, self.buf
        self.torch.cuda.empty_cache()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------- chunk sweeps
# the op kinds of chunk programs (one-qubit special forms and general 2x2,
# fused two-qubit blocks, phase segments of every shape, SWAP relabels,
# sweeps fed by the merge booster) at sizes where every CTA runs several chunks
CASES22 = {
    "diag_heavy22": lambda: C.diag_heavy(22, 300, 3),
    "layered22": lambda: C.layered(22, 12, 1),
    "qft22_swaps": lambda: C.qft(22, 5),
    "qaoa22": lambda: C.qaoa(22, 2, 3),
    "qaoa24p4": lambda: C.qaoa(24, 4, 7),
    "mixed22": lambda: C.random_mixed(22, 300, 11),
    "mixed23": lambda: C.random_mixed(23, 400, 12),
    "supremacy22": lambda: C.supremacy(22, 8, 13),
    "rzz_full22": lambda: C.rzz_full(22, 14),   # a fused diagonal sweep fed by the booster
}
_oracle_cache = {}


def _oracle(name):
    if name not in _oracle_cache:
        c = CASES22[name]()
        _oracle_cache[name] = (c, oracle.run(c))
    return _oracle_cache[name]


@pytest.mark.parametrize("shape", [(12, 4), (12, 5), (13, 5)], ids=["C12RB4", "C12RB5", "C13RB5"])
@pytest.mark.parametrize("name", sorted(CASES22))
def test_specialised_sweeps_loop_over_chunks(name, shape):
    """svs_chunk_jit / svs_diag_jit against the oracle and the interpreter
    where a CTA processes several chunks (tiles) per launch: chunks of 2^12
    amplitudes on 128 or 256 threads (two or three CTAs per SM) and of 2^13
    on 256 threads (one CTA per SM)."""
    cq, rb = shape
    c, exp = _oracle(name)
    assert (1 << (c.n - cq)) > 3 * _sm_count()   # more chunks than resident CTAs
    got, st = _run(c, S.SIM_C64, S.default_options(flags=BASE | S.SIM_F_JIT, register_bits=rb, chunk_qubits=cq))
    assert st["chunk_ops"] + st["diag_ops"] > 0
    _check64(got, exp)
    ref, st_ref = _run(c, S.SIM_C64, S.default_options(flags=BASE, register_bits=rb, chunk_qubits=cq))
    st.pop("plan_ms"), st_ref.pop("plan_ms")
    assert st == st_ref
    assert float(np.max(np.abs(got - ref))) <= 1e-6


@pytest.fixture(scope="module")
def config1():
    """The 28-qubit diagonal-heavy stream (H on every qubit + 500 gates) and
    its complex128 oracle state (4 GiB, gate by gate on the host cores)."""
    c = C.diag_heavy(28, 500, 1)
    return c, oracle.run(c)


def _chunked_check(got, exp, tol, fid_min=None, step=1 << 24):
    """max |got - exp| and the fidelity, over slices (no full-size temporaries)."""
    err, ov, ng, ne = 0.0, 0j, 0.0, 0.0
    for lo in range(0, exp.size, step):
        g = got[lo:lo + step].astype(np.complex128)
        e = exp[lo:lo + step]
        err = max(err, float(np.max(np.abs(g - e))))
        ov += np.vdot(e, g)
        ng += float(np.vdot(g, g).real)
        ne += float(np.vdot(e, e).real)
    assert err <= tol, err
    if fid_min is not None:
        assert abs(ov) ** 2 / (ng * ne) >= fid_min
    return err


def test_config1_28q_specialised_against_oracle(config1):
    """The bench's workload in the bench's configuration (merge booster,
    diagonal detector, cache blocking, fusion, specialised chunk kernels at
    32 amplitudes per thread): every amplitude against the oracle."""
    c, exp = config1
    got, st = _run(c, S.SIM_C64, S.default_options(flags=BASE | S.SIM_F_JIT))
    assert st["sweeps"] == 7 and st["diag_fused"] > 0
    _chunked_check(got, exp, TOL64, FID64)


def test_config1_28q_complex128_against_oracle(config1):
    """The same stream in complex128 (double-float chunk sweeps): 1e-12."""
    c, exp = config1
    got, st = _run(c, S.SIM_C128, S.default_options())
    assert st["chunk_ops"] > 0
    _chunked_check(got, exp, TOL128)


# ---------------------------------------------------------------- dense blocks
DENSE = [(S.SIM_C64, S.SIM_DENSE_SPLIT_TF32, TOL64), (S.SIM_C64, S.SIM_DENSE_FP32, TOL64),
         (S.SIM_C128, S.SIM_DENSE_DOUBLE_FLOAT, TOL128), (S.SIM_C128, S.SIM_DENSE_FP64, TOL128)]


@pytest.mark.parametrize("dtype,prec,tol", DENSE, ids=["tf32x3", "fp32", "double-float", "fp64"])
def test_dense_blocks_loop_over_tiles(dtype, prec, tol):
    """Dense 5-qubit blocks at 24 qubits: 2^19 columns, so each tensor-core
    CTA runs about 13 tiles (mbarrier phase flips, TMEM reuse, the prefetched
    next tile) and each CUDA-core CTA several column blocks."""
    c = C.layered(24, 4, 4)
    exp = oracle.run(c)
    opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG, dense_precision=prec)
    got, st = _run(c, dtype, opt)
    assert st["dense_ops"] > 0
    assert (1 << (24 - 5)) // 128 > 2 * _sm_count() * 4
    got = got.astype(np.complex128)
    err = float(np.max(np.abs(got - exp)))
    assert err <= tol, err
    if dtype == S.SIM_C64:
        assert _fid(exp, got) >= FID64


@pytest.mark.parametrize("dtype,prec,tol", DENSE, ids=["tf32x3", "fp32", "double-float", "fp64"])
def test_single_dense_block_22q(dtype, prec, tol):
    """One Haar-random 32x32 block on scattered qubits of a random 22-qubit
    state (1024 tensor-core tiles on 2 x SMs CTAs)."""
    rng = np.random.default_rng(2022)
    n = 22
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    g = C.Gate("unitary", (17, 2, 9, 21, 5), matrix=C.haar_unitary(rng, 32))
    c = C.Circuit(n, [g])
    exp = oracle.run(c, state=psi)
    with S.Sim(n, dtype) as s:
        s.set_state(psi)
        s.apply(c.gates, S.default_options(flags=S.SIM_F_TC, dense_precision=prec))
        assert s.stats()["dense_ops"] == 1
        got = s.get_state().astype(np.complex128)
    err = float(np.max(np.abs(got - exp)))
    # amplitudes of a random 22-qubit state are ~5e-4: the block's error
    # stays well below the circuit tolerance
    assert err <= tol * 0.1, err


# ---------------------------------------------------------------- closed forms
def _qft_factors(n, x):
    """QFT|x> = 2^(-n/2) sum_y e^{2 pi i x y / 2^n} |y>: with y = h 2^m + l
    (m = n // 2) the phase is x h 2^m + x l turns of 2^-n, so a_y =
    2^(-n/2) f_hi[h] f_lo[l]; the products x h 2^m and x l are reduced
    modulo 2^n in integers before the one rounding to an angle."""
    m = n // 2
    mod = (1 << n) - 1
    l = np.arange(1 << m, dtype=np.uint64)
    h = np.arange(1 << (n - m), dtype=np.uint64)
    tl = ((np.uint64(x) * l) & np.uint64(mod)).astype(np.float64) / float(1 << n)
    th = ((np.uint64(x) * (h << np.uint64(m))) & np.uint64(mod)).astype(np.float64) / float(1 << n)
    return m, np.exp(2j * np.pi * th), np.exp(2j * np.pi * tl) * 2.0 ** (-n / 2)


@pytest.mark.parametrize("jit", [False, True], ids=["interpreter", "specialised"])
def test_qft30_every_amplitude_closed_form(jit):
    """The 30-qubit circuit-level QFT workload (480 gates, reversal SWAPs as
    relabellings) on a random basis state: all 2^30 amplitudes against the
    closed form, complex64 (amplitudes 2^-15: the error is also bounded
    relative to that magnitude)."""
    n = 30
    c = C.qft(n, 2)
    m, f_hi, f_lo = _qft_factors(n, c.basis)
    opt = S.default_options(flags=S.default_options().flags | (S.SIM_F_JIT if jit else 0))
    amp = 2.0 ** (-n / 2)
    with DeviceState(n, S.SIM_C64) as d:
        d.sim.reset(c.basis)
        d.sim.apply(c.gates, opt)
        d.sync()
        step = 1 << 24
        rows = step >> m

        def part(lo):
            g = d.slice(lo, lo + step)
            h0 = lo >> m
            e = np.outer(f_hi[h0:h0 + rows], f_lo).reshape(-1)
            return float(np.max(np.abs(g - e))), np.vdot(e, g), float(np.vdot(g, g).real), \
                float(np.vdot(e, e).real)

        with ThreadPoolExecutor(8) as ex:
            res = list(ex.map(part, range(0, 1 << n, step)))
    err = max(r[0] for r in res)
    ov = sum(r[1] for r in res)
    ng, ne = sum(r[2] for r in res), sum(r[3] for r in res)
    assert err <= TOL64 and err <= 1e-3 * amp, err
    assert abs(ov) ** 2 / (ng * ne) >= FID64


def _sample_indices(n, seed, count=1 << 16):
    rng = np.random.default_rng(seed)
    rand = rng.integers(0, 1 << n, size=count, dtype=np.int64)
    start = int(rng.integers(0, (1 << n) - count))
    return np.unique(np.concatenate([rand, np.arange(start, start + count, dtype=np.int64),
                                     np.array([0, (1 << n) - 1], np.int64)]))


def test_qft33_complex128_sampled_closed_form():
    """The 33-qubit complex128 QFT (128 GiB): a seeded sample of 2^16 random
    indices and a run of 2^16 consecutive ones against the closed form, at
    the complex128 tolerance."""
    n = 33
    c = C.qft(n, 2)
    m, f_hi, f_lo = _qft_factors(n, c.basis)
    idx = _sample_indices(n, 33)
    exp = f_hi[idx >> m] * f_lo[idx & ((1 << m) - 1)]
    with DeviceState(n, S.SIM_C128) as d:
        d.sim.reset(c.basis)
        d.sim.apply(c.gates)
        got = d.gather(idx)
    err = float(np.max(np.abs(got - exp)))
    assert err <= TOL128, err


def test_rzz_full34_sampled_closed_form():
    """RZZ on all 561 pairs of 34 qubits after H on every qubit: a_x =
    2^-17 exp(-i/2 sum_{a<b} theta_ab s_a s_b) with s_q = 1 - 2 x_q (each RZZ
    is exp(-i theta Z_a Z_b / 2)).  One fused write-only phase sweep of 128
    GiB; a seeded sample of indices against that closed form."""
    n = 34
    c = C.rzz_full(n)
    theta = np.zeros((n, n))
    for g in c.gates:
        if g.kind == "rzz":
            a, b = g.qubits
            theta[a, b] += g.params[0]
    idx = _sample_indices(n, 34)
    s = 1.0 - 2.0 * ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)
    phase = -0.5 * np.einsum("ia,ab,ib->i", s, theta, s)
    amp = 2.0 ** (-n / 2)
    exp = amp * np.exp(1j * phase)
    with DeviceState(n, S.SIM_C64) as d:
        d.sim.reset(0)
        d.sim.apply(c.gates)
        assert d.sim.stats()["sweeps"] == 1
        got = d.gather(idx)
    err = float(np.max(np.abs(got - exp)))
    assert err <= TOL64 and err <= 1e-4 * amp, err / amp
    assert abs(np.vdot(exp, got)) ** 2 / (np.vdot(got, got).real * np.vdot(exp, exp).real) >= FID64
