"""Cache-blocked dense-block sweeps (K6 inside K4): complex64 states, 5-qubit
blocks in split-TF32 on the tensor cores, several blocks per pass over the
state, against the oracle.

- Sizes from one chunk (12 qubits: one CTA) through one chunk per CTA (20
  qubits: 256 chunks on 2 x 152 CTAs) to CTAs that loop over chunks (22-23
  qubits), where the next chunk's loads, the B-image copies between chunks
  and the reuse of tensor memory all run.
- A sweep of one block (its B image stays in shared memory across chunks).
- Equality with one sweep per block (the separate tensor-core kernel).
"""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]

BLOCKED = S.SIM_F_TC | S.SIM_F_DIAG | S.SIM_F_BLOCK
SEPARATE = S.SIM_F_TC | S.SIM_F_DIAG


def fid(a, b):
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def run(c, flags, state=None):
    opt = S.default_options(flags=flags, dense_precision=S.SIM_DENSE_SPLIT_TF32)
    with S.Sim(c.n, S.SIM_C64) as s:
        if state is None:
            s.reset(c.basis)
        else:
            s.set_state(state)
        s.profile_enable(True)
        s.apply(c.gates, opt)
        st = s.stats()
        prof = s.profile_read()
        return s.get_state().astype(np.complex128), st, prof


def plan_ops(c, flags):
    p = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, S.default_options(flags=flags))
    return [op for op in p["ops"] if op["op"] == "dense_chunk"]


CASES = [
    ("layered12", lambda: C.layered(12, 6, 3)),
    ("layered14", lambda: C.layered(14, 8, 5)),
    ("mixed14", lambda: C.random_mixed(14, 160, 9, max_k=3)),
    ("qft13", lambda: C.qft(13, 5)),
    ("layered20", lambda: C.layered(20, 6, 4)),
    ("supremacy20", lambda: C.supremacy(20, 8, 6)),
    ("layered22", lambda: C.layered(22, 6, 7)),
    ("mixed23", lambda: C.random_mixed(23, 220, 11, max_k=3)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matches_oracle(name, make):
    c = make()
    ops = plan_ops(c, BLOCKED)
    assert ops, "no cache-blocked dense sweep in the plan"
    exp = oracle.run(c)
    got, st, prof = run(c, BLOCKED)
    assert prof["dense"]["launches"] == len(ops)
    err = np.max(np.abs(got - exp))
    assert err <= 1e-5, err
    assert fid(exp, got) >= 1 - 1e-6
    assert abs(np.linalg.norm(got) - 1) <= 1e-5


@pytest.mark.parametrize("n", [12, 20, 22])
@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4), (4, 5, 9, 10, 11), (7, 1, 6, 11, 5)])
def test_one_block_sweep(n, targets):
    """One Haar 5-qubit unitary on a random state: a sweep holding one block,
    whose B image stays in shared memory for every chunk of the CTA."""
    rng = np.random.default_rng(n * 100 + sum(targets))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    c = C.Circuit(n, [C.Gate("unitary", targets, matrix=C.haar_unitary(rng, 32))])
    ops = plan_ops(c, BLOCKED)
    assert len(ops) == 1 and len(ops[0]["blocks"]) == 1
    exp = oracle.run(c, state=psi)
    got, st, _ = run(c, BLOCKED, state=psi)
    assert st["dense_ops"] == 1
    assert np.max(np.abs(got - exp)) <= 1e-6


def test_equals_one_sweep_per_block():
    """Cache-blocked block sweeps against one sweep per block (k_dense5_tc):
    both are split-TF32 products of the same circuit, so the states agree to
    complex64 rounding."""
    c = C.layered(18, 10, 8)
    a, sa, _ = run(c, BLOCKED)
    b, sb, _ = run(c, SEPARATE)
    assert sa["sweeps"] < sb["sweeps"]
    assert np.max(np.abs(a - b)) <= 2e-6


def test_bounded_waits_self_test():
    """Both tensor-core kernels: with the MMA issue suppressed every wait
    gives up, the status word is set, the state is untouched, and a normal
    launch afterwards is exact."""
    lib = S.load()
    assert lib.sim_selftest_wait_timeout() == S.SIM_OK, (lib.sim_global_error() or b"").decode()
