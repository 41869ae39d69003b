"""Failure paths, with the failure made on the host (sim_fault_inject): an
allocation that the device refuses returns SIM_ENOMEM, a launch that fails
returns SIM_ECUDA, and the handle or server that saw the failure stays
usable -- its next circuit is exact.  No GPU fault is involved: an armed
allocation never reaches cudaMalloc and an armed launch is never made."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]


@pytest.fixture(autouse=True)
def disarm():
    yield
    S.fault_inject(S.SIM_FAULT_ALLOC, 0)
    S.fault_inject(S.SIM_FAULT_LAUNCH, 0)


def _exact(s, c, tol=2e-5):
    s.reset(c.basis)
    s.apply(c.gates)
    got = s.get_state().astype(np.complex128)
    assert np.max(np.abs(got - oracle.run(c))) <= tol


def test_create_reports_enomem_then_recovers():
    """sim_create allocates the state, then its read-out buffers: refusing the
    first, the second or the fifth of those fails the create with SIM_ENOMEM
    (freeing what it had taken), and the next create is exact."""
    for skip in (0, 1, 4):
        S.fault_inject(S.SIM_FAULT_ALLOC, 1, skip=skip)
        with pytest.raises(S.SimError) as e:
            S.Sim(14, S.SIM_C64)
        assert e.value.code == S.SIM_ENOMEM
        S.fault_inject(S.SIM_FAULT_ALLOC, 0)
        with S.Sim(14, S.SIM_C64) as s:
            _exact(s, C.random_mixed(14, 60, 3 + skip))


def test_apply_reports_enomem_for_booster_buffers_then_recovers():
    """The merge booster's sub-state buffers are allocated on the first apply
    that needs them: refused, the apply fails with SIM_ENOMEM; the next one
    allocates them and is exact."""
    c = C.diag_heavy(18, 120, 4)
    with S.Sim(18, S.SIM_C64) as s:
        S.fault_inject(S.SIM_FAULT_ALLOC, 1)
        s.reset(c.basis)
        with pytest.raises(S.SimError) as e:
            s.apply(c.gates)
        assert e.value.code == S.SIM_ENOMEM
        _exact(s, c)


def test_launch_failure_reports_ecuda_then_recovers():
    c = C.random_mixed(16, 150, 5)
    with S.Sim(16, S.SIM_C64) as s:
        for k in (1, 3):
            S.fault_inject(S.SIM_FAULT_LAUNCH, 0)
            s.reset(c.basis)
            s.apply(c.gates)       # nothing armed: fine
            S.fault_inject(S.SIM_FAULT_LAUNCH, k)
            s.reset(c.basis)
            with pytest.raises(S.SimError) as e:
                s.apply(c.gates)
            assert e.value.code == S.SIM_ECUDA
            S.fault_inject(S.SIM_FAULT_LAUNCH, 0)
            _exact(s, c)


def test_server_worker_allocation_failure_is_reported_per_request():
    """A worker whose state buffer is refused fails that request with
    SIM_ENOMEM and serves the next one."""
    a, b = C.diag_heavy(17, 60, 1), C.diag_heavy(17, 60, 2)
    with S.Server(1 << 30, n_streams=1) as srv:
        S.fault_inject(S.SIM_FAULT_ALLOC, 1)
        ra = srv.poll(srv.submit(a, 4, [1]))
        rb = srv.poll(srv.submit(b, 4, [1]))
        st = srv.stats()
    assert ra["status"] == S.SIM_ENOMEM
    assert rb["status"] == 0 and st["failed"] == 1
    np.testing.assert_allclose(rb["expect"], oracle.expectation_z(oracle.run(b), [1]), atol=2e-5)
