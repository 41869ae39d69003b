"""sim_expectation_noalloc: the expectation entry point for callers that
cannot allocate device memory (it keeps its partial sums in a fixed device
array inside the library).  Its results must match sim_expectation's, the
allocating entry point, on consecutive calls that share that array, and the
oracle's <Z-string> of the oracle's own state within the same tolerance.

Collected last on purpose (file name) so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_lib")]


@pytest.mark.parametrize("dtype,tol", [(S.SIM_C64, 2e-5), (S.SIM_C128, 1e-12)])
def test_noalloc_matches_allocating_entry_point(dtype, tol):
    import torch
    n = 15
    c = C.random_mixed(n, 120, 77, max_k=2)
    first = [(1 << 0) | (1 << 7), (1 << 3) | (1 << 14), 1 << 9, (1 << n) - 1]
    second = [(1 << 2) | (1 << 5), (1 << 11), (1 << 1) | (1 << 4) | (1 << 13), 0, 0b1010101010, 1 << 14,
              (1 << 6) | (1 << 8)]
    ref_state = oracle.run(c)
    with S.Sim(n, dtype) as s:
        s.reset(c.basis)
        s.apply(c.gates)
        state_ptr, stream = s.device()
        for masks in (first, second):     # two calls in a row share the fixed array
            expect = s.expectation(masks)
            ref = oracle.expectation_z(ref_state, masks)
            dm = torch.tensor(np.array(masks, dtype=np.uint64).view(np.int64), device="cuda")
            out = torch.full((len(masks),), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            S.expectation_noalloc(state_ptr, n, dtype, dm.data_ptr(), len(masks), out.data_ptr(), stream)
            s.sync()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, expect, atol=tol, rtol=0)
            np.testing.assert_allclose(got, ref, atol=tol, rtol=0)


def test_noalloc_rejects_bad_arguments():
    import torch
    with S.Sim(10, S.SIM_C64) as s:
        s.apply([C.Gate("h", (0,))])
        state_ptr, stream = s.device()
        dm = torch.zeros(17, dtype=torch.int64, device="cuda")
        out = torch.zeros(17, dtype=torch.float64, device="cuda")
        with pytest.raises(S.SimError) as e:
            S.expectation_noalloc(state_ptr, 10, S.SIM_C64, dm.data_ptr(), 17, out.data_ptr(), stream)
        assert e.value.code == S.SIM_EINVAL
        with pytest.raises(S.SimError):
            S.expectation_noalloc(state_ptr, 10, S.SIM_C64, dm.data_ptr(), 0, out.data_ptr(), stream)
