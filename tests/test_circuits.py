"""Input generators: the batched Haar U(2) draw is the Mezzadri QR method, and
the workload recipes have the shapes they state."""
import numpy as np

from paper_2604_12256_gb300 import circuits as C


def test_haar_batch_is_qr_with_phase_correction():
    """Same Ginibre draws through numpy's QR and Mezzadri's R-diagonal phase
    correction give the same unitaries."""
    U = C.haar_u2_batch(np.random.default_rng(5), 64)
    rng = np.random.default_rng(5)
    z = (rng.standard_normal((64, 2, 2)) + 1j * rng.standard_normal((64, 2, 2))) / np.sqrt(2.0)
    for i in range(64):
        q, r = np.linalg.qr(z[i])
        d = np.diagonal(r)
        np.testing.assert_allclose(U[i], q * (d / np.abs(d))[None, :], atol=1e-14)


def test_haar_batch_statistics():
    """Unitary to rounding; |U00|^2 is uniform on [0, 1] and arg det U uniform
    on (-pi, pi] under the Haar measure on U(2)."""
    U = C.haar_u2_batch(np.random.default_rng(0), 100000)
    eye = np.einsum("nij,nkj->nik", U, U.conj())
    assert np.abs(eye - np.eye(2)).max() < 1e-14
    p = np.abs(U[:, 0, 0]) ** 2
    np.testing.assert_allclose(np.quantile(p, [0.25, 0.5, 0.75]), [0.25, 0.5, 0.75], atol=0.01)
    ph = np.angle(np.linalg.det(U))
    assert abs(ph.mean()) < 0.03 and abs(ph.std() - np.pi / np.sqrt(3)) < 0.02


def test_workload_shapes():
    c = C.diag_heavy(28, 500, 1)
    assert len(c.gates) == 528 and all(g.kind == "h" for g in c.gates[:28])
    kinds = [g.kind for g in c.gates[28:]]
    frac = sum(k in ("rz", "cp", "rzz") for k in kinds) / len(kinds)
    assert 0.74 < frac < 0.86
    q = C.qft(30, 2)
    assert sum(g.kind == "h" for g in q.gates) == 30 and sum(g.kind == "cp" for g in q.gates) == 435
    assert sum(g.kind == "swap" for g in q.gates) == 15
    a = C.qaoa(30, 4, 3)
    assert len(a.gates) == 30 + 4 * (45 + 30)
    lay = C.layered(14, 20, 0)
    assert len(lay.gates) == 20 * 14 + 10 * 7 + 10 * 6
