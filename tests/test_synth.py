"""The seeded input generators: unitarity, det = 1, the closed-form SU(3)
exponential against an eigendecomposition, determinism of the seeds."""
import numpy as np

from paper_2202_07388_gb300 import synth


def test_expi_matches_eigendecomposition():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((4000, 3, 3)) + 1j * rng.standard_normal((4000, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    h -= (np.trace(h, axis1=-2, axis2=-1).real / 3.0)[:, None, None] * np.eye(3)
    h[0] = 0.0                                   # Q = 0
    h[1] = np.diag([1.0, 1.0, -2.0])             # degenerate eigenvalues
    h[2] = -h[1]
    for eps in (0.01, 0.3, 0.6, 1.0, 2.5):
        w, v = np.linalg.eigh(eps * h)
        ref = (v * np.exp(1j * w)[:, None, :]) @ np.conj(np.swapaxes(v, -1, -2))
        assert np.max(np.abs(synth.expi_hermitian3(eps * h) - ref)) < 1e-13


def test_gauge_links_are_su3_and_seeded():
    u = synth.make_gauge((2, 2, 4, 2), 0.6, 7)
    m = u.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(m @ np.conj(np.swapaxes(m, -1, -2)) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(m) - 1.0)) < 1e-14
    assert np.array_equal(u, synth.make_gauge((2, 2, 4, 2), 0.6, 7))
    assert not np.array_equal(u, synth.make_gauge((2, 2, 4, 2), 0.6, 8))
    # chunked generation draws the same stream
    assert np.array_equal(u, synth.make_gauge((2, 2, 4, 2), 0.6, 7, chunk=5))


def test_u1_and_point_sources():
    u = synth.make_gauge((2, 2, 2, 2), 0.5, 1)
    a = synth.make_u1_field((2, 2, 2, 2), 0.2, 2)
    u3 = synth.apply_u1(u, a, 2.0 / 3.0)
    det = np.linalg.det(u3.reshape(-1, 3, 3)).reshape(a.shape)
    assert np.max(np.abs(det - np.exp(2j * a))) < 1e-13
    ps = synth.make_point_sources((2, 2, 2, 2))
    assert ps.shape == (12, 2, 2, 2, 2, 4, 3) and ps.sum() == 12
    assert ps[5, 0, 0, 0, 0, 1, 2] == 1.0
