"""Pins of the oracle's parallel-transport layers: exact gauge equivariance,
the adjoint identity of the transports, and central finite differences of
the loss against the hand-written backward pass."""
import numpy as np

from oracle import ptc
from paper_2202_07388_gb300 import synth

DIMS = (4, 2, 2, 4)


def _weights(seed, cout, cin):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ptc.NPATH, cout, cin, 4, 4))
            + 1j * rng.standard_normal((ptc.NPATH, cout, cin, 4, 4))) * 0.2


def test_transport_adjoint_identity():
    u = synth.make_gauge(DIMS, 0.6, 1)
    a, b = synth.make_source(DIMS, 2), synth.make_source(DIMS, 3)
    for p in range(ptc.NPATH):
        lhs = np.vdot(ptc.transport(u, a, p), b)
        rhs = np.vdot(a, ptc.transport_adjoint(u, b, p))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_ptc_gauge_equivariance():
    u = synth.make_gauge(DIMS, 0.6, 4)
    lam = synth.random_gauge_transform(DIMS, 5)
    up = synth.gauge_transform(u, lam)
    w1, w2 = _weights(6, 2, 1), _weights(7, 1, 2)
    psi = synth.make_source(DIMS, 8)
    rot = lambda v: np.einsum("...ab,...sb->...sa", lam, v)
    y, _ = ptc.forward(u, w1, w2, psi)
    yp, _ = ptc.forward(up, w1, w2, rot(psi))
    assert np.max(np.abs(yp - rot(y))) < 1e-12


def test_identity_weights_give_identity_map():
    u = synth.make_gauge(DIMS, 0.6, 9)
    w1 = np.zeros((ptc.NPATH, 2, 1, 4, 4), complex)
    w2 = np.zeros((ptc.NPATH, 1, 2, 4, 4), complex)
    w1[0, 0, 0] = np.eye(4)
    w2[0, 0, 0] = np.eye(4)
    psi = synth.make_source(DIMS, 10)
    y, _ = ptc.forward(u, w1, w2, psi)
    assert np.max(np.abs(y - psi)) == 0


def test_backward_matches_finite_differences():
    u = synth.make_gauge(DIMS, 0.6, 11)
    w1, w2 = _weights(12, 2, 1), _weights(13, 1, 2)
    r, e = synth.make_source(DIMS, 14), synth.make_source(DIMS, 15)
    _, g1, g2 = ptc.backward(u, w1, w2, r, e)
    rng = np.random.default_rng(16)
    h = 1e-6
    for which, w, g in (("w1", w1, g1), ("w2", w2, g2)):
        for _ in range(12):
            idx = tuple(rng.integers(0, n) for n in w.shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                wp, wm = w.copy(), w.copy()
                wp[idx] += h * unit
                wm[idx] -= h * unit
                if which == "w1":
                    fd = (ptc.loss(u, wp, w2, r, e) - ptc.loss(u, wm, w2, r, e)) / (2 * h)
                else:
                    fd = (ptc.loss(u, w1, wp, r, e) - ptc.loss(u, w1, wm, r, e)) / (2 * h)
                an = g[idx].real if part == "re" else g[idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, idx, part, fd, an)
