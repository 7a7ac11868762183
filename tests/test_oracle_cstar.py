"""Pins of the oracle's C* boundary conditions (orbifold form, oracle.cstar).

What fixes them independently of the oracle's own formulas:
* without doubling and twists the operator is the pinned periodic one;
* the free field on the doubled, twisted lattice: plane waves whose momenta
  satisfy the twisted periodicity are eigenvectors with the closed-form
  eigenvalue m0 + sum(1 - cos p) + i sum g_mu sin p;
* the charge-conjugation structure: with the mirror half holding U^*, the
  operator commutes with the antilinear map (M chi)(x) = K chi(x + L1 e1)^*
  (K g_mu^* K^-1 = g_mu); a mirror half holding U instead breaks it;
* gamma5-hermiticity and gauge covariance on the twisted lattice."""
import numpy as np
import pytest

from oracle import cstar, dirac
from paper_2202_07388_gb300 import synth

M0 = dirac.kappa_to_m0(0.13)


def test_no_twist_reduces_to_the_periodic_operator():
    dims = (4, 4, 2, 6)
    u = synth.make_gauge(dims, 0.5, 3)
    psi = synth.make_source(dims, 4)
    a0 = dirac.clover_field(u, M0, 1.2)
    a1 = cstar.clover_field(u, M0, 1.2, 0)
    assert np.array_equal(a0, a1)
    assert np.allclose(cstar.dw(u, a1, psi, 0), dirac.dw(u, a0, psi), rtol=0, atol=1e-14)


@pytest.mark.parametrize("cs", [1, 2, 3])
def test_free_field_plane_waves_on_the_twisted_lattice(cs):
    dims = (4, 6, 4, 6)                      # physical; doubled x1 extent 12
    dd = (dims[0], 2 * dims[1], dims[2], dims[3])
    u = np.broadcast_to(np.eye(3), dd + (4, 3, 3)).astype(np.complex128).copy()
    a = cstar.clover_field(u, M0, 1.0, cs)
    assert np.allclose(a, (4 + M0) * np.eye(12))          # no field strength
    g = dirac.gamma_matrices()
    rng = np.random.default_rng(5)
    x = np.indices(dd)
    for _ in range(4):
        n = rng.integers(0, 6, size=4)
        p1 = 2 * np.pi * n[1] / dd[1]
        p = np.array([(2 * n[0] + 1) * np.pi / dd[0], p1, 0.0, 0.0])
        for mu in (2, 3):
            # twisted: psi(x + L_mu e_mu) = psi(x + L1 e1), i.e. exp(i p_mu L_mu) = exp(i p1 L1)
            shift = p1 * dims[1] if cstar.twisted(mu, cs) else 0.0
            p[mu] = (2 * np.pi * n[mu] + shift) / dd[mu]
        spin = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * np.tensordot(p, x, axes=(0, 0)))
        psi = phase[..., None, None] * spin
        got = cstar.dw(u, a, psi, cs)
        mat = (M0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(np.sin(p[m]) * g[m] for m in range(4))
        want = phase[..., None, None] * (mat @ spin)
        assert np.allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("cs", [1, 2, 3])
def test_charge_conjugation_mirror_commutes(cs):
    dims = (4, 4, 4, 2)
    u = cstar.double_links(synth.make_gauge(dims, 0.6, 7))
    a = cstar.clover_field(u, M0, 1.3, cs)
    k = cstar.charge_conjugation_matrix()
    g = dirac.gamma_matrices()
    for m in range(4):
        assert np.allclose(k @ np.conj(g[m]) @ np.linalg.inv(k), g[m])
    chi = synth.make_source(u.shape[:4], 8)
    lhs = cstar.dw(u, a, cstar.mirror(chi, k), cs)
    rhs = cstar.mirror(cstar.dw(u, a, chi, cs), k)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-13)
    # a mirror half that is not the charge conjugate breaks the symmetry
    ub = np.concatenate([u[:, :dims[1]], u[:, :dims[1]]], axis=1)
    ab = cstar.clover_field(ub, M0, 1.3, cs)
    bad = cstar.dw(ub, ab, cstar.mirror(chi, k), cs) - cstar.mirror(cstar.dw(ub, ab, chi, cs), k)
    assert np.abs(bad).max() > 1e-2


@pytest.mark.parametrize("cs", [1, 3])
def test_gamma5_hermiticity_and_gauge_covariance(cs):
    dims = (4, 4, 2, 4)
    u = cstar.double_links(synth.make_gauge(dims, 0.6, 9))
    dd = u.shape[:4]
    a = cstar.clover_field(u, M0, 1.1, cs)
    phi, psi = synth.make_source(dd, 10), synth.make_source(dd, 11)
    lhs = np.vdot(phi, cstar.dw_dagger(u, a, psi, cs))
    rhs = np.vdot(cstar.dw(u, a, phi, cs), psi)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lam = synth.random_gauge_transform(dd, 12)
    up = np.empty_like(u)
    for mu in range(4):
        lam_f = cstar.shift(lam, mu, +1, cs)          # Lambda(x + mu) on the twisted lattice
        up[..., mu, :, :] = lam @ u[..., mu, :, :] @ np.conj(np.swapaxes(lam_f, -1, -2))
    ap = cstar.clover_field(up, M0, 1.1, cs)
    rot = lambda v: np.matmul(v, np.swapaxes(lam, -1, -2))  # noqa: E731  (Lambda psi per site)
    assert np.allclose(cstar.dw(up, ap, rot(psi), cs), rot(cstar.dw(u, a, psi, cs)), rtol=0, atol=1e-12)
