"""Pins of the FP64 oracle's Dirac operator against facts fixed by the
mathematics: Clifford algebra, the free-field dispersion relation,
gamma5-hermiticity, gauge covariance, closed forms of the clover term, the
sparsity of the assembled matrix (Sec. 2: about 2 % non-zeros) and the
even-odd Schur complement (Sec. 3, Fig. 3)."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.oracle_cases import gauge_case, rand_spinor


def test_clifford_algebra_and_gamma5():
    g = dirac.gamma_matrices()
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))
    assert np.allclose(dirac.gamma5(), np.diag([1, 1, -1, -1]))
    # sigma_{mu nu} is block diagonal in chirality in this basis
    for m in range(4):
        for n in range(4):
            s = dirac.sigma_munu(m, n)
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3), (3, 1, 1, 0)])
def test_free_field_plane_wave(n):
    """U = 1: D e^{ipx} u = [m0 + sum(1 - cos p) + i sum g_mu sin p] e^{ipx} u,
    with antiperiodic time momenta p0 = (2 n0 + 1) pi / T."""
    dims = (8, 4, 4, 6)
    u = np.zeros(dims + (4, 3, 3), complex)
    u[...] = np.eye(3)
    m0 = dirac.kappa_to_m0(0.13)
    a = dirac.clover_field(u, m0, 1.0)
    p = [(2 * n[0] + 1) * np.pi / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)]
    x = np.indices(dims)
    phase = np.exp(1j * sum(p[mu] * x[mu] for mu in range(4)))
    rng = np.random.default_rng(7)
    spin_col = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi = phase[..., None, None] * spin_col
    g = dirac.gamma_matrices()
    mom = (m0 + sum(1 - np.cos(pm) for pm in p)) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
    expect = phase[..., None, None] * (mom @ spin_col)
    got = dirac.dw(u, a, psi)
    assert np.max(np.abs(got - expect)) < 1e-12
    # free D^dag D eigenvalue on this mode
    dd = dirac.dw_dagger(u, a, got)
    lam = (m0 + sum(1 - np.cos(pm) for pm in p)) ** 2 + sum(np.sin(pm) ** 2 for pm in p)
    assert np.max(np.abs(dd - lam * psi)) < 1e-11


def test_gamma5_hermiticity_dense():
    """gamma5 D gamma5 = D^dag as dense matrices on a 2^4 lattice."""
    dims = (2, 2, 2, 2)
    u, a, ainv = gauge_case(dims, 0.5, 11, 0.13, 1.0)
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), dims)
    g5 = np.kron(np.eye(16), np.kron(dirac.gamma5(), np.eye(3)))
    assert np.max(np.abs(g5 @ m @ g5 - m.conj().T)) < 1e-13


def test_gamma5_hermiticity_random_vectors():
    u, a, ainv = gauge_case()
    dims = u.shape[:4]
    phi, psi = rand_spinor(dims, 3), rand_spinor(dims, 4)
    lhs = np.vdot(phi, dirac.dw(u, a, psi))
    rhs = np.vdot(dirac.dw_dagger(u, a, phi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    pe, qe = dirac.even_part(phi), dirac.even_part(psi)
    lhs = np.vdot(pe, dirac.dw_hat(u, a, ainv, qe))
    rhs = np.vdot(dirac.dw_hat_dagger(u, a, ainv, pe), qe)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_covariance():
    """D[U'] (Lambda psi) = Lambda D[U] psi, U' = Lambda U Lambda^dag(x+mu)."""
    dims = (4, 4, 2, 6)
    u = synth.make_gauge(dims, 0.5, 21)
    lam = synth.random_gauge_transform(dims, 22)
    up = synth.gauge_transform(u, lam)
    m0, csw = dirac.kappa_to_m0(0.135), 1.3
    a, ap = dirac.clover_field(u, m0, csw), dirac.clover_field(up, m0, csw)
    psi = rand_spinor(dims, 23)
    rot = lambda v: np.einsum("...ab,...sb->...sa", lam, v)
    lhs = dirac.dw(up, ap, rot(psi))
    rhs = rot(dirac.dw(u, a, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_clover_vanishes_on_pure_gauge():
    dims = (4, 2, 4, 2)
    one = np.zeros(dims + (4, 3, 3), complex)
    one[...] = np.eye(3)
    u = synth.gauge_transform(one, synth.random_gauge_transform(dims, 5))
    f = dirac.field_strength(u)
    assert max(np.max(np.abs(v)) for v in f.values()) < 1e-13
    m0 = dirac.kappa_to_m0(0.13)
    a = dirac.clover_field(u, m0, 1.0)
    assert np.max(np.abs(a - (4 + m0) * np.eye(12))) < 1e-13


@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 3)])
def test_clover_constant_abelian_field(plane):
    """Constant U(1) flux theta in one plane: F = i sin(theta) there and
    A = (4 + m0) - (c_sw / 2) sin(theta) sigma_{mu nu} (x) 1_colour."""
    mu, nu = plane
    dims = (4, 6, 2, 4)
    theta = 2 * np.pi * 1 / (dims[mu] * dims[nu])
    x = np.indices(dims)
    u = np.zeros(dims + (4, 3, 3), complex)
    u[...] = np.eye(3)
    ph_nu = np.exp(1j * theta * x[mu])
    u[..., nu, :, :] = ph_nu[..., None, None] * np.eye(3)
    edge = x[mu] == dims[mu] - 1
    ph_mu = np.where(edge, np.exp(-1j * theta * dims[mu] * x[nu]), 1.0)
    u[..., mu, :, :] = ph_mu[..., None, None] * np.eye(3)
    f = dirac.field_strength(u)
    assert np.max(np.abs(f[(mu, nu)] - 1j * np.sin(theta) * np.eye(3))) < 1e-13
    for (m, n), v in f.items():
        if {m, n} != {mu, nu}:
            assert np.max(np.abs(v)) < 1e-13
    m0, csw = dirac.kappa_to_m0(0.135), 1.7
    a = dirac.clover_field(u, m0, csw)
    expect = (4 + m0) * np.eye(12) - 0.5 * csw * np.sin(theta) * np.kron(dirac.sigma_munu(mu, nu), np.eye(3))
    assert np.max(np.abs(a - expect)) < 1e-13


def test_clover_hermitian_chiral_blocks():
    u, a, _ = gauge_case()
    assert np.max(np.abs(a - np.conj(np.swapaxes(a, -1, -2)))) < 1e-14
    assert np.max(np.abs(a[..., :6, 6:])) < 1e-14 and np.max(np.abs(a[..., 6:, :6])) < 1e-14


def test_sparsity_matches_paper():
    """Sec. 2: the 4^4 operator as a CSR matrix has about 2 % non-zeros.
    Chiral basis: 8 hops x (2 spin x 3 colour) + 6 clover = 54 per row."""
    u, a, _ = gauge_case()
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), (4, 4, 4, 4))
    nnz_row = (np.abs(m) > 1e-15).sum(axis=1)
    assert np.all(nnz_row == 54)
    frac = nnz_row.sum() / m.size
    assert abs(frac - 54 / 3072) < 1e-12 and 0.015 < frac < 0.025


def test_schur_complement_dense():
    """Dhat equals the dense Schur complement D_ee - D_eo D_oo^-1 D_oe, and
    solving the even system then reconstructing the odd part solves D x = b."""
    dims = (2, 2, 2, 2)
    u, a, ainv = gauge_case(dims, 0.6, 12, 0.13, 1.0)
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), dims)
    odd = np.repeat(dirac.parity_mask(dims).reshape(-1), 12)
    ev = ~odd
    s = m[np.ix_(ev, ev)] - m[np.ix_(ev, odd)] @ np.linalg.solve(m[np.ix_(odd, odd)], m[np.ix_(odd, ev)])
    mh = dirac.assemble_dense(lambda v: dirac.dw_hat(u, a, ainv, v), dims)
    assert np.max(np.abs(mh[np.ix_(ev, ev)] - s)) < 1e-13
    assert np.max(np.abs(mh[:, odd])) == 0 and np.max(np.abs(mh[odd, :])) == 0
    b = rand_spinor(dims, 13)
    bh = dirac.schur_source(u, a, ainv, b)
    xe = np.linalg.solve(s, bh.reshape(-1)[ev])
    xfull = np.zeros(b.size, complex)
    xfull[ev] = xe
    x = dirac.schur_reconstruct_odd(u, a, ainv, b, xfull.reshape(b.shape))
    assert np.max(np.abs(x.reshape(-1) - np.linalg.solve(m, b.reshape(-1)))) < 1e-12


def test_dw_site_matches_field():
    u, a, _ = gauge_case()
    psi = rand_spinor(u.shape[:4], 9)
    full = dirac.dw(u, a, psi)
    for x in [(0, 0, 0, 0), (3, 1, 2, 3), (3, 3, 3, 3), (1, 0, 3, 2)]:
        assert np.max(np.abs(dirac.dw_site(u, a, psi, x) - full[x])) < 1e-13


def test_clover_site_matches_field():
    dims = (6, 4, 2, 4)
    u = synth.make_gauge(dims, 0.6, 17)
    m0 = dirac.kappa_to_m0(0.135)
    a = dirac.clover_field(u, m0, 1.3)
    for x in [(0, 0, 0, 0), (5, 3, 1, 3), (2, 0, 1, 2), (5, 0, 0, 3)]:
        assert np.max(np.abs(dirac.clover_site(u, m0, 1.3, x) - a[x])) < 1e-14


def test_operator_condition_small_lattice():
    """The smallest singular value of D on the 4^4 workload is well away from
    zero (kappa = 0.13), so solves to 1e-10 are meaningful."""
    u, a, _ = gauge_case()
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), (4, 4, 4, 4))
    sv = np.linalg.svd(m, compute_uv=False)
    assert sv.min() > 1e-2 and sv.max() < 20
