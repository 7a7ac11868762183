"""Pins of the oracle's Schroedinger-functional time boundaries (openQCD
boundary type 1, used for the 4^4 matrix of Fig. 4, Sec. 2 footnote) and of
the QCD+QED clover term with separate SU(3) and U(1) coefficients (Sec. 1):
the free-field solution at zero spatial momentum (closed form by forward /
backward substitution), gamma5-hermiticity and gauge covariance, the dense
Schur complement, and reductions of the QED clover to the U(3) clover and to
the constant-flux closed form."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth


def _active_idx(dims, even_only=False):
    act = np.ones(dims, bool)
    act[0] = False
    if even_only:
        act &= ~dirac.parity_mask(dims)
    return np.repeat(act.reshape(-1), 12)


@pytest.mark.parametrize("cf", [1.0, 1.37])
def test_sf_free_field_zero_momentum_closed_form(cf):
    """U = 1, a spatially constant source: with P+- = (1 +- g0)/2 the operator
    is d(x0) psi - P- psi(x0 + 1) - P+ psi(x0 - 1), d = 1 + m0 (m0 + c_F at
    x0 = 1, T-1), fields zero at x0 = 0, T.  So P+ psi follows from forward
    and P- psi from backward substitution."""
    dims = (7, 2, 2, 2)
    t = dims[0]
    u = np.zeros(dims + (4, 3, 3), complex)
    u[...] = np.eye(3)
    m0 = dirac.kappa_to_m0(0.121)
    a = dirac.clover_field_sf(u, m0, 1.3, cf)
    rng = np.random.default_rng(5)
    eta_t = rng.standard_normal((t, 4, 3)) + 1j * rng.standard_normal((t, 4, 3))
    eta_t[0] = 0.0
    eta = np.broadcast_to(eta_t[:, None, None, None], dims + (4, 3)).copy()
    # dense solve on the active sites
    m = dirac.assemble_dense(lambda v: dirac.dw_sf(u, a, v), dims)
    act = _active_idx(dims)
    x = np.zeros(m.shape[0], complex)
    x[act] = np.linalg.solve(m[np.ix_(act, act)], eta.reshape(-1)[act])
    psi = x.reshape(dims + (4, 3))
    g0 = dirac.gamma_matrices()[0]
    pp, pm = (np.eye(4) + g0) / 2, (np.eye(4) - g0) / 2
    d = np.full(t, 1.0 + m0)
    d[1] = d[t - 1] = m0 + cf
    chi_p = np.zeros((t + 1, 4, 3), complex)
    for x0 in range(1, t):
        chi_p[x0] = (pp @ eta_t[x0] + chi_p[x0 - 1]) / d[x0]
    chi_m = np.zeros((t + 1, 4, 3), complex)
    for x0 in range(t - 1, 0, -1):
        chi_m[x0] = (pm @ eta_t[x0] + chi_m[x0 + 1]) / d[x0]
    expect = chi_p[:t] + chi_m[:t]
    for x0 in range(t):
        assert np.max(np.abs(psi[x0] - expect[x0][None, None, None])) < 1e-12, x0


def test_sf_output_and_input_at_the_boundary():
    dims = (6, 4, 2, 4)
    u = synth.make_gauge_sf(dims, 0.4, 11)
    a = dirac.clover_field_sf(u, dirac.kappa_to_m0(0.13), 1.1, 1.2)
    psi = synth.make_source(dims, 12)
    out = dirac.dw_sf(u, a, psi)
    assert np.max(np.abs(out[0])) == 0.0
    junk = psi.copy()
    junk[0] = synth.make_source(dims, 13)[0]
    assert np.array_equal(dirac.dw_sf(u, a, junk), out)
    # the boundary links are the identity
    assert np.array_equal(u[0, ..., 1:, :, :], np.broadcast_to(np.eye(3), u[0, ..., 1:, :, :].shape))


def test_sf_gamma5_hermiticity_and_schur_complement():
    """On the active sites D_sf is gamma5-hermitian, and Dhat_sf is the dense
    Schur complement D_ee - D_eo D_oo^{-1} D_oe of D_sf over active sites."""
    dims = (4, 2, 2, 2)
    u = synth.make_gauge_sf(dims, 0.5, 21)
    a = dirac.clover_field_sf(u, dirac.kappa_to_m0(0.13), 1.0, 1.15)
    ainv = np.linalg.inv(a)
    m = dirac.assemble_dense(lambda v: dirac.dw_sf(u, a, v), dims)
    act = _active_idx(dims)
    ma = m[np.ix_(act, act)]
    g5 = np.kron(np.eye(int(act.sum()) // 12), np.kron(dirac.gamma5(), np.eye(3)))
    assert np.max(np.abs(g5 @ ma @ g5 - ma.conj().T)) < 1e-13
    ev = _active_idx(dims, even_only=True)
    od = act & ~ev
    schur = m[np.ix_(ev, ev)] - m[np.ix_(ev, od)] @ np.linalg.solve(m[np.ix_(od, od)], m[np.ix_(od, ev)])
    mh = dirac.assemble_dense(lambda v: dirac.dw_hat_sf(u, a, ainv, v), dims)
    assert np.max(np.abs(mh[np.ix_(ev, ev)] - schur)) < 1e-12
    assert np.max(np.abs(mh[~ev])) == 0.0 and np.max(np.abs(mh[:, ~ev])) == 0.0
    mhd = dirac.assemble_dense(lambda v: dirac.dw_hat_sf_dagger(u, a, ainv, v), dims)
    assert np.max(np.abs(mhd[np.ix_(ev, ev)] - schur.conj().T)) < 1e-12


def test_sf_gauge_covariance():
    dims = (6, 2, 4, 2)
    u = synth.make_gauge_sf(dims, 0.4, 31)
    lam = synth.random_gauge_transform(dims, 32)
    ug = synth.gauge_transform(u, lam)
    m0 = dirac.kappa_to_m0(0.13)
    a, ag = dirac.clover_field_sf(u, m0, 1.2, 1.3), dirac.clover_field_sf(ug, m0, 1.2, 1.3)
    psi = synth.make_source(dims, 33)
    lpsi = np.einsum("...ab,...sb->...sa", lam, psi)
    lhs = dirac.dw_sf(ug, ag, lpsi)
    rhs = np.einsum("...ab,...sb->...sa", lam, dirac.dw_sf(u, a, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_qed_clover_reductions():
    """SU(3) links = 1: the separate-coefficient clover is the U(3) clover of
    the charged U(1) links with c_sw = c_sw^QED; A = 0: it is the SU(3)
    clover with c_sw."""
    dims = (4, 4, 2, 4)
    au = synth.make_u1_field(dims, 0.3, 41)
    q = -1.0 / 3.0
    m0 = dirac.kappa_to_m0(0.135)
    one = np.zeros(dims + (4, 3, 3), complex)
    one[...] = np.eye(3)
    a1 = dirac.clover_field_qed(one, au, q, m0, 1.9, 0.7)
    assert np.max(np.abs(a1 - dirac.clover_field(synth.apply_u1(one, au, q), m0, 0.7))) < 1e-13
    u = synth.make_gauge(dims, 0.4, 42)
    a2 = dirac.clover_field_qed(u, np.zeros(dims + (4,)), q, m0, 1.9, 0.7)
    assert np.max(np.abs(a2 - dirac.clover_field(u, m0, 1.9))) < 1e-13


def test_qed_clover_constant_flux_closed_form():
    """A constant U(1) flux theta in the (1, 2) plane: the U(1) part of the
    clover term is -(c_sw^QED / 2) sin(q theta) sigma_12 (x) 1_colour."""
    dims = (2, 4, 6, 2)
    mu, nu = 1, 2
    q = 2.0 / 3.0
    theta = 2 * np.pi / (q * dims[mu] * dims[nu])   # q theta = one flux quantum over the plane
    x = np.indices(dims)
    au = np.zeros(dims + (4,))
    au[..., nu] = theta * x[mu]
    edge = x[mu] == dims[mu] - 1
    au[..., mu] = np.where(edge, -theta * dims[mu] * x[nu], 0.0)
    one = np.zeros(dims + (4, 3, 3), complex)
    one[...] = np.eye(3)
    m0, cq = dirac.kappa_to_m0(0.13), 1.4
    a = dirac.clover_field_qed(one, au, q, m0, 2.0, cq)
    expect = (4 + m0) * np.eye(12) - 0.5 * cq * np.sin(q * theta) * np.kron(dirac.sigma_munu(mu, nu), np.eye(3))
    assert np.max(np.abs(a - expect)) < 1e-12


def test_sf_cgne_matches_dense_solve():
    """CGNE on the Schroedinger-functional Schur system reaches the dense
    solution of the normal equations on the active even sites (brute force
    on 4 x 2^3)."""
    from oracle import solvers
    dims = (4, 2, 2, 2)
    u = synth.make_gauge_sf(dims, 0.4, 51)
    a = dirac.clover_field_sf(u, dirac.kappa_to_m0(0.13), 1.0, 1.2)
    ainv = np.linalg.inv(a)
    eta = dirac.sf_project(dirac.even_part(synth.make_source(dims, 52)))
    dh = lambda v: dirac.dw_hat_sf(u, a, ainv, v)
    dhd = lambda v: dirac.dw_hat_sf_dagger(u, a, ainv, v)
    res = solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-12, 500, "fp64")
    m = dirac.assemble_dense(dh, dims)
    ev = _active_idx(dims, even_only=True)
    n = m[np.ix_(ev, ev)]
    x = np.linalg.solve(n.conj().T @ n, eta.reshape(-1)[ev])
    assert res.converged
    assert np.max(np.abs(res.x.reshape(-1)[ev] - x)) < 1e-9 * np.max(np.abs(x))
    assert np.max(np.abs(res.x.reshape(-1)[~ev])) == 0.0
