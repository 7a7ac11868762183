"""GPU parity of the Schroedinger-functional time boundaries (openQCD boundary
type 1, the boundaries of the matrices of Sec. 2) and of the QCD+QED clover
term with separate SU(3) and U(1) coefficients (Sec. 1) against the FP64
oracle: operators in every storage type, the multi-rhs kernels, CGNE (with a
precision ladder) and SAP-GCR solves checked with the oracle's operators."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import TOL, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

CF = 1.23


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def _sf_case(dims, eps, seed, kappa, csw):
    u = synth.make_gauge_sf(dims, eps, seed)
    a = dirac.clover_field_sf(u, dirac.kappa_to_m0(kappa), csw, CF)
    return u, a, np.linalg.inv(a)


def _sf_handle(dims, u, kappa, csw, fmt):
    oq = _oq()
    h = oq.Handle(dims, bc_t=0)
    h.gauge_upload(to_dev(u), fmt)
    h.clover_build(kappa, csw, cF=CF)
    return h


SF_CASES = [((6, 4, 2, 6), 0.5, 2, 0.135, 1.0),     # Vh = 144 (ragged)
            ((8, 6, 4, 10), 0.5, 3, 0.1365, 1.3)]   # Vh = 960


@pytest.mark.parametrize("case", SF_CASES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("fmt", [0, 1])
def test_sf_operators(case, prec, fmt):
    """Dw, Dhat and their adjoints with SF boundaries; the x0 = 0 slice of the
    input is ignored (set to junk) and that of the output is exactly zero."""
    oq = _oq()
    dims, eps, seed, kappa, csw = case
    u, a, ainv = _sf_case(dims, eps, seed, kappa, csw)
    h = _sf_handle(dims, u, kappa, csw, fmt)
    n = 2
    psi = synth.make_source(dims, seed + 600, nrhs=n)
    for dagger in (False, True):
        pin, pout = h.new_packed(prec, nrhs=n), h.new_packed(prec, nrhs=n)
        h.pack(to_dev(psi), pin, prec, nrhs=n)
        h.dw(pin, pout, prec, nrhs=n, dagger=dagger)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, prec, nrhs=n)
        got = from_dev(out, psi.shape)
        for k in range(n):
            ref = dirac.dw_sf_dagger(u, a, psi[k]) if dagger else dirac.dw_sf(u, a, psi[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)
            assert np.max(np.abs(got[k][0])) == 0.0
        ev = np.stack([dirac.even_part(p) for p in psi])
        pin, pout = h.new_packed(prec, oq.EVEN, nrhs=n), h.new_packed(prec, oq.EVEN, nrhs=n)
        h.pack(to_dev(ev), pin, prec, oq.EVEN, nrhs=n)
        h.dw_hat(pin, pout, prec, nrhs=n, dagger=dagger)
        out = to_dev(np.zeros_like(ev))
        h.unpack(pout, out, prec, oq.EVEN, nrhs=n)
        got = from_dev(out, ev.shape)
        for k in range(n):
            ref = (dirac.dw_hat_sf_dagger if dagger else dirac.dw_hat_sf)(u, a, ainv, ev[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)
            assert np.max(np.abs(got[k][0])) == 0.0


@pytest.mark.parametrize("prec,nr,cap", [(1, 2, 1), (3, 4, 0), (2, 2, 0)])
def test_sf_multi_rhs_kernels(prec, nr, cap):
    oq = _oq()
    dims, eps, seed, kappa, csw = SF_CASES[1]
    u, a, ainv = _sf_case(dims, eps, seed, kappa, csw)
    h = _sf_handle(dims, u, kappa, csw, oq.LINK_12)
    n = 5
    for mode in (0, 1, 2):
        h.tune_set(prec, mode, n, 32, 1, nr=nr, regcap=cap)
    ev = np.stack([dirac.even_part(p) for p in synth.make_source(dims, 700, nrhs=n)])
    pin, pout = h.new_packed(prec, oq.EVEN, nrhs=n), h.new_packed(prec, oq.EVEN, nrhs=n)
    h.pack(to_dev(ev), pin, prec, oq.EVEN, nrhs=n)
    h.dw_hat(pin, pout, prec, nrhs=n)
    out = to_dev(np.zeros_like(ev))
    h.unpack(pout, out, prec, oq.EVEN, nrhs=n)
    got = from_dev(out, ev.shape)
    for k in range(n):
        assert rel_err(got[k], dirac.dw_hat_sf(u, a, ainv, ev[k])) < TOL[prec], k


def _normal_residual_sf(u, a, ainv, eta, x):
    ax = dirac.dw_hat_sf_dagger(u, a, ainv, dirac.dw_hat_sf(u, a, ainv, x))
    return np.linalg.norm((eta - ax).reshape(-1)) / np.linalg.norm(eta.reshape(-1))


@pytest.mark.parametrize("kw", [dict(sdtype=1), dict(sdtype=3), dict(sdtype=0), dict(ladder=(3, 1, 0))])
def test_sf_cgne(kw):
    """CGNE on the SF Schur system to a binary64 residual of 1e-10 checked
    with the oracle's SF operator; the solution vanishes at x0 = 0."""
    oq = _oq()
    dims, eps, seed, kappa, csw = SF_CASES[1]
    u, a, ainv = _sf_case(dims, eps, seed, kappa, csw)
    h = _sf_handle(dims, u, kappa, csw, oq.LINK_12)
    n = 2
    eta = np.stack([dirac.sf_project(dirac.even_part(e)) for e in synth.make_source(dims, 710, nrhs=n)])
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, **kw), nrhs=n)
    assert rc == oq.OK
    x = from_dev(psi, eta.shape)
    for k in range(n):
        assert st[k]["converged"]
        check_residual(_normal_residual_sf(u, a, ainv, eta[k], x[k]), st[k]["true_rel_res"])
        assert np.max(np.abs(x[k][0])) == 0.0


@pytest.mark.parametrize("ncy,nmr", [(0, 0), (4, 5)])
def test_sf_sap_gcr(ncy, nmr):
    """SAP-preconditioned GCR on the full SF operator (blocks of 4^4 that
    touch the boundary slice included) to 1e-10, checked with the oracle."""
    oq = _oq()
    dims = (8, 8, 8, 8)
    kappa, csw = 0.135, 1.0
    u, a, _ = _sf_case(dims, 0.5, 5, kappa, csw)
    h = _sf_handle(dims, u, kappa, csw, oq.LINK_12)
    eta = dirac.sf_project(synth.make_source(dims, 720))
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=500, nkv=12, ncy=ncy, nmr=nmr,
                                                          bs=(4, 4, 4, 4)))
    assert rc == oq.OK and st[0]["converged"]
    x = from_dev(psi, eta.shape)
    r = np.linalg.norm((eta - dirac.dw_sf(u, a, x)).reshape(-1)) / np.linalg.norm(eta.reshape(-1))
    check_residual(r, st[0]["true_rel_res"])
    assert np.max(np.abs(x[0])) == 0.0


QED_DIMS = (6, 4, 4, 6)


@pytest.mark.parametrize("prec", [0, 1, 3, 4])
@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("bc_t", [-1, 0])
def test_qed_clover(prec, split, bc_t):
    """QCD+QED upload (SU(3) links, U(1) potential, charge q): hopping with the
    U(3) links U exp(i q A), clover with c_sw F^{SU(3)} + c_sw^QED F^{U(1)}
    (split) or c_sw F^{U(3)}; also on SF lattices."""
    oq = _oq()
    dims = QED_DIMS
    kappa, csw, cq, q = 0.135, 1.1, 0.8, -1.0 / 3.0
    u = synth.make_gauge_sf(dims, 0.5, 61) if bc_t == 0 else synth.make_gauge(dims, 0.5, 61)
    au = synth.make_u1_field(dims, 0.3, 62)
    if bc_t == 0:
        au[0, ..., 1:] = 0.0    # zero U(1) boundary field as well
    u3 = synth.apply_u1(u, au, q)
    m0 = dirac.kappa_to_m0(kappa)
    a = dirac.clover_field_qed(u, au, q, m0, csw, cq) if split else dirac.clover_field(u3, m0, csw)
    if bc_t == 0:
        for x0 in {1, dims[0] - 1}:
            a[x0] += (CF - 1.0) * np.eye(12)
    h = oq.Handle(dims, bc_t=bc_t)
    h.gauge_upload_qed(to_dev(u), to_dev(au), q)
    h.clover_build(kappa, csw, cF=CF if bc_t == 0 else None, csw_qed=cq if split else None)
    psi = synth.make_source(dims, 63)
    pin, pout = h.new_packed(prec), h.new_packed(prec)
    h.pack(to_dev(psi), pin, prec)
    h.dw(pin, pout, prec)
    out = to_dev(np.zeros_like(psi))
    h.unpack(pout, out, prec)
    got = from_dev(out, psi.shape)
    ref = dirac.dw_sf(u3, a, psi) if bc_t == 0 else dirac.dw(u3, a, psi)
    assert rel_err(got, ref) < TOL[prec]


def test_boundary_rejections():
    oq = _oq()
    dims = (4, 4, 4, 4)
    with pytest.raises(oq.OqError):
        oq.Handle(dims, bc_t=3)                      # 2 is a time-split sub-domain (OQ_BC_HALO)
    h = oq.Handle(dims, bc_t=0)
    h.gauge_upload(to_dev(synth.make_gauge_sf(dims, 0.3, 1)), oq.LINK_12)
    with pytest.raises(oq.OqError):
        h.clover_build(0.13, 1.0, csw_qed=1.0)      # no U(1) field uploaded
