"""C* boundary conditions on the GPU (openQ*D, Sec. 1; orbifold form) against
the oracle (oracle.cstar): the library doubles the lattice in x1 from the
physical links (complex-conjugate mirror half) and shifts x1 on the wrapped
x2 / x3 hops.  Dw and Dhat with their adjoints in every storage type, the
multi-rhs kernels (plain, capped, staged), the mixed-precision CGNE and
SAP-GCR to 1e-10, and the QCD+QED links (mirror angles negated)."""
import numpy as np
import pytest

from oracle import cstar, dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import TOL, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.135, 1.2


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def _case(dims, cs, seed):
    u = synth.make_gauge(dims, 0.5, seed)
    ud = cstar.double_links(u)
    a = cstar.clover_field(ud, dirac.kappa_to_m0(KAPPA), CSW, cs)
    return u, ud, a, np.linalg.inv(a)


def _handle(dims, u, cs, fmt):
    oq = _oq()
    h = oq.Handle(dims, cstar=cs)
    h.gauge_upload(to_dev(u), fmt)
    h.clover_build(KAPPA, CSW)
    return h


@pytest.mark.parametrize("cs", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("fmt", [0, 1])
def test_cstar_dw_and_dhat(cs, prec, fmt):
    oq = _oq()
    dims = (4, 6, 4, 6)
    u, ud, a, ainv = _case(dims, cs, 31)
    h = _handle(dims, u, cs, fmt)
    dd = h.dims[0]
    assert dd == (4, 12, 4, 6)
    psi = synth.make_source(dd, 32)
    for dagger in (False, True):
        pin, pout = h.new_packed(prec), h.new_packed(prec)
        h.pack(to_dev(psi), pin, prec)
        h.dw(pin, pout, prec, dagger=dagger)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, prec)
        ref = cstar.dw_dagger(ud, a, psi, cs) if dagger else cstar.dw(ud, a, psi, cs)
        assert rel_err(from_dev(out, psi.shape), ref) < TOL[prec], dagger
        ev = dirac.even_part(psi)
        pin, pout = h.new_packed(prec, oq.EVEN), h.new_packed(prec, oq.EVEN)
        h.pack(to_dev(ev), pin, prec, oq.EVEN)
        h.dw_hat(pin, pout, prec, dagger=dagger)
        out = to_dev(np.zeros_like(ev))
        h.unpack(pout, out, prec, oq.EVEN)
        ref = cstar.dw_hat_dagger(ud, a, ainv, ev, cs) if dagger else cstar.dw_hat(ud, a, ainv, ev, cs)
        assert rel_err(from_dev(out, ev.shape), ref) < TOL[prec], dagger
    h.close()


@pytest.mark.parametrize("cs", [2, 3])
@pytest.mark.parametrize("nr,cap", [(2, 0), (2, 1), (2, 2), (4, 2), (2, 3)])
def test_cstar_multi_rhs_kernels(cs, nr, cap):
    """The multi-rhs kernel computes its neighbour indices itself (32-bit
    strides): the shifted wraps of x2 and x3 there."""
    oq = _oq()
    dims = (4, 4, 6, 8)
    u, ud, a, ainv = _case(dims, cs, 41)
    h = _handle(dims, u, cs, oq.LINK_12)
    nrhs = 5
    for mode in (0, 1, 2):
        h.tune_set(oq.F16, mode, nrhs, 64, 1, nr=nr, regcap=cap, link_fmt=oq.LINK_12)
    dd = h.dims[0]
    psi = synth.make_source(dd, 42, nrhs=nrhs)
    for dagger in (False, True):
        pin, pout = h.new_packed(oq.F16, nrhs=nrhs), h.new_packed(oq.F16, nrhs=nrhs)
        h.pack(to_dev(psi), pin, oq.F16, nrhs=nrhs)
        h.dw(pin, pout, oq.F16, nrhs=nrhs, dagger=dagger)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, oq.F16, nrhs=nrhs)
        got = from_dev(out, psi.shape)
        ev = np.stack([dirac.even_part(p) for p in psi])
        pe, qe = h.new_packed(oq.F16, oq.EVEN, nrhs=nrhs), h.new_packed(oq.F16, oq.EVEN, nrhs=nrhs)
        h.pack(to_dev(ev), pe, oq.F16, oq.EVEN, nrhs=nrhs)
        h.dw_hat(pe, qe, oq.F16, nrhs=nrhs, dagger=dagger)
        oe = to_dev(np.zeros_like(ev))
        h.unpack(qe, oe, oq.F16, oq.EVEN, nrhs=nrhs)
        gote = from_dev(oe, ev.shape)
        for k in range(nrhs):
            ref = cstar.dw_dagger(ud, a, psi[k], cs) if dagger else cstar.dw(ud, a, psi[k], cs)
            assert rel_err(got[k], ref) < TOL[oq.F16], (k, dagger)
            ref = cstar.dw_hat_dagger(ud, a, ainv, ev[k], cs) if dagger else cstar.dw_hat(ud, a, ainv, ev[k], cs)
            assert rel_err(gote[k], ref) < TOL[oq.F16], (k, dagger)
    h.close()


@pytest.mark.parametrize("cs", [1, 3])
def test_cstar_cgne_and_sap_gcr(cs):
    oq = _oq()
    dims = (8, 8, 8, 8)                        # doubled x1 extent 16: the x1 shift of 8 is 2 blocks of 4
    u, ud, a, ainv = _case(dims, cs, 51)
    h = _handle(dims, u, cs, oq.LINK_12)
    dd = h.dims[0]
    eta = dirac.even_part(synth.make_source(dd, 52))
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, sdtype=oq.F16))
    assert rc == oq.OK and st[0]["converged"]
    x = from_dev(psi, eta.shape)
    ax = cstar.dw_hat_dagger(ud, a, ainv, cstar.dw_hat(ud, a, ainv, x, cs), cs)
    check_residual(np.linalg.norm(eta - ax) / np.linalg.norm(eta), st[0]["true_rel_res"])
    src = synth.make_source(dd, 53)
    psi = to_dev(np.zeros_like(src))
    rc, st = h.sap_gcr(to_dev(src), psi, oq.SolverParams(res=1e-10, nmx=500, nkv=12, ncy=4, nmr=4,
                                                         bs=(4, 4, 4, 4), sdtype=oq.F32))
    assert rc == oq.OK and st[0]["converged"]
    x = from_dev(psi, src.shape)
    check_residual(np.linalg.norm(src - cstar.dw(ud, a, x, cs)) / np.linalg.norm(src), st[0]["true_rel_res"])
    # a block layout whose x1 shift is an odd number of blocks would break the colouring
    rc, _ = h.sap_gcr(to_dev(src), psi, oq.SolverParams(res=1e-10, nmx=5, ncy=1, nmr=1, bs=(4, 8, 2, 4),
                                                        sdtype=oq.F32), check=False)
    assert rc == (oq.ERR_ARG if cs >= 2 else oq.OK) or (cs < 2 and rc == oq.ERR_NOCONV)
    h.close()


def test_cstar_qed_links():
    """U(3) links with C*: the mirror half gets exp(-i q A) times U^* (the
    charge-conjugate photon field flips sign)."""
    oq = _oq()
    dims = (4, 4, 4, 6)
    cs, q = 3, -1.0 / 3.0
    u = synth.make_gauge(dims, 0.5, 61)
    A = synth.make_u1_field(dims, 0.3, 62)
    ud = cstar.double_links(u) * np.exp(1j * q * cstar.double_angles(A))[..., None, None]
    a = cstar.clover_field(ud, dirac.kappa_to_m0(KAPPA), CSW, cs)
    h = oq.Handle(dims, cstar=cs)
    h.gauge_upload_qed(to_dev(u), to_dev(np.ascontiguousarray(A)), q)
    h.clover_build(KAPPA, CSW)
    psi = synth.make_source(h.dims[0], 63)
    pin, pout = h.new_packed(oq.F64), h.new_packed(oq.F64)
    h.pack(to_dev(psi), pin, oq.F64)
    h.dw(pin, pout, oq.F64)
    out = to_dev(np.zeros_like(psi))
    h.unpack(pout, out, oq.F64)
    assert rel_err(from_dev(out, psi.shape), cstar.dw(ud, a, psi, cs)) < TOL[oq.F64]
    h.close()
