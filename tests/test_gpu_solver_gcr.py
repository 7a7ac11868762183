"""GPU SAP and SAP-preconditioned flexible GCR (Sec. 3, 3.1, 3.2) against
the FP64 oracle: SAP applications element by element (binary32 arithmetic,
1e-5), GCR / SAP-GCR solutions checked with the oracle's own operator to a
binary64 relative residual of 1e-10, the adaptive variant, and the error
paths."""
import numpy as np
import pytest

from oracle import dirac, solvers
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import oracle_case, make_handle, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def _true_res(u, a, eta, x):
    r = eta - dirac.dw(u, a, x)
    return np.linalg.norm(r.reshape(-1)) / np.linalg.norm(eta.reshape(-1))


@pytest.mark.parametrize("dims,bs,ncy,nmr", [((8, 8, 8, 8), (4, 4, 4, 4), 2, 3),
                                             ((4, 4, 4, 4), (2, 2, 2, 2), 1, 5),
                                             ((8, 4, 4, 8), (2, 2, 2, 4), 3, 2)])
@pytest.mark.parametrize("link_fmt", [0, 1])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_sap_apply_matches_oracle(dims, bs, ncy, nmr, link_fmt, kernel):
    """Every SAP block kernel: operands in shared memory (0), global operands
    with one (1) or two (2) blocks per SM."""
    oq = _oq()
    u, a, ainv = oracle_case(dims, 0.5, 21, 0.1365, 1.0)
    rho = synth.make_source(dims, 22)
    ref = solvers.sap(u, a, rho, bs, ncy, nmr)
    h = make_handle(dims, u, 0.1365, 1.0, link_fmt)
    h.set_option(oq.OPT_SAP_KERNEL, kernel)
    prho, pphi = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(to_dev(rho), prho, oq.F32)
    h.sap_apply(prho, pphi, oq.SolverParams(ncy=ncy, nmr=nmr, bs=bs))
    out = to_dev(np.zeros_like(rho))
    h.unpack(pphi, out, oq.F32)
    assert rel_err(from_dev(out, rho.shape), ref) < 1e-5


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("ncy,alpha,tol_frac", [(1, 0.5, 0.0), (1, 0.6, 0.0), (1, 0.9, 0.05), (2, 0.5, 0.0)])
def test_adaptive_sap_apply_matches_oracle(kernel, ncy, alpha, tol_frac):
    """The adaptive MR exits of Sec. 3.2 (after >= 4 steps when the block
    residual exceeds alpha times the previous one, when it grew, or below
    mr_tol = tol_frac ||rho|| / n_blocks; at most 20 steps) element by element
    against the oracle's SAP with binary32 storage (the block decisions taken
    on binary32 residuals on both sides), for every block kernel.  On this
    field alpha = 0.5 stops every block at 4 steps, 0.6 after 8 to 10, and the
    tolerance after 7 or 8."""
    oq = _oq()
    dims, bs = (8, 8, 8, 8), (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.5, 23, 0.1365, 1.0)
    rho = synth.make_source(dims, 24)
    nblk = int(np.prod([d // b for d, b in zip(dims, bs)]))
    mr_tol = tol_frac * np.linalg.norm(rho) / nblk
    info = {}
    ref = solvers.sap(u, a, rho, bs, ncy, 20, adaptive=True, alpha=alpha, mr_tol=mr_tol, store="fp32", info=info)
    assert info["cycles"] == ncy               # the cycle test (not applied by oq_sap_apply) never stops early
    steps = np.concatenate(info["mr_steps"])
    assert steps.min() < 20                    # the exit rules did act
    h = make_handle(dims, u, 0.1365, 1.0, oq.LINK_12)
    h.set_option(oq.OPT_SAP_KERNEL, kernel)
    prho, pphi = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(to_dev(rho), prho, oq.F32)
    h.sap_apply(prho, pphi, oq.SolverParams(ncy=ncy, nmr=20, bs=bs, adaptive=1, alpha=alpha), mr_tol=mr_tol)
    out = to_dev(np.zeros_like(rho))
    h.unpack(pphi, out, oq.F32)
    assert rel_err(from_dev(out, rho.shape), ref) < 1e-5


@pytest.mark.parametrize("ncy,nmr,bs", [(0, 0, (4, 4, 4, 4)), (2, 4, (2, 2, 2, 2)), (4, 5, (4, 4, 4, 4))])
def test_sap_gcr_converges_to_binary64_residual(ncy, nmr, bs):
    oq = _oq()
    dims = (8, 8, 8, 8) if bs[0] == 4 else (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.5, 31, 0.1365, 1.0)
    eta = synth.make_source(dims, 32)
    h = make_handle(dims, u, 0.1365, 1.0, oq.LINK_12)
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=500, nkv=12, ncy=ncy, nmr=nmr, bs=bs,
                                                         sdtype=oq.F32))
    assert rc == oq.OK, st
    x = from_dev(psi, eta.shape)
    check_residual(_true_res(u, a, eta, x), st[0]["true_rel_res"])
    assert st[0]["converged"] and st[0]["true_rel_res"] <= 1e-10
    assert st[0]["restarts"] >= 2   # binary32 Krylov vectors: binary64 restarts carry the accuracy


def test_sap_reduces_gcr_steps_and_matches_oracle_solution():
    oq = _oq()
    dims = (8, 8, 8, 8)
    u, a, ainv = oracle_case(dims, 0.5, 41, 0.1365, 1.0)
    eta = synth.make_source(dims, 42)
    h = make_handle(dims, u, 0.1365, 1.0, oq.LINK_12)
    steps = {}
    for ncy in (0, 4):
        psi = to_dev(np.zeros_like(eta))
        rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=1000, nkv=16, ncy=ncy, nmr=5,
                                                             bs=(4, 4, 4, 4), sdtype=oq.F32))
        assert rc == oq.OK
        steps[ncy] = st[0]["steps"]
    assert steps[4] < steps[0] / 3
    ref = solvers.fgcr(lambda v: dirac.dw(u, a, v), lambda v: v, eta, 1e-11, 2000, 16)
    x = from_dev(psi, eta.shape)
    assert rel_err(x, ref.x) < 1e-8


@pytest.mark.parametrize("kernel", [0, 2])
def test_adaptive_sap_gcr(kernel):
    """Sec. 3.2: ncy, nmr are maxima (20, 20), alpha = 0.9."""
    oq = _oq()
    dims = (8, 8, 8, 8)
    u, a, ainv = oracle_case(dims, 0.5, 51, 0.1365, 1.0)
    eta = synth.make_source(dims, 52)
    h = make_handle(dims, u, 0.1365, 1.0, oq.LINK_12)
    h.set_option(oq.OPT_SAP_KERNEL, kernel)
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=300, nkv=16, ncy=20, nmr=20,
                                                         bs=(4, 4, 4, 4), sdtype=oq.F32, adaptive=1, alpha=0.9))
    assert rc == oq.OK
    check_residual(_true_res(u, a, eta, from_dev(psi, eta.shape)), st[0]["true_rel_res"])
    s = st[0]
    assert 1.0 <= s["mr_avg"] <= 20.0
    assert s["steps"] <= s["cycles"] <= 20 * s["steps"]


def test_gcr_argument_and_convergence_errors():
    oq = _oq()
    dims = (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.3, 1, 0.13, 1.0)
    eta = synth.make_source(dims, 61)
    h = make_handle(dims, u, 0.13, 1.0, oq.LINK_12)
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=3, nkv=8, ncy=1, nmr=2, bs=(2, 2, 2, 2),
                                                         sdtype=oq.F32))
    assert rc == oq.ERR_NOCONV and st[0]["steps"] == 3 and not st[0]["converged"]
    # odd number of blocks in a direction: rejected before any work
    rc, _ = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(ncy=1, nmr=2, bs=(4, 2, 2, 2), sdtype=oq.F32),
                      check=False)
    assert rc == oq.ERR_ARG


def test_autotuner_picks_valid_shapes_and_keeps_results():
    oq = _oq()
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.1365, 1.3)
    h = make_handle(dims, u, 0.1365, 1.3, oq.LINK_12)
    psi = synth.make_source(dims, 71, nrhs=4)
    for prec in (1, 3):
        shapes = h.autotune(prec, nrhs=4)
        for mode, (bx, by, ms, fmt, nr, cap) in shapes.items():
            assert bx % 32 == 0 and bx * by <= (256 if nr == 1 else 128) and ms > 0
            assert fmt in ("12-real", "18-real") and nr in (1, 2, 4) and cap in (0, 1, 2, 3)
            assert cap < 2 or (nr > 1 and fmt == "12-real")       # staged hops: multi-rhs, 12-real links
            assert cap != 3 or nr == 2
        # pass 2 is tuned once per epilogue; epi 0 is what oq_tune_get reports
        epis = h.tuned_epilogues(prec, nrhs=4)
        assert epis["store"] == shapes[2]
        for bx, by, ms, fmt, nr, cap in epis.values():
            assert bx % 32 == 0 and ms > 0 and (cap < 2 or (nr > 1 and fmt == "12-real"))
        pin, pout = h.new_packed(prec, nrhs=4), h.new_packed(prec, nrhs=4)
        h.pack(to_dev(psi), pin, prec, nrhs=4)
        h.dw(pin, pout, prec, nrhs=4)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, prec, nrhs=4)
        got = from_dev(out, psi.shape)
        for k in range(4):
            assert rel_err(got[k], dirac.dw(u, a, psi[k])) < (1e-5 if prec == 1 else 2e-3)


@pytest.mark.parametrize("dims,bs,ncy,nmr", [((8, 8, 8, 8), (4, 4, 4, 4), 2, 3),
                                             ((4, 4, 4, 4), (2, 2, 2, 2), 1, 5),
                                             ((8, 4, 4, 8), (2, 2, 2, 4), 3, 2)])
@pytest.mark.parametrize("link_fmt", [0, 1])
def test_sap_eo_block_solver_matches_oracle(dims, bs, ncy, nmr, link_fmt):
    """The even-odd reduced block solver (MR on each block's Schur
    complement, odd sites solved afterwards) against the oracle's, element
    by element."""
    oq = _oq()
    u, a, ainv = oracle_case(dims, 0.5, 23, 0.1365, 1.0)
    rho = synth.make_source(dims, 24)
    ref = solvers.sap(u, a, rho, bs, ncy, nmr, eo=True, ainv=ainv)
    h = make_handle(dims, u, 0.1365, 1.0, link_fmt)
    prho, pphi = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(to_dev(rho), prho, oq.F32)
    h.sap_apply(prho, pphi, oq.SolverParams(ncy=ncy, nmr=nmr, bs=bs, sap_eo=1))
    out = to_dev(np.zeros_like(rho))
    h.unpack(pphi, out, oq.F32)
    assert rel_err(from_dev(out, rho.shape), ref) < 1e-5


@pytest.mark.parametrize("adaptive", [0, 1])
def test_sap_eo_gcr(adaptive):
    """SAP-GCR with the even-odd block solver to a binary64 residual of 1e-10
    (checked with the oracle's operator), in fewer GCR steps than with MR on
    the full block operator at the same MR count."""
    oq = _oq()
    dims = (8, 8, 8, 8)
    u, a, ainv = oracle_case(dims, 0.5, 53, 0.1365, 1.0)
    eta = synth.make_source(dims, 54)
    h = make_handle(dims, u, 0.1365, 1.0, oq.LINK_12)
    steps = {}
    for eo in (0, 1):
        psi = to_dev(np.zeros_like(eta))
        prm = oq.SolverParams(res=1e-10, nmx=500, nkv=16, ncy=4 if not adaptive else 20,
                              nmr=4 if not adaptive else 20, bs=(4, 4, 4, 4), sdtype=oq.F32, adaptive=adaptive,
                              alpha=0.9, sap_eo=eo)
        rc, st = h.sap_gcr(to_dev(eta), psi, prm)
        assert rc == oq.OK
        check_residual(_true_res(u, a, eta, from_dev(psi, eta.shape)), st[0]["true_rel_res"])
        steps[eo] = st[0]["steps"]
    if not adaptive:
        assert steps[1] <= steps[0]


def test_sap_eo_needs_even_bs3():
    oq = _oq()
    dims = (4, 4, 4, 6)
    u, a, ainv = oracle_case(dims, 0.3, 25, 0.13, 1.0)
    h = make_handle(dims, u, 0.13, 1.0, oq.LINK_12)
    prho, pphi = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(to_dev(synth.make_source(dims, 26)), prho, oq.F32)
    with pytest.raises(oq.OqError):
        h.sap_apply(prho, pphi, oq.SolverParams(ncy=1, nmr=2, bs=(2, 2, 2, 3), sap_eo=1))
    h.sap_apply(prho, pphi, oq.SolverParams(ncy=1, nmr=2, bs=(2, 2, 2, 3)))
