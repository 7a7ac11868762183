"""Uneven batch: QCD+QED operators (U(3) = SU(3) x U(1) links with charges
2/3 and -1/3) on lattices of three sizes solved by one batched CGNE
(persistent tile-list launches, graph-captured regular iterations).  Every
solution is checked with the FP64 oracle's operator (binary64 residual of the
normal equations <= 1e-10), and the batch agrees with one-system solves."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

LATS = [(4, 4, 4, 4), (6, 4, 4, 8), (8, 6, 6, 8)]
CHARGES = [2.0 / 3.0, -1.0 / 3.0]
KAPPA, CSW = 0.135, 1.0


def _systems():
    out = []
    for k, dims in enumerate(LATS):
        su3 = synth.make_gauge(dims, 0.5, 400 + k)
        a_u1 = synth.make_u1_field(dims, 0.2, 450 + k)
        for q in CHARGES:
            u = synth.apply_u1(su3, a_u1, q)
            a = dirac.clover_field(u, dirac.kappa_to_m0(KAPPA), CSW)
            ainv = np.linalg.inv(a)
            eta = dirac.even_part(synth.make_source(dims, 470 + k))
            out.append((dims, u, a, ainv, eta))
    return out


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_uneven_batch_cgne(prec):
    from paper_2202_07388_gb300 import oq
    systems = _systems()
    h = oq.Handle([s[0] for s in systems])
    for lat, (dims, u, a, ainv, eta) in enumerate(systems):
        h.gauge_upload(to_dev(u), oq.LINK_18, lat=lat)
        h.clover_build(KAPPA, CSW, lat=lat)
    etas = [to_dev(s[4]) for s in systems]
    psis = [to_dev(np.zeros_like(s[4])) for s in systems]
    prm = oq.SolverParams(res=1e-10, nmx=5000, sdtype=prec)
    rc, st = h.cgne_batch(list(range(len(systems))), etas, psis, prm)
    assert rc == oq.OK, st
    for k, (dims, u, a, ainv, eta) in enumerate(systems):
        x = from_dev(psis[k], eta.shape)
        r = eta - dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, x))
        check_residual(np.linalg.norm(r) / np.linalg.norm(eta), st[k]["true_rel_res"])
        assert st[k]["converged"]
        # the same system alone
        psi1 = to_dev(np.zeros_like(eta))
        rc1, st1 = h.cgne(etas[k], psi1, prm, lat=k)
        assert rc1 == oq.OK
        assert abs(st1[0]["steps"] - st[k]["steps"]) <= 2
        assert rel_err(from_dev(psi1, eta.shape), x) < 1e-8
    # repeated calls give identical results (graph replay is deterministic)
    psis2 = [to_dev(np.zeros_like(s[4])) for s in systems]
    rc2, st2 = h.cgne_batch(list(range(len(systems))), etas, psis2, prm)
    assert rc2 == oq.OK
    for k in range(len(systems)):
        assert np.array_equal(psis2[k].cpu().numpy(), psis[k].cpu().numpy())
    h.close()


def test_batch_rejects_mixed_link_formats():
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 4, 4)
    u = synth.make_gauge(dims, 0.5, 1)
    h = oq.Handle([dims, dims])
    h.gauge_upload(to_dev(u), oq.LINK_18, lat=0)
    h.gauge_upload(to_dev(u), oq.LINK_12, lat=1)
    for lat in (0, 1):
        h.clover_build(KAPPA, CSW, lat=lat)
    eta = to_dev(dirac.even_part(synth.make_source(dims, 2)))
    psi = [to_dev(np.zeros(dims + (4, 3), complex)) for _ in range(2)]
    rc, _ = h.cgne_batch([0, 1], [eta, eta], psi, oq.SolverParams(sdtype=1), check=False)
    assert rc == oq.ERR_ARG
    h.close()
