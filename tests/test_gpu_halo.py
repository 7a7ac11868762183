"""Time-split sub-domains on the GPU (Sec. 3: the lattice divided into local
lattices), R parts held in one process and exchanged in place
(``LoopbackComm``): the faces packed by ``oq_face_pack`` and consumed by
``oq_dw_apply_halo`` / ``oq_dhat_pass``.

Binary64: the split Dw, Dhat and Dhat^dag equal the unsplit library
operator bit for bit (the same arithmetic, only the sender of the boundary
projection changes) and the oracle to rounding; binary32 / binary16 agree with
the oracle within the storage tolerance.  The distributed binary64 CGNE
reaches an oracle-checked true residual of 1e-10 and the unsplit CGNE's
solution.  Whole-lattice entry points refuse a sub-domain."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import halo, synth
from tests.gpu_cases import TOL, oracle_case, make_handle, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.1365, 1.3


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def _parts(split, u, link_fmt):
    oq = _oq()
    hs = []
    for r in range(split.nparts):
        h = oq.Handle(split.local_dims, bc_t=oq.BC_HALO)
        h.gauge_upload_halo(to_dev(np.ascontiguousarray(split.ext_links(u, r))), link_fmt)
        h.clover_build(KAPPA, CSW)
        hs.append(h)
    return hs


def _pack_parts(split, hs, field, prec, subset, nrhs=1):
    oq = _oq()
    out = []
    for r, h in enumerate(hs):
        loc = np.ascontiguousarray(field[:, split.start(r):split.start(r) + split.tl] if nrhs > 1
                                   else split.local(field, r))
        p = h.new_packed(prec, subset, nrhs=nrhs)
        h.pack(to_dev(loc), p, prec, subset, nrhs=nrhs)
        out.append(p)
    return out


def _unpack_parts(split, hs, packed, prec, subset, shape_loc, nrhs=1):
    res = []
    shape = ((nrhs,) if nrhs > 1 else ()) + shape_loc
    for h, p in zip(hs, packed):
        c = to_dev(np.zeros(shape, np.complex128))
        h.unpack(p, c, prec, subset, nrhs=nrhs)
        res.append(from_dev(c, shape))
    if nrhs > 1:
        return np.concatenate(res, axis=1)
    return split.gather(res)


@pytest.mark.parametrize("dims,nparts", [((8, 4, 4, 6), 2), ((8, 6, 4, 4), 4), ((12, 4, 6, 4), 3)])
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_split_dw_and_dhat(dims, nparts, prec):
    oq = _oq()
    u, a, ainv = oracle_case(dims, 0.5, 7, KAPPA, CSW)
    split = halo.TimeSplit(dims, nparts)
    hs = _parts(split, u, oq.LINK_12)
    comm = halo.LoopbackComm(nparts)
    nrhs = 2
    psi = synth.make_source(dims, 70, nrhs=nrhs)
    shape_loc = split.local_dims + (4, 3)
    whole = make_handle(dims, u, KAPPA, CSW, oq.LINK_12)
    for dagger in (False, True):
        # full operator: faces of both parities (subset FULL)
        ins = _pack_parts(split, hs, psi, prec, oq.FULL, nrhs)
        outs = [h.new_packed(prec, oq.FULL, nrhs=nrhs) for h in hs]
        fp = [h.new_faces(prec, nrhs, parities=2) for h in hs]
        fn = [h.new_faces(prec, nrhs, parities=2) for h in hs]
        for h, x, a_, b_ in zip(hs, ins, fp, fn):
            h.face_pack(x, a_, b_, prec, oq.FULL, nrhs=nrhs, dagger=dagger)
        from_next, from_prev = comm.exchange(fp, fn)
        for r, (h, x, y) in enumerate(zip(hs, ins, outs)):
            sn, sp = split.signs(r)
            h.dw_halo(x, y, prec, oq.Handle.halo(from_next[r], from_prev[r], sn, sp), nrhs=nrhs, dagger=dagger)
        got = _unpack_parts(split, hs, outs, prec, oq.FULL, shape_loc, nrhs)
        pw, qw = whole.new_packed(prec, nrhs=nrhs), whole.new_packed(prec, nrhs=nrhs)
        whole.pack(to_dev(psi), pw, prec, nrhs=nrhs)
        whole.dw(pw, qw, prec, nrhs=nrhs, dagger=dagger)
        cw = to_dev(np.zeros_like(psi))
        whole.unpack(qw, cw, prec, nrhs=nrhs)
        want = from_dev(cw, psi.shape)
        for k in range(nrhs):
            ref = dirac.dw_dagger(u, a, psi[k]) if dagger else dirac.dw(u, a, psi[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)
        if prec == oq.F64:
            assert np.array_equal(got, want), "split binary64 Dw differs from the unsplit one"
        # Dhat: two passes, one exchange each
        ev = np.stack([dirac.even_part(p) for p in psi])
        op = halo.GpuSplitDhat(split, range(nparts), hs, comm, prec=prec, nrhs=nrhs)
        xs = _pack_parts(split, hs, ev, prec, oq.EVEN, nrhs)
        ys = op.new_field()
        op.dhat(xs, ys, dagger=dagger)
        got = _unpack_parts(split, hs, ys, prec, oq.EVEN, shape_loc, nrhs)
        pe, qe = whole.new_packed(prec, oq.EVEN, nrhs=nrhs), whole.new_packed(prec, oq.EVEN, nrhs=nrhs)
        whole.pack(to_dev(ev), pe, prec, oq.EVEN, nrhs=nrhs)
        whole.dw_hat(pe, qe, prec, nrhs=nrhs, dagger=dagger)
        ce = to_dev(np.zeros_like(ev))
        whole.unpack(qe, ce, prec, oq.EVEN, nrhs=nrhs)
        want = from_dev(ce, ev.shape)
        for k in range(nrhs):
            ref = dirac.dw_hat_dagger(u, a, ainv, ev[k]) if dagger else dirac.dw_hat(u, a, ainv, ev[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)
        if prec == oq.F64:
            assert np.array_equal(got, want), "split binary64 Dhat differs from the unsplit one"
    for h in hs:
        h.close()
    whole.close()


@pytest.mark.parametrize("nparts", [2, 4])
def test_split_cgne_binary64(nparts):
    oq = _oq()
    dims = (8, 6, 4, 6)
    u, a, ainv = oracle_case(dims, 0.5, 9, KAPPA, CSW)
    split = halo.TimeSplit(dims, nparts)
    hs = _parts(split, u, oq.LINK_12)
    comm = halo.LoopbackComm(nparts)
    op = halo.GpuSplitDhat(split, range(nparts), hs, comm, prec=oq.F64, nrhs=1)
    eta = dirac.even_part(synth.make_source(dims, 90))
    etas = _pack_parts(split, hs, eta, oq.F64, oq.EVEN)
    xs = op.new_field()
    st = halo.split_cgne(op, comm, etas, xs, res=1e-10, nmx=5000)
    x = _unpack_parts(split, hs, xs, oq.F64, oq.EVEN, split.local_dims + (4, 3))
    normal = lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v))  # noqa: E731
    rel = np.linalg.norm(eta - normal(x)) / np.linalg.norm(eta)
    assert st[0]["converged"]
    check_residual(rel, st[0]["true_rel_res"])
    # the unsplit binary64 CGNE of the library reaches the same solution
    whole = make_handle(dims, u, KAPPA, CSW, oq.LINK_12)
    psi = to_dev(np.zeros_like(eta))
    rc, sw = whole.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, sdtype=oq.F64))
    assert rc == oq.OK
    xw = from_dev(psi, eta.shape)
    assert np.linalg.norm(x - xw) <= 1e-8 * np.linalg.norm(xw)
    assert abs(st[0]["steps"] - sw[0]["steps"]) <= 2
    for h in hs:
        h.close()
    whole.close()


def test_sub_domain_refuses_whole_lattice_calls():
    oq = _oq()
    dims = (8, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.5, 7, KAPPA, CSW)
    split = halo.TimeSplit(dims, 2)
    h = _parts(split, u, oq.LINK_12)[0]
    x, y = h.new_packed(oq.F32, oq.EVEN), h.new_packed(oq.F32, oq.EVEN)
    x.zero_()
    from paper_2202_07388_gb300.oq import lib, _ptr, _stream
    assert lib().oq_dw_hat_apply(h.h, 0, oq.F32, _ptr(x), _ptr(y), 1, 0, _stream()) == oq.ERR_STATE
    assert h.dhat_pass(1, x, None, y, oq.F32, halo=None, check=False) == oq.ERR_STATE
    f = h.new_faces(oq.F32)
    assert h.dhat_pass(1, x, None, y, oq.F32, halo=oq.Handle.halo(f, f, 2.0, 1.0), check=False) == oq.ERR_ARG
    assert h.face_bytes(oq.DF64) == 0
    rc, _ = h.cgne(to_dev(np.zeros(split.local_dims + (4, 3), np.complex128)),
                   to_dev(np.zeros(split.local_dims + (4, 3), np.complex128)), oq.SolverParams(), check=False)
    assert rc == oq.ERR_STATE
    # a whole lattice cannot take sub-domain links
    w = make_handle(dims, u, KAPPA, CSW, oq.LINK_12)
    assert lib().oq_gauge_upload_halo(w.h, 0, _ptr(to_dev(u)), oq.LINK_12, _stream()) == oq.ERR_STATE
    h.close()
    w.close()
