"""GPU parity of the multi-right-hand-side stencil (2 or 4 right-hand sides
per thread, packed two-lane binary32 arithmetic, with and without the
register cap, and with the hop operands staged in shared memory) against
the FP64 oracle, pinned with oq_tune_set: full Dw,
Dhat and their adjoints for every binary32-arithmetic storage type and both
link formats, on ragged site counts and right-hand-side counts that are not
multiples of the per-thread count; the fused CG epilogue through a batched
CGNE solve to a binary64 residual of 1e-10."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import TOL, oracle_case, make_handle, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

CASES = [((6, 4, 2, 6), 0.5, 2, 0.135, 1.0),       # Vh = 144: ragged tail for every bx
         ((8, 6, 4, 10), 0.5, 3, 0.1365, 1.3)]     # Vh = 960


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def torch_equal(x, y):
    import torch
    return bool(torch.equal(x, y))


def unpack(h, packed, shape, n, even=False):
    oq = _oq()
    out = to_dev(np.zeros(shape, dtype=np.complex128))
    if even:
        h.unpack(packed, out, oq.DF64, oq.EVEN, nrhs=n)
    else:
        h.unpack(packed, out, oq.DF64, nrhs=n)
    return out


def _pin(h, prec, nrhs, bx, by, nr, cap, fmt):
    for mode in (0, 1, 2):
        h.tune_set(prec, mode, nrhs, bx, by, nr=nr, regcap=cap, link_fmt=fmt)


SHAPES = [(2, 5, 64, 2), (4, 5, 32, 1), (4, 8, 128, 1), (2, 2, 32, 1)]
# (regcap, link format): regcap 2 and 3 stage the hop operands (12-real links);
# regcap 3 (the staged kernel at 168 registers) exists for 2 rhs per thread
CAPS = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 1), (3, 1)]
LAUNCHES = [sh + cf for sh in SHAPES for cf in CAPS if not (cf[0] == 3 and sh[0] != 2)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("nr,nrhs,bx,by,cap,fmt", LAUNCHES)
def test_multi_rhs_dw_and_dw_hat(case, prec, nr, nrhs, bx, by, cap, fmt):
    oq = _oq()
    dims, eps, seed, kappa, csw = case
    u, a, ainv = oracle_case(dims, eps, seed, kappa, csw)
    h = make_handle(dims, u, kappa, csw, oq.LINK_12)
    _pin(h, prec, nrhs, bx, by, nr, cap, fmt)
    psi = synth.make_source(dims, seed + 400, nrhs=nrhs)
    for dagger in (False, True):
        pin, pout = h.new_packed(prec, nrhs=nrhs), h.new_packed(prec, nrhs=nrhs)
        h.pack(to_dev(psi), pin, prec, nrhs=nrhs)
        h.dw(pin, pout, prec, nrhs=nrhs, dagger=dagger)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, prec, nrhs=nrhs)
        got = from_dev(out, psi.shape)
        for k in range(nrhs):
            ref = dirac.dw_dagger(u, a, psi[k]) if dagger else dirac.dw(u, a, psi[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)
        ev = np.stack([dirac.even_part(p) for p in psi])
        pin, pout = h.new_packed(prec, oq.EVEN, nrhs=nrhs), h.new_packed(prec, oq.EVEN, nrhs=nrhs)
        h.pack(to_dev(ev), pin, prec, oq.EVEN, nrhs=nrhs)
        h.dw_hat(pin, pout, prec, nrhs=nrhs, dagger=dagger)
        out = to_dev(np.zeros_like(ev))
        h.unpack(pout, out, prec, oq.EVEN, nrhs=nrhs)
        got = from_dev(out, ev.shape)
        for k in range(nrhs):
            ref = dirac.dw_hat_dagger(u, a, ainv, ev[k]) if dagger else dirac.dw_hat(u, a, ainv, ev[k])
            assert rel_err(got[k], ref) < TOL[prec], (k, dagger)


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("nr,cap", [(2, 0), (4, 1), (2, 2), (4, 2), (2, 3)])
def test_multi_rhs_cgne_epilogues(prec, nr, cap):
    """The norm and CG-update epilogues of the multi-rhs kernel inside the
    batched CGNE: 5 right-hand sides (a ragged group), every one to a binary64
    normal-equation residual of 1e-10, the same step counts as the one-rhs
    kernel up to rounding."""
    oq = _oq()
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.135, 1.0)
    n = 5
    eta = np.stack([dirac.even_part(e) for e in synth.make_source(dims, 91, nrhs=n)])
    steps = {}
    for variant in ("one", "multi"):
        h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
        if variant == "multi":
            _pin(h, prec, n, 32, 1, nr, cap, -1)
        else:
            _pin(h, prec, n, 64, 1, 1, 0, -1)
        psi = to_dev(np.zeros_like(eta))
        rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, sdtype=prec), nrhs=n)
        assert rc == oq.OK
        x = from_dev(psi, eta.shape)
        for k in range(n):
            ax = dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, x[k]))
            r = np.linalg.norm((eta[k] - ax).reshape(-1)) / np.linalg.norm(eta[k].reshape(-1))
            assert st[k]["converged"], (variant, k, r)
            check_residual(r, st[k]["true_rel_res"])
        steps[variant] = [s["steps"] for s in st]
    for a_, b_ in zip(steps["one"], steps["multi"]):
        assert abs(a_ - b_) <= 3


def test_tune_set_rejects_inadmissible_launches():
    oq = _oq()
    dims = (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.3, 1, 0.13, 1.0)
    h = make_handle(dims, u, 0.13, 1.0, oq.LINK_12)
    assert h.tune_set(oq.F16, 1, 4, 48, 1, check=False) == oq.ERR_ARG            # bx not a multiple of 32
    assert h.tune_set(oq.F16, 1, 4, 128, 2, nr=2, check=False) == oq.ERR_ARG     # 256 threads with nr > 1
    assert h.tune_set(oq.F64, 1, 4, 64, 1, nr=2, check=False) == oq.ERR_ARG      # binary64: one rhs per thread
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=3, check=False) == oq.ERR_ARG
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=2, link_fmt=0, check=False) == oq.ERR_ARG  # staged: 12-real
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=2, link_fmt=1) == oq.OK
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=3) == oq.OK     # staged, 168 registers
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=4, regcap=3, check=False) == oq.ERR_ARG   # 2 rhs per thread only
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=4, check=False) == oq.ERR_ARG
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=1, regcap=1, check=False) == oq.ERR_ARG   # cap: nr > 1 or DF64
    assert h.tune_set(oq.DF64, 1, 4, 128, 2, nr=1, regcap=1, check=False) == oq.ERR_ARG  # capped: <= 128 threads
    assert h.tune_set(oq.DF64, 1, 4, 64, 2, nr=1, regcap=1) == oq.OK
    assert h.tune_set(oq.DF64, 1, 4, 64, 2, nr=1, regcap=2) == oq.OK
    assert h.tune_set(oq.DF64, 1, 4, 64, 2, nr=1, regcap=3, check=False) == oq.ERR_ARG
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=2) == oq.OK      # staged on the uploaded 12-real links
    assert h.tune_set(oq.F16, 1, 4, 64, 1, nr=4, regcap=1) == oq.OK
    assert h.tune_get(oq.F16, 1, 4)[4:] == (4, 1)
    # a pinned pass-2 launch serves every epilogue
    assert h.tune_set(oq.F16, 2, 4, 64, 1, nr=2, regcap=2) == oq.OK
    assert all(v[:2] == (64, 1) and v[4:] == (2, 2) for v in h.tuned_epilogues(oq.F16, nrhs=4).values())
    assert oq.lib().oq_tune_get_epi(h.h, 0, oq.F16, 2, 3, 4, *[oq.C.byref(oq.C.c_int()) for _ in range(2)],
                                    oq.C.byref(oq.C.c_float()), None, None, None) == oq.ERR_ARG
    h2 = make_handle(dims, u, 0.13, 1.0, oq.LINK_18)
    assert h2.tune_set(oq.F32, 1, 1, 64, 1, link_fmt=oq.LINK_12, check=False) == oq.ERR_ARG
    assert h2.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=2, check=False) == oq.ERR_ARG  # staged: 12-real links
    assert h2.tune_set(oq.F16, 1, 4, 64, 1, nr=2, regcap=3, check=False) == oq.ERR_ARG


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("cap", [0, 1, 2])
def test_double_float_kernels_pinned(case, cap):
    """Double-float storage and arithmetic (one rhs per thread), with and
    without the register cap, pinned with oq_tune_set: Dw, Dhat and their
    adjoints within 1e-12 of the FP64 oracle for 3 right-hand sides."""
    oq = _oq()
    dims, eps, seed, kappa, csw = case
    u, a, ainv = oracle_case(dims, eps, seed, kappa, csw)
    h = make_handle(dims, u, kappa, csw, oq.LINK_12)
    n = 3
    for mode in (0, 1, 2):
        h.tune_set(oq.DF64, mode, n, 32, 2, nr=1, regcap=cap)
    psi = synth.make_source(dims, seed + 500, nrhs=n)
    ev = np.stack([dirac.even_part(p) for p in psi])
    for dagger in (False, True):
        pin, pout = h.new_packed(oq.DF64, nrhs=n), h.new_packed(oq.DF64, nrhs=n)
        h.pack(to_dev(psi), pin, oq.DF64, nrhs=n)
        h.dw(pin, pout, oq.DF64, nrhs=n, dagger=dagger)
        out = to_dev(np.zeros_like(psi))
        h.unpack(pout, out, oq.DF64, nrhs=n)
        got = from_dev(out, psi.shape)
        for k in range(n):
            ref = dirac.dw_dagger(u, a, psi[k]) if dagger else dirac.dw(u, a, psi[k])
            assert rel_err(got[k], ref) < TOL[4]
        pin, pout = h.new_packed(oq.DF64, oq.EVEN, nrhs=n), h.new_packed(oq.DF64, oq.EVEN, nrhs=n)
        h.pack(to_dev(ev), pin, oq.DF64, oq.EVEN, nrhs=n)
        h.dw_hat(pin, pout, oq.DF64, nrhs=n, dagger=dagger)
        out = to_dev(np.zeros_like(ev))
        h.unpack(pout, out, oq.DF64, oq.EVEN, nrhs=n)
        got = from_dev(out, ev.shape)
        for k in range(n):
            ref = dirac.dw_hat_dagger(u, a, ainv, ev[k]) if dagger else dirac.dw_hat(u, a, ainv, ev[k])
            assert rel_err(got[k], ref) < TOL[4]


def _df64_outputs(h, psi, ev, n):
    """Packed double-float Dw, Dhat and their adjoints of n right-hand sides."""
    oq = _oq()
    outs = []
    for dagger in (False, True):
        pin, pout = h.new_packed(oq.DF64, nrhs=n), h.new_packed(oq.DF64, nrhs=n)
        h.pack(to_dev(psi), pin, oq.DF64, nrhs=n)
        h.dw(pin, pout, oq.DF64, nrhs=n, dagger=dagger)
        outs.append(pout.clone())
        pin, pout = h.new_packed(oq.DF64, oq.EVEN, nrhs=n), h.new_packed(oq.DF64, oq.EVEN, nrhs=n)
        h.pack(to_dev(ev), pin, oq.DF64, oq.EVEN, nrhs=n)
        h.dw_hat(pin, pout, oq.DF64, nrhs=n, dagger=dagger)
        outs.append(pout.clone())
    return outs


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("bx,by,cap", [(32, 1, 0), (64, 2, 0), (32, 2, 1)])
def test_double_float_two_rhs_per_thread(case, bx, by, cap):
    """Double-float passes with two right-hand sides per thread (packed
    two-lane arithmetic, links and clover loaded once): bit for bit the
    one-rhs kernel's Dw, Dhat and adjoints for 5 right-hand sides (a ragged
    pair), and within 1e-12 of the FP64 oracle."""
    oq = _oq()
    dims, eps, seed, kappa, csw = case
    u, a, ainv = oracle_case(dims, eps, seed, kappa, csw)
    h = make_handle(dims, u, kappa, csw, oq.LINK_12)
    n = 5
    psi = synth.make_source(dims, seed + 600, nrhs=n)
    ev = np.stack([dirac.even_part(p) for p in psi])
    for mode in (0, 1, 2):
        h.tune_set(oq.DF64, mode, n, 32, 2, nr=1, regcap=0)
    one = _df64_outputs(h, psi, ev, n)
    for mode in (0, 1, 2):
        h.tune_set(oq.DF64, mode, n, bx, by, nr=2, regcap=cap)
    assert h.tune_get(oq.DF64, 1, n)[4:] == (2, cap)
    two = _df64_outputs(h, psi, ev, n)
    for k, (x1, x2) in enumerate(zip(one, two)):
        assert torch_equal(x1, x2), k
    outs = iter(two)
    for dagger in (False, True):
        got = from_dev(unpack(h, next(outs), psi.shape, n), psi.shape)
        for k in range(n):
            ref = dirac.dw_dagger(u, a, psi[k]) if dagger else dirac.dw(u, a, psi[k])
            assert rel_err(got[k], ref) < TOL[4]
        got = from_dev(unpack(h, next(outs), ev.shape, n, even=True), ev.shape)
        for k in range(n):
            ref = dirac.dw_hat_dagger(u, a, ainv, ev[k]) if dagger else dirac.dw_hat(u, a, ainv, ev[k])
            assert rel_err(got[k], ref) < TOL[4]
    assert h.tune_set(oq.DF64, 1, n, 128, 2, nr=2, regcap=0, check=False) == oq.ERR_ARG   # <= 128 threads
    assert h.tune_set(oq.DF64, 1, n, 64, 1, nr=2, regcap=2, check=False) == oq.ERR_ARG   # regcap 0 / 1
    assert h.tune_set(oq.DF64, 1, n, 64, 1, nr=4, check=False) == oq.ERR_ARG
    assert h.tune_set(oq.DF64, 1, 1, 64, 1, nr=2, check=False) == oq.ERR_ARG             # nr > nrhs


def test_double_float_resets_two_rhs_per_thread_same_solve():
    """The batched F16 CGNE with double-float resets gives the same solution
    bit for bit, and the same steps and resets, whether its double-float
    reset passes run one or two right-hand sides per thread."""
    oq = _oq()
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.135, 1.0)
    n = 5
    eta = np.stack([dirac.even_part(e) for e in synth.make_source(dims, 93, nrhs=n)])
    runs = []
    for nr in (1, 2):
        h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
        for mode in (0, 1, 2):
            h.tune_set(oq.DF64, mode, n, 32, 2, nr=nr, regcap=0)
        psi = to_dev(np.zeros_like(eta))
        rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, sdtype=oq.F16), nrhs=n)
        assert rc == oq.OK and all(s["converged"] for s in st)
        assert max(s["resets"] for s in st) >= 2      # intermediate double-float resets ran
        runs.append((from_dev(psi, eta.shape), [(s["steps"], s["resets"]) for s in st]))
    assert runs[0][1] == runs[1][1]
    assert np.array_equal(runs[0][0], runs[1][0])
    x = runs[1][0]
    for k in range(n):
        ax = dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, x[k]))
        r = np.linalg.norm((eta[k] - ax).reshape(-1)) / np.linalg.norm(eta[k].reshape(-1))
        assert r <= 1.05e-10


def test_profile_separates_passes_and_adjoints():
    """oq_profile_start/stop: one entry per (pass, epilogue, type, rhs per
    thread, link format, adjoint), with its launch count and bytes."""
    oq = _oq()
    dims = (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.3, 1, 0.13, 1.0)
    h = make_handle(dims, u, 0.13, 1.0, oq.LINK_12)
    ev = dirac.even_part(synth.make_source(dims, 5))
    pin, pout = h.new_packed(oq.F32, oq.EVEN), h.new_packed(oq.F32, oq.EVEN)
    h.pack(to_dev(ev), pin, oq.F32, oq.EVEN)
    h.profile_start()
    for _ in range(3):
        h.dw_hat(pin, pout, oq.F32)
    h.dw_hat(pin, pout, oq.F32, dagger=True)
    prof = h.profile_stop()
    got = {(p["mode"], p["dag"]): p for p in prof}
    assert got[(1, 0)]["launches"] == 3 and got[(2, 0)]["launches"] == 3
    assert got[(1, 1)]["launches"] == 1 and got[(2, 1)]["launches"] == 1
    assert all(p["bytes"] > 0 and p["total_ms"] > 0 for p in prof)
