"""GPU CGNE storage-type sweep (Fig. 4 analog, Sec. 2) and the precision
ladder proposed after it, against the FP64 oracle.  The 4^4 case and the
oracle's step / reset counts are those of tests/golden/fig4_sweep_4x4x4x4.txt
(written by make_fig4_sweep.py); the GPU's regular steps use binary32
arithmetic where the oracle rounds binary64 arithmetic to the storage type,
so counts agree up to a few steps and one reset."""
import os

import numpy as np
import pytest

from oracle import dirac, solvers
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import oracle_case, make_handle, to_dev, from_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DIMS = (4, 4, 4, 4)
ORACLE_NAME = {"F64": "fp64", "F32": "fp32", "BF16": "bf16", "F16": "fp16"}


def _oq():
    from paper_2202_07388_gb300 import oq
    return oq


def _rows():
    rows = {}
    for line in open(os.path.join(GOLDEN, "fig4_sweep_4x4x4x4.txt")):
        if line.strip() and line[0] != "#":
            f = line.split()
            rows[f[0]] = dict(status=int(f[1]), resets=int(f[2]), first=int(f[3]), conv=int(f[4]),
                              phases=f[6].split(","))
    return rows


def _case():
    u, a, ainv = oracle_case(DIMS, 0.3, 1, 0.13, 1.0)
    eta = dirac.even_part(synth.make_source(DIMS, 34))
    return u, a, ainv, eta


def _normal_residual(u, a, ainv, eta, x):
    ax = dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, x))
    return np.linalg.norm((eta - ax).reshape(-1)) / np.linalg.norm(eta.reshape(-1))


def _solve(h, eta, **kw):
    oq = _oq()
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-12, nmx=3000, **kw))
    return rc, st[0], from_dev(psi, eta.shape)


@pytest.mark.parametrize("df64", [1, 0])
def test_fig4_sweep_on_gpu(df64):
    """Every GPU storage type to the 1e-12 target of Fig. 4 with the reset
    count of the oracle (+-1) and its regular steps (+-4); the binary64 run
    within 1e-10 of the oracle's solution."""
    oq = _oq()
    u, a, ainv, eta = _case()
    rows = _rows()
    h = make_handle(DIMS, u, 0.13, 1.0, oq.LINK_12)
    h.set_option(oq.OPT_DF64_RESETS, df64)
    ref64 = solvers.cgne(lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v)),
                         eta, 1e-12, 3000, "fp64")
    for name, prec in (("fp64", oq.F64), ("fp32", oq.F32), ("bf16", oq.BF16), ("fp16", oq.F16)):
        rc, st, x = _solve(h, eta, sdtype=prec)
        assert rc == oq.OK and st["converged"], name
        assert _normal_residual(u, a, ainv, eta, x) <= 1.05e-12, name
        assert abs(st["resets"] - rows[name]["resets"]) <= 1, (name, st)
        assert abs(st["steps"] - rows[name]["status"]) <= 4, (name, st)
        assert st["ladder_steps"] == [st["steps"], 0, 0, 0]
        if prec == oq.F64:
            assert np.linalg.norm((x - ref64.x).reshape(-1)) <= 1e-10 * np.linalg.norm(ref64.x.reshape(-1))


@pytest.mark.parametrize("name,types", [("ladder_fp16_fp32_fp64", ("F16", "F32", "F64")),
                                        ("ladder_fp16_fp32", ("F16", "F32")),
                                        ("ladder_bf16_fp32_fp64", ("BF16", "F32", "F64"))])
def test_ladder_matches_oracle(name, types):
    """The ladder on the GPU: the same phases as the oracle's ladder (the
    regular steps spent in each type agree to +-2, so every switch happens at
    the same reset), its reset count, and a binary64 residual of 1e-12."""
    oq = _oq()
    u, a, ainv, eta = _case()
    row = _rows()[name]
    h = make_handle(DIMS, u, 0.13, 1.0, oq.LINK_12)
    lad = tuple(getattr(oq, t) for t in types)
    rc, st, x = _solve(h, eta, ladder=lad)
    assert rc == oq.OK and st["converged"]
    assert _normal_residual(u, a, ainv, eta, x) <= 1.05e-12
    assert st["resets"] == row["resets"]
    ref = solvers.cgne(lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v)), eta, 1e-12, 3000,
                       ncomp=1536, ladder=solvers.precision_ladder(tuple(ORACLE_NAME[t] for t in types)))
    # regular steps per type in the oracle: between its resets
    bounds = [0] + ref.reset_at
    per = {}
    for i, t in enumerate(ref.phases):
        per[t] = per.get(t, 0) + bounds[i + 1] - bounds[i]
    names = [ORACLE_NAME[t] for t in types]
    for i, t in enumerate(names):
        assert abs(st["ladder_steps"][i] - per.get(t, 0)) <= 2, (t, st["ladder_steps"], per)
    assert sum(st["ladder_steps"]) == st["steps"]


def test_ladder_multi_rhs_parks_until_the_phase_changes():
    """Right-hand sides that qualify for the next type at different resets:
    each one runs, within the 3-rhs call, the same inner solves as alone
    (the same steps in each type and resets, up to rounding), and reaches
    1e-12."""
    oq = _oq()
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.135, 1.0)
    n = 3
    # a Gaussian source, a point source (a different convergence history) and
    # the Gaussian source times 1e3 (the same relative history as the first)
    gauss = dirac.even_part(synth.make_source(dims, 88))
    point = dirac.even_part(synth.make_point_sources(dims)[0])
    eta = np.stack([gauss, point, 1e3 * gauss])
    h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
    prm = oq.SolverParams(res=1e-12, nmx=5000, ladder=(oq.F16, oq.F32, oq.F64))
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.cgne(to_dev(eta), psi, prm, nrhs=n)
    assert rc == oq.OK
    x = from_dev(psi, eta.shape)
    for k in range(n):
        assert _normal_residual(u, a, ainv, eta[k], x[k]) <= 1.05e-12, k
        psi1 = to_dev(np.zeros_like(eta[k]))
        rc1, st1 = h.cgne(to_dev(eta[k]), psi1, prm)
        assert rc1 == oq.OK
        # alone the reductions may run over another CTA shape (rounding): +-2 steps
        assert abs(st[k]["resets"] - st1[0]["resets"]) <= 1, (k, st[k], st1[0])
        for i in range(4):
            assert abs(st[k]["ladder_steps"][i] - st1[0]["ladder_steps"][i]) <= 2, (k, st[k], st1[0])


def test_ladder_rejections():
    oq = _oq()
    u, a, ainv, eta = _case()
    h = make_handle(DIMS, u, 0.13, 1.0, oq.LINK_12)
    psi = to_dev(np.zeros_like(eta))
    rc, _ = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-12, nmx=100, ladder=(oq.F16, 9)), check=False)
    assert rc == oq.ERR_ARG
    with pytest.raises(ValueError):
        oq.SolverParams(ladder=(1, 1, 1, 1, 1)).c()
    rc, _ = h.cgne_batch([0], [to_dev(eta)], [psi], oq.SolverParams(res=1e-12, nmx=100, ladder=(oq.F16,)),
                         check=False)
    assert rc == oq.ERR_ARG


def test_ladder_switch_constant():
    """ladder_c scales the switch thresholds (c eps of the current type): with
    c = 100 binary16 is left after its first reset (residual ~1e-2 < 100 eps);
    the GPU follows the oracle ladder with the same constant."""
    oq = _oq()
    u, a, ainv, eta = _case()
    h = make_handle(DIMS, u, 0.13, 1.0, oq.LINK_12)
    rc, st, x = _solve(h, eta, ladder=(oq.F16, oq.F32, oq.F64), ladder_c=100.0)
    assert rc == oq.OK and st["converged"]
    assert _normal_residual(u, a, ainv, eta, x) <= 1.05e-12
    ref = solvers.cgne(lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v)), eta, 1e-12, 3000,
                       ncomp=1536, ladder=solvers.precision_ladder(("fp16", "fp32", "fp64"), c=100.0))
    assert ref.phases[0] == "fp16" and ref.phases[1] != "fp16"
    bounds = [0] + ref.reset_at
    per = {}
    for i, t in enumerate(ref.phases):
        per[t] = per.get(t, 0) + bounds[i + 1] - bounds[i]
    for i, t in enumerate(("fp16", "fp32", "fp64")):
        assert abs(st["ladder_steps"][i] - per.get(t, 0)) <= 2, (t, st["ladder_steps"], per)
