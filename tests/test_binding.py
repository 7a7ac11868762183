"""Host logic of the ctypes binding (CPU only, no library call): solver
parameters marshal into the C struct as the header documents them, and
status structs unmarshal into dictionaries with every field."""
import pytest

from paper_2202_07388_gb300 import oq


def test_solver_params_marshal_ladder_and_defaults():
    p = oq.SolverParams().c()
    assert p.nladder == 0 and p.sap_eo == 0 and p.ladder_c == 0.0   # zero-initialised: no ladder
    assert p.sdtype == oq.F32 and p.res == 1e-10 and tuple(p.bs) == (4, 4, 4, 4)
    q = oq.SolverParams(ladder=(oq.F16, oq.F32, oq.F64), ladder_c=3.0, sap_eo=1, bs=(2, 2, 2, 4)).c()
    assert q.nladder == 3 and list(q.ladder)[:3] == [oq.F16, oq.F32, oq.F64]
    assert q.ladder_c == 3.0 and q.sap_eo == 1 and tuple(q.bs) == (2, 2, 2, 4)
    with pytest.raises(ValueError):
        oq.SolverParams(ladder=(1, 1, 1, 1, 1)).c()


def test_status_dict_has_every_field():
    s = oq.OqStatus()
    s.steps, s.resets, s.converged, s.true_rel_res = 41, 3, 1, 9.5e-11
    s.ladder_steps[0], s.ladder_steps[1] = 16, 25
    s.nn_fallback = 1
    d = oq.status_dict(s)
    assert d["steps"] == 41 and d["resets"] == 3 and d["converged"] is True
    assert d["ladder_steps"] == [16, 25, 0, 0] and d["nn_fallback"] == 1
    assert set(d) >= {"restarts", "true_rel_res", "cycles", "mr_avg"}


def test_clover_params_struct():
    c = oq.OqCloverParams(0.135, 1.0, 1.1, 0.8, 1)
    assert (c.kappa, c.csw, c.cF, c.csw_qed, c.qed_split) == (0.135, 1.0, 1.1, 0.8, 1)
