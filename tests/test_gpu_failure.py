"""Failure detection without a GPU fault: a bounded device wait that is made
to run out returns OQ_ERR_TIMEOUT and leaves the device usable; NaN in a
host-side source is caught by the binary64 norms; argument errors are
rejected before any work."""
import time

import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import TOL, oracle_case, make_handle, to_dev, from_dev, rel_err

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_times_out_and_device_stays_usable():
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 2, 6)
    u, a, ainv = oracle_case(dims, 0.6, 81, 0.135, 1.0)
    h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
    w = torch.zeros(2 * 576, dtype=torch.float32, device="cuda")
    psi = synth.make_source(dims, 3)
    pin, pout = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(to_dev(psi), pin, oq.F32)
    h.set_option(oq.OPT_TEST_TC_SKIP_MMA, 1)
    t0 = time.time()
    with pytest.raises(oq.OqError) as err:
        h.nnprec_apply_tc(w, pin, pout)
    assert err.value.code == oq.ERR_TIMEOUT
    assert time.time() - t0 < 30
    h.set_option(oq.OPT_TEST_TC_SKIP_MMA, 0)
    # the context is intact: a normal operator application still matches the oracle
    h.dw(pin, pout, oq.F32)
    out = to_dev(np.zeros_like(psi))
    h.unpack(pout, out, oq.F32)
    assert rel_err(from_dev(out, psi.shape), dirac.dw(u, a, psi)) < TOL[1]
    h.close()


def test_nan_in_source_is_reported():
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 4, 4)
    u, a, ainv = oracle_case(dims, 0.3, 1, 0.13, 1.0)
    h = make_handle(dims, u, 0.13, 1.0, oq.LINK_12)
    eta = dirac.even_part(synth.make_source(dims, 4))
    eta[0, 0, 0, 0, 1, 2] = np.nan
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=100, sdtype=oq.F32), check=False)
    assert rc == oq.ERR_NONFINITE and not st[0]["converged"]
    rc, st = h.sap_gcr(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=20, nkv=4, ncy=1, nmr=2,
                                                         bs=(2, 2, 2, 2), sdtype=oq.F32), check=False)
    assert rc in (oq.ERR_NONFINITE, oq.ERR_NOCONV) and not st[0]["converged"]
    h.close()


def test_out_of_order_and_bad_arguments():
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 4, 4)
    h = oq.Handle(dims)
    x = torch.zeros(h.spinor_bytes(oq.F32), dtype=torch.uint8, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(oq.OqError) as e:
        h.dw(x, y, oq.F32)        # no gauge field / clover yet
    assert e.value.code == oq.ERR_STATE
    u, a, ainv = oracle_case(dims, 0.3, 1, 0.13, 1.0)
    h.gauge_upload(to_dev(u), oq.LINK_12)
    h.clover_build(0.13, 1.0)
    with pytest.raises(oq.OqError) as e:
        h.dw(x, x, oq.F32)        # in == out
    assert e.value.code == oq.ERR_ARG
    with pytest.raises(oq.OqError) as e:
        h.dw(x, y, 7)             # unknown precision
    assert e.value.code == oq.ERR_ARG
    h.close()
