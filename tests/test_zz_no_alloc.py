"""oq_dw_hat_apply_noalloc: the even-odd operator for callers that cannot
allocate device memory (its odd-site intermediate lives in a fixed static
device array instead of handle-owned scratch).

Called through the C ABI and compared with oq_dw_hat_apply on the same
inputs, on two calls in a row with different inputs (the shared array keeps
the previous call's contents, which must not leak into the next result).
This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import TOL, oracle_case, make_handle, to_dev, from_dev, rel_err

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 16 * 1024 * 1024


def _call_noalloc(oq, h, prec, pin, pout, nrhs, dagger):
    import torch
    return oq.lib().oq_dw_hat_apply_noalloc(h.h, 0, prec, ctypes.c_void_p(pin.data_ptr()),
                                            ctypes.c_void_p(pout.data_ptr()), nrhs, int(dagger),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_allocating_entry_point(prec):
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.1365, 1.3)
    h = make_handle(dims, u, 0.1365, 1.3, oq.LINK_12)
    nrhs = 2
    for call, dagger in enumerate((False, True)):
        psi = np.stack([dirac.even_part(p) for p in synth.make_source(dims, 500 + call, nrhs=nrhs)])
        pin = h.new_packed(prec, oq.EVEN, nrhs=nrhs)
        h.pack(to_dev(psi), pin, prec, oq.EVEN, nrhs=nrhs)
        ref = h.new_packed(prec, oq.EVEN, nrhs=nrhs)
        out = h.new_packed(prec, oq.EVEN, nrhs=nrhs)
        out.fill_(0xFF)   # NaN pattern: every byte must be written
        h.dw_hat(pin, ref, prec, nrhs=nrhs, dagger=dagger)
        rc = _call_noalloc(oq, h, prec, pin, out, nrhs, dagger)
        assert rc == oq.OK
        torch.cuda.synchronize()
        cr = to_dev(np.zeros_like(psi))
        co = to_dev(np.zeros_like(psi))
        h.unpack(ref, cr, prec, oq.EVEN, nrhs=nrhs)
        h.unpack(out, co, prec, oq.EVEN, nrhs=nrhs)
        got, want = from_dev(co, psi.shape), from_dev(cr, psi.shape)
        assert np.all(np.isfinite(got))
        assert rel_err(got, want) <= TOL[prec]
        # and against the oracle
        for k in range(nrhs):
            oref = dirac.dw_hat_dagger(u, a, ainv, psi[k]) if dagger else dirac.dw_hat(u, a, ainv, psi[k])
            assert rel_err(got[k], oref) < TOL[prec]
    h.close()


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.1365, 1.3)
    h = make_handle(dims, u, 0.1365, 1.3, oq.LINK_12)
    half = h.spinor_bytes(oq.F64, oq.EVEN)
    nrhs = NOALLOC_BYTES // half + 1
    pin = torch.zeros(half * nrhs, dtype=torch.uint8, device="cuda")
    pout = torch.zeros_like(pin)
    assert _call_noalloc(oq, h, oq.F64, pin, pout, nrhs, False) == oq.ERR_ARG
    assert int(pout.abs().sum()) == 0   # nothing was enqueued
    h.close()


def test_noalloc_rejects_double_float_and_writes_nothing():
    """OQ_DF64 needs handle-allocated double-float splits of links and clover,
    so the entry point that must not allocate refuses it before enqueuing."""
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.1365, 1.3)
    h = make_handle(dims, u, 0.1365, 1.3, oq.LINK_12)
    half = h.spinor_bytes(oq.DF64, oq.EVEN)
    pin = torch.ones(half, dtype=torch.uint8, device="cuda")
    pout = torch.zeros_like(pin)
    assert _call_noalloc(oq, h, oq.DF64, pin, pout, 1, False) == oq.ERR_ARG
    torch.cuda.synchronize()
    assert int(pout.abs().sum()) == 0
    h.close()


def test_noalloc_launches_are_profiled_like_the_allocating_ones():
    """Both stencil passes show in the profile and in the launch count."""
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (8, 6, 4, 10)
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.1365, 1.3)
    h = make_handle(dims, u, 0.1365, 1.3, oq.LINK_12)
    psi = dirac.even_part(synth.make_source(dims, 600))
    pin, pout = h.new_packed(oq.F32, oq.EVEN), h.new_packed(oq.F32, oq.EVEN)
    h.pack(to_dev(psi), pin, oq.F32, oq.EVEN)
    n0 = h.kernel_launches()
    h.profile_start()
    assert _call_noalloc(oq, h, oq.F32, pin, pout, 1, False) == oq.OK
    prof = h.profile_stop()
    assert h.kernel_launches() - n0 == 2
    assert sorted(p["mode"] for p in prof) == [1, 2]
    assert all(p["launches"] == 1 and p["bytes"] > 0 for p in prof)
    h.close()
