"""The stencil profile counts the bytes of right-hand sides that a launch
actually acts on.

The CGNE (Sec. 2) launches its regular steps in chunks and gates off, on the
device, every right-hand side whose state left the step's mode; a launch in
which none is live moves no operand.  Checked: every profile entry's bytes are
its live launches x (links + clover) + its live right-hand-side launches x
(spinor and epilogue vectors), by the algorithmic byte count written out here;
the CG-update kernel acted on exactly the regular steps the solver reports;
gated launches exist in a chunked solve and add no bytes."""
import numpy as np
import pytest

from oracle import dirac
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import oracle_case, make_handle, to_dev

pytestmark = pytest.mark.gpu


def _parts(p, vh):
    """(bytes once per launch, bytes per live right-hand side) of one stencil launch."""
    sp = {0: 8, 1: 4, 2: 2, 3: 2, 4: 8}[p["prec"]]
    wide = p["prec"] in (0, 4)
    su = 8 if wide else 4
    ru = 12 if (not wide and p["link_fmt"] == 1) else 18
    sites = vh * (2 if p["mode"] == 0 else 1)
    if p["mode"] == 0:
        spin, links = 48 * sp, 4 * ru * su
    else:
        spin, links = (48 if p["mode"] == 1 else 72) * sp, 8 * ru * su
    if p["epi"] == 2:   # CG update: read p, r, x; write r, x (x binary32, binary64 for binary64 storage)
        spin += 72 * sp + 48 * (8 if p["prec"] == 0 else 4)
    if p["epi"] == 3:   # reset residual: read eta
        spin += 24 * sp
    return sites * (links + 72 * su), sites * spin


@pytest.mark.parametrize("prec", [1, 3])
def test_profile_charges_only_live_right_hand_sides(prec):
    from paper_2202_07388_gb300 import oq
    dims = (8, 6, 4, 10)
    vh = int(np.prod(dims)) // 2
    u, a, ainv = oracle_case(dims, 0.5, 3, 0.135, 1.0)
    h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
    n = 3
    eta = np.stack([dirac.even_part(e) for e in synth.make_source(dims, 91, nrhs=n)])
    eta[1] *= 1e3      # different scales and sources: the right-hand sides stop at different steps
    psi = to_dev(np.zeros_like(eta))
    h.profile_start()
    rc, st = h.cgne(to_dev(eta), psi, oq.SolverParams(res=1e-10, nmx=5000, sdtype=prec), nrhs=n)
    prof = h.profile_stop()
    assert rc == oq.OK
    steps = sum(s["steps"] for s in st)
    gated = 0
    for p in prof:
        fixed, per = _parts(p, vh)
        assert p["bytes"] == pytest.approx(p["launches"] * fixed + p["rhs_launches"] * per, rel=1e-12), p
        assert p["launches"] <= p["rhs_launches"] <= n * p["launches"]
        gated += p["gated_launches"]
        if p["prec"] == prec and p["epi"] == 2:
            assert p["rhs_launches"] == steps           # one live rhs-launch per regular step
            assert max(s["steps"] for s in st) <= p["launches"] <= steps
    assert any(p["prec"] == prec and p["epi"] == 2 for p in prof)
    assert gated > 0      # the chunked loop did launch steps with nothing live
    h.close()
