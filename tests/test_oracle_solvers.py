"""Pins of the oracle's solvers: brute-force dense solves on 2^4 and 4^4
lattices, the Krylov least-squares property of GCR, exact-block SAP against
the dense multiplicative Schwarz formula (Sec. 3, Fig. 3), the storage-type
behaviour of CGNE with reset steps (Sec. 2), and Table 1 format limits."""
import os

import numpy as np
import pytest

from oracle import dirac, solvers, precision
from tests.oracle_cases import gauge_case, rand_spinor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _even_ops(u, a, ainv):
    dh = lambda v: dirac.dw_hat(u, a, ainv, v)
    dhd = lambda v: dirac.dw_hat_dagger(u, a, ainv, v)
    return dh, dhd


def test_table1_limits_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_limits.txt")) if l.strip() and l[0] != "#"]
    for name, fmax, fmin, fsmin, eps in rows:
        lim = precision.format_limits(name)
        for key, printed in (("f_max", fmax), ("f_min", fmin), ("f_smin", fsmin), ("eps", eps)):
            got = float(f"{lim[key]:.1e}")
            assert got == float(printed), (name, key, lim[key], printed)


def test_rounding_matches_hardware_formats():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))
    assert np.array_equal(precision.round_real(x, "fp32"), x.astype(np.float32).astype(np.float64))
    assert np.array_equal(precision.round_real(x, "fp16"), x.astype(np.float16).astype(np.float64))
    # bf16 = fp32 with the low 16 mantissa bits rounded away; check the
    # values that are exact in fp32 against a bit-level RNE
    xf = x.astype(np.float32)
    bits = xf.view(np.uint32).astype(np.uint64)
    rnd = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    expect = rnd.astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.array_equal(precision.round_real(xf.astype(np.float64), "bf16"), expect)
    assert precision.round_real(np.array([70000.0]), "fp16")[0] == np.inf
    assert precision.round_real(np.array([6e-8]), "fp16")[0] == 2.0 ** -24


def test_cgne_fp64_matches_dense_solve():
    dims = (2, 2, 2, 2)
    u, a, ainv = gauge_case(dims, 0.5, 31, 0.13, 1.0)
    dh, dhd = _even_ops(u, a, ainv)
    mh = dirac.assemble_dense(dh, dims)
    eta = dirac.even_part(rand_spinor(dims, 32))
    res = solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-12, 500, "fp64")
    ev = ~np.repeat(dirac.parity_mask(dims).reshape(-1), 12)
    n = mh[np.ix_(ev, ev)]
    x = np.linalg.solve(n.conj().T @ n, eta.reshape(-1)[ev])
    assert res.converged and res.resets == 1
    assert np.max(np.abs(res.x.reshape(-1)[ev] - x)) < 1e-10 * np.max(np.abs(x))


@pytest.mark.parametrize("store,max_resets", [("fp32", 4), ("bf16", 40), ("fp16", 30)])
def test_cgne_mixed_precision_reaches_binary64_residual(store, max_resets):
    """Whatever the storage type, reset steps carry the exact residual to
    1e-10 (Sec. 2); lower precision costs more resets (Sec. 2, eq. 1)."""
    u, a, ainv = gauge_case()
    dh, dhd = _even_ops(u, a, ainv)
    eta = dirac.even_part(rand_spinor(u.shape[:4], 33))
    r = solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-10, 2000, store, ncomp=12 * 128)
    assert r.converged and r.rel_res <= 1e-10
    assert 1 <= r.resets <= max_resets


def test_cgne_reset_count_ordering():
    """Sec. 2: bfloat16 needs more reset steps than binary16 (more mantissa),
    which needs more than binary32."""
    u, a, ainv = gauge_case()
    dh, dhd = _even_ops(u, a, ainv)
    eta = dirac.even_part(rand_spinor(u.shape[:4], 34))
    out = {s: solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-12, 3000, s, ncomp=1536) for s in ("fp32", "fp16", "bf16")}
    assert out["bf16"].resets > out["fp16"].resets > out["fp32"].resets
    f64 = solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-12, 3000, "fp64")
    assert f64.status <= out["fp32"].status <= out["bf16"].status


def test_cgne_history_exact_vs_recursive():
    """Fig. 4a/4b: the exact and recursive residuals agree until round-off
    accumulates; in binary64 they stay together to ~1e-10."""
    u, a, ainv = gauge_case()
    dh, dhd = _even_ops(u, a, ainv)
    eta = dirac.even_part(rand_spinor(u.shape[:4], 35))
    r = solvers.cgne(lambda v: dhd(dh(v)), eta, 1e-10, 500, "fp64", history=True)
    ex = np.array([h[1] for h in r.history])
    rc = np.array([h[2] for h in r.history])
    assert np.max(np.abs(ex - rc) / ex) < 1e-3


def test_gcr_krylov_least_squares_property():
    """Unpreconditioned GCR without restart minimises ||rho0 - D z|| over
    z in K_k(D, rho0): compare with a dense least-squares solve."""
    dims = (2, 2, 2, 2)
    u, a, _ = gauge_case(dims, 0.5, 41, 0.13, 1.0)
    d = lambda v: dirac.dw(u, a, v)
    m = dirac.assemble_dense(d, dims)
    eta = rand_spinor(dims, 42)
    b = eta.reshape(-1)
    for k in (1, 3, 6):
        r = solvers.fgcr(d, lambda v: v, eta, 1e-30, k, k + 1)
        kry = np.stack([np.linalg.matrix_power(m, j) @ b for j in range(k)], axis=1)
        z, *_ = np.linalg.lstsq(m @ kry, b, rcond=None)
        best = np.linalg.norm(b - m @ kry @ z) / np.linalg.norm(b)
        assert abs(r.res_history[-1] - best) < 1e-10
        assert abs(r.rel_res - best) < 1e-10


def test_gcr_and_sap_gcr_match_dense_solve():
    dims = (4, 4, 4, 4)
    u, a, _ = gauge_case()
    d = lambda v: dirac.dw(u, a, v)
    eta = rand_spinor(dims, 43)
    m = dirac.assemble_dense(d, dims)
    x = solvers.dense_solve(m, eta)
    plain = solvers.fgcr(d, lambda v: v, eta, 1e-11, 400, 16)
    assert plain.converged and np.max(np.abs(plain.x - x)) < 1e-9
    pre = lambda v: solvers.sap(u, a, v, (2, 2, 2, 2), 2, 4)
    sg = solvers.fgcr(d, pre, eta, 1e-11, 100, 8)
    assert sg.converged and np.max(np.abs(sg.x - x)) < 1e-9
    assert sg.status < plain.status


def test_sap_exact_blocks_equal_multiplicative_schwarz():
    """With (nearly) exact block solves one SAP cycle is
    phi_b = D_bb^-1 rho_b ; phi = phi_b + D_ww^-1 (rho - D phi_b)_w."""
    dims = (4, 4, 4, 4)
    u, a, _ = gauge_case()
    d = lambda v: dirac.dw(u, a, v)
    m = dirac.assemble_dense(d, dims)
    _, colour, _ = solvers.block_index(dims, (2, 2, 2, 2))
    blk = np.repeat(colour.reshape(-1) == 0, 12)
    wht = ~blk
    rho = rand_spinor(dims, 44).reshape(-1)
    phi = np.zeros_like(rho)
    phi[blk] = np.linalg.solve(m[np.ix_(blk, blk)], rho[blk])
    rr = rho - m @ phi
    phi[wht] += np.linalg.solve(m[np.ix_(wht, wht)], rr[wht])
    got = solvers.sap(u, a, rho.reshape(dims + (4, 3)), (2, 2, 2, 2), 1, 200)
    assert np.max(np.abs(got.reshape(-1) - phi)) < 1e-10 * np.max(np.abs(phi))
    # same-colour blocks are decoupled: P_b D P_b is block diagonal
    bid, _, _ = solvers.block_index(dims, (2, 2, 2, 2))
    bsite = np.repeat(bid.reshape(-1), 12)
    mb = m[np.ix_(blk, blk)]
    same = bsite[blk][:, None] == bsite[blk][None, :]
    assert np.max(np.abs(mb[~same])) == 0


def test_adaptive_sap_exit_rules():
    """Sec. 3.2: at least one cycle, never more than the caps, fewer MR steps
    for a smaller alpha, and exit 3 stops every block at once when the
    tolerance is huge."""
    u, a, _ = gauge_case()
    rho = rand_spinor(u.shape[:4], 45)
    info = {}
    solvers.sap(u, a, rho, (2, 2, 2, 2), 20, 20, adaptive=True, alpha=0.9, info=info)
    assert 1 <= info["cycles"] <= 20
    steps_09 = np.concatenate(info["mr_steps"]).mean()
    assert all(s.max() <= 20 and s.min() >= 1 for s in info["mr_steps"])
    info7 = {}
    solvers.sap(u, a, rho, (2, 2, 2, 2), 20, 20, adaptive=True, alpha=0.3, info=info7)
    assert np.concatenate(info7["mr_steps"]).mean() <= steps_09
    info_t = {}
    solvers.sap(u, a, rho, (2, 2, 2, 2), 20, 20, adaptive=True, mr_tol=1e30, info=info_t)
    assert all(s.max() == 1 for s in info_t["mr_steps"])


def test_sap_gcr_adaptive_converges():
    u, a, _ = gauge_case()
    d = lambda v: dirac.dw(u, a, v)
    eta = rand_spinor(u.shape[:4], 46)
    nb = 128
    pre = lambda v: solvers.sap(u, a, v, (2, 2, 2, 2), 20, 20, adaptive=True, alpha=0.9,
                                mr_tol=1e-10 * solvers.norm(eta) / nb)
    r = solvers.fgcr(d, pre, eta, 1e-10, 60, 8)
    assert r.converged and r.rel_res <= 1e-10


def test_gcr_fp32_krylov_vectors_restart_to_binary64():
    u, a, _ = gauge_case()
    d = lambda v: dirac.dw(u, a, v)
    eta = rand_spinor(u.shape[:4], 47)
    pre = lambda v: solvers.sap(u, a, v, (2, 2, 2, 2), 1, 4, store="fp32")
    r = solvers.fgcr(d, pre, eta, 1e-10, 200, 6, store="fp32")
    assert r.converged and r.rel_res <= 1e-10 and r.restarts >= 2
