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


# ---------------------------------------------------------------------------
# Fig. 4 storage-type sweep and the precision ladder (Sec. 2)
# ---------------------------------------------------------------------------

def _fig4_case():
    u, a, ainv = gauge_case()
    dh, dhd = _even_ops(u, a, ainv)
    eta = dirac.even_part(rand_spinor(u.shape[:4], 34))
    return (lambda v: dhd(dh(v))), eta


def _read_rows(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and line[0] != "#":
            f = line.split()
            rows[f[0]] = f[1:]
    return rows


def test_fig4_reset_counts_match_the_paper():
    """Sec. 2 (after Fig. 4): binary32 -> tensorfloat32 -> bfloat16 each cost
    4 more reset steps; the reset counts (2, 6, 10) are those the paper
    states.  The reset rule (delta ~ 10 eps of the type) decides them."""
    apply_a, eta = _fig4_case()
    paper = _read_rows("fig4_paper_counts.txt")
    got = {t: solvers.cgne(apply_a, eta, 1e-12, 3000, t, ncomp=1536) for t in ("fp32", "tf32", "bf16")}
    for t, r in got.items():
        assert r.converged and r.rel_res <= 1e-12
        assert r.resets == int(paper[t][1]), (t, r.resets)
    # the less precision, the more regular steps (the paper: +1 each; here a few)
    assert got["fp32"].status <= got["tf32"].status <= got["bf16"].status
    assert got["bf16"].status - got["fp32"].status <= 10


def test_fig4_hierarchy_and_first_resets():
    """Sec. 2, the step hierarchy binary64 < binary32 <= tensorfloat32 <=
    {binary16, bfloat16}, and the order of the first reset: bfloat16 first,
    then binary16 and tensorfloat32 together (both 10 mantissa bits), then
    binary32; binary64 never resets before the end."""
    apply_a, eta = _fig4_case()
    r = {t: solvers.cgne(apply_a, eta, 1e-12, 3000, t, ncomp=1536) for t in ("fp64", "fp32", "tf32", "bf16", "fp16")}
    assert r["fp64"].status < r["fp32"].status <= r["tf32"].status <= min(r["bf16"].status, r["fp16"].status)
    first = {t: v.reset_at[0] for t, v in r.items()}
    assert first["bf16"] < first["fp16"] == first["tf32"] < first["fp32"] < first["fp64"]
    assert r["fp64"].resets == 1 and r["fp64"].reset_at == [r["fp64"].status]


def test_fig4_unscaled_binary16_stalls():
    """Sec. 2: cast to binary16 as it is (no per-reset scale), the residual
    components leave binary16's range and CG stalls far above the 1e-12
    target; with the scale the same type converges."""
    apply_a, eta = _fig4_case()
    r = solvers.cgne(apply_a, eta, 1e-12, 300, "fp16", ncomp=1536, scaled=False)
    assert not r.converged and r.status == 300 and 1e-8 < r.rel_res < 1e-4
    assert solvers.cgne(apply_a, eta, 1e-12, 300, "fp16", ncomp=1536).converged


def test_ladder_single_type_equals_plain_cgne():
    """A one-type ladder is the plain CGNE of that type, bit for bit; a
    ladder whose switch values are never reached runs only its first type."""
    apply_a, eta = _fig4_case()
    plain = solvers.cgne(apply_a, eta, 1e-12, 3000, "bf16", ncomp=1536)
    for lad in ([("bf16", 0.0)], [("bf16", 1e-30), ("fp32", 0.0)]):
        r = solvers.cgne(apply_a, eta, 1e-12, 3000, ncomp=1536, ladder=lad)
        assert np.array_equal(r.x, plain.x) and r.status == plain.status and r.resets == plain.resets
        assert set(r.phases) == {"bf16"}


def test_ladder_switch_rule():
    """Precision ladder (Sec. 2, after Fig. 4): binary16 until the binary64
    residual is below eps(binary16), binary32 until below eps(binary32), then
    binary64.  Up to the switch the run is the plain binary16 run (same
    history); each phase starts at the first reset that passes its switch
    value; the ladder needs fewer regular and reset steps than binary16 alone
    and reaches the same target."""
    apply_a, eta = _fig4_case()
    lad = solvers.precision_ladder(("fp16", "fp32", "fp64"))
    assert lad == [("fp16", 2.0 ** -10), ("fp32", 2.0 ** -23), ("fp64", 0.0)]
    r = solvers.cgne(apply_a, eta, 1e-12, 3000, ncomp=1536, ladder=lad, history=True)
    p16 = solvers.cgne(apply_a, eta, 1e-12, 3000, "fp16", ncomp=1536, history=True)
    assert r.converged and r.rel_res <= 1e-12
    assert r.phases == sorted(r.phases, key=["fp16", "fp32", "fp64"].index)
    n16 = r.phases.count("fp16")
    assert 1 <= n16 < len(r.phases)
    cut = r.reset_at[n16 - 1]
    assert r.history[:cut] == p16.history[:cut]
    # the exact residual at every reset decides the next phase
    ex = {h[0]: h[1] for h in r.history}
    for i, t in enumerate(r.phases[1:], start=1):
        rel = ex[r.reset_at[i - 1]]
        prev_sw = dict(lad)[r.phases[i - 1]]
        assert (t != r.phases[i - 1]) == (rel <= prev_sw), (i, t, rel)
    assert r.status < p16.status and r.resets < p16.resets


def test_fig4_sweep_fixture_is_current():
    """The stored sweep (written by make_fig4_sweep.py from the oracle, read by
    the GPU parity tests) matches the oracle as it stands."""
    rows = _read_rows("fig4_sweep_4x4x4x4.txt")
    apply_a, eta = _fig4_case()
    for name, kw in (("bf16", dict(store="bf16")),
                     ("ladder_fp16_fp32_fp64", dict(ladder=solvers.precision_ladder(("fp16", "fp32", "fp64"))))):
        r = solvers.cgne(apply_a, eta, 1e-12, 3000, ncomp=1536, **kw)
        assert (r.status, r.resets, r.reset_at[0]) == tuple(int(v) for v in rows[name][:3])
        assert ",".join(r.phases) == rows[name][5]


# ---------------------------------------------------------------------------
# even-odd reduced block solver of SAP (Sec. 3)
# ---------------------------------------------------------------------------

def test_sap_eo_exact_blocks_equal_multiplicative_schwarz():
    """With exact block solves the even-odd reduced block solver gives the
    same SAP cycle as the plain one: the dense multiplicative Schwarz formula."""
    dims = (4, 4, 4, 4)
    u, a, ainv = gauge_case()
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), dims)
    _, colour, _ = solvers.block_index(dims, (2, 2, 2, 2))
    blk = np.repeat(colour.reshape(-1) == 0, 12)
    wht = ~blk
    rho = rand_spinor(dims, 45).reshape(-1)
    phi = np.zeros_like(rho)
    phi[blk] = np.linalg.solve(m[np.ix_(blk, blk)], rho[blk])
    rr = rho - m @ phi
    phi[wht] += np.linalg.solve(m[np.ix_(wht, wht)], rr[wht])
    got = solvers.sap(u, a, rho.reshape(dims + (4, 3)), (2, 2, 2, 2), 1, 100, eo=True, ainv=ainv)
    assert np.max(np.abs(got.reshape(-1) - phi)) < 1e-10 * np.max(np.abs(phi))


@pytest.mark.parametrize("nmr", [1, 3])
def test_sap_eo_block_solve_against_dense_schur_complement(nmr):
    """One colour of 2^4 blocks on 4^4: the block correction solves the odd
    block equations exactly, and its even part is nmr MR steps on the dense
    Schur complement S = D_ee - D_eo D_oo^-1 D_oe of the colour's block
    matrix, started from rhat = r_e - D_eo D_oo^-1 r_o (all blocks of the
    colour at once, one omega per block)."""
    dims = (4, 4, 4, 4)
    bs = (2, 2, 2, 2)
    u, a, ainv = gauge_case()
    m = dirac.assemble_dense(lambda v: dirac.dw(u, a, v), dims)
    bid, colour, nblk = solvers.block_index(dims, bs)
    odd = dirac.parity_mask(dims)
    sel = colour == 1
    r = np.where(sel[..., None, None], rand_spinor(dims, 46), 0.0)
    d, st = solvers.eo_block_solve(u, a, ainv, r, sel[..., None, None], (sel & ~odd)[..., None, None],
                                   (sel & odd)[..., None, None], bid, sel, nblk, nmr, False, 0.9, 0.0, "fp64")
    assert np.all(st[np.unique(bid[sel])] == nmr)
    c = np.repeat(sel.reshape(-1), 12)
    ev = np.repeat((sel & ~odd).reshape(-1), 12)
    od = np.repeat((sel & odd).reshape(-1), 12)
    mc = m.copy()
    mc[~c, :] = 0.0
    mc[:, ~c] = 0.0
    res = r.reshape(-1) - mc @ d.reshape(-1)
    assert np.max(np.abs(res[od])) < 1e-12 * np.max(np.abs(r))
    assert np.max(np.abs(d.reshape(-1)[~c])) == 0.0
    see = mc[np.ix_(ev, ev)] - mc[np.ix_(ev, od)] @ np.linalg.solve(mc[np.ix_(od, od)], mc[np.ix_(od, ev)])
    rb = r.reshape(-1)
    rhat = rb[ev] - mc[np.ix_(ev, od)] @ np.linalg.solve(mc[np.ix_(od, od)], rb[od])
    site_blk = np.repeat(bid.reshape(-1), 12)[ev]
    x = np.zeros_like(rhat)
    rr = rhat.copy()
    for _ in range(nmr):
        p = see @ rr
        om = np.zeros(nblk, complex)
        for b in np.unique(site_blk):
            k = site_blk == b
            om[b] = np.vdot(p[k], rr[k]) / np.vdot(p[k], p[k]).real
        x = x + om[site_blk] * rr
        rr = rr - om[site_blk] * p
    assert np.max(np.abs(d.reshape(-1)[ev] - x)) < 1e-12 * np.max(np.abs(x))


def test_sap_eo_converges_faster_per_mr_step():
    """The reduced block operator is better conditioned: with the same MR
    step count, one SAP cycle with the even-odd block solver leaves a smaller
    residual than with MR on the full block operator."""
    dims = (4, 4, 4, 4)
    u, a, ainv = gauge_case()
    rho = rand_spinor(dims, 47)
    res = {}
    for eo in (False, True):
        phi = solvers.sap(u, a, rho, (2, 2, 2, 2), 1, 4, eo=eo, ainv=ainv)
        res[eo] = solvers.norm(rho - dirac.dw(u, a, phi)) / solvers.norm(rho)
    assert res[True] < res[False]
