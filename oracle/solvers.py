"""FP64 reference solvers (test infrastructure).

* ``cgne``   - conjugate gradient on the normal equations with reset steps
               (Sec. 2 and the caption of Fig. 4): regular steps run in a
               "small" storage type (emulated by rounding every stored
               vector, Table 1), all reductions are binary64 (Sec. 2, 2.1),
               and a reset step recomputes the exact residual b - A x in
               binary64 once the recursively updated residual has dropped by
               about the machine epsilon of the storage type.
* ``sap``    - Schwarz alternating procedure (Sec. 3, Figs. 2-3): the lattice
               is cut into blocks coloured like a chessboard; one Schwarz
               cycle solves all blocks of one colour, then all of the other,
               each block problem D_i delta = r_i by a few minimal-residual
               (MR) steps with the current global residual as right-hand side.
               ``adaptive=True`` is the variant of Sec. 3.2 (cycle and MR
               counts chosen on the fly, with the three MR exit rules).
* ``fgcr``   - flexible GCR with restarts (Sec. 3.1, Table 2 settings res,
               nmx, nkv), the preconditioner applied to every new residual.
* ``dense_solve`` - brute-force LU solve of an assembled operator.

Where the paper does not spell out a detail, the reading used here is noted
at the spot (reset threshold, scaling of the small-type vectors, Gram-Schmidt
variant, block colouring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .precision import round_complex, machine_eps
from . import dirac

__all__ = [
    "vdot",
    "norm",
    "CgneResult",
    "cgne",
    "precision_ladder",
    "default_reset_delta",
    "block_index",
    "sap",
    "eo_block_solve",
    "fgcr",
    "GcrResult",
    "dense_solve",
    "mr_block",
]


def vdot(a, b) -> complex:
    """<a, b> = sum conj(a) b, accumulated in binary64."""
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def norm(a) -> float:
    return float(np.sqrt(np.vdot(a.reshape(-1), a.reshape(-1)).real))


def default_reset_delta(store: str) -> float:
    """Reset when the recursive residual has dropped by ~10 x eps of the type.

    The paper states only "roughly the machine epsilon of the data type"
    (Fig. 4 caption).  Ten times epsilon, capped at 0.1, is the reading used
    throughout (binary32: 1.2e-6, bfloat16: 0.078, binary16: 0.0098).
    """
    if store == "fp64":
        return 0.0
    return min(0.1, 10.0 * machine_eps(store))


@dataclass
class CgneResult:
    x: np.ndarray
    status: int               # regular CG steps (the value of ``status``)
    resets: int               # reset steps (the bracketed number in Fig. 4)
    converged: bool
    rel_res: float            # exact ||eta - A x|| / ||eta|| (binary64)
    history: list = field(default_factory=list)   # (step, exact, recursive)
    phases: list = field(default_factory=list)    # storage type of every inner solve
    reset_at: list = field(default_factory=list)  # value of status at every reset step


def precision_ladder(types=("fp16", "fp32", "fp64"), c=1.0):
    """The precision ladder of Sec. 2 (after Fig. 4): start the small-type CG
    in the first type and move to the next one once the relative residual has
    fallen below c times the machine epsilon of the current type (the paper
    asks for a threshold that scales with epsilon; c = 1 is the reading used
    by default).  Returns (type, switch_below) pairs; the last type never
    switches.
    """
    return [(t, c * machine_eps(t) if k + 1 < len(types) else 0.0) for k, t in enumerate(types)]


def cgne(apply_a, eta, res, nmx, store="fp64", delta=None, history=False,
         ncomp=None, ladder=None, scaled=True) -> CgneResult:
    """Solve A x = eta, A = Dhat^dag Dhat, by CG with binary64 reset steps.

    ``apply_a`` applies A in binary64.  The small type ``store`` is emulated
    by rounding every stored vector of a regular step (x_s, r_s, p and the
    operator output q); arithmetic and reductions stay binary64.

    Between resets the small-type CG solves A x_s = r / s for the current
    exact residual r, scaled by s = ||r|| / sqrt(n) so that the stored
    components are O(1) (the per-vector scale that keeps binary16 inside its
    range); n = ``ncomp`` complex components (default: all of ``eta``).
    ``scaled=False`` takes s = 1 instead: the residual is cast to the small
    type as it is, which is what the paper's simulation did (Fig. 4: binary16
    then stalls once the residual components leave its range).  A reset adds
    s * x_s to the binary64 solution and recomputes the residual exactly.  A reset is triggered when the recursive residual
    has fallen below delta times its value at the last reset, or below the
    target, or when ``nmx`` regular steps have been used.

    ``ladder`` (optional, see ``precision_ladder``): the storage type of each
    inner solve is chosen at its start from the relative binary64 residual:
    the ladder moves to its next type while the residual is below the
    current type's switch value; delta is then that type's default.
    """
    stages = list(ladder) if ladder is not None else [(store, 0.0)]
    stage = 0
    store = stages[0][0]
    fixed_delta = delta
    if delta is None:
        delta = default_reset_delta(store)

    def rnd(v):
        return round_complex(v, store)

    n = eta.size if ncomp is None else int(ncomp)
    eta_norm = norm(eta)
    tol = res * eta_norm
    x = np.zeros_like(eta)
    r = eta.copy()
    rn = eta_norm
    status = 0
    resets = 0
    hist = []
    phases = []
    reset_at = []
    if rn <= tol or rn == 0.0:
        return CgneResult(x, 0, 0, True, rn / eta_norm if eta_norm else 0.0, hist, phases, reset_at)
    while True:
        while stage + 1 < len(stages) and rn <= stages[stage][1] * eta_norm:
            stage += 1
        if stages[stage][0] != store:
            store = stages[stage][0]
            delta = fixed_delta if fixed_delta is not None else default_reset_delta(store)
        phases.append(store)
        s = rn / np.sqrt(n) if scaled else 1.0
        rs = rnd(r / s)
        p = rs.copy()
        xs = np.zeros_like(eta)
        rr = norm(rs) ** 2
        rn_start = np.sqrt(rr)
        while True:
            q = rnd(apply_a(p))
            pq = vdot(p, q).real
            alpha = rr / pq
            xs = rnd(xs + alpha * p)
            rs = rnd(rs - alpha * q)
            rr_new = norm(rs) ** 2
            status += 1
            if history:
                exact = norm(eta - apply_a(x + s * xs)) / eta_norm
                hist.append((status, exact, np.sqrt(rr_new) * s / eta_norm))
            if (np.sqrt(rr_new) <= delta * rn_start or np.sqrt(rr_new) * s <= tol
                    or status >= nmx):
                break
            beta = rr_new / rr
            p = rnd(rs + beta * p)
            rr = rr_new
        # reset step, binary64
        x = x + s * xs
        r = eta - apply_a(x)
        rn = norm(r)
        resets += 1
        reset_at.append(status)
        if rn <= tol:
            return CgneResult(x, status, resets, True, rn / eta_norm, hist, phases, reset_at)
        if status >= nmx:
            return CgneResult(x, status, resets, False, rn / eta_norm, hist, phases, reset_at)


# ---------------------------------------------------------------------------
# Schwarz alternating procedure
# ---------------------------------------------------------------------------

def block_index(dims, bs):
    """Block number and colour of every site.

    Blocks are bs[0] x ... x bs[3] boxes; their grid is numbered
    lexicographically (time slowest).  The colour of a block is the parity of
    the sum of its grid coordinates, so neighbouring blocks always differ in
    colour (Fig. 2); this needs an even number of blocks in every direction.
    Returns (bid, colour_of_site, n_blocks).
    """
    dims = tuple(dims)
    nb = tuple(d // b for d, b in zip(dims, bs))
    for d, b, m in zip(dims, bs, nb):
        if d % b or m % 2:
            raise ValueError("each lattice extent must hold an even number of blocks")
    idx = np.indices(dims)
    bc = [idx[mu] // bs[mu] for mu in range(4)]
    bid = ((bc[0] * nb[1] + bc[1]) * nb[2] + bc[2]) * nb[3] + bc[3]
    colour = (bc[0] + bc[1] + bc[2] + bc[3]) % 2
    return bid, colour, int(np.prod(nb))


def _block_sum(z, bid, nblk):
    """Per-block sum of a complex site field (summed over spin and colour)."""
    zs = z.reshape(z.shape[:4] + (-1,)).sum(axis=-1)
    re = np.bincount(bid.reshape(-1), weights=zs.real.reshape(-1), minlength=nblk)
    im = np.bincount(bid.reshape(-1), weights=zs.imag.reshape(-1), minlength=nblk)
    return re + 1j * im


def mr_block(apply_dc, b, bid, sel_site, nblk, nmr, adaptive=False, alpha=0.9,
             tol=0.0, store="fp64"):
    """Minimal-residual steps on every block of one colour at once.

    ``apply_dc`` applies the colour-restricted operator P_c D P_c, which is
    the direct sum of the block operators D_i (Dirichlet boundaries) because
    blocks of one colour never touch.  Per block: x = 0, r = b; each step
    p = D_i r, omega = <p, r>/<p, p>, x += omega r, r -= omega p.

    With ``adaptive`` a block stops when (a) after at least 4 steps its
    residual norm exceeds alpha times the previous one, (b) its residual
    norm grew, or (c) it fell below ``tol`` (Sec. 3.2); ``nmr`` is then the
    maximal step count.  The last step is kept in every case.
    Returns (x, r, steps_per_block).
    """
    def rnd(v):
        return round_complex(v, store)

    x = np.zeros_like(b)
    r = rnd(b)
    active = np.zeros(nblk, dtype=bool)
    blocks_here = np.unique(bid[sel_site])
    active[blocks_here] = True
    steps = np.zeros(nblk, dtype=np.int64)
    rn_prev = np.sqrt(_block_sum(np.abs(r) ** 2, bid, nblk).real)
    for k in range(1, nmr + 1):
        if not active.any():
            break
        p = rnd(apply_dc(r))
        pr = _block_sum(np.conj(p) * r, bid, nblk)
        pp = _block_sum(np.abs(p) ** 2, bid, nblk).real
        omega = np.where(active & (pp > 0), pr / np.where(pp > 0, pp, 1.0), 0.0)
        om_site = omega[bid][..., None, None]
        x = rnd(x + om_site * r)
        r = rnd(r - om_site * p)
        steps += active
        rn_new = np.sqrt(_block_sum(np.abs(r) ** 2, bid, nblk).real)
        if adaptive:
            stop = ((k >= 4) & (rn_new > alpha * rn_prev)) | (rn_new > rn_prev) | (rn_new < tol)
            active &= ~stop
        rn_prev = rn_new
    return x, r, steps


def eo_block_solve(u, a, ainv, r, mask, mask_e, mask_o, bid, sel, nblk, nmr, adaptive, alpha, mr_tol, store,
                   bc_t=-1.0):
    """Approximate solution of D_i delta = r_i on every block of one colour
    through the block's even-odd Schur complement (the even-odd reduced block
    solver of openQCD's SAP, Sec. 3):

        rhat_e  = r_e - D_eo A_oo^{-1} r_o
        Dhat_i  = A_ee - D_eo A_oo^{-1} D_oe        (MR on the even block sites)
        delta_o = A_oo^{-1} (r_o - D_oe delta_e)

    with D_eo, D_oe the hops inside the blocks (Dirichlet boundaries).
    Returns (delta, steps_per_block)."""
    def hop_c(v):
        # in-block hopping part of D: the colour's blocks never touch
        return np.where(mask, -0.5 * dirac.hopping(u, np.where(mask, v, 0.0), bc_t), 0.0)

    def on(m, v):
        return np.where(m, v, 0.0)

    r_e, r_o = on(mask_e, r), on(mask_o, r)
    rhat = r_e - on(mask_e, hop_c(dirac.apply_site_matrix(ainv, r_o)))

    def apply_dhat(v):
        v = on(mask_e, v)
        t = on(mask_o, dirac.apply_site_matrix(ainv, on(mask_o, hop_c(v))))
        return on(mask_e, dirac.apply_site_matrix(a, v) - hop_c(t))

    d_e, _, st = mr_block(apply_dhat, rhat, bid, sel, nblk, nmr, adaptive, alpha, mr_tol, store)
    d_e = on(mask_e, d_e)
    d_o = on(mask_o, dirac.apply_site_matrix(ainv, r_o - on(mask_o, hop_c(d_e))))
    return d_e + d_o, st


def sap(u, a, rho, bs, ncy, nmr, bc_t=-1.0, adaptive=False, alpha=0.9, mr_tol=0.0,
        store="fp64", info=None, eo=False, ainv=None):
    """Approximate D^{-1} rho by SAP (Sec. 3), starting from phi = 0.

    One cycle: for colour 0 ("black") then colour 1 ("white"): take the
    current global residual r = rho - D phi, solve every block of that
    colour by MR, add the block corrections to phi.  ``adaptive`` ends the
    cycles once a cycle did not lower ||rho - D phi|| (at least one cycle;
    ``ncy`` is then the maximum) and switches on the MR exit rules with
    ``mr_tol`` = res ||eta|| / n_blocks.  ``eo`` runs the MR steps on the
    blocks' even-odd Schur complements instead (``eo_block_solve``; ``ainv``
    the per-site inverse of ``a``).
    """
    dims = rho.shape[:4]
    bid, colour, nblk = block_index(dims, bs)
    odd = dirac.parity_mask(dims)
    if eo and ainv is None:
        ainv = np.linalg.inv(a)
    phi = np.zeros_like(rho)
    prev = norm(rho)
    cycles = 0
    mr_steps = []
    for _ in range(ncy):
        for c in (0, 1):
            sel = colour == c
            mask = sel[..., None, None]

            def apply_dc(v, mask=mask):
                return np.where(mask, dirac.dw(u, a, np.where(mask, v, 0.0), bc_t), 0.0)

            r = np.where(mask, rho - dirac.dw(u, a, phi, bc_t), 0.0)
            if eo:
                mask_e = (sel & ~odd)[..., None, None]
                mask_o = (sel & odd)[..., None, None]
                dx, st = eo_block_solve(u, a, ainv, r, mask, mask_e, mask_o, bid, sel, nblk, nmr, adaptive,
                                        alpha, mr_tol, store, bc_t)
            else:
                dx, _, st = mr_block(apply_dc, r, bid, sel, nblk, nmr, adaptive, alpha, mr_tol, store)
            phi = round_complex(phi + dx, store)
            mr_steps.append(st[np.unique(bid[sel])])
        cycles += 1
        if adaptive:
            now = norm(rho - dirac.dw(u, a, phi, bc_t))
            if not now < prev:
                break
            prev = now
    if info is not None:
        info["cycles"] = cycles
        info["mr_steps"] = mr_steps
    return phi


# ---------------------------------------------------------------------------
# Flexible GCR
# ---------------------------------------------------------------------------

@dataclass
class GcrResult:
    x: np.ndarray
    status: int            # GCR steps
    restarts: int
    converged: bool
    rel_res: float         # exact ||eta - D x|| / ||eta|| (binary64)
    res_history: list = field(default_factory=list)


def fgcr(apply_d, precond, eta, res, nmx, nkv, x0=None, store="fp64") -> GcrResult:
    """Flexible GCR for D x = eta (Sec. 3.1, Table 2).

    Per step k < nkv: phi_k = M rho_k, chi_k = D phi_k, chi_k is made
    orthogonal to chi_0..chi_{k-1} (modified Gram-Schmidt, coefficients
    a_lk), b_k = ||chi_k||, chi_k /= b_k, c_k = <chi_k, rho_k>,
    rho_{k+1} = rho_k - c_k chi_k.  At a restart (k = nkv, convergence of
    the recursive residual, or nmx steps) the coefficients beta solve the
    triangular system b_l beta_l + sum_{m>l} a_lm beta_m = c_l, the binary64
    solution is updated by sum beta_l phi_l and the residual is recomputed
    exactly (the "large" type).  The Krylov vectors live in ``store``.
    """
    def rnd(v):
        return round_complex(v, store)

    eta_norm = norm(eta)
    tol = res * eta_norm
    x = np.zeros_like(eta) if x0 is None else x0.astype(np.complex128).copy()
    rho_d = eta - apply_d(x)
    status = 0
    restarts = 0
    hist = [norm(rho_d) / eta_norm]
    while True:
        if norm(rho_d) <= tol:
            return GcrResult(x, status, restarts, True, norm(rho_d) / eta_norm, hist)
        if status >= nmx:
            return GcrResult(x, status, restarts, False, norm(rho_d) / eta_norm, hist)
        rho = rnd(rho_d)
        phis, chis = [], []
        a = np.zeros((nkv, nkv), dtype=np.complex128)
        b = np.zeros(nkv)
        c = np.zeros(nkv, dtype=np.complex128)
        k_used = 0
        for k in range(nkv):
            phi = rnd(precond(rho))
            chi = apply_d(phi)
            for l in range(k):
                a[l, k] = vdot(chis[l], chi)
                chi = chi - a[l, k] * chis[l]
            b[k] = norm(chi)
            chi = rnd(chi / b[k])
            c[k] = vdot(chi, rho)
            rho = rnd(rho - c[k] * chi)
            phis.append(phi)
            chis.append(chi)
            status += 1
            k_used = k + 1
            hist.append(norm(rho) / eta_norm)
            if norm(rho) <= tol or status >= nmx:
                break
        beta = np.zeros(k_used, dtype=np.complex128)
        for l in range(k_used - 1, -1, -1):
            s = c[l] - sum(a[l, m] * beta[m] for m in range(l + 1, k_used))
            beta[l] = s / b[l]
        for l in range(k_used):
            x = x + beta[l] * phis[l]
        rho_d = eta - apply_d(x)
        restarts += 1


def dense_solve(m: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Brute force: LU solve of an assembled operator."""
    return np.linalg.solve(m, b.reshape(-1)).reshape(b.shape)
