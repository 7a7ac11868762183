"""FP64 Wilson-clover Dirac operator by direct definition (test infrastructure).

The paper (Sec. 1) names the operator only: O(a)-improved Wilson fermions,
whose application to a spinor field is the SpMV-like kernel that dominates
the solvers (Sec. 1, footnote 1).  The definition written out here is the
standard one in openQCD normalisation:

    (D psi)(x) = A(x) psi(x)
                 - 1/2 sum_mu [ U_mu(x) (1 - g_mu) psi(x + mu)
                               + U_mu(x - mu)^dag (1 + g_mu) psi(x - mu) ]

    A(x) = (4 + m0) + c_sw * (i/4) * sum_{mu != nu} sigma_{mu nu} F_{mu nu}(x),
    m0   = 1/(2 kappa) - 4,
    F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{nu mu}(x)) / 8   (clover of 4 plaquettes),
    sigma_{mu nu} = (i/2) [g_mu, g_nu].

Gamma matrices are in the chiral basis
    g_0 = [[0, -1], [-1, 0]],   g_k = [[0, -i s_k], [i s_k, 0]],
so that g_5 = g_0 g_1 g_2 g_3 = diag(1, 1, -1, -1).  Time is antiperiodic for
fermions: a hop across the x0 = T-1 <-> 0 face picks up a factor -1; the
clover term uses the links themselves (no sign).

Even/odd ordering (Sec. 3, Fig. 3): parity(x) = (x0 + x1 + x2 + x3) mod 2,
even sites first.  The even-odd reduced operator is the Schur complement

    Dhat = D_ee - D_eo D_oo^{-1} D_oe       (acting on even sites).

Everything here works on full-lattice canonical arrays (see the module
``paper_2202_07388_gb300.synth`` for the layout); an "even" field is a full
array that vanishes on odd sites.  No step is blocked, fused or reordered.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gamma_matrices",
    "gamma5",
    "sigma_munu",
    "kappa_to_m0",
    "shift_spinor",
    "shift_link",
    "hopping",
    "field_strength",
    "clover_field",
    "apply_site_matrix",
    "dw",
    "dw_dagger",
    "parity_mask",
    "even_part",
    "odd_part",
    "dw_hat",
    "dw_hat_dagger",
    "schur_source",
    "schur_reconstruct_odd",
    "assemble_dense",
    "dw_site",
    "apply_gamma5",
    "sf_project",
    "clover_field_sf",
    "dw_sf",
    "dw_sf_dagger",
    "dw_hat_sf",
    "dw_hat_sf_dagger",
    "clover_field_qed",
]


def gamma_matrices() -> np.ndarray:
    """g_0..g_3 in the chiral basis, shape (4, 4, 4)."""
    z = np.zeros((2, 2), dtype=np.complex128)
    i2 = np.eye(2, dtype=np.complex128)
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    g0 = np.block([[z, -i2], [-i2, z]])
    gk = [np.block([[z, -1j * s], [1j * s, z]]) for s in (s1, s2, s3)]
    return np.stack([g0] + gk)


def gamma5() -> np.ndarray:
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma_munu(mu: int, nu: int) -> np.ndarray:
    g = gamma_matrices()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def kappa_to_m0(kappa: float) -> float:
    """openQCD normalisation: diagonal term 4 + m0 = 1/(2 kappa)."""
    return 1.0 / (2.0 * kappa) - 4.0


def shift_spinor(psi: np.ndarray, mu: int, d: int, bc_t: float = -1.0) -> np.ndarray:
    """Return f(x) = psi(x + d*mu) with the fermion time boundary factor.

    ``psi`` has lattice axes 0..3 (possibly more trailing axes).  For mu = 0
    a hop across the time boundary is multiplied by ``bc_t`` (-1 for
    antiperiodic, +1 for periodic).
    """
    out = np.roll(psi, -d, axis=mu)
    if mu == 0 and bc_t != 1.0:
        t = psi.shape[0]
        if d == +1:
            out[t - 1] = bc_t * out[t - 1]
        else:
            out[0] = bc_t * out[0]
    return out


def shift_link(u_mu: np.ndarray, nu: int, d: int) -> np.ndarray:
    """Return f(x) = u_mu(x + d*nu) (periodic; links carry no boundary sign)."""
    return np.roll(u_mu, -d, axis=nu)


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def _spin_mul(p: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(p psi)[s, a] = sum_t p[s, t] psi[t, a] for a 4x4 spin matrix p."""
    return np.einsum("st,...ta->...sa", p, psi)


def _colour_mul(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(u psi)[s, a] = sum_b u[a, b] psi[s, b] for site-dependent u."""
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def hopping(u: np.ndarray, psi: np.ndarray, bc_t: float = -1.0) -> np.ndarray:
    """H psi = sum_mu [U_mu(x)(1-g_mu)psi(x+mu) + U_mu(x-mu)^dag (1+g_mu) psi(x-mu)]."""
    g = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros_like(psi)
    for mu in range(4):
        u_mu = u[..., mu, :, :]
        fwd = shift_spinor(psi, mu, +1, bc_t)
        bwd = shift_spinor(psi, mu, -1, bc_t)
        u_back = shift_link(u_mu, mu, -1)
        out += _colour_mul(u_mu, _spin_mul(one - g[mu], fwd))
        out += _colour_mul(_dag(u_back), _spin_mul(one + g[mu], bwd))
    return out


def field_strength(u: np.ndarray) -> dict:
    """F_{mu nu}(x) = (Q_{mu nu} - Q_{mu nu}^dag)/8 for all mu != nu.

    Q_{mu nu}(x) is the sum of the four plaquettes in the (mu, nu) plane that
    start and end at x, each traversed counter-clockwise; Q_{nu mu} = Q^dag.
    """
    f = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um = u[..., mu, :, :]
            un = u[..., nu, :, :]
            um_xn = shift_link(um, nu, +1)             # U_mu(x+nu)
            un_xm = shift_link(un, mu, +1)             # U_nu(x+mu)
            um_bm = shift_link(um, mu, -1)             # U_mu(x-mu)
            un_bm = shift_link(un, mu, -1)             # U_nu(x-mu)
            um_bm_xn = shift_link(um_bm, nu, +1)       # U_mu(x-mu+nu)
            um_bn = shift_link(um, nu, -1)             # U_mu(x-nu)
            un_bn = shift_link(un, nu, -1)             # U_nu(x-nu)
            um_bm_bn = shift_link(um_bm, nu, -1)       # U_mu(x-mu-nu)
            un_bm_bn = shift_link(un_bm, nu, -1)       # U_nu(x-mu-nu)
            un_xm_bn = shift_link(un_xm, nu, -1)       # U_nu(x+mu-nu)
            q = um @ un_xm @ _dag(um_xn) @ _dag(un)
            q = q + un @ _dag(um_bm_xn) @ _dag(un_bm) @ um_bm
            q = q + _dag(um_bm) @ _dag(un_bm_bn) @ um_bm_bn @ un_bn
            q = q + _dag(un_bn) @ um_bn @ un_xm_bn @ _dag(um)
            fmn = (q - _dag(q)) / 8.0
            f[(mu, nu)] = fmn
            f[(nu, mu)] = -fmn
    return f


def clover_field(u: np.ndarray, m0: float, csw: float) -> np.ndarray:
    """A(x) as a 12x12 matrix per site, index = 3*spin + colour."""
    dims = u.shape[:4]
    f = field_strength(u)
    a = np.zeros(dims + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            s = sigma_munu(mu, nu)
            a += (csw * 0.25j) * np.einsum("st,...ab->...satb", s, f[(mu, nu)]).reshape(dims + (12, 12))
    a += (4.0 + m0) * np.eye(12)
    return a


def apply_site_matrix(a: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(A psi)(x) for a per-site 12x12 matrix field."""
    shp = psi.shape
    v = psi.reshape(shp[:-2] + (12, 1))
    return np.matmul(a, v).reshape(shp)


def dw(u: np.ndarray, a: np.ndarray, psi: np.ndarray, bc_t: float = -1.0) -> np.ndarray:
    """D psi = A psi - 1/2 H psi."""
    return apply_site_matrix(a, psi) - 0.5 * hopping(u, psi, bc_t)


def apply_gamma5(psi: np.ndarray) -> np.ndarray:
    return _spin_mul(gamma5(), psi)


def dw_dagger(u, a, psi, bc_t=-1.0):
    """D^dag psi = g5 D g5 psi (gamma5-hermiticity, pinned in the tests)."""
    return apply_gamma5(dw(u, a, apply_gamma5(psi), bc_t))


def parity_mask(dims) -> np.ndarray:
    """Boolean mask, True on odd sites."""
    x = np.indices(tuple(dims)).sum(axis=0)
    return (x % 2) == 1


def even_part(psi: np.ndarray) -> np.ndarray:
    out = psi.copy()
    out[parity_mask(psi.shape[:4])] = 0.0
    return out


def odd_part(psi: np.ndarray) -> np.ndarray:
    out = psi.copy()
    out[~parity_mask(psi.shape[:4])] = 0.0
    return out


def _hop_term(u, psi, bc_t):
    """The off-diagonal part of D: -1/2 H."""
    return -0.5 * hopping(u, psi, bc_t)


def dw_hat(u, a, ainv, psi_e, bc_t=-1.0):
    """Dhat psi_e = A_ee psi_e - D_eo A_oo^{-1} D_oe psi_e (even sites only).

    ``ainv`` is the per-site inverse of ``a`` (only its odd sites are used).
    """
    psi_e = even_part(psi_e)
    t_o = odd_part(_hop_term(u, psi_e, bc_t))          # D_oe psi_e
    t_o = odd_part(apply_site_matrix(ainv, t_o))       # D_oo^{-1} D_oe psi_e
    s_e = even_part(_hop_term(u, t_o, bc_t))           # D_eo (...)
    return even_part(apply_site_matrix(a, psi_e)) - s_e


def dw_hat_dagger(u, a, ainv, psi_e, bc_t=-1.0):
    return apply_gamma5(dw_hat(u, a, ainv, apply_gamma5(psi_e), bc_t))


def schur_source(u, a, ainv, b, bc_t=-1.0):
    """bhat = b_e - D_eo D_oo^{-1} b_o (right-hand side of the even system)."""
    t_o = odd_part(apply_site_matrix(ainv, odd_part(b)))
    return even_part(b) - even_part(_hop_term(u, t_o, bc_t))


def schur_reconstruct_odd(u, a, ainv, b, x_e, bc_t=-1.0):
    """x_o = D_oo^{-1} (b_o - D_oe x_e); returns the full solution x_e + x_o."""
    rhs = odd_part(b) - odd_part(_hop_term(u, even_part(x_e), bc_t))
    return even_part(x_e) + odd_part(apply_site_matrix(ainv, rhs))


def assemble_dense(op, dims) -> np.ndarray:
    """Dense matrix of a linear map on spinor fields by applying it to unit vectors."""
    dims = tuple(dims)
    n = int(np.prod(dims)) * 12
    m = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(dims + (4, 3), dtype=np.complex128)
    flat = e.reshape(-1)
    for j in range(n):
        flat[j] = 1.0
        m[:, j] = op(e).reshape(-1)
        flat[j] = 0.0
    return m


def clover_site(u, m0, csw, x) -> np.ndarray:
    """A(x) (12x12) at one site from the four plaquette leaves around x.

    Same definition as ``clover_field``, evaluated at a single site with
    explicit index arithmetic, for checking samples of very large lattices.
    """
    dims = u.shape[:4]

    def link(y, mu):
        return u[tuple(c % d for c, d in zip(y, dims)) + (mu,)]

    x = tuple(int(c) for c in x)
    a = (4.0 + m0) * np.eye(12, dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            e_mu = [0, 0, 0, 0]
            e_nu = [0, 0, 0, 0]
            e_mu[mu] = 1
            e_nu[nu] = 1
            add = lambda y, s, t: tuple(y[k] + s * e_mu[k] + t * e_nu[k] for k in range(4))
            q = (link(x, mu) @ link(add(x, 1, 0), nu) @ _dag(link(add(x, 0, 1), mu)) @ _dag(link(x, nu))
                 + link(x, nu) @ _dag(link(add(x, -1, 1), mu)) @ _dag(link(add(x, -1, 0), nu)) @ link(add(x, -1, 0), mu)
                 + _dag(link(add(x, -1, 0), mu)) @ _dag(link(add(x, -1, -1), nu)) @ link(add(x, -1, -1), mu)
                 @ link(add(x, 0, -1), nu)
                 + _dag(link(add(x, 0, -1), nu)) @ link(add(x, 0, -1), mu) @ link(add(x, 1, -1), nu)
                 @ _dag(link(x, mu)))
            f = (q - _dag(q)) / 8.0
            a += (csw * 0.25j) * np.kron(sigma_munu(mu, nu), f)
    return a


def dw_site(u, a, psi, x, bc_t=-1.0) -> np.ndarray:
    """(D psi)(x) at one site by explicit loops over the 8 neighbours.

    Used to check sampled outputs of very large lattices.  Returns (4, 3).
    """
    g = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    dims = psi.shape[:4]
    x = tuple(int(c) for c in x)
    out = (a[x] @ psi[x].reshape(12)).reshape(4, 3)
    for mu in range(4):
        xf = list(x)
        xf[mu] = (x[mu] + 1) % dims[mu]
        xb = list(x)
        xb[mu] = (x[mu] - 1) % dims[mu]
        sf = bc_t if (mu == 0 and x[0] == dims[0] - 1) else 1.0
        sb = bc_t if (mu == 0 and x[0] == 0) else 1.0
        pf = (one - g[mu]) @ psi[tuple(xf)] * sf
        pb = (one + g[mu]) @ psi[tuple(xb)] * sb
        uf = u[x + (mu,)]
        ub = u[tuple(xb) + (mu,)]
        out = out - 0.5 * (pf @ uf.T + pb @ np.conj(ub))
    return out


# ---------------------------------------------------------------------------
# Schroedinger-functional time boundaries (openQCD boundary type 1, the
# boundary conditions of the 4^4 matrix of Fig. 4, Sec. 2 footnote)
# ---------------------------------------------------------------------------
#
# The stored time slices are x0 = 0 .. T-1.  Quark fields live on the active
# slices 1 <= x0 <= T-1 and vanish at x0 = 0 and x0 = T; the operator maps
# active fields to active fields.  The gauge links at the boundaries (the
# spatial links of slice 0, which by periodicity also stand for those of
# slice T) enter only through the clover leaves of slices 1 and T-1.  The
# boundary-improvement term adds (c_F - 1) to the diagonal at x0 = 1 and
# x0 = T-1.

def sf_project(psi: np.ndarray) -> np.ndarray:
    """Set the x0 = 0 slice to zero (the field there vanishes)."""
    out = psi.copy()
    out[0] = 0.0
    return out


def clover_field_sf(u: np.ndarray, m0: float, csw: float, cf: float) -> np.ndarray:
    """The clover field plus the boundary term (c_F - 1) at x0 = 1, T-1."""
    a = clover_field(u, m0, csw)
    t = u.shape[0]
    for x0 in {1, t - 1}:
        a[x0] += (cf - 1.0) * np.eye(12)
    return a


def dw_sf(u, a, psi):
    """D psi for Schroedinger-functional boundaries: the fields at x0 = 0 and
    x0 = T are zero (input and output), so no hop crosses x0 = 0 <-> T-1 and
    the output at x0 = 0 is zero.  ``a`` from ``clover_field_sf``."""
    return sf_project(dw(u, a, sf_project(psi), bc_t=0.0))


def dw_sf_dagger(u, a, psi):
    return apply_gamma5(dw_sf(u, a, apply_gamma5(psi)))


def dw_hat_sf(u, a, ainv, psi_e):
    """The even-odd Schur complement of ``dw_sf`` on the active even sites:
    A_ee psi_e - D_eo A_oo^{-1} D_oe psi_e with every intermediate field
    vanishing at x0 = 0."""
    psi_e = sf_project(even_part(psi_e))
    t_o = sf_project(odd_part(_hop_term(u, psi_e, 0.0)))
    t_o = odd_part(apply_site_matrix(ainv, t_o))
    s_e = even_part(_hop_term(u, t_o, 0.0))
    return sf_project(even_part(apply_site_matrix(a, psi_e)) - s_e)


def dw_hat_sf_dagger(u, a, ainv, psi_e):
    return apply_gamma5(dw_hat_sf(u, a, ainv, apply_gamma5(psi_e)))


# ---------------------------------------------------------------------------
# QCD+QED clover term with separate coefficients (openQ*D, Sec. 1)
# ---------------------------------------------------------------------------

def clover_field_qed(u_su3, a_u1, q, m0, csw, csw_qed):
    """A(x) = (4 + m0) + (i/4) sum_{mu != nu} sigma_{mu nu}
                 [c_sw F^{SU(3)}_{mu nu}(x) + c_sw^{QED} F^{U(1)}_{mu nu}(x) 1_colour]

    F^{SU(3)} is the clover-leaf field strength of the SU(3) links,
    F^{U(1)} that of the charged U(1) links exp(i q A_mu(x)) (the same
    clover-leaf formula applied to the phases).  The hopping term uses the
    product links U_mu(x) exp(i q A_mu(x)).
    """
    dims = u_su3.shape[:4]
    z = np.exp(1j * q * np.asarray(a_u1))[..., None, None] * np.eye(3)
    f3 = field_strength(u_su3)
    f1 = field_strength(z)
    a = np.zeros(dims + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            s = sigma_munu(mu, nu)
            f = csw * f3[(mu, nu)] + csw_qed * f1[(mu, nu)]
            a += 0.25j * np.einsum("st,...ab->...satb", s, f).reshape(dims + (12, 12))
    a += (4.0 + m0) * np.eye(12)
    return a
