"""C* boundary conditions in the orbifold form (test infrastructure).

openQ*D (Sec. 1 of the paper) runs QCD+QED with C* spatial boundary
conditions: across the boundary of a C* direction k the fields continue as
their charge conjugates; for the gauge field U_mu(x + L_k k) = U_mu(x)^*.
The orbifold form, the one this oracle states and the library implements:

* the lattice is doubled in x1, extent 2 L1; its second half holds the
  charge-conjugate copy of the gauge field, U_mu(x + L1 e1) = U_mu(x)^*
  (and for a U(1) field A_mu(x + L1 e1) = -A_mu(x));
* the doubled lattice is periodic in x1 with period 2 L1 (C* in x1);
* for C* in x2 (x3 likewise) the point x + L2 e2 is the point x + L1 e1 of
  the doubled lattice: a step across the x2 boundary also moves x1 by L1;
* on the doubled lattice the Dirac operator is the ordinary Wilson-clover
  operator of ``dirac`` (same normalisation, gamma basis and clover leaves)
  for these links and this neighbour relation.

Here every shift is written out with that neighbour relation; the Dirac
algebra (gamma matrices, sigma_{mu nu}, the per-site matrix product) is
taken from ``dirac``.  Nothing is blocked or reordered.
"""
from __future__ import annotations

import numpy as np

from . import dirac


def double_links(u: np.ndarray) -> np.ndarray:
    """Physical links (T, L1, L2, L3, 4, 3, 3) -> links of the doubled lattice
    (T, 2 L1, L2, L3, 4, 3, 3): the second half is the complex conjugate."""
    return np.concatenate([u, np.conj(u)], axis=1)


def double_angles(a: np.ndarray) -> np.ndarray:
    """U(1) angles A_mu(x) (T, L1, L2, L3, 4) -> doubled lattice, second half -A."""
    return np.concatenate([a, -a], axis=1)


def twisted(mu: int, cstar: int) -> bool:
    """Does a step across the x_mu boundary move x1 by half the doubled extent?"""
    return (mu == 2 and cstar >= 2) or (mu == 3 and cstar >= 3)


def shift(f: np.ndarray, mu: int, d: int, cstar: int, bc_t: float = 1.0) -> np.ndarray:
    """g(x) = f(x + d mu) on the doubled lattice (axes 0..3 are the lattice).

    A step that leaves through the x_mu boundary re-enters on the other side
    and, for a twisted direction, in the other copy (x1 + L1 mod 2 L1); for
    mu = 0 it picks up the fermion factor bc_t (1 for links)."""
    out = np.roll(f, -d, axis=mu)
    L = f.shape[mu]
    edge = L - 1 if d == +1 else 0            # the sites whose neighbour wrapped
    idx = [slice(None)] * f.ndim
    idx[mu] = edge
    idx = tuple(idx)
    if twisted(mu, cstar):
        # the slab at the edge keeps axes 0 and 1 (mu >= 2): its x1 is axis 1
        h = f.shape[1] // 2
        out[idx] = np.roll(out[idx], -h, axis=1)
    if mu == 0 and bc_t != 1.0:
        out[idx] = bc_t * out[idx]
    return out


def hopping(u: np.ndarray, psi: np.ndarray, cstar: int, bc_t: float = -1.0) -> np.ndarray:
    """H psi = sum_mu [U_mu(x)(1 - g_mu) psi(x + mu) + U_mu(x - mu)^dag (1 + g_mu) psi(x - mu)]."""
    g = dirac.gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros_like(psi)
    for mu in range(4):
        u_mu = u[..., mu, :, :]
        fwd = shift(psi, mu, +1, cstar, bc_t)
        bwd = shift(psi, mu, -1, cstar, bc_t)
        u_back = shift(u_mu, mu, -1, cstar)
        # colour product with U: psi @ U^T
        out += np.matmul(np.einsum("st,...ta->...sa", one - g[mu], fwd), np.swapaxes(u_mu, -1, -2))
        # colour product with U^dag: psi @ (U^dag)^T = psi @ conj(U)
        out += np.matmul(np.einsum("st,...ta->...sa", one + g[mu], bwd), np.conj(u_back))
    return out


def field_strength(u: np.ndarray, cstar: int) -> dict:
    """F_{mu nu}(x) = (Q_{mu nu} - Q_{mu nu}^dag) / 8 from the four plaquettes
    in the (mu, nu) plane through x (counter-clockwise), twisted shifts."""
    def dag(m):
        return np.conj(np.swapaxes(m, -1, -2))

    def at(m, *steps):
        for mu, d in steps:
            m = shift(m, mu, d, cstar)
        return m

    f = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um, un = u[..., mu, :, :], u[..., nu, :, :]
            leaf1 = um @ at(un, (mu, 1)) @ dag(at(um, (nu, 1))) @ dag(un)
            leaf2 = un @ dag(at(um, (mu, -1), (nu, 1))) @ dag(at(un, (mu, -1))) @ at(um, (mu, -1))
            leaf3 = dag(at(um, (mu, -1))) @ dag(at(un, (mu, -1), (nu, -1))) @ at(um, (mu, -1), (nu, -1)) \
                @ at(un, (nu, -1))
            leaf4 = dag(at(un, (nu, -1))) @ at(um, (nu, -1)) @ at(un, (mu, 1), (nu, -1)) @ dag(um)
            q = leaf1 + leaf2 + leaf3 + leaf4
            f[(mu, nu)] = (q - dag(q)) / 8.0
            f[(nu, mu)] = -f[(mu, nu)]
    return f


def clover_field(u: np.ndarray, m0: float, csw: float, cstar: int) -> np.ndarray:
    """A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} F_{mu nu}(x), 12 x 12 per site."""
    dims = u.shape[:4]
    f = field_strength(u, cstar)
    a = np.zeros(dims + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                s = dirac.sigma_munu(mu, nu)
                a += (csw * 0.25j) * np.einsum("st,...ab->...satb", s, f[(mu, nu)]).reshape(dims + (12, 12))
    return a + (4.0 + m0) * np.eye(12)


def dw(u, a, psi, cstar, bc_t=-1.0):
    """D psi = A psi - 1/2 H psi on the doubled lattice."""
    return dirac.apply_site_matrix(a, psi) - 0.5 * hopping(u, psi, cstar, bc_t)


def dw_dagger(u, a, psi, cstar, bc_t=-1.0):
    return dirac.apply_gamma5(dw(u, a, dirac.apply_gamma5(psi), cstar, bc_t))


def dw_hat(u, a, ainv, psi_e, cstar, bc_t=-1.0):
    """Dhat = D_ee - D_eo D_oo^-1 D_oe on the even sites of the doubled lattice."""
    psi_e = dirac.even_part(psi_e)
    t_o = dirac.odd_part(-0.5 * hopping(u, psi_e, cstar, bc_t))
    t_o = dirac.odd_part(dirac.apply_site_matrix(ainv, t_o))
    return dirac.even_part(dirac.apply_site_matrix(a, psi_e) + 0.5 * hopping(u, t_o, cstar, bc_t))


def dw_hat_dagger(u, a, ainv, psi_e, cstar, bc_t=-1.0):
    return dirac.apply_gamma5(dw_hat(u, a, ainv, dirac.apply_gamma5(psi_e), cstar, bc_t))


def charge_conjugation_matrix() -> np.ndarray:
    """K with K g_mu^* K^-1 = g_mu for every mu (in the chiral basis of
    ``dirac``: g0, g2 real, g1, g3 imaginary, so K = g1 g3)."""
    g = dirac.gamma_matrices()
    return g[1] @ g[3]


def mirror(chi: np.ndarray, k: np.ndarray) -> np.ndarray:
    """(M chi)(x) = K chi(x + L1 e1)^*: the charge-conjugate copy, moved by half the doubled extent."""
    h = chi.shape[1] // 2
    return np.einsum("st,...ta->...sa", k, np.conj(np.roll(chi, -h, axis=1)))
