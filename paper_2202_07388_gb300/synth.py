"""Seeded synthetic inputs: gauge fields, sources and gauge transformations.

This module only draws inputs. It holds none of the solver or operator
arithmetic, and it is the one piece of code that both the CUDA path (through
the tests and the benchmark) and the FP64 oracle consume.

Canonical host layout (shared by every producer and consumer of these arrays):

* lattice dims ``L = (L0, L1, L2, L3)``, ``L0`` = time, slowest index;
  site index ``x = ((x0*L1 + x1)*L2 + x2)*L3 + x3``.
* gauge field ``U[x0, x1, x2, x3, mu, a, b]`` complex128, ``mu = 0..3``
  (``mu = 0`` is time), ``a, b`` colour row/column.
* spinor ``psi[x0, x1, x2, x3, s, a]`` complex128, ``s`` spin (chiral basis
  index 0..3), ``a`` colour.

Gauge links follow the recipe U = exp(i*eps*H), H Gaussian Hermitian
traceless, reunitarised; an optional U(1) factor exp(i*q*A_mu(x)) with
A_mu(x) ~ N(0, sigma^2) turns them into U(3) = SU(3) x U(1) links (QCD+QED).
Random numbers come from NumPy's PCG64 seeded with the given seed, so both
sides of every comparison see the same bits.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "make_gauge",
    "make_u1_field",
    "apply_u1",
    "make_source",
    "make_point_sources",
    "random_gauge_transform",
    "gauge_transform",
    "volume",
]


def volume(dims) -> int:
    d = tuple(int(v) for v in dims)
    return d[0] * d[1] * d[2] * d[3]


def expi_hermitian3(q: np.ndarray) -> np.ndarray:
    """exp(i Q) for a batch of Hermitian traceless 3x3 matrices Q.

    Cayley-Hamilton closed form exp(iQ) = f0 + f1 Q + f2 Q^2 with the
    coefficients of Morningstar and Peardon (Phys. Rev. D 69 (2004) 054501,
    Sec. III), written from those formulas; c0 < 0 uses
    f_j(-c0) = (-1)^j conj(f_j(c0)).  Checked against an eigendecomposition
    in the tests.
    """
    q2 = q @ q
    c0 = np.trace(q2 @ q, axis1=-2, axis2=-1).real / 3.0
    c1 = 0.5 * np.trace(q2, axis1=-2, axis2=-1).real
    neg = c0 < 0
    c0max = 2.0 * (c1 / 3.0) ** 1.5
    ratio = np.where(c0max > 0, np.abs(c0) / np.where(c0max > 0, c0max, 1.0), 0.0)
    theta = np.arccos(np.clip(ratio, -1.0, 1.0))
    u = np.sqrt(c1 / 3.0) * np.cos(theta / 3.0)
    w = np.sqrt(c1) * np.sin(theta / 3.0)
    w2 = w * w
    xi0 = np.where(np.abs(w) > 0.05, np.sin(w) / np.where(w != 0, w, 1.0),
                   1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)))
    e2iu = np.exp(2j * u)
    emiu = np.exp(-1j * u)
    cw = np.cos(w)
    uu = u * u
    h0 = (uu - w2) * e2iu + emiu * (8.0 * uu * cw + 2j * u * (3.0 * uu + w2) * xi0)
    h1 = 2.0 * u * e2iu - emiu * (2.0 * u * cw - 1j * (3.0 * uu - w2) * xi0)
    h2 = e2iu - emiu * (cw + 3j * u * xi0)
    den = 9.0 * uu - w2
    tiny = den < 1e-12  # Q ~ 0
    den = np.where(tiny, 1.0, den)
    f0, f1, f2 = h0 / den, h1 / den, h2 / den
    f0 = np.where(neg, np.conj(f0), f0)
    f1 = np.where(neg, -np.conj(f1), f1)
    f2 = np.where(neg, np.conj(f2), f2)
    f0 = np.where(tiny, 1.0, f0)
    f1 = np.where(tiny, 1j, f1)
    f2 = np.where(tiny, -0.5, f2)
    return f0[..., None, None] * np.eye(3) + f1[..., None, None] * q + f2[..., None, None] * q2


def _random_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """n matrices exp(i*eps*H), H = (A + A^dag)/2 - tr/3, A complex Gaussian."""
    z = rng.standard_normal((n, 2, 3, 3))  # 18 draws per link, link by link
    a = z[:, 0] + 1j * z[:, 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    return _reunitarise(expi_hermitian3(eps * h))


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1; row 2 = conj(row0 x row1) (det = 1)."""
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def make_gauge(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """SU(3) gauge field of shape dims + (4, 3, 3), complex128.

    Links are drawn site by site in canonical order (x, then mu), in chunks
    so that large lattices stay within host memory limits.
    """
    dims = tuple(int(v) for v in dims)
    n = volume(dims) * 4
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = _random_su3(rng, e - s, eps)
    return out.reshape(dims + (4, 3, 3))


def make_gauge_sf(dims, eps: float, seed: int) -> np.ndarray:
    """SU(3) field for Schroedinger-functional boundaries with zero boundary
    fields: ``make_gauge`` with the spatial links of slice x0 = 0 (the
    boundary at x0 = 0 and, by periodicity, at x0 = T) set to the identity."""
    u = make_gauge(dims, eps, seed)
    u[0, :, :, :, 1:] = np.eye(3)
    return u


def make_u1_field(dims, sigma: float, seed: int) -> np.ndarray:
    """Real U(1) gauge potential A_mu(x) ~ N(0, sigma^2), shape dims + (4,)."""
    dims = tuple(int(v) for v in dims)
    rng = np.random.default_rng(seed)
    return sigma * rng.standard_normal(dims + (4,))


def apply_u1(u: np.ndarray, a: np.ndarray, q: float) -> np.ndarray:
    """U(3) links: U_mu(x) * exp(i*q*A_mu(x))."""
    return u * np.exp(1j * q * a)[..., None, None]


def make_source(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian complex spinor field(s): re, im ~ N(0, 1/2) per component."""
    dims = tuple(int(v) for v in dims)
    rng = np.random.default_rng(seed)
    shape = dims + (4, 3) if nrhs is None else (nrhs,) + dims + (4, 3)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def make_point_sources(dims, site=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 spin-colour point sources delta_{x,site} delta_{(s,a),(s0,a0)}.

    Shape (12,) + dims + (4, 3); source j has spin j // 3 and colour j % 3.
    """
    dims = tuple(int(v) for v in dims)
    out = np.zeros((12,) + dims + (4, 3), dtype=np.complex128)
    for j in range(12):
        out[(j,) + tuple(site) + (j // 3, j % 3)] = 1.0
    return out


def random_gauge_transform(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """Random SU(3) matrix Lambda(x) per site, shape dims + (3, 3)."""
    dims = tuple(int(v) for v in dims)
    rng = np.random.default_rng(seed)
    return _random_su3(rng, volume(dims), eps).reshape(dims + (3, 3))


def gauge_transform(u: np.ndarray, lam: np.ndarray):
    """U'_mu(x) = Lambda(x) U_mu(x) Lambda(x+mu)^dag (periodic site wrap).

    Returns the transformed links. Spinors transform as psi' = Lambda psi,
    which callers apply with ``np.einsum('...ab,...sb->...sa', lam, psi)``.
    """
    out = np.empty_like(u)
    for mu in range(4):
        lam_fwd = np.roll(lam, -1, axis=mu)
        out[..., mu, :, :] = lam @ u[..., mu, :, :] @ np.conj(np.swapaxes(lam_fwd, -1, -2))
    return out
