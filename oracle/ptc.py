"""Gauge-equivariant parallel-transport layers, FP64 (test infrastructure).

Not part of the paper: the learned preconditioner is a two-layer linear
network of parallel-transport convolutions (PTC).  A layer maps C_in spinor
fields to C_out spinor fields by

    out_{c'}(x) = sum_{p in P} sum_c W^{(p)}_{c' c} (T_p psi_c)(x),

with the 9 paths P = {identity, +mu, -mu (mu = 0..3)}, the parallel
transports

    (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),
    (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu),

(times the fermion time-boundary factor on hops across the time boundary,
as in the Dirac operator) and W^{(p)}_{c' c} a complex 4x4 matrix acting on
spin only.  Because W never touches colour and T_p moves a spinor together
with the links, psi -> Lambda psi, U -> Lambda U Lambda^dag(x+mu) maps the
output to Lambda out exactly (gauge equivariance).

Weights are stored as an array W[p, c', c, s, t], p = 0 (identity),
p = 1 + 2 mu (+mu), p = 2 + 2 mu (-mu).

Gradients use the real-gradient convention g = dL/dRe(W) + i dL/dIm(W),
which is what finite differences on the real and imaginary parts measure.
"""
from __future__ import annotations

import numpy as np

from .dirac import shift_spinor, shift_link

__all__ = ["NPATH", "transport", "transport_adjoint", "ptc_layer", "ptc_layer_backward",
           "forward", "loss", "backward"]

NPATH = 9


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _colour_mul(u, psi):
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def transport(u, psi, p, bc_t=-1.0):
    """T_p psi for one spinor field psi (dims + (4, 3))."""
    if p == 0:
        return psi.copy()
    mu = (p - 1) // 2
    if (p - 1) % 2 == 0:
        return _colour_mul(u[..., mu, :, :], shift_spinor(psi, mu, +1, bc_t))
    u_back = shift_link(u[..., mu, :, :], mu, -1)
    return _colour_mul(_dag(u_back), shift_spinor(psi, mu, -1, bc_t))


def transport_adjoint(u, g, p, bc_t=-1.0):
    """T_p^dag g, written out from <T_p a, b> = <a, T_p^dag b>.

    For p = +mu: (T^dag g)(y) = U_mu(y - mu)^dag g(y - mu) (times the boundary
    factor of the hop y - mu -> y); for p = -mu: (T^dag g)(y) = U_mu(y) g(y + mu).
    """
    if p == 0:
        return g.copy()
    mu = (p - 1) // 2
    if (p - 1) % 2 == 0:
        u_back = shift_link(u[..., mu, :, :], mu, -1)
        return _colour_mul(_dag(u_back), shift_spinor(g, mu, -1, bc_t))
    return _colour_mul(u[..., mu, :, :], shift_spinor(g, mu, +1, bc_t))


def ptc_layer(u, w, fields, bc_t=-1.0):
    """One PTC layer: fields (C_in,) + dims + (4, 3) -> (C_out,) + dims + (4, 3)."""
    npath, cout, cin = w.shape[:3]
    out = np.zeros((cout,) + fields.shape[1:], dtype=np.complex128)
    for p in range(npath):
        for c in range(cin):
            tp = transport(u, fields[c], p, bc_t)
            for co in range(cout):
                out[co] += np.einsum("st,...ta->...sa", w[p, co, c], tp)
    return out


def ptc_layer_backward(u, w, fields, grad_out, bc_t=-1.0):
    """Gradients of one layer given g = grad_out (real-gradient convention).

    For a real loss L and y = layer(x): grad_W[p, c', c] = sum_x g_{c'}(x)
    (T_p x_c)(x)^dag (spin outer product, summed over colour) and
    grad_x_c = sum_p T_p^dag sum_{c'} W^{(p)dag}_{c' c} g_{c'}.
    """
    npath, cout, cin = w.shape[:3]
    gw = np.zeros_like(w)
    gx = np.zeros_like(fields)
    for p in range(npath):
        for c in range(cin):
            tp = transport(u, fields[c], p, bc_t)
            for co in range(cout):
                gw[p, co, c] = np.einsum("ijklsa,ijklta->st", grad_out[co], np.conj(tp))
        for c in range(cin):
            acc = np.zeros_like(fields[c])
            for co in range(cout):
                acc += np.einsum("ts,...ta->...sa", np.conj(w[p, co, c]), grad_out[co])
            gx[c] += transport_adjoint(u, acc, p, bc_t)
    return gw, gx


def forward(u, w1, w2, psi, bc_t=-1.0):
    """Two layers 1 -> C_hidden -> 1 with no activation.  Returns (y, h)."""
    h = ptc_layer(u, w1, psi[None], bc_t)
    y = ptc_layer(u, w2, h, bc_t)
    return y[0], h


def loss(u, w1, w2, r, e, bc_t=-1.0) -> float:
    """||M r - e||^2 / ||e||^2 for one (residual, error) pair."""
    y, _ = forward(u, w1, w2, r, bc_t)
    return float(np.vdot(y - e, y - e).real / np.vdot(e, e).real)


def backward(u, w1, w2, r, e, bc_t=-1.0):
    """(loss, grad_w1, grad_w2) for one pair."""
    y, h = forward(u, w1, w2, r, bc_t)
    en = np.vdot(e, e).real
    gy = 2.0 * (y - e) / en
    gw2, gh = ptc_layer_backward(u, w2, h, gy[None], bc_t)
    gw1, _ = ptc_layer_backward(u, w1, r[None], gh, bc_t)
    return float(np.vdot(y - e, y - e).real / en), gw1, gw2
