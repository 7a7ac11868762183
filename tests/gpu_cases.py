"""Shared set-up of the GPU parity tests: seeded inputs (synth), the oracle
on the CPU, and the library through its C ABI on cuda:0."""
import functools

import numpy as np

from oracle import dirac
from paper_2202_07388_gb300 import synth

# relative L2 error vs the FP64 oracle, per storage type (4: binary64 storage,
# double-float arithmetic, ~48-bit significands)
TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 2e-3, 4: 1e-12}


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if np.iscomplexobj(a):
        return torch.from_numpy(a.view(np.float64).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


def from_dev(t, shape):
    v = t.cpu().numpy().view(np.complex128)
    return v.reshape(shape)


@functools.lru_cache(maxsize=8)
def oracle_case(dims, eps, seed, kappa, csw):
    u = synth.make_gauge(dims, eps, seed)
    a = dirac.clover_field(u, dirac.kappa_to_m0(kappa), csw)
    ainv = np.linalg.inv(a)
    return u, a, ainv


def make_handle(dims, u, kappa, csw, link_fmt):
    from paper_2202_07388_gb300 import oq
    h = oq.Handle(dims)
    ud = to_dev(u)
    h.gauge_upload(ud, link_fmt)
    h.clover_build(kappa, csw)
    return h


def rel_err(got, ref):
    return float(np.linalg.norm((got - ref).reshape(-1)) / np.linalg.norm(ref.reshape(-1)))


def check_residual(oracle_res, reported, target=1e-10, rel=1e-3):
    """The binary64 relative residual recomputed by the oracle meets the
    target, and the solver's own report of it agrees to `rel` (relative)."""
    assert oracle_res <= target * (1 + rel), (oracle_res, target)
    assert abs(oracle_res - reported) <= rel * oracle_res, (oracle_res, reported)
