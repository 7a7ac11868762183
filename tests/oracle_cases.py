"""Small seeded lattices shared by the oracle pin tests (CPU only)."""
import functools

import numpy as np

from oracle import dirac
from paper_2202_07388_gb300 import synth


@functools.lru_cache(maxsize=None)
def gauge_case(dims=(4, 4, 4, 4), eps=0.3, seed=1, kappa=0.13, csw=1.0):
    u = synth.make_gauge(dims, eps, seed)
    m0 = dirac.kappa_to_m0(kappa)
    a = dirac.clover_field(u, m0, csw)
    ainv = np.linalg.inv(a)
    return u, a, ainv


def rand_spinor(dims, seed):
    return synth.make_source(dims, seed)
