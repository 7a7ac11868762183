"""Host-side layout contracts of the C ABI (CPU only): the even-site
canonical layout of oq_cgne_solve_even puts the even site of lexicographic
index n at n // 2, which is a bijection onto 0 .. V/2 - 1 (the sites of one
parity alternate along x3 when L3 is even), for every admissible lattice."""
import itertools

import numpy as np
import pytest


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 6, 2), (6, 4, 2, 8), (8, 6, 4, 10)])
def test_even_site_index_is_a_bijection(dims):
    lex = np.arange(int(np.prod(dims)))
    parity = np.indices(dims).sum(axis=0).reshape(-1) % 2
    for p in (0, 1):
        half = lex[parity == p] // 2
        assert np.array_equal(np.sort(half), np.arange(lex.size // 2))
        # order preserving: the layout keeps the lexicographic order of the sites
        assert np.all(np.diff(half) > 0)


def test_even_site_gather_roundtrip():
    dims = (4, 2, 2, 6)
    rng = np.random.default_rng(3)
    full = rng.standard_normal(dims + (4, 3)) + 1j * rng.standard_normal(dims + (4, 3))
    even = (np.indices(dims).sum(axis=0) % 2) == 0
    full[~even] = 0.0
    flat = full.reshape(-1, 12)
    half = np.zeros((flat.shape[0] // 2, 12), complex)
    for n, x in enumerate(itertools.product(*[range(d) for d in dims])):
        if sum(x) % 2 == 0:
            half[n // 2] = flat[n]
    back = np.zeros_like(flat)
    back[np.nonzero(even.reshape(-1))[0]] = half
    assert np.array_equal(back, flat)
