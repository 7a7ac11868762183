"""Host logic of the time-split sub-domains (Sec. 3: one local lattice per
process), on CPU.

The decomposition (slices, extended link slices, boundary signs) is checked
directly.  Then two gloo ranks run the product driver -- ``TimeSplit``,
``DistComm`` (point-to-point faces, binary64 all-reduce) and ``split_cgne``
-- over a NumPy stand-in for the GPU sub-domain operator written in this file
from the oracle: each part applies the oracle's hopping term on its slab
extended by one ghost slice per side, filled with the neighbour's boundary
slice (times the boundary factor), pass by pass as the GPU does.  The split
Dhat must equal the oracle's unsplit Dhat slab by slab, and the distributed
CGNE must reach the unsplit oracle solution."""
import os
import socket

import numpy as np
import pytest

from oracle import dirac, solvers
from paper_2202_07388_gb300 import halo, synth

DIMS = (8, 4, 4, 4)
KAPPA, CSW, EPS, SEED = 0.13, 1.0, 0.3, 11


def test_time_split_decomposition():
    s = halo.TimeSplit((8, 4, 4, 6), 2)
    assert s.local_dims == (4, 4, 4, 6)
    assert s.slices(1) == [4, 5, 6, 7]
    assert s.ext_slices(0) == [7, 0, 1, 2, 3, 4] and s.ext_slices(1) == [3, 4, 5, 6, 7, 0]
    # antiperiodic: only the hops across the global boundary (last part <-> first) carry -1
    assert s.signs(0) == (1.0, -1.0) and s.signs(1) == (-1.0, 1.0)
    s4 = halo.TimeSplit((8, 4, 4, 6), 4, bc_t=1)
    assert [s4.signs(r) for r in range(4)] == [(1.0, 1.0)] * 4
    assert s4.prev(0) == 3 and s4.next(3) == 0
    u = np.arange(8 * 3).reshape(8, 3)
    assert np.array_equal(s.gather([s.local(u, r) for r in range(2)]), u)
    with pytest.raises(ValueError):
        halo.TimeSplit((8, 4, 4, 4), 3)          # 8 slices do not split in 3
    with pytest.raises(ValueError):
        halo.TimeSplit((6, 4, 4, 4), 2)          # odd local extent breaks the parities


def test_loopback_exchange_routes_faces():
    c = halo.LoopbackComm(3)
    fn, fp = c.exchange(["p0", "p1", "p2"], ["n0", "n1", "n2"])
    assert fn == ["p1", "p2", "p0"] and fp == ["n2", "n0", "n1"]


class NumpyPart:
    """The oracle's Dhat on one part (test stand-in for GpuSplitDhat)."""

    def __init__(self, split, r, u, comm):
        self.split, self.r, self.comm, self.nrhs = split, r, comm, 1
        self.u_ext = split.ext_links(u, r)
        a_ext = dirac.clover_field(self.u_ext, dirac.kappa_to_m0(KAPPA), CSW)
        self.a = a_ext[1:-1]
        self.ainv = np.linalg.inv(self.a)
        self.sn, self.sp = split.signs(r)

    def _ghosted_hop(self, x):
        """-1/2 H x on the slab, the neighbours' boundary slices as ghosts."""
        import torch
        first = torch.from_numpy(np.ascontiguousarray(x[0]).view(np.float64))
        last = torch.from_numpy(np.ascontiguousarray(x[-1]).view(np.float64))
        (fn,), (fp,) = self.comm.exchange([first], [last])
        nxt = fn.numpy().view(np.complex128).reshape(x.shape[1:])
        prv = fp.numpy().view(np.complex128).reshape(x.shape[1:])
        ext = np.concatenate([self.sp * prv[None], x, self.sn * nxt[None]], axis=0)
        return -0.5 * dirac.hopping(self.u_ext, ext, bc_t=1.0)[1:-1]

    def dhat(self, x, dagger=False):
        if dagger:
            return dirac.apply_gamma5(self.dhat(dirac.apply_gamma5(x)))
        t = dirac.odd_part(dirac.apply_site_matrix(self.ainv, dirac.odd_part(self._ghosted_hop(x))))
        return dirac.even_part(dirac.apply_site_matrix(self.a, x) - self._ghosted_hop(t))

    # the operator interface of split_cgne (one local part)
    def new_field(self):
        return [np.zeros(self.split.local_dims + (4, 3), np.complex128)]

    def normal(self, xs, ys):
        ys[0][...] = self.dhat(self.dhat(xs[0]), dagger=True)

    def dot_local(self, xs, ys):
        return np.array([np.vdot(xs[0], ys[0])])

    def axpby(self, a, xs, b, ys):
        ys[0][...] = a[0] * xs[0] + b[0] * ys[0]

    def copy(self, src, dst):
        dst[0][...] = src[0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        split = halo.TimeSplit(DIMS, world)
        u = synth.make_gauge(DIMS, EPS, SEED)
        comm = halo.DistComm()
        part = NumpyPart(split, rank, u, comm)
        psi = dirac.even_part(synth.make_source(DIMS, SEED + 1))
        dh = part.dhat(split.local(psi, rank))
        dhd = part.dhat(split.local(psi, rank), dagger=True)
        eta = [np.ascontiguousarray(split.local(psi, rank))]
        x = part.new_field()
        st = halo.split_cgne(part, comm, eta, x, res=1e-11, nmx=2000)
        out[rank] = (dh, dhd, x[0], st[0])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_dhat_and_cgne():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    split = halo.TimeSplit(DIMS, world)
    u = synth.make_gauge(DIMS, EPS, SEED)
    a = dirac.clover_field(u, dirac.kappa_to_m0(KAPPA), CSW)
    ainv = np.linalg.inv(a)
    psi = dirac.even_part(synth.make_source(DIMS, SEED + 1))
    ref = dirac.dw_hat(u, a, ainv, psi)
    refd = dirac.dw_hat_dagger(u, a, ainv, psi)
    for r in range(world):
        dh, dhd, _, _ = res[r]
        assert np.allclose(dh, split.local(ref, r), rtol=0, atol=1e-13 * np.abs(ref).max())
        assert np.allclose(dhd, split.local(refd, r), rtol=0, atol=1e-13 * np.abs(refd).max())
    # the distributed CGNE against the unsplit operator and the oracle's own CGNE
    x = split.gather([res[r][2] for r in range(world)])
    normal = lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v))  # noqa: E731
    rel = np.linalg.norm(psi - normal(x)) / np.linalg.norm(psi)
    assert rel <= 1.05e-11
    for r in range(world):
        st = res[r][3]
        assert st["converged"] and abs(st["true_rel_res"] - rel) <= 1e-3 * rel
    ref_x = solvers.cgne(normal, psi, 1e-11, 2000, "fp64").x
    assert np.linalg.norm(x - ref_x) <= 1e-9 * np.linalg.norm(ref_x)
    assert res[0][3]["steps"] == res[1][3]["steps"]
