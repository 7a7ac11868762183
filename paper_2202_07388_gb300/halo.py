"""Time-split sub-domains and the distributed CGNE over them.

The paper (Sec. 3) runs openQ*D on a lattice divided into local lattices,
one per process; every application of the Dirac operator exchanges the
boundary values with the neighbouring processes, and the solvers' scalar
products are global sums.  Here the lattice is split along time into R
parts of T_loc = T / R slices (T_loc even, so the even-odd parities of a
part are the global ones).  Per operator pass and part, two faces of
12 reals per boundary site move (the library packs and consumes them,
``oq_face_pack`` / ``oq_dhat_pass``):

* to the previous part: the projected half spinors of the first slice;
* to the next part: the link-transported half spinors of the last slice.

Moving the faces is the communicator's job:

* ``LoopbackComm`` holds all R parts in one process (one GPU): a part's
  received faces are the other parts' packed buffers;
* ``DistComm`` holds one part per process and moves the faces with
  ``torch.distributed`` point-to-point messages (NCCL for device tensors,
  gloo for host tensors) and sums scalar products with an all-reduce in
  binary64.

``split_cgne`` is the CG on the normal equations (Sec. 2, ``cgne()``) in
binary64 over such parts: every vector step is local, every scalar product
is a global binary64 sum, and the solution is checked against the binary64
true residual at the end.  The operator it is given decides where the work
runs; ``GpuSplitDhat`` runs every step in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import oq


class TimeSplit:
    """Split of a T x L1 x L2 x L3 lattice into ``nparts`` time slabs."""

    def __init__(self, dims, nparts, bc_t=-1):
        T = int(dims[0])
        if nparts < 1 or T % nparts:
            raise ValueError(f"T = {T} does not split into {nparts} parts")
        tl = T // nparts
        if tl % 2 or tl < 2:
            raise ValueError(f"local time extent {tl} must be even and >= 2")
        if bc_t not in (-1, 1):
            raise ValueError("time boundary must be periodic (+1) or antiperiodic (-1)")
        self.dims = tuple(int(d) for d in dims)
        self.nparts = nparts
        self.tl = tl
        self.bc_t = bc_t
        self.local_dims = (tl,) + self.dims[1:]

    def start(self, r):
        return r * self.tl

    def slices(self, r):
        """Global time slices of part r."""
        return list(range(self.start(r), self.start(r) + self.tl))

    def ext_slices(self, r):
        """The slices of part r with one more on each side (periodic in T):
        the links a part needs for its clover term."""
        T = self.dims[0]
        return [(self.start(r) + k) % T for k in range(-1, self.tl + 1)]

    def prev(self, r):
        return (r - 1) % self.nparts

    def next(self, r):
        return (r + 1) % self.nparts

    def signs(self, r):
        """(sign_next, sign_prev): the boundary factor of part r's hops across
        its last / first face (the global time boundary lies between the last
        part and the first)."""
        sn = float(self.bc_t) if r == self.nparts - 1 else 1.0
        sp = float(self.bc_t) if r == 0 else 1.0
        return sn, sp

    # canonical arrays have time as their first axis
    def local(self, field, r):
        return field[self.start(r):self.start(r) + self.tl]

    def ext_links(self, links, r):
        return links[self.ext_slices(r)]

    def gather(self, parts):
        """Stack the parts' canonical arrays back into the global one."""
        if isinstance(parts[0], np.ndarray):
            return np.concatenate(parts, axis=0)
        import torch
        return torch.cat(list(parts), dim=0)


class LoopbackComm:
    """All parts in this process: faces are handed over, sums are local."""

    def __init__(self, nparts):
        self.nparts = nparts

    def exchange(self, to_prev, to_next):
        """to_prev[r], to_next[r]: the faces part r packed for its neighbours.
        Returns (from_next, from_prev) per part."""
        n = self.nparts
        return [to_prev[(r + 1) % n] for r in range(n)], [to_next[(r - 1) % n] for r in range(n)]

    def allreduce(self, local):
        return np.asarray(local)


class DistComm:
    """One part per process of a ``torch.distributed`` group (rank r holds
    part r).  Faces travel as point-to-point messages, scalar products as a
    binary64 all-reduce."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.nparts = 1
        self._recv = {}

    def _buffers(self, like):
        key = (tuple(like.shape), like.dtype, str(like.device))
        if key not in self._recv:
            import torch
            self._recv[key] = (torch.empty_like(like), torch.empty_like(like))
        return self._recv[key]

    def exchange(self, to_prev, to_next):
        (tp,), (tn,) = to_prev, to_next
        if self.size == 1:
            return [tp], [tn]
        d = self.dist
        prv, nxt = (self.rank - 1) % self.size, (self.rank + 1) % self.size
        from_next, from_prev = self._buffers(tp)
        # tag 0: faces travelling to the previous rank, tag 1: to the next one
        ops = [d.P2POp(d.isend, tp, prv, self.group, 0), d.P2POp(d.isend, tn, nxt, self.group, 1),
               d.P2POp(d.irecv, from_next, nxt, self.group, 0), d.P2POp(d.irecv, from_prev, prv, self.group, 1)]
        for w in d.batch_isend_irecv(ops):
            w.wait()
        return [from_next], [from_prev]

    def allreduce(self, local):
        import torch
        v = np.asarray(local)
        flat = np.concatenate([v.real.reshape(-1), v.imag.reshape(-1)]) if np.iscomplexobj(v) else v.reshape(-1)
        t = torch.tensor(flat, dtype=torch.float64)
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, group=self.group)
        out = t.cpu().numpy()
        if np.iscomplexobj(v):
            n = v.size
            return (out[:n] + 1j * out[n:]).reshape(v.shape)
        return out.reshape(v.shape)


class GpuSplitDhat:
    """Dhat and Dhat^dag Dhat over the local parts of a time split, on the GPU.

    ``handles[k]`` is a library handle of part ``parts[k]`` (a lattice of
    ``split.local_dims`` created with bc_t = OQ_BC_HALO, links uploaded with
    ``gauge_upload_halo`` and the clover built).  Fields are lists of packed
    even half fields (one per local part, ``nrhs`` right-hand sides)."""

    def __init__(self, split, parts, handles, comm, prec=oq.F64, nrhs=1):
        self.split, self.parts, self.handles, self.comm = split, list(parts), list(handles), comm
        self.prec, self.nrhs = prec, nrhs
        self.t = [h.new_packed(prec, oq.ODD, nrhs=nrhs) for h in handles]
        self.u = [h.new_packed(prec, oq.EVEN, nrhs=nrhs) for h in handles]
        self.fprev = [h.new_faces(prec, nrhs) for h in handles]
        self.fnext = [h.new_faces(prec, nrhs) for h in handles]

    def new_field(self):
        import torch
        return [torch.zeros(h.spinor_bytes(self.prec, oq.EVEN) * self.nrhs, dtype=torch.uint8, device="cuda")
                for h in self.handles]

    def _exchange(self, fields, subset, dagger):
        for h, f, a, b in zip(self.handles, fields, self.fprev, self.fnext):
            h.face_pack(f, a, b, self.prec, subset, nrhs=self.nrhs, dagger=dagger)
        if isinstance(self.comm, DistComm):
            import torch
            torch.cuda.current_stream().synchronize()   # faces complete before another stream reads them
        from_next, from_prev = self.comm.exchange(self.fprev, self.fnext)
        halos = []
        for r, h, fn, fp in zip(self.parts, self.handles, from_next, from_prev):
            sn, sp = self.split.signs(r)
            halos.append(oq.Handle.halo(fn, fp, sn, sp))
        return halos

    def dhat(self, xs, ys, dagger=False):
        halos = self._exchange(xs, oq.EVEN, dagger)
        for h, x, t, hl in zip(self.handles, xs, self.t, halos):
            h.dhat_pass(1, x, None, t, self.prec, halo=hl, nrhs=self.nrhs, dagger=dagger)
        halos = self._exchange(self.t, oq.ODD, dagger)
        for h, x, t, y, hl in zip(self.handles, xs, self.t, ys, halos):
            h.dhat_pass(2, t, x, y, self.prec, halo=hl, nrhs=self.nrhs, dagger=dagger)

    def normal(self, xs, ys):
        """ys = Dhat^dag Dhat xs."""
        self.dhat(xs, self.u)
        self.dhat(self.u, ys, dagger=True)

    def dot_local(self, xs, ys):
        return sum(h.dot(x, y, self.prec, oq.EVEN, nrhs=self.nrhs) for h, x, y in zip(self.handles, xs, ys))

    def axpby(self, a, xs, b, ys):
        for h, x, y in zip(self.handles, xs, ys):
            h.axpby(a, x, b, y, self.prec, oq.EVEN, nrhs=self.nrhs)

    def copy(self, src, dst):
        for s, d in zip(src, dst):
            d.copy_(s)


def split_cgne(op, comm, etas, psis, res=1e-10, nmx=10000):
    """Binary64 CGNE (Sec. 2) on the parts of a split: solves
    Dhat^dag Dhat psi = eta for every right-hand side, starting from psi = 0.
    ``op`` provides normal / dot_local / axpby / copy / new_field over the
    local parts; ``comm.allreduce`` makes each scalar product global.  Stops
    when every right-hand side's recursive residual is below res ||eta||,
    then recomputes the true residual.  Returns one status dict per rhs."""
    n = op.nrhs
    gdot = lambda a, b: comm.allreduce(op.dot_local(a, b))  # noqa: E731
    r, p, q = op.new_field(), op.new_field(), op.new_field()
    zero, one = [0.0] * n, [1.0] * n
    op.axpby(zero, etas, zero, psis)           # psi = 0
    op.copy(etas, r)
    op.copy(etas, p)
    rr = gdot(r, r).real
    eta_n = np.sqrt(rr)
    live = eta_n > 0
    steps = np.zeros(n, dtype=int)
    for _ in range(nmx):
        if not live.any():
            break
        op.normal(p, q)
        pq = gdot(p, q).real
        alpha = np.where(live & (pq > 0), rr / np.where(pq > 0, pq, 1.0), 0.0)
        op.axpby(alpha, p, one, psis)
        op.axpby(-alpha, q, one, r)
        rr_new = gdot(r, r).real
        steps += live
        live = live & (np.sqrt(rr_new) > res * eta_n)
        beta = np.where(live, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        op.axpby(one, r, beta, p)
        rr = rr_new
    # true residual eta - A psi
    op.normal(psis, q)
    op.copy(etas, r)
    op.axpby([-1.0] * n, q, one, r)
    true = np.sqrt(gdot(r, r).real) / np.where(eta_n > 0, eta_n, 1.0)
    return [{"steps": int(steps[k]), "true_rel_res": float(true[k]), "converged": bool(true[k] <= res)}
            for k in range(n)]
