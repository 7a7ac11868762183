"""The learned preconditioner on the GPU: forward layers and gradients
against the FP64 oracle (with the same bfloat16-rounded weights), and the
gain tests: a network trained on the GPU (own forward/backward kernels, Adam)
on (residual, error) pairs from the binary64 solver lowers its loss, cuts
the flexible-GCR step count relative to GCR without it, and reaches the
target residual in less time than SAP-GCR, its fallback and judge."""
import numpy as np
import pytest

from oracle import dirac, ptc
from paper_2202_07388_gb300 import synth
from tests.gpu_cases import oracle_case, make_handle, to_dev, from_dev, rel_err, check_residual

pytestmark = pytest.mark.gpu

NW1 = 9 * 2 * 1 * 16
NW2 = 9 * 1 * 2 * 16


def _bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _weights(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal(2 * (NW1 + NW2)) * scale).astype(np.float32)
    return w


def _split(w32):
    """binary32 master (re, im interleaved) -> oracle complex arrays of the bf16-rounded weights."""
    wr = _bf16(w32).astype(np.float64)
    c = wr[0::2] + 1j * wr[1::2]
    return c[:NW1].reshape(9, 2, 1, 4, 4), c[NW1:].reshape(9, 1, 2, 4, 4)


def _wdev(w32):
    import torch
    return torch.from_numpy(w32.copy()).cuda()


def _packed(h, oq, fields):
    import torch
    n = fields.shape[0]
    out = h.new_packed(oq.F32, nrhs=n)
    h.pack(to_dev(fields), out, oq.F32, nrhs=n)
    return out


@pytest.mark.parametrize("link_fmt", [0, 1])
def test_ptc_forward_matches_oracle(link_fmt):
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 2, 6)
    u, a, ainv = oracle_case(dims, 0.6, 81, 0.135, 1.0)
    h = make_handle(dims, u, 0.135, 1.0, link_fmt)
    w = _weights(82)
    w1, w2 = _split(w)
    psi = synth.make_source(dims, 83)
    ref, _ = ptc.forward(u, w1, w2, psi)
    pin = _packed(h, oq, psi[None])
    pout = h.new_packed(oq.F32)
    h.nnprec_apply(_wdev(w), pin, pout)
    out = to_dev(np.zeros_like(psi))
    h.unpack(pout, out, oq.F32)
    assert rel_err(from_dev(out, psi.shape), ref) < 1e-5


@pytest.mark.parametrize("dims,link_fmt", [((4, 4, 2, 6), 0), ((4, 4, 2, 6), 1), ((8, 8, 4, 8), 1)])
def test_ptc_tensor_core_forward_matches_oracle(dims, link_fmt):
    """tcgen05 channel contraction (bfloat16 operands, binary32 accumulation
    in tensor memory): 1e-2 relative, from rounding the transported inputs
    and the hidden fields to bfloat16; V = 192 leaves a ragged 128-site tile."""
    from paper_2202_07388_gb300 import oq
    u, a, ainv = oracle_case(dims, 0.6, 81, 0.135, 1.0)
    h = make_handle(dims, u, 0.135, 1.0, link_fmt)
    w = _weights(87)
    w1, w2 = _split(w)
    psi = synth.make_source(dims, 88)
    ref, _ = ptc.forward(u, w1, w2, psi)
    pin = _packed(h, oq, psi[None])
    pout, pcc = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.nnprec_apply_tc(_wdev(w), pin, pout)
    h.nnprec_apply(_wdev(w), pin, pcc)
    out, occ = to_dev(np.zeros_like(psi)), to_dev(np.zeros_like(psi))
    h.unpack(pout, out, oq.F32)
    h.unpack(pcc, occ, oq.F32)
    got = from_dev(out, psi.shape)
    assert rel_err(got, ref) < 1e-2
    assert rel_err(got, from_dev(occ, psi.shape)) < 1e-2


def test_ptc_gradient_matches_oracle():
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (4, 4, 2, 6)
    u, a, ainv = oracle_case(dims, 0.6, 81, 0.135, 1.0)
    h = make_handle(dims, u, 0.135, 1.0, oq.LINK_12)
    w = _weights(84)
    w1, w2 = _split(w)
    n = 2
    r = synth.make_source(dims, 85, nrhs=n)
    e = synth.make_source(dims, 86, nrhs=n)
    # oracle: mean loss and gradient over the pairs (inputs rounded to binary32 as the GPU sees them)
    r32 = r.astype(np.complex64).astype(np.complex128)
    e32 = e.astype(np.complex64).astype(np.complex128)
    loss, g1, g2 = 0.0, 0.0, 0.0
    for k in range(n):
        lk, a1, a2 = ptc.backward(u, w1, w2, r32[k], e32[k])
        loss += lk / n
        g1 = g1 + a1 / n
        g2 = g2 + a2 / n
    grad = torch.zeros(2 * (NW1 + NW2), dtype=torch.float64, device="cuda")
    gl = h.nnprec_grad(_wdev(w), _packed(h, oq, r), _packed(h, oq, e), n, grad)
    gg = grad.cpu().numpy()
    gc = gg[0::2] + 1j * gg[1::2]
    assert abs(gl - loss) < 1e-5 * loss
    assert rel_err(gc[:NW1].reshape(g1.shape), g1) < 1e-4
    assert rel_err(gc[NW1:].reshape(g2.shape), g2) < 1e-4


def test_trained_network_cuts_gcr_steps():
    import torch
    from paper_2202_07388_gb300 import oq
    dims = (8, 8, 8, 8)
    kappa = 0.1365
    u, a, ainv = oracle_case(dims, 0.5, 91, kappa, 1.0)
    h = make_handle(dims, u, kappa, 1.0, oq.LINK_12)
    # training pairs from the binary64 solver: e = D^-1 r
    ntrain = 12
    r = synth.make_source(dims, 92, nrhs=ntrain)
    e = np.zeros_like(r)
    prm = oq.SolverParams(res=1e-10, nmx=2000, nkv=16, ncy=4, nmr=5, bs=(4, 4, 4, 4), sdtype=oq.F32)
    for k in range(ntrain):
        psi = to_dev(np.zeros_like(r[k]))
        rc, _ = h.sap_gcr(to_dev(r[k]), psi, prm)
        assert rc == oq.OK
        e[k] = from_dev(psi, r[k].shape)
    # start: M = identity / (4 + m0) on the direct path, small random elsewhere
    w = _weights(93, scale=0.01)
    c0 = 1.0 / (2 * kappa)
    wc = w[0::2] + 1j * w[1::2]
    W1 = wc[:NW1].reshape(9, 2, 1, 4, 4)
    W2 = wc[NW1:].reshape(9, 1, 2, 4, 4)
    W1[0, 0, 0] += np.eye(4)
    W2[0, 0, 0] += np.eye(4) / c0
    wc = np.concatenate([W1.reshape(-1), W2.reshape(-1)])
    w = np.empty(2 * wc.size, np.float32)
    w[0::2], w[1::2] = wc.real, wc.imag
    wd = _wdev(w)
    rp, ep = _packed(h, oq, r), _packed(h, oq, e)
    losses = h.nnprec_train(wd, rp, ep, ntrain, 0.01, 150)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0]
    # held-out source: flexible GCR with the trained network vs without it
    eta = synth.make_source(dims, 99)
    gprm = oq.SolverParams(res=1e-10, nmx=2000, nkv=16, ncy=0, sdtype=oq.F32)
    psi0 = to_dev(np.zeros_like(eta))
    rc0, st0 = h.sap_gcr(to_dev(eta), psi0, gprm)
    psi1 = to_dev(np.zeros_like(eta))
    rc1, st1 = h.nn_gcr(wd, to_dev(eta), psi1, gprm)
    assert rc0 == oq.OK and rc1 == oq.OK
    x = from_dev(psi1, eta.shape)
    res = np.linalg.norm(eta - dirac.dw(u, a, x)) / np.linalg.norm(eta)
    check_residual(res, st1[0]["true_rel_res"])
    assert st1[0]["steps"] < st0[0]["steps"]     # binary32 CUDA-core network (default)
    h.set_option(oq.OPT_NN_TENSOR_CORES, 1)
    psi2 = to_dev(np.zeros_like(eta))
    rc2, st2 = h.nn_gcr(wd, to_dev(eta), psi2, gprm)
    assert rc2 == oq.OK and st2[0]["steps"] < st0[0]["steps"]   # tcgen05 network
    x2 = from_dev(psi2, eta.shape)
    check_residual(np.linalg.norm(eta - dirac.dw(u, a, x2)) / np.linalg.norm(eta), st2[0]["true_rel_res"])


def _timed_min(fn, reps=3):
    """Best of reps CUDA-event timings of fn() on the current stream (ms) and its last result."""
    import torch
    best, out = None, None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best, out


def test_trained_network_against_sap_gcr():
    """The comparison the learned preconditioner is judged by: on a 16^4
    lattice at kappa = 0.1365 a network trained on the GPU (12 pairs from the
    binary64 SAP-GCR solver, 150 Adam steps) preconditions flexible GCR, and
    SAP-GCR with the Table 2 style settings (4^4 blocks, 5 MR steps, 4
    cycles, 16 Krylov vectors) solves the same held-out source.  Both reach a
    binary64 residual of 1e-10 (recomputed by the oracle and equal to the
    reported one within 1e-3 relative); the network keeps the whole solve (no
    fallback to SAP) and reaches the target in less time than SAP-GCR."""
    from paper_2202_07388_gb300 import oq
    dims = (16, 16, 16, 16)
    kappa = 0.1365
    u, a, ainv = oracle_case(dims, 0.5, 191, kappa, 1.0)
    h = make_handle(dims, u, kappa, 1.0, oq.LINK_12)
    for p in (oq.F32, oq.F64):
        h.autotune(p, nrhs=1)
    sap = oq.SolverParams(res=1e-10, nmx=2000, nkv=16, ncy=4, nmr=5, bs=(4, 4, 4, 4), sdtype=oq.F32)
    ntrain = 12
    r = synth.make_source(dims, 192, nrhs=ntrain)
    e = np.zeros_like(r)
    for k in range(ntrain):
        psi = to_dev(np.zeros_like(r[k]))
        rc, _ = h.sap_gcr(to_dev(r[k]), psi, sap)
        assert rc == oq.OK
        e[k] = from_dev(psi, r[k].shape)
    wc = np.zeros(NW1 + NW2, complex)
    W1 = wc[:NW1].reshape(9, 2, 1, 4, 4)
    W2 = wc[NW1:].reshape(9, 1, 2, 4, 4)
    W1[0, 0, 0] = np.eye(4)
    W2[0, 0, 0] = np.eye(4) * (2 * kappa)
    w = np.empty(2 * wc.size, np.float32)
    w[0::2], w[1::2] = wc.real, wc.imag
    wd = _wdev(w)
    losses = h.nnprec_train(wd, _packed(h, oq, r), _packed(h, oq, e), ntrain, 0.01, 150)
    assert losses[-1] < 0.8 * losses[0]
    eta = synth.make_source(dims, 199)
    plain = oq.SolverParams(res=1e-10, nmx=2000, nkv=16, ncy=0, sdtype=oq.F32)
    results = {}
    for name, run in (("nn_gcr", lambda x: h.nn_gcr(wd, to_dev(eta), x, plain)),
                      ("sap_gcr", lambda x: h.sap_gcr(to_dev(eta), x, sap))):
        x = to_dev(np.zeros_like(eta))
        ms, (rc, st) = _timed_min(lambda: run(x))
        assert rc == oq.OK and st[0]["converged"], name
        xs = from_dev(x, eta.shape)
        res = np.linalg.norm(eta - dirac.dw(u, a, xs)) / np.linalg.norm(eta)
        assert res <= 1e-10 * (1 + 1e-3) and abs(res - st[0]["true_rel_res"]) <= 1e-3 * res, name
        results[name] = (ms, st[0])
    assert results["nn_gcr"][1]["nn_fallback"] == 0
    assert results["nn_gcr"][0] < results["sap_gcr"][0], results
    h.close()


def _direct_path_network(w1, w2):
    """Weights with only the identity path: M = w2 w1 (4x4 spin matrices)."""
    w = np.zeros(2 * (NW1 + NW2), np.float32)
    wc = w[0::2] + 1j * w[1::2]
    W1 = wc[:NW1].reshape(9, 2, 1, 4, 4)
    W2 = wc[NW1:].reshape(9, 1, 2, 4, 4)
    W1[0, 0, 0] = w1
    W2[0, 0, 0] = w2
    wc = np.concatenate([W1.reshape(-1), W2.reshape(-1)])
    w[0::2], w[1::2] = wc.real, wc.imag
    return _wdev(w)


def test_useless_network_falls_back_to_sap():
    """A network whose output lies in half of the space (M = the projector
    on the upper chirality): D M spans half the space, so a restart cycle
    cannot halve the residual of a Gaussian source (the rest keeps ~1/sqrt(2)
    of it); SAP takes over, the solve reaches 1e-10 and reports the fallback.
    M = 2 kappa (a scaled identity) keeps the network for the whole solve."""
    from paper_2202_07388_gb300 import oq
    dims = (8, 8, 8, 8)
    kappa = 0.1365
    u, a, ainv = oracle_case(dims, 0.5, 95, kappa, 1.0)
    h = make_handle(dims, u, kappa, 1.0, oq.LINK_12)
    eta = synth.make_source(dims, 96)
    gprm = oq.SolverParams(res=1e-10, nmx=2000, nkv=8, ncy=2, nmr=4, bs=(4, 4, 4, 4), sdtype=oq.F32)
    wd = _direct_path_network(np.diag([1.0, 1.0, 0.0, 0.0]), np.eye(4))
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.nn_gcr(wd, to_dev(eta), psi, gprm)
    assert rc == oq.OK and st[0]["converged"]
    assert st[0]["nn_fallback"] == 1 and st[0]["cycles"] > 0
    x = from_dev(psi, eta.shape)
    check_residual(np.linalg.norm(eta - dirac.dw(u, a, x)) / np.linalg.norm(eta), st[0]["true_rel_res"])
    psi = to_dev(np.zeros_like(eta))
    rc, st = h.nn_gcr(_direct_path_network(np.eye(4), np.eye(4) * (2 * kappa)), to_dev(eta), psi, gprm)
    assert rc == oq.OK and st[0]["nn_fallback"] == 0 and st[0]["cycles"] == 0
