"""Thin ctypes binding of the C ABI in ``include/oq.h``.

Only argument marshalling happens here: every step of every operator and
solver runs in ``liboq.so``.  Device buffers are torch tensors (PyTorch is
used for memory and streams only); a tensor is passed by its data pointer
and the current torch CUDA stream is passed as the library's stream.

The shared library is loaded on first use.  If it has not been built the
load raises: there is no fallback to any other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liboq.so")

F64, F32, BF16, F16, DF64 = 0, 1, 2, 3, 4
LINK_18, LINK_12 = 0, 1
EVEN, ODD, FULL = 0, 1, 2
PREC = {"fp64": F64, "fp32": F32, "bf16": BF16, "fp16": F16, "df64": DF64}
OPT_DF64_RESETS, OPT_TEST_TC_SKIP_MMA, OPT_NN_TENSOR_CORES, OPT_SAP_KERNEL, OPT_HISTORY = 1, 2, 3, 4, 5

BC_HALO = 2   # bc_t of a time-split sub-domain

OK = 0
ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_NONFINITE, ERR_NOCONV, ERR_STATE = -1, -2, -3, -4, -5, -6, -7


class OqLattice(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("bc_t", C.c_int), ("cstar", C.c_int)]


class OqSolverParams(C.Structure):
    _fields_ = [
        ("res", C.c_double), ("nmx", C.c_int), ("nkv", C.c_int), ("ncy", C.c_int), ("nmr", C.c_int),
        ("bs", C.c_int * 4), ("sdtype", C.c_int), ("delta", C.c_double), ("adaptive", C.c_int),
        ("alpha", C.c_double), ("nladder", C.c_int), ("ladder", C.c_int * 4), ("ladder_c", C.c_double),
        ("sap_eo", C.c_int),
    ]


class OqCloverParams(C.Structure):
    _fields_ = [("kappa", C.c_double), ("csw", C.c_double), ("cF", C.c_double), ("csw_qed", C.c_double),
                ("qed_split", C.c_int)]


class OqStatus(C.Structure):
    _fields_ = [("steps", C.c_int), ("resets", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("true_rel_res", C.c_double), ("cycles", C.c_int), ("mr_avg", C.c_double),
                ("ladder_steps", C.c_int * 4), ("nn_fallback", C.c_int)]


class OqHalo(C.Structure):
    _fields_ = [("from_next", C.c_void_p), ("from_prev", C.c_void_p), ("sign_next", C.c_double),
                ("sign_prev", C.c_double)]


class OqKernelTime(C.Structure):
    _fields_ = [("mode", C.c_int), ("epi", C.c_int), ("prec", C.c_int), ("launches", C.c_int),
                ("total_ms", C.c_double), ("bytes", C.c_double), ("nr", C.c_int), ("link_fmt", C.c_int),
                ("dag", C.c_int), ("gated_launches", C.c_int), ("gated_ms", C.c_double),
                ("rhs_launches", C.c_longlong)]


_lib = None

# name -> (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "oq_create": (C.c_int, [C.POINTER(_P), C.POINTER(OqLattice), C.c_int]),
    "oq_destroy": (C.c_int, [_P]),
    "oq_error_string": (C.c_char_p, [C.c_int]),
    "oq_spinor_bytes": (C.c_size_t, [_P, C.c_int, C.c_int, C.c_int]),
    "oq_gauge_upload": (C.c_int, [_P, C.c_int, _P, C.c_int, _P]),
    "oq_clover_build": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, _P]),
    "oq_gauge_upload_qed": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, _P]),
    "oq_clover_build_ex": (C.c_int, [_P, C.c_int, C.POINTER(OqCloverParams), _P]),
    "oq_spinor_pack": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_double, C.c_int, _P]),
    "oq_spinor_unpack": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_double, C.c_int, _P]),
    "oq_dw_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, _P]),
    "oq_dw_hat_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, _P]),
    "oq_dw_hat_apply_noalloc": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, _P]),
    "oq_norm2": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int, C.POINTER(C.c_double), _P]),
    "oq_dot": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, C.POINTER(C.c_double), _P]),
    "oq_cgne_solve": (C.c_int, [_P, C.c_int, C.POINTER(OqSolverParams), _P, _P, C.c_int,
                                C.POINTER(OqStatus), _P]),
    "oq_cgne_solve_even": (C.c_int, [_P, C.c_int, C.POINTER(OqSolverParams), _P, _P, C.c_int,
                                     C.POINTER(OqStatus), _P]),
    "oq_sap_gcr_solve": (C.c_int, [_P, C.c_int, C.POINTER(OqSolverParams), _P, _P, C.c_int,
                                   C.POINTER(OqStatus), _P]),
    "oq_sap_apply": (C.c_int, [_P, C.c_int, C.POINTER(OqSolverParams), _P, _P, C.c_double, _P]),
    "oq_cgne_solve_batch": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(OqSolverParams),
                                      C.POINTER(_P), C.POINTER(_P), C.POINTER(OqStatus), _P]),
    "oq_nnprec_apply": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "oq_nnprec_apply_tc": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "oq_nnprec_grad": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int, _P, C.POINTER(C.c_double), _P]),
    "oq_nnprec_train": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int, C.c_double, C.c_int,
                                  C.POINTER(C.c_double), _P]),
    "oq_nn_gcr_solve": (C.c_int, [_P, C.c_int, C.POINTER(OqSolverParams), _P, _P, _P, C.c_int,
                                  C.POINTER(OqStatus), _P]),
    "oq_set_option": (C.c_int, [_P, C.c_int, C.c_int]),
    "oq_autotune": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P]),
    "oq_tune_get": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int)]),
    "oq_tune_get_epi": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "oq_tune_set": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                              C.c_int]),
    "oq_gauge_upload_halo": (C.c_int, [_P, C.c_int, _P, C.c_int, _P]),
    "oq_face_bytes": (C.c_size_t, [_P, C.c_int, C.c_int]),
    "oq_face_pack": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int, C.c_int, _P, _P, _P]),
    "oq_dw_apply_halo": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, C.POINTER(OqHalo), _P]),
    "oq_dhat_pass": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int, C.POINTER(OqHalo), _P]),
    "oq_axpby": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), _P, C.POINTER(C.c_double), _P,
                           C.c_int, _P]),
    "oq_solve_history": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
    "oq_profile_start": (C.c_int, [_P]),
    "oq_kernel_launches": (C.c_longlong, [_P]),
    "oq_profile_stop": (C.c_int, [_P, C.POINTER(OqKernelTime), C.c_int, C.POINTER(C.c_int)]),
}


def lib():
    """Load liboq.so (once).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2202_07388_gb300.build.build() "
                               "(the CUDA library is required, there is no fallback)")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(handle, name)
            f.restype = res
            f.argtypes = args
        _lib = handle
    return _lib


def exported_symbols():
    return list(_SIGS)


class OqError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lib().oq_error_string(code).decode()} ({code})")


def _check(code, where):
    if code != OK:
        raise OqError(code, where)
    return code


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class SolverParams:
    res: float = 1e-10
    nmx: int = 10000
    nkv: int = 16
    ncy: int = 4
    nmr: int = 5
    bs: tuple = (4, 4, 4, 4)
    sdtype: int = F32
    delta: float = 0.0
    adaptive: int = 0
    alpha: float = 0.9
    ladder: tuple = ()        # CGNE precision ladder, e.g. (F16, F32, F64); () = sdtype throughout
    ladder_c: float = 0.0     # switch constant (x eps of the current type); <= 0: 1
    sap_eo: int = 0           # SAP block solver on the even-odd Schur complement

    def c(self):
        p = OqSolverParams()
        p.res, p.nmx, p.nkv, p.ncy, p.nmr = self.res, self.nmx, self.nkv, self.ncy, self.nmr
        for k in range(4):
            p.bs[k] = self.bs[k]
        p.sdtype, p.delta, p.adaptive, p.alpha = self.sdtype, self.delta, self.adaptive, self.alpha
        if len(self.ladder) > 4:
            raise ValueError("a precision ladder has at most 4 types")
        p.nladder = len(self.ladder)
        for k, t in enumerate(self.ladder):
            p.ladder[k] = t
        p.ladder_c = self.ladder_c
        p.sap_eo = self.sap_eo
        return p


def status_dict(s: OqStatus) -> dict:
    return {"steps": s.steps, "resets": s.resets, "restarts": s.restarts, "converged": bool(s.converged),
            "true_rel_res": s.true_rel_res, "cycles": s.cycles, "mr_avg": s.mr_avg,
            "ladder_steps": list(s.ladder_steps), "nn_fallback": s.nn_fallback}


class Handle:
    """One library handle over one or more lattices (``dims`` tuples)."""

    def __init__(self, lattices, bc_t=-1, cstar=0):
        """cstar: C* boundaries in that many spatial directions; the handle's
        fields then live on the lattice doubled in x1 (self.dims holds it)."""
        if isinstance(lattices[0], int):
            lattices = [lattices]
        n = len(lattices)
        arr = (OqLattice * n)()
        for k, d in enumerate(lattices):
            for mu in range(4):
                arr[k].L[mu] = int(d[mu])
            arr[k].bc_t = bc_t
            arr[k].cstar = cstar
        h = C.c_void_p()
        _check(lib().oq_create(C.byref(h), arr, n), "oq_create")
        self.h = h
        self.dims = [tuple(int(v) * (2 if (cstar and mu == 1) else 1) for mu, v in enumerate(d)) for d in lattices]

    def close(self):
        if self.h:
            lib().oq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # sizes -------------------------------------------------------------
    def spinor_bytes(self, prec, subset=FULL, lat=0):
        return int(lib().oq_spinor_bytes(self.h, lat, prec, subset))

    def new_packed(self, prec, subset=FULL, nrhs=1, lat=0):
        import torch
        n = self.spinor_bytes(prec, subset, lat) * nrhs
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    # setup -------------------------------------------------------------
    def gauge_upload(self, u_dev, link_fmt=LINK_12, lat=0, stream=None):
        _check(lib().oq_gauge_upload(self.h, lat, _ptr(u_dev), link_fmt, _stream(stream)), "oq_gauge_upload")

    def gauge_upload_qed(self, u_dev, a_dev, q, lat=0, stream=None):
        """SU(3) links and U(1) potential A_mu(x) with charge q (U(3) hopping links)."""
        _check(lib().oq_gauge_upload_qed(self.h, lat, _ptr(u_dev), _ptr(a_dev), q, _stream(stream)),
               "oq_gauge_upload_qed")

    def clover_build(self, kappa, csw, lat=0, stream=None, cF=None, csw_qed=None):
        """cF: Schroedinger-functional boundary coefficient; csw_qed: separate
        coefficient of the U(1) field strength (after gauge_upload_qed)."""
        if cF is None and csw_qed is None:
            _check(lib().oq_clover_build(self.h, lat, kappa, csw, _stream(stream)), "oq_clover_build")
            return
        p = OqCloverParams(kappa, csw, 1.0 if cF is None else cF, 0.0 if csw_qed is None else csw_qed,
                           0 if csw_qed is None else 1)
        _check(lib().oq_clover_build_ex(self.h, lat, C.byref(p), _stream(stream)), "oq_clover_build_ex")

    # layouts -----------------------------------------------------------
    def pack(self, canon_dev, packed_dev, prec, subset=FULL, scale=1.0, nrhs=1, lat=0, stream=None):
        _check(lib().oq_spinor_pack(self.h, lat, prec, subset, _ptr(canon_dev), _ptr(packed_dev), scale, nrhs,
                                    _stream(stream)), "oq_spinor_pack")

    def unpack(self, packed_dev, canon_dev, prec, subset=FULL, scale=1.0, nrhs=1, lat=0, stream=None):
        _check(lib().oq_spinor_unpack(self.h, lat, prec, subset, _ptr(packed_dev), _ptr(canon_dev), scale, nrhs,
                                      _stream(stream)), "oq_spinor_unpack")

    # operators ---------------------------------------------------------
    def dw(self, in_dev, out_dev, prec, nrhs=1, dagger=False, lat=0, stream=None):
        _check(lib().oq_dw_apply(self.h, lat, prec, _ptr(in_dev), _ptr(out_dev), nrhs, int(dagger),
                                 _stream(stream)), "oq_dw_apply")

    def dw_hat(self, in_dev, out_dev, prec, nrhs=1, dagger=False, lat=0, stream=None):
        _check(lib().oq_dw_hat_apply(self.h, lat, prec, _ptr(in_dev), _ptr(out_dev), nrhs, int(dagger),
                                     _stream(stream)), "oq_dw_hat_apply")

    def norm2(self, x_dev, prec, subset=FULL, nrhs=1, lat=0, stream=None):
        out = (C.c_double * nrhs)()
        _check(lib().oq_norm2(self.h, lat, prec, subset, _ptr(x_dev), nrhs, out, _stream(stream)), "oq_norm2")
        return np.array(out[:])

    def dot(self, x_dev, y_dev, prec, subset=FULL, nrhs=1, lat=0, stream=None):
        out = (C.c_double * (2 * nrhs))()
        _check(lib().oq_dot(self.h, lat, prec, subset, _ptr(x_dev), _ptr(y_dev), nrhs, out, _stream(stream)),
               "oq_dot")
        v = np.array(out[:])
        return v[0::2] + 1j * v[1::2]

    # time-split sub-domains ------------------------------------------
    def gauge_upload_halo(self, u_ext_dev, link_fmt=LINK_12, lat=0, stream=None):
        """Links of T_loc + 2 slices (one beyond each face) of a sub-domain lattice."""
        _check(lib().oq_gauge_upload_halo(self.h, lat, _ptr(u_ext_dev), link_fmt, _stream(stream)),
               "oq_gauge_upload_halo")

    def face_bytes(self, prec, lat=0):
        return int(lib().oq_face_bytes(self.h, lat, prec))

    def new_faces(self, prec, nrhs=1, parities=1, lat=0):
        import torch
        return torch.empty(self.face_bytes(prec, lat) * nrhs * parities, dtype=torch.uint8, device="cuda")

    def face_pack(self, in_dev, to_prev, to_next, prec, subset, nrhs=1, dagger=False, lat=0, stream=None):
        _check(lib().oq_face_pack(self.h, lat, prec, subset, _ptr(in_dev), nrhs, int(dagger), _ptr(to_prev),
                                  _ptr(to_next), _stream(stream)), "oq_face_pack")

    @staticmethod
    def halo(from_next, from_prev, sign_next=1.0, sign_prev=1.0):
        return OqHalo(_ptr(from_next).value, _ptr(from_prev).value, float(sign_next), float(sign_prev))

    def dw_halo(self, in_dev, out_dev, prec, halo: OqHalo, nrhs=1, dagger=False, lat=0, stream=None):
        _check(lib().oq_dw_apply_halo(self.h, lat, prec, _ptr(in_dev), _ptr(out_dev), nrhs, int(dagger),
                                      C.byref(halo), _stream(stream)), "oq_dw_apply_halo")

    def dhat_pass(self, pass_, in_dev, in2_dev, out_dev, prec, halo=None, nrhs=1, dagger=False, lat=0,
                  stream=None, check=True):
        rc = lib().oq_dhat_pass(self.h, lat, prec, pass_, _ptr(in_dev), _ptr(in2_dev) if in2_dev is not None
                                else None, _ptr(out_dev), nrhs, int(dagger),
                                C.byref(halo) if halo is not None else None, _stream(stream))
        if check:
            _check(rc, "oq_dhat_pass")
        return rc

    def axpby(self, a, x_dev, b, y_dev, prec, subset=FULL, nrhs=1, lat=0, stream=None):
        """y = a x + b y per right-hand side (a, b: sequences of nrhs reals)."""
        av = (C.c_double * nrhs)(*[float(v) for v in a])
        bv = (C.c_double * nrhs)(*[float(v) for v in b])
        _check(lib().oq_axpby(self.h, lat, prec, subset, av, _ptr(x_dev), bv, _ptr(y_dev), nrhs, _stream(stream)),
               "oq_axpby")

    # solvers -----------------------------------------------------------
    def cgne(self, eta_dev, psi_dev, params: SolverParams, nrhs=1, lat=0, stream=None, check=True):
        st = (OqStatus * nrhs)()
        p = params.c()
        rc = lib().oq_cgne_solve(self.h, lat, C.byref(p), _ptr(eta_dev), _ptr(psi_dev), nrhs, st, _stream(stream))
        if check and rc not in (OK, ERR_NOCONV):
            _check(rc, "oq_cgne_solve")
        return rc, [status_dict(s) for s in st]

    def cgne_even(self, eta_dev, psi_dev, params: SolverParams, nrhs=1, lat=0, stream=None, check=True):
        """oq_cgne_solve on even-site canonical fields (V/2 sites each, index lex // 2)."""
        st = (OqStatus * nrhs)()
        p = params.c()
        rc = lib().oq_cgne_solve_even(self.h, lat, C.byref(p), _ptr(eta_dev), _ptr(psi_dev), nrhs, st,
                                      _stream(stream))
        if check and rc not in (OK, ERR_NOCONV):
            _check(rc, "oq_cgne_solve_even")
        return rc, [status_dict(s) for s in st]

    def cgne_batch(self, lats, etas, psis, params: SolverParams, stream=None, check=True):
        n = len(lats)
        la = (C.c_int * n)(*lats)
        ep = (_P * n)(*[t.data_ptr() for t in etas])
        pp = (_P * n)(*[t.data_ptr() for t in psis])
        st = (OqStatus * n)()
        p = params.c()
        rc = lib().oq_cgne_solve_batch(self.h, n, la, C.byref(p), ep, pp, st, _stream(stream))
        if check and rc not in (OK, ERR_NOCONV):
            _check(rc, "oq_cgne_solve_batch")
        return rc, [status_dict(s) for s in st]

    def sap_gcr(self, eta_dev, psi_dev, params: SolverParams, nrhs=1, lat=0, stream=None, check=True):
        st = (OqStatus * nrhs)()
        p = params.c()
        rc = lib().oq_sap_gcr_solve(self.h, lat, C.byref(p), _ptr(eta_dev), _ptr(psi_dev), nrhs, st,
                                    _stream(stream))
        if check and rc not in (OK, ERR_NOCONV):
            _check(rc, "oq_sap_gcr_solve")
        return rc, [status_dict(s) for s in st]

    # learned preconditioner -------------------------------------------
    def nnprec_apply(self, weights, in_packed, out_packed, lat=0, stream=None):
        _check(lib().oq_nnprec_apply(self.h, lat, _ptr(weights), _ptr(in_packed), _ptr(out_packed),
                                     _stream(stream)), "oq_nnprec_apply")

    def nnprec_apply_tc(self, weights, in_packed, out_packed, lat=0, stream=None):
        _check(lib().oq_nnprec_apply_tc(self.h, lat, _ptr(weights), _ptr(in_packed), _ptr(out_packed),
                                        _stream(stream)), "oq_nnprec_apply_tc")

    def nnprec_grad(self, weights, r_packed, e_packed, n, grad, lat=0, stream=None):
        loss = C.c_double()
        _check(lib().oq_nnprec_grad(self.h, lat, _ptr(weights), _ptr(r_packed), _ptr(e_packed), n, _ptr(grad),
                                    C.byref(loss), _stream(stream)), "oq_nnprec_grad")
        return loss.value

    def nnprec_train(self, weights, r_packed, e_packed, n, lr, steps, lat=0, stream=None):
        losses = (C.c_double * steps)()
        _check(lib().oq_nnprec_train(self.h, lat, _ptr(weights), _ptr(r_packed), _ptr(e_packed), n, lr, steps,
                                     losses, _stream(stream)), "oq_nnprec_train")
        return np.array(losses[:])

    def nn_gcr(self, weights, eta_dev, psi_dev, params: SolverParams, nrhs=1, lat=0, stream=None, check=True):
        st = (OqStatus * nrhs)()
        p = params.c()
        rc = lib().oq_nn_gcr_solve(self.h, lat, C.byref(p), _ptr(weights), _ptr(eta_dev), _ptr(psi_dev), nrhs,
                                   st, _stream(stream))
        if check and rc not in (OK, ERR_NOCONV):
            _check(rc, "oq_nn_gcr_solve")
        return rc, [status_dict(s) for s in st]

    def sap_apply(self, rho_packed, phi_packed, params: SolverParams, mr_tol=0.0, lat=0, stream=None):
        p = params.c()
        _check(lib().oq_sap_apply(self.h, lat, C.byref(p), _ptr(rho_packed), _ptr(phi_packed), mr_tol,
                                  _stream(stream)), "oq_sap_apply")

    def set_option(self, key, value):
        _check(lib().oq_set_option(self.h, key, int(value)), "oq_set_option")

    def solve_history(self, rhs=0):
        """Diagnostics of the last CGNE solve run with OPT_HISTORY: (recursive, resets) for one
        right-hand side, recursive[k-1] = ||r_rec|| / ||eta|| after regular step k, resets an
        (n, 2) array of (steps before the reset, relative residual of the reset)."""
        import numpy as np
        n = C.c_int()
        _check(lib().oq_solve_history(self.h, rhs, 0, None, 0, C.byref(n)), "oq_solve_history")
        rec = np.zeros(n.value)
        _check(lib().oq_solve_history(self.h, rhs, 0, rec.ctypes.data_as(C.POINTER(C.c_double)), n.value,
                                      C.byref(n)), "oq_solve_history")
        _check(lib().oq_solve_history(self.h, rhs, 1, None, 0, C.byref(n)), "oq_solve_history")
        rst = np.zeros(2 * n.value)
        _check(lib().oq_solve_history(self.h, rhs, 1, rst.ctypes.data_as(C.POINTER(C.c_double)), 2 * n.value,
                                      C.byref(n)), "oq_solve_history")
        return rec, rst.reshape(-1, 2)

    # tuning ------------------------------------------------------------
    def autotune(self, prec, nrhs=1, lat=0, stream=None):
        """Tune the stencil launches of (lat, prec, nrhs); returns per mode (0 Dw, 1 Dhat pass 1,
        2 Dhat pass 2) the chosen (bx, by, ms, link format, rhs per thread, register cap)."""
        _check(lib().oq_autotune(self.h, lat, prec, nrhs, _stream(stream)), "oq_autotune")
        return {mode: self.tune_get(prec, mode, nrhs, lat) for mode in (0, 1, 2)}

    def tuned_epilogues(self, prec, nrhs=1, lat=0):
        """Pass 2's chosen launch per epilogue (store, norm, cg) after autotune."""
        return {name: self.tune_get(prec, 2, nrhs, lat, epi) for epi, name in enumerate(("store", "norm", "cg"))}

    def tune_get(self, prec, mode, nrhs=1, lat=0, epi=0):
        """The launch chosen for (prec, mode, nrhs); for pass 2 (mode 2) per epilogue
        (epi 0 store, 1 store and norm, 2 CGNE update)."""
        bx, by, ms, fmt, nr, cap = C.c_int(), C.c_int(), C.c_float(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().oq_tune_get_epi(self.h, lat, prec, mode, epi, nrhs, C.byref(bx), C.byref(by), C.byref(ms),
                                     C.byref(fmt), C.byref(nr), C.byref(cap)), "oq_tune_get_epi")
        return (bx.value, by.value, ms.value, "12-real" if fmt.value == LINK_12 else "18-real", nr.value, cap.value)

    def tune_set(self, prec, mode, nrhs, bx, by, nr=1, regcap=0, link_fmt=-1, lat=0, check=True):
        rc = lib().oq_tune_set(self.h, lat, prec, mode, nrhs, bx, by, nr, regcap, link_fmt)
        if check:
            _check(rc, "oq_tune_set")
        return rc

    # instrumentation ---------------------------------------------------
    def profile_start(self):
        _check(lib().oq_profile_start(self.h), "oq_profile_start")

    def kernel_launches(self):
        return int(lib().oq_kernel_launches(self.h))

    def profile_stop(self):
        buf = (OqKernelTime * 64)()
        n = C.c_int()
        _check(lib().oq_profile_stop(self.h, buf, 64, C.byref(n)), "oq_profile_stop")
        return [{"mode": b.mode, "epi": b.epi, "prec": b.prec, "launches": b.launches, "total_ms": b.total_ms,
                 "bytes": b.bytes, "nr": b.nr, "link_fmt": b.link_fmt, "dag": b.dag,
                 "gated_launches": b.gated_launches, "gated_ms": b.gated_ms, "rhs_launches": b.rhs_launches}
                for b in buf[: n.value]]
