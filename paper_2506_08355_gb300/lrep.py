"""ctypes binding of liblrep (include/lrep.h, include/lrep_ops.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Host arrays are numpy float64 (column-major blocks are
Fortran-ordered n x c arrays); device arrays are torch CUDA tensors laid
out as (c, ld) row-major, i.e. column j of the block is row j of the
tensor (``device_block``).  The library is loaded on first use; a missing
library raises RuntimeError (no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, NOT_CONVERGED = 0, 1
ERR = {-1: "ERR_ARG", -2: "ERR_NOMEM", -3: "ERR_CUDA", -4: "ERR_NOT_SPD",
       -5: "ERR_BREAKDOWN", -6: "ERR_TIMEOUT", -7: "ERR_STATE", -8: "ERR_CALLBACK"}
MEM_HOST, MEM_DEVICE_COPY, MEM_DEVICE_BORROW = 0, 1, 2
FORM_AB, FORM_KM = 0, 1
OP_K, OP_M, OP_B = 0, 1, 2
PREC_FP64, PREC_MIXED_BF16X3, PREC_FP64_SLICED, PREC_MIXED_SLICED = 0, 1, 2, 3
(Q_NCONV, Q_EIGVALS, Q_X, Q_Y, Q_U, Q_V, Q_RESID, Q_ITERS, Q_MATVECS, Q_TIMINGS,
 Q_BIORTH_ERR, Q_HISTORY, Q_REBIORTHS, Q_PROFILE, Q_PROFILE_CG, Q_PROFILE_CLASSES) = range(16)
PROFILE_CLASSES = ("prod_cg", "prod_f64", "gram", "update", "small", "cg_vec", "alg1", "other")


class Options(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("precision", C.c_int32),
                ("s", C.c_int32), ("ngs", C.c_int32), ("cg_maxit", C.c_int32),
                ("cg_tol", C.c_double), ("maxit", C.c_int32),
                ("discard_tol", C.c_double), ("seed", C.c_uint64),
                ("refresh_every", C.c_int32), ("rebiorth_tol", C.c_double),
                ("verbose", C.c_int32), ("profile", C.c_int32)]


APPLY_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.c_int64, C.c_int32,
                       C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p)

EXPORTS = {
    # name: (restype, argtypes)
    "lrep_default_options": (None, [C.POINTER(Options)]),
    "lrep_create_dense": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p]),
    "lrep_create_csr": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "lrep_create_stencil": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32,
                                      C.c_int32, C.c_double, C.c_double, C.c_void_p,
                                      C.c_void_p, C.c_int32, C.c_void_p]),
    "lrep_create_spectral": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32,
                                       C.c_int32, C.c_void_p, C.c_double, C.c_void_p,
                                       C.c_void_p, C.c_int32, C.c_void_p]),
    "lrep_create_operator": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, APPLY_FN,
                                       C.c_void_p, C.c_void_p]),
    "lrep_set_nullspace": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.c_int32]),
    "lrep_find_nullspace": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                      C.c_void_p, C.c_int64, C.c_int32,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lrep_set_mass_dense": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32]),
    "lrep_set_mass_csr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int32]),
    "lrep_set_mass_callback": (C.c_int, [C.c_void_p, C.c_int32]),
    "lrep_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "lrep_set_start": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_int32]),
    "lrep_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double]),
    "lrep_solve_begin": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double]),
    "lrep_solve_advance": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32)]),
    "lrep_query": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32]),
    "lrep_last_error": (C.c_char_p, [C.c_void_p]),
    "lrep_destroy": (C.c_int, [C.c_void_p]),
    "lrep_footprint": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
    "lrep_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int32, C.c_void_p]),
    "lrep_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                     C.c_double, C.POINTER(C.c_uint64)]),
    "lrep_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32]),
    "lrep_server_destroy": (C.c_int, [C.c_void_p]),
    "lrep_server_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lrep_op_gram_sliced": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                      C.c_void_p]),
    "lrep_op_update_sliced": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                        C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                        C.c_double, C.c_void_p, C.c_int64, C.c_void_p]),
    "lrep_op_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                C.c_void_p, C.c_int64]),
    "lrep_op_apply_cg": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.c_int64]),
    "lrep_op_cg": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                             C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                             C.POINTER(C.c_int32)]),
    "lrep_op_gram": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                               C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "lrep_op_update": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                 C.c_int64, C.c_void_p]),
    "lrep_op_small_lrep": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.POINTER(C.c_int32), C.c_void_p]),
    "lrep_op_biorth": (C.c_int, [C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_double, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.POINTER(C.c_int32), C.c_void_p]),
    "lrep_op_residuals": (C.c_int, [C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "lrep_op_philox_normal": (C.c_int, [C.c_int64, C.c_int32, C.c_uint64, C.c_int32,
                                        C.c_void_p, C.c_int64, C.c_void_p]),
    "lrep_launch_count": (C.c_int64, []),
    "lrep_op_gram_noalloc": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                       C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded liblrep (raises RuntimeError when it was not built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("liblrep.so is not built (%s); run "
                               "python -m paper_2506_08355_gb300.build" % path)
        L = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class LrepError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (ERR.get(status, status), msg))
        self.status = status


def _check(status, handle=None):
    if status < 0:
        msg = lib().lrep_last_error(handle)
        raise LrepError(status, msg.decode() if msg else "")
    return status


def default_options(**kw) -> Options:
    o = Options()
    lib().lrep_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ----------------------------------------------------------- array helpers


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _host_block(a):
    """Fortran float64 copy of a host block and its leading dimension."""
    a = np.asfortranarray(np.asarray(a, dtype=np.float64))
    if a.ndim == 1:
        a = a.reshape(-1, 1, order="F")
    return a, a.shape[0]


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def device_block(n, c, like=None):
    """Empty device block: torch tensor (c, n) whose row j is column j."""
    import torch
    dev = like.device if like is not None else "cuda"
    return torch.empty((c, n), dtype=torch.float64, device=dev)


def block_arg(a, n):
    """(pointer, ld, mem) of a block given as numpy (n x c) or torch (c, ld)."""
    if _is_torch(a):
        if a.dim() == 1:
            return _ptr(a), max(n, a.shape[0]), MEM_DEVICE_COPY
        assert a.stride(1) == 1, "device blocks are (c, ld) with unit row stride"
        return _ptr(a), a.stride(0) if a.shape[0] > 1 else max(n, a.shape[1]), MEM_DEVICE_COPY
    h, ld = _host_block(a)
    return h, ld, MEM_HOST


# ------------------------------------------------------------------ problem


class Problem:
    """One LREP instance (dense, CSR, stencil or callback operator)."""

    def __init__(self, handle, n, keep=()):
        self.h = handle
        self.n = n
        self._keep = list(keep)

    # constructors --------------------------------------------------------
    @classmethod
    def dense(cls, P1, P2, form=FORM_KM, borrow=False, stream=None):
        h = C.c_void_p()
        if _is_torch(P1):
            n = P1.shape[0]
            mem = MEM_DEVICE_BORROW if borrow else MEM_DEVICE_COPY
            st = lib().lrep_create_dense(C.byref(h), n, _ptr(P1), _ptr(P2), P1.stride(0),
                                         form, mem, _stream(stream))
            keep = (P1, P2) if borrow else ()
        else:
            a, ld = _host_block(P1)
            b, _ = _host_block(P2)
            n = a.shape[0]
            st = lib().lrep_create_dense(C.byref(h), n, _ptr(a), _ptr(b), ld, form,
                                         MEM_HOST, _stream(stream))
            keep = ()
        _check(st)
        return cls(h, n, keep)

    @classmethod
    def csr(cls, n, csr1, csr2, form=FORM_KM, stream=None):
        h = C.c_void_p()
        arrs = []
        for (rp, ci, va) in (csr1, csr2):
            arrs += [np.ascontiguousarray(rp, dtype=np.int64),
                     np.ascontiguousarray(ci, dtype=np.int32),
                     np.ascontiguousarray(va, dtype=np.float64)]
        st = lib().lrep_create_csr(C.byref(h), n, form, *[_ptr(a) for a in arrs],
                                   MEM_HOST, _stream(stream))
        _check(st)
        return cls(h, n)

    @classmethod
    def stencil(cls, nx, ny, nz, h_grid, lap_coef, dK, dM, stream=None):
        h = C.c_void_p()
        dk = np.ascontiguousarray(dK, dtype=np.float64)
        dm = np.ascontiguousarray(dM, dtype=np.float64)
        st = lib().lrep_create_stencil(C.byref(h), nx, ny, nz, h_grid, lap_coef,
                                       _ptr(dk), _ptr(dm), MEM_HOST, _stream(stream))
        _check(st)
        return cls(h, nx * ny * nz)

    @classmethod
    def spectral(cls, nx, ny, nz, lengths, lap_coef, dK, dM, stream=None):
        """Periodic Fourier spectral operator (lrep_create_spectral):
        K = lap_coef * Lap_F + diag(dK), M = lap_coef * Lap_F + diag(dM) on an
        nx*ny*nz grid of a box with side lengths ``lengths``."""
        h = C.c_void_p()
        L = np.ascontiguousarray(lengths, dtype=np.float64)
        if L.shape != (3,):
            raise ValueError("lengths must hold three box lengths")
        dk = np.ascontiguousarray(dK, dtype=np.float64)
        dm = np.ascontiguousarray(dM, dtype=np.float64)
        st = lib().lrep_create_spectral(C.byref(h), nx, ny, nz, _ptr(L), lap_coef,
                                        _ptr(dk), _ptr(dm), MEM_HOST, _stream(stream))
        _check(st)
        return cls(h, nx * ny * nz)

    @classmethod
    def operator(cls, n, fn, stream=None):
        """fn(op, ncols, X_ptr, ldx, Y_ptr, ldy, stream_ptr) -> int."""
        def tramp(user, op, nn, nc, X, ldx, Y, ldy, st):
            try:
                return int(fn(op, nc, X, ldx, Y, ldy, st) or 0)
            except Exception:  # reported as LREP_ERR_CALLBACK
                return 1
        cb = APPLY_FN(tramp)
        h = C.c_void_p()
        _check(lib().lrep_create_operator(C.byref(h), n, cb, None, _stream(stream)))
        return cls(h, n, keep=(cb,))

    # configuration -------------------------------------------------------
    def set_nullspace(self, X0, Y0=None):
        if X0 is None:
            _check(lib().lrep_set_nullspace(self.h, 0, None, None, self.n, MEM_HOST), self.h)
            return
        x, ldx, mem = block_arg(X0, self.n)
        r = x.shape[1] if not _is_torch(X0) else (X0.shape[0] if X0.dim() > 1 else 1)
        y = None
        if Y0 is not None:
            y, _, _ = block_arg(Y0, self.n)
        _check(lib().lrep_set_nullspace(self.h, r, _ptr(x), _ptr(y), ldx, mem), self.h)

    def find_nullspace(self, r_max=8, tol=1e-10, maxit=2000):
        """Basis of N(K) by LOBPCG on the GPU, installed as the nullspace;
        returns (X0 as an n x r numpy array, iterations)."""
        r, it = C.c_int32(), C.c_int32()
        out = np.zeros((max(r_max, 1), self.n), dtype=np.float64)
        _check(lib().lrep_find_nullspace(self.h, r_max, tol, maxit, _ptr(out), self.n, MEM_HOST,
                                         C.byref(r), C.byref(it)), self.h)
        return out[: r.value].T.copy(), it.value

    def set_mass(self, Bm=None, borrow=False):
        """Mass matrix B of the generalized LREP: a dense (n, n) array or
        device tensor for dense problems, a CSR triple for CSR problems,
        True for a callback problem (the callback is asked for op OP_B);
        None clears it."""
        L = lib()
        if isinstance(Bm, bool):
            _check(L.lrep_set_mass_callback(self.h, int(Bm)), self.h)
        elif Bm is None:
            st = L.lrep_set_mass_dense(self.h, None, self.n, MEM_HOST)
            if st < 0:
                st = L.lrep_set_mass_csr(self.h, None, None, None, MEM_HOST)
            _check(st, self.h)
        elif isinstance(Bm, tuple):
            rp, ci, va = (np.ascontiguousarray(Bm[0], dtype=np.int64),
                          np.ascontiguousarray(Bm[1], dtype=np.int32),
                          np.ascontiguousarray(Bm[2], dtype=np.float64))
            self._keep.extend([rp, ci, va])
            _check(L.lrep_set_mass_csr(self.h, _ptr(rp), _ptr(ci), _ptr(va), MEM_HOST), self.h)
        elif _is_torch(Bm):
            mem = MEM_DEVICE_BORROW if borrow else MEM_DEVICE_COPY
            if borrow:
                self._keep.append(Bm)
            _check(L.lrep_set_mass_dense(self.h, _ptr(Bm), Bm.stride(0), mem), self.h)
        else:
            b, ld = _host_block(Bm)
            _check(L.lrep_set_mass_dense(self.h, _ptr(b), ld, MEM_HOST), self.h)

    def set_options(self, **kw):
        o = default_options(**kw)
        _check(lib().lrep_set_options(self.h, C.byref(o)), self.h)

    def set_start(self, U0, V0):
        u, ld, mem = block_arg(U0, self.n)
        v, _, _ = block_arg(V0, self.n)
        c = u.shape[1] if not _is_torch(U0) else U0.shape[0]
        _check(lib().lrep_set_start(self.h, c, _ptr(u), _ptr(v), ld, mem), self.h)

    def solve(self, nev, block, tol):
        return _check(lib().lrep_solve(self.h, nev, block, tol), self.h)

    def solve_begin(self, nev, block, tol):
        """Start a solve to be advanced batch by batch (lrep_solve_begin)."""
        return _check(lib().lrep_solve_begin(self.h, nev, block, tol), self.h)

    def solve_advance(self, locks=1):
        """Run outer iterations until `locks` more lock events or the end of
        the solve (lrep_solve_advance); returns (status, pairs locked so far,
        done)."""
        done, locked = C.c_int32(), C.c_int32()
        st = _check(lib().lrep_solve_advance(self.h, locks, C.byref(locked), C.byref(done)),
                    self.h)
        return st, locked.value, bool(done.value)

    # results -------------------------------------------------------------
    def _q_scalar(self, what, ctype):
        v = ctype()
        _check(lib().lrep_query(self.h, what, C.byref(v), C.sizeof(v), MEM_HOST), self.h)
        return v.value

    def nconv(self):
        return self._q_scalar(Q_NCONV, C.c_int32)

    def _q_array(self, what, count, shape=None):
        out = np.zeros(count, dtype=np.float64)
        if count:
            _check(lib().lrep_query(self.h, what, _ptr(out), out.nbytes, MEM_HOST), self.h)
        return out if shape is None else out.reshape(shape, order="F")

    def eigvals(self):
        return self._q_array(Q_EIGVALS, self.nconv())

    def vectors(self, which=Q_X):
        k = self.nconv()
        return self._q_array(which, self.n * k, (self.n, k))

    def vectors_device(self, which=Q_X):
        import torch
        k = self.nconv()
        out = torch.empty((k, self.n), dtype=torch.float64, device="cuda")
        if k:
            _check(lib().lrep_query(self.h, which, C.c_void_p(out.data_ptr()),
                                    out.numel() * 8, MEM_DEVICE_COPY), self.h)
        return out

    def residuals(self):
        return self._q_array(Q_RESID, self.nconv())

    def iters(self):
        return self._q_scalar(Q_ITERS, C.c_int32)

    def matvecs(self):
        return self._q_scalar(Q_MATVECS, C.c_int64)

    def timings(self):
        return self._q_array(Q_TIMINGS, 5)

    def biorth_err(self):
        return self._q_scalar(Q_BIORTH_ERR, C.c_double)

    def history(self):
        return self._q_array(Q_HISTORY, self.iters())

    def rebiorths(self):
        return self._q_scalar(Q_REBIORTHS, C.c_int32)

    def footprint(self, nev, block):
        """Device bytes a solve needs beyond the operator (server admission)."""
        v = C.c_int64()
        _check(lib().lrep_footprint(self.h, nev, block, C.byref(v)), self.h)
        return v.value

    def profile(self):
        """(product seconds, product launches, flops, algorithmic bytes)."""
        return self._q_array(Q_PROFILE, 4)

    def profile_cg(self):
        """profile() restricted to the CG-operator products."""
        return self._q_array(Q_PROFILE_CG, 4)

    def profile_classes(self):
        """{class: (device seconds, timed spans)} of the last profiled solve
        (options.profile), classes as in PROFILE_CLASSES."""
        v = self._q_array(Q_PROFILE_CLASSES, 2 * len(PROFILE_CLASSES))
        return {name: (float(v[2 * i]), int(v[2 * i + 1]))
                for i, name in enumerate(PROFILE_CLASSES)}

    # op level --------------------------------------------------------------
    def apply(self, op, X, Y, cg=False):
        """Y = op(X) for device blocks X, Y (torch (c, ld))."""
        f = lib().lrep_op_apply_cg if cg else lib().lrep_op_apply
        _check(f(self.h, op, X.shape[0], _ptr(X), _ld(X), _ptr(Y), _ld(Y)), self.h)

    def cg(self, op, B, X, tol, maxit):
        """X <- CG solution of op X = B (device blocks (c, ld)), zero start,
        the problem's CG operator (lrep_op_cg); returns the iterations run."""
        it = C.c_int32()
        _check(lib().lrep_op_cg(self.h, op, B.shape[0], _ptr(B), _ld(B), _ptr(X), _ld(X),
                                tol, maxit, C.byref(it)), self.h)
        return it.value

    def close(self):
        if self.h:
            lib().lrep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- op level


def _ld(t):
    """Leading dimension of a (c, ld) device block (size-1 dims carry no
    meaningful stride)."""
    return t.stride(0) if t.shape[0] > 1 else t.shape[1]


def _st(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _stream(stream)


def gram(A, B, G, stream=None, sliced=False):
    """G (b, a) tensor <- A^T B for device blocks A (a, n), B (b, n);
    sliced: float64 accuracy on the tensor cores (lrep_op_gram_sliced)."""
    n = A.shape[1]
    f = lib().lrep_op_gram_sliced if sliced else lib().lrep_op_gram
    _check(f(n, A.shape[0], B.shape[0], _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(G), _ld(G),
             _st(stream)))


def update(A, B, Cm, alpha, beta, stream=None, sliced=False):
    """Cm <- alpha Cm + beta A B for device A (k, n), B (c, k), Cm (c, n);
    sliced: float64 accuracy on the tensor cores (lrep_op_update_sliced)."""
    n = A.shape[1]
    f = lib().lrep_op_update_sliced if sliced else lib().lrep_op_update
    _check(f(n, A.shape[0], Cm.shape[0], alpha, _ptr(A), _ld(A), _ptr(B), _ld(B), beta,
             _ptr(Cm), _ld(Cm), _st(stream)))


def small_lrep(Kh, Mh, lam, Xh, Yh, stream=None):
    d = Kh.shape[0]
    info = C.c_int32()
    _check(lib().lrep_op_small_lrep(d, _ptr(Kh), _ptr(Mh), _ld(Kh), _ptr(lam),
                                    _ptr(Xh), _ptr(Yh), _ld(Xh), C.byref(info),
                                    _st(stream)))
    return info.value


def biorth(W, Z, P, Q, tau=1e-10, stream=None):
    n = W.shape[1]
    kept = C.c_int32()
    _check(lib().lrep_op_biorth(n, W.shape[0], _ptr(W), _ptr(Z), _ld(W), tau,
                                _ptr(P), _ptr(Q), _ld(P), C.byref(kept), _st(stream)))
    return kept.value


def residuals(X, Y, KX, MY, lam, eps, stream=None):
    n = X.shape[1]
    _check(lib().lrep_op_residuals(n, X.shape[0], _ptr(X), _ptr(Y), _ptr(KX), _ptr(MY),
                                   _ld(X), _ptr(lam), _ptr(eps), _st(stream)))


def launch_count():
    """Kernels launched by the library in this process."""
    return lib().lrep_launch_count()


def philox_normal(n, ncols, seed, stream_id, out, stream=None):
    _check(lib().lrep_op_philox_normal(n, ncols, seed, stream_id, _ptr(out), _ld(out),
                                       _st(stream)))


class Server:
    def __init__(self, hbm_budget_bytes, max_slots, stream=None):
        self.h = C.c_void_p()
        _check(lib().lrep_server_create(C.byref(self.h), hbm_budget_bytes, max_slots,
                                        _stream(stream)))

    def submit(self, problem, nev, block, tol):
        t = C.c_uint64()
        _check(lib().lrep_server_submit(self.h, problem.h, nev, block, tol, C.byref(t)),
               problem.h)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        return lib().lrep_server_wait(self.h, ticket, timeout_ms)

    def stats(self):
        """(batched small-LREP launches, problems in them, largest batch)."""
        out = np.zeros(3, dtype=np.int64)
        _check(lib().lrep_server_stats(self.h, _ptr(out)))
        return tuple(int(v) for v in out)

    def close(self):
        if self.h:
            lib().lrep_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
