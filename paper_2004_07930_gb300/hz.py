"""Thin ctypes binding of the C ABI in include/hz.h (argument marshalling only).

Every step of the solve runs in libhz.so; this module only converts NumPy /
torch buffers to pointers. It raises if the library has not been built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ECUDA, HZ_EINTERNAL, HZ_ESINGULAR, HZ_ENOTCONV, HZ_EBREAKDOWN = range(8)
HZ_COARSE_NONE, HZ_COARSE_GMRES, HZ_COARSE_DIRECT = 0, 1, 2
HZ_PREC_FP64, HZ_PREC_MIXED = 0, 1

EXPORTS = ["hz_default_options", "hz_setup", "hz_ndof", "hz_dof_coords", "hz_get_info", "hz_solve",
           "hz_solve_rhs", "hz_apply_A", "hz_apply_prec", "hz_matrix_csr", "hz_free", "hz_strerror",
           "hz_last_error", "hz_profile_begin", "hz_profile_end", "hz_apply_A_noalloc", "hz_server_create",
           "hz_server_submit", "hz_server_step", "hz_server_fetch", "hz_server_pending", "hz_server_free",
           "hz_receiver_operator", "hz_fwi_gradient", "hz_column_stats", "hz_krylov_basis",
           "hz_server_column_bytes"]
HZ_NOALLOC_MAX_ENTRIES = 1048576  # complex entries per work block of hz_apply_A_noalloc (n * s)


class HzMesh(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("nv", C.c_int64), ("tets", C.c_void_p), ("ne", C.c_int64),
                ("bfaces", C.c_void_p), ("bface_tag", C.c_void_p), ("nbf", C.c_int64)]


class HzOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rtol", C.c_double), ("maxit", C.c_int32), ("restart", C.c_int32),
                ("max_block", C.c_int32), ("coarse_mode", C.c_int32), ("coarse_inner_its", C.c_int32),
                ("leaf_size", C.c_int32), ("pivot_tau", C.c_double), ("verbose", C.c_int32),
                ("use_graphs", C.c_int32), ("tensor_cores", C.c_int32), ("overlap", C.c_int32),
                ("coarse_fp32", C.c_int32), ("debug_bounds", C.c_int32), ("block_arnoldi", C.c_int32),
                ("persistent_sweeps", C.c_int32), ("factor_fp32", C.c_int32),
                ("recycle", C.c_int32), ("emulate_fp64", C.c_int32), ("coarse_leaf_size", C.c_int32)]


class HzStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("ncols", C.c_int32), ("max_rel_residual", C.c_double), ("solve_seconds", C.c_double),
                ("setup_seconds", C.c_double), ("factor_seconds", C.c_double), ("perturbed_pivots", C.c_int32)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HzInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_imag", C.c_int64), ("nparts", C.c_int32),
                ("sub_rows", C.c_int64), ("n_coarse", C.c_int64), ("nnz_coarse", C.c_int64),
                ("factor_entries", C.c_int64), ("coarse_factor_entries", C.c_int64),
                ("front_entries", C.c_int64), ("max_front", C.c_int32), ("nfronts", C.c_int32),
                ("nlevels", C.c_int32), ("perturbed_pivots", C.c_int32), ("device_bytes", C.c_double),
                ("kernel_launches", C.c_int64), ("factor_ldlt_seconds", C.c_double),
                ("factor_inverse_seconds", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HzPhaseTime(C.Structure):
    _fields_ = [("name", C.c_char_p), ("calls", C.c_int64), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


_LIB = None


def library_path():
    return _build.LIB


def load():
    """Load libhz.so (built by paper_2004_07930_gb300.build); raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libhz.so is not built (%s); run paper_2004_07930_gb300.build.build()" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.hz_default_options.argtypes = [C.POINTER(HzOptions)]
    lib.hz_setup.argtypes = [C.POINTER(HzMesh), P, C.c_double, P, C.c_int32, C.POINTER(HzMesh),
                             C.POINTER(HzOptions), P, C.POINTER(P)]
    lib.hz_ndof.argtypes = [P, C.POINTER(C.c_int64)]
    lib.hz_dof_coords.argtypes = [P, P]
    lib.hz_get_info.argtypes = [P, C.POINTER(HzInfo)]
    lib.hz_solve.argtypes = [P, P, P, C.c_int32, P, C.c_int32, C.POINTER(HzStats)]
    lib.hz_solve_rhs.argtypes = [P, P, C.c_int32, C.c_int32, P, C.c_int32, C.POINTER(HzStats)]
    lib.hz_apply_A.argtypes = [P, P, P, C.c_int32, C.c_int32]
    lib.hz_apply_prec.argtypes = [P, P, P, C.c_int32, C.c_int32]
    lib.hz_matrix_csr.argtypes = [P, P, P, P]
    lib.hz_apply_A_noalloc.argtypes = [P, P, P, C.c_int32, P]
    lib.hz_server_create.argtypes = [P, C.c_int32, C.POINTER(P)]
    lib.hz_server_column_bytes.argtypes = [P, C.POINTER(C.c_double)]
    lib.hz_server_submit.argtypes = [P, C.c_int64, P, P, C.c_int32]
    lib.hz_server_step.argtypes = [P, P, C.c_int32, C.POINTER(C.c_int32)]
    lib.hz_server_fetch.argtypes = [P, C.c_int64, P, C.POINTER(HzStats)]
    lib.hz_server_pending.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.hz_server_free.argtypes = [P]
    lib.hz_server_free.restype = None
    lib.hz_receiver_operator.argtypes = [P, P, C.c_int32, P, P]
    lib.hz_fwi_gradient.argtypes = [P, P, P, C.c_int32, P, C.c_int32, P, P, P, P, C.POINTER(HzStats)]
    lib.hz_column_stats.argtypes = [P, P, P, C.c_int32, C.POINTER(C.c_int32)]
    lib.hz_krylov_basis.argtypes = [P, P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.hz_profile_begin.argtypes = [P]
    lib.hz_profile_end.argtypes = [P, C.POINTER(HzPhaseTime), C.c_int32, C.POINTER(C.c_int32)]
    lib.hz_free.argtypes = [P]
    lib.hz_free.restype = None
    lib.hz_strerror.argtypes = [C.c_int]
    lib.hz_strerror.restype = C.c_char_p
    lib.hz_last_error.argtypes = []
    lib.hz_last_error.restype = C.c_char_p
    _LIB = lib
    return lib


class HzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (msg, code, ""))
        self.code = code
        self.msg = msg

    def __str__(self):
        return "hz error %d: %s" % (self.code, self.msg)


def _check(rc):
    if rc != HZ_OK:
        lib = load()
        raise HzError(rc, "%s: %s" % (lib.hz_strerror(rc).decode(), lib.hz_last_error().decode()))


def default_options(**kw):
    o = HzOptions()
    load().hz_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _mesh(bundle, keep):
    xyz = np.ascontiguousarray(bundle["xyz"], dtype=np.float64)
    tets = np.ascontiguousarray(bundle["tets"], dtype=np.int32)
    bf = np.ascontiguousarray(bundle["bfaces"], dtype=np.int32).reshape(-1, 3)
    bt = np.ascontiguousarray(bundle["btags"], dtype=np.int32).reshape(-1)
    keep.extend([xyz, tets, bf, bt])
    return HzMesh(xyz.ctypes.data, len(xyz), tets.ctypes.data, len(tets), bf.ctypes.data, bt.ctypes.data, len(bt))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Solver:
    """One mesh + frequency; owns the device factors until close()."""

    def __init__(self, fine, velocity, freq, elem_part, nparts, coarse=None, options=None, stream=None):
        lib = load()
        keep = []
        fm = _mesh(fine, keep)
        cm = _mesh(coarse, keep) if coarse is not None else None
        vel = np.ascontiguousarray(velocity, dtype=np.float64)
        part = np.ascontiguousarray(elem_part, dtype=np.int32)
        opt = options if options is not None else default_options()
        if coarse is None and options is None:
            opt.coarse_mode = HZ_COARSE_NONE
        ctx = C.c_void_p()
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = lib.hz_setup(C.byref(fm), vel.ctypes.data, float(freq), part.ctypes.data, int(nparts),
                          C.byref(cm) if cm is not None else None, C.byref(opt), st, C.byref(ctx))
        _check(rc)
        self._ctx = ctx
        self._lib = lib
        self.options = opt
        n = C.c_int64()
        _check(lib.hz_ndof(ctx, C.byref(n)))
        self.n = n.value
        self.ne = len(vel)

    @classmethod
    def from_problem(cls, prob, options=None, stream=None, **kw):
        opt = options if options is not None else default_options(**kw)
        coarse = prob.get("coarse") if opt.coarse_mode != HZ_COARSE_NONE else None
        return cls(prob["fine"], prob["velocity"], prob["freq"], prob["elem_part"], prob["nparts"],
                   coarse=coarse, options=opt, stream=stream)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.hz_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def coords(self):
        out = np.empty((self.n, 3), dtype=np.float64)
        _check(self._lib.hz_dof_coords(self._ctx, out.ctypes.data))
        return out

    def info(self):
        i = HzInfo()
        _check(self._lib.hz_get_info(self._ctx, C.byref(i)))
        return i.asdict()

    def matrix_csr(self):
        import scipy.sparse as sp

        nnz = self.info()["nnz"]
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.complex128)
        _check(self._lib.hz_matrix_csr(self._ctx, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return sp.csr_matrix((val, col, rp), shape=(self.n, self.n))

    def column_stats(self):
        """(rel_residual [ncols], iterations [ncols]) of every column of the
        last solve call, in source order (FWI: forward columns, then adjoint)."""
        nc = C.c_int32()
        _check(self._lib.hz_column_stats(self._ctx, None, None, 0, C.byref(nc)))
        res = np.empty(nc.value, dtype=np.float64)
        its = np.empty(nc.value, dtype=np.int32)
        _check(self._lib.hz_column_stats(self._ctx, res.ctypes.data, its.ctypes.data, nc.value, C.byref(nc)))
        return res, its

    def krylov_basis(self):
        """Basis of the last restart cycle: array [nblocks, ncols, n] complex."""
        nb, nc = C.c_int32(), C.c_int32()
        _check(self._lib.hz_krylov_basis(self._ctx, None, 0, C.byref(nb), C.byref(nc)))
        V = np.empty((nb.value, nc.value, self.n), dtype=np.complex128)
        _check(self._lib.hz_krylov_basis(self._ctx, V.ctypes.data, nb.value, C.byref(nb), C.byref(nc)))
        return V

    def profile_begin(self):
        _check(self._lib.hz_profile_begin(self._ctx))

    def profile_end(self):
        """{phase: {calls, ms, flops, bytes}} since profile_begin()."""
        arr = (HzPhaseTime * 16)()
        cnt = C.c_int32()
        _check(self._lib.hz_profile_end(self._ctx, arr, 16, C.byref(cnt)))
        return {arr[i].name.decode(): dict(calls=arr[i].calls, ms=arr[i].ms, flops=arr[i].flops,
                                           bytes=arr[i].bytes) for i in range(cnt.value)}

    # ---- block calls: arrays [s, n] complex128 (NumPy on host, torch on device)
    def _io(self, X):
        if _is_torch(X):
            import torch

            assert X.dtype == torch.complex128 and X.is_contiguous()
            Y = torch.empty_like(X)
            return X.data_ptr(), Y, Y.data_ptr(), 1, X.shape[0] if X.dim() == 2 else 1
        X = np.ascontiguousarray(X, dtype=np.complex128)
        Y = np.empty_like(X)
        return X.ctypes.data, Y, Y.ctypes.data, 0, X.shape[0] if X.ndim == 2 else 1

    def apply_A(self, X):
        xp, Y, yp, dev, s = self._io(X)
        _check(self._lib.hz_apply_A(self._ctx, xp, yp, s, dev))
        return Y

    def apply_prec(self, X):
        xp, Y, yp, dev, s = self._io(X)
        _check(self._lib.hz_apply_prec(self._ctx, xp, yp, s, dev))
        return Y

    def solve_rhs(self, F, raise_on_notconv=True):
        xp, U, up, dev, s = self._io(F)
        st = HzStats()
        rc = self._lib.hz_solve_rhs(self._ctx, xp, s, dev, up, dev, C.byref(st))
        if rc != HZ_ENOTCONV or raise_on_notconv:
            _check(rc)
        return U, st.asdict()

    def solve(self, src_xyz, src_amp=None, out=None, raise_on_notconv=True):
        """Wavefields [ns, n] for point sources; `out` may be a device
        torch.complex128 tensor [ns, n] (else a NumPy array is returned)."""
        src = np.ascontiguousarray(src_xyz, dtype=np.float64).reshape(-1, 3)
        ns = len(src)
        amp = np.ones(ns, dtype=np.complex128) if src_amp is None else \
            np.ascontiguousarray(src_amp, dtype=np.complex128).reshape(-1)
        if out is None:
            U = np.empty((ns, self.n), dtype=np.complex128)
            up, dev = U.ctypes.data, 0
        else:
            U = out
            up, dev = (out.data_ptr(), 1) if _is_torch(out) else (out.ctypes.data, 0)
        st = HzStats()
        rc = self._lib.hz_solve(self._ctx, src.ctypes.data, amp.ctypes.data, ns, up, dev, C.byref(st))
        if rc != HZ_ENOTCONV or raise_on_notconv:
            _check(rc)
        return U, st.asdict()

    def column_bytes(self):
        """Device bytes one server slot (right-hand-side column) costs on this solver."""
        b = C.c_double()
        _check(self._lib.hz_server_column_bytes(self._ctx, C.byref(b)))
        return b.value

    def receiver_operator(self, rec_xyz):
        """(idx [nr, 20] int32, w [nr, 20]): receiver k samples
        sum_i w[k, i] u[idx[k, i]] (idx -1: no entry)."""
        rec = np.ascontiguousarray(rec_xyz, dtype=np.float64).reshape(-1, 3)
        idx = np.empty((len(rec), 20), dtype=np.int32)
        w = np.empty((len(rec), 20), dtype=np.float64)
        _check(self._lib.hz_receiver_operator(self._ctx, rec.ctypes.data, len(rec), idx.ctypes.data, w.ctypes.data))
        return idx, w

    def fwi_gradient(self, src_xyz, rec_xyz, d_obs=None, src_amp=None, raise_on_notconv=True):
        """(chi, grad [ne], d_syn [ns, nr], stats): least-squares misfit of
        the receiver data and its gradient with respect to the per-element
        squared slowness (adjoint state, on the device)."""
        src = np.ascontiguousarray(src_xyz, dtype=np.float64).reshape(-1, 3)
        rec = np.ascontiguousarray(rec_xyz, dtype=np.float64).reshape(-1, 3)
        ns, nr = len(src), len(rec)
        amp = np.ones(ns, dtype=np.complex128) if src_amp is None else \
            np.ascontiguousarray(src_amp, dtype=np.complex128).reshape(-1)
        dp = None
        if d_obs is not None:
            d_obs = np.ascontiguousarray(d_obs, dtype=np.complex128).reshape(ns, nr)
            dp = d_obs.ctypes.data
        chi = C.c_double()
        grad = np.empty(self.ne, dtype=np.float64)
        dsyn = np.empty((ns, nr), dtype=np.complex128)
        st = HzStats()
        rc = self._lib.hz_fwi_gradient(self._ctx, src.ctypes.data, amp.ctypes.data, ns, rec.ctypes.data, nr, dp,
                                       C.byref(chi), grad.ctypes.data, dsyn.ctypes.data, C.byref(st))
        if rc != HZ_ENOTCONV or raise_on_notconv:
            _check(rc)
        return chi.value, grad, dsyn, st.asdict()


class Server:
    """Continuous-batching request loop on one Solver (mesh + frequency):
    `slots` right-hand-side columns shared by the queued requests."""

    def __init__(self, solver, slots):
        self.solver = solver
        self._lib = solver._lib
        h = C.c_void_p()
        _check(self._lib.hz_server_create(solver._ctx, int(slots), C.byref(h)))
        self._h = h
        self.slots = slots

    def submit(self, request_id, src_xyz, src_amp=None):
        src = np.ascontiguousarray(src_xyz, dtype=np.float64).reshape(-1, 3)
        amp = np.ones(len(src), dtype=np.complex128) if src_amp is None else \
            np.ascontiguousarray(src_amp, dtype=np.complex128).reshape(-1)
        _check(self._lib.hz_server_submit(self._h, int(request_id), src.ctypes.data, amp.ctypes.data, len(src)))

    def step(self, cap=4096):
        """One restart cycle; returns the ids of the requests that finished
        (at most cap; the others come with the next steps)."""
        done = np.empty(max(cap, 1), dtype=np.int64)
        nd = C.c_int32()
        _check(self._lib.hz_server_step(self._h, done.ctypes.data, int(cap), C.byref(nd)))
        return done[: nd.value].tolist()

    def fetch(self, request_id, ns):
        u = np.empty((ns, self.solver.n), dtype=np.complex128)
        st = HzStats()
        rc = self._lib.hz_server_fetch(self._h, int(request_id), u.ctypes.data, C.byref(st))
        if rc not in (HZ_OK, HZ_ENOTCONV):
            _check(rc)
        return u, st.asdict()

    def pending(self):
        q, a = C.c_int32(), C.c_int32()
        _check(self._lib.hz_server_pending(self._h, C.byref(q), C.byref(a)))
        return q.value, a.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hz_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
