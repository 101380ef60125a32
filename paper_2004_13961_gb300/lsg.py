"""Thin ctypes binding of the C ABI in include/lsg.h (argument marshalling only).

Every computation happens in the CUDA library liblsg.so; this module only turns
torch tensors / numpy arrays into pointers and streams.  Importing it loads the
library and raises if the CUDA extension is missing or cannot be built -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:  # torch provides device memory and streams; load it first so one CUDA runtime is shared
    import torch
except Exception:  # pragma: no cover - torch is always present in this project
    torch = None

from . import build as _build

FP64, MIXED_TF32, MIXED_BF16 = 0, 1, 2
SETUP_KEEP_M = 1
SETUP_PROFILE = 2
SETUP_AUTOTUNE = 4
SETUP_CONST_PRECOND = 8
SETUP_SHARED_GPU = 16

EXPORT_GAUSS_X, EXPORT_GAUSS_W, EXPORT_AHAT, EXPORT_BHAT = 0, 1, 2, 3
EXPORT_BAND_S, EXPORT_BAND_M, EXPORT_M, EXPORT_LU = 4, 5, 6, 7
EXPORT_AHAT_Y, EXPORT_AHAT_Z, EXPORT_CONST_EIG = 8, 9, 10

Q_UNKNOWNS, Q_GRID, Q_HALF_WIDTH, Q_SLOTS, Q_LEVELS, Q_DEVICE_BYTES, Q_NNZ, Q_PRECISION, Q_ASSEMBLE_US, Q_ILU_US = \
    range(10)
(Q_SWEEP_L_US, Q_SWEEP_L_CALLS, Q_SWEEP_U_US, Q_SWEEP_U_CALLS, Q_KX_US, Q_KX_CALLS, Q_KX_LO_US,
 Q_KX_LO_CALLS) = range(10, 18)
Q_CONST_US, Q_CONST_CALLS, Q_PRECOND_KIND = 18, 19, 20

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_ILU_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_NONFINITE = \
    0, -1, -2, -3, -4, -5, -6, -7

# every symbol the header declares (checked by the ABI test)
SYMBOLS = [
    "lsg_version", "lsg_status_string", "lsg_last_error", "lsg_kernel_launches", "lsg_gauss", "lsg_gauss_noalloc", "lsg_footprint_bytes",
    "lsg_setup", "lsg_setup_ex", "lsg_setup_problem", "lsg_load_vector", "lsg_apply_A", "lsg_apply_A_lowp", "lsg_apply_Minv",
    "lsg_pcg_solve",
    "lsg_eval", "lsg_export_count", "lsg_export", "lsg_query", "lsg_destroy", "lsg_set_wait_budget",
    "lsg_autotune_transforms", "lsg_transform_tiles", "lsg_set_transform_tiles",
    "lsg_batch_solve",
    "lsg_server_create", "lsg_server_set_aging", "lsg_server_submit", "lsg_server_poll", "lsg_server_drain",
    "lsg_server_release", "lsg_server_destroy",
]


class LsgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return dict(iters=self.iters, outer_iters=self.outer_iters, relres=self.relres,
                    relres_true=self.relres_true, status=self.status)


class LsgProblem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int), ("Q", ctypes.c_int),
                ("a", ctypes.c_void_p * 3), ("b", ctypes.c_void_p), ("ta", (ctypes.c_int * 3) * 3),
                ("tb", ctypes.c_int * 3), ("precision", ctypes.c_int), ("flags", ctypes.c_uint)]


class LsgRequest(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("d", ctypes.c_int), ("N", ctypes.c_int), ("T", ctypes.c_int),
                ("Q", ctypes.c_int), ("precision", ctypes.c_int), ("rtol", ctypes.c_double),
                ("kmax", ctypes.c_int), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("f", ctypes.c_void_p)]


class LsgResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("info", LsgInfo), ("latency_ms", ctypes.c_double),
                ("u", ctypes.POINTER(ctypes.c_double)), ("n", ctypes.c_longlong)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load liblsg.so (building it in-tree when stale); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
    L = ctypes.CDLL(_build.LIB, mode=ctypes.RTLD_GLOBAL)
    vp, ci, cd, cll, cu = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_uint
    L.lsg_version.restype = ci
    L.lsg_status_string.restype = ctypes.c_char_p
    L.lsg_status_string.argtypes = [ci]
    L.lsg_last_error.restype = ctypes.c_char_p
    L.lsg_kernel_launches.restype = cll
    L.lsg_gauss.argtypes = [ci, vp, vp]
    L.lsg_gauss_noalloc.argtypes = [ci, vp, vp]
    L.lsg_footprint_bytes.argtypes = [ci, ci, ci, ci, ci]
    L.lsg_footprint_bytes.restype = ctypes.c_size_t
    L.lsg_setup.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, vp, vp, ci, vp]
    L.lsg_setup_ex.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, vp, vp, ci, cu, vp]
    L.lsg_setup_problem.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(LsgProblem), vp]
    for name in ("lsg_load_vector", "lsg_apply_A", "lsg_apply_A_lowp", "lsg_apply_Minv", "lsg_eval"):
        getattr(L, name).argtypes = [vp, vp, vp, vp]
    L.lsg_pcg_solve.argtypes = [vp, vp, vp, cd, ci, ctypes.POINTER(LsgInfo), vp]
    L.lsg_export_count.argtypes = [vp, ci]
    L.lsg_export_count.restype = cll
    L.lsg_export.argtypes = [vp, ci, vp]
    L.lsg_query.argtypes = [vp, ci]
    L.lsg_query.restype = cll
    L.lsg_destroy.argtypes = [vp]
    L.lsg_set_wait_budget.argtypes = [vp, cll]
    L.lsg_autotune_transforms.argtypes = [vp, ci, ctypes.POINTER(ci)]
    L.lsg_transform_tiles.argtypes = [vp, ctypes.POINTER(ci)]
    L.lsg_set_transform_tiles.argtypes = [vp, ctypes.POINTER(ci)]
    L.lsg_batch_solve.argtypes = [ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), cd, ci,
                                  ctypes.POINTER(LsgInfo), vp]
    L.lsg_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ci]
    L.lsg_server_set_aging.argtypes = [vp, cd]
    L.lsg_server_submit.argtypes = [vp, ctypes.POINTER(LsgRequest)]
    L.lsg_server_poll.argtypes = [vp, ctypes.POINTER(LsgResult), ci, ctypes.POINTER(ci)]
    L.lsg_server_drain.argtypes = [vp]
    L.lsg_server_release.argtypes = [vp, ctypes.POINTER(LsgResult)]
    L.lsg_server_destroy.argtypes = [vp]
    _lib = L
    return L


class LsgError(RuntimeError):
    def __init__(self, status, where=""):
        L = load(False)
        msg = L.lsg_status_string(status).decode()
        last = L.lsg_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}) {last}".strip())
        self.status = status


def _check(status, where):
    if status != OK:
        raise LsgError(status, where)
    return status


def _ptr(a):
    """Pointer of a contiguous float64 torch tensor (CPU or CUDA) or numpy array."""
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous float64 array")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is None:
        if torch is not None and torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if torch is not None and isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _like(ref, n):
    if torch is not None and isinstance(ref, torch.Tensor):
        return torch.empty(n, dtype=torch.float64, device=ref.device)
    return np.empty(n, dtype=np.float64)


def kernel_launches() -> int:
    return int(load().lsg_kernel_launches())


def gauss(Q: int):
    L = load()
    x = np.zeros(Q)
    w = np.zeros(Q)
    _check(L.lsg_gauss(Q, _ptr(x), _ptr(w)), "lsg_gauss")
    return x, w


def gauss_noalloc(Q: int):
    """Gauss rule through the entry point that allocates no device memory."""
    L = load()
    x = np.zeros(Q)
    w = np.zeros(Q)
    _check(L.lsg_gauss_noalloc(Q, _ptr(x), _ptr(w)), "lsg_gauss_noalloc")
    return x, w


def footprint_bytes(d, N, T, Q=0, precision=FP64) -> int:
    return int(load().lsg_footprint_bytes(d, N, T, Q, precision))


class Context:
    """An lsg_ctx: tables, coefficient samples, M's ILU(0) factors and workspaces."""

    def __init__(self, d, N, T, a, b, Q=None, precision=FP64, keep_M=False, stream=None, allow_breakdown=False,
                 profile=False, autotune=False, ta=None, tb=None, const_precond=False, shared_gpu=False):
        """A context for lsg_setup_ex (one coefficient a, one degree T), or -- when `a` is a list
        of d per-direction coefficients or the degrees ta (d x d: ta[j][i] of a_j in direction
        i) and tb (d) are given -- for lsg_setup_problem (T unused then)."""
        L = load()
        self._L = L
        self.d, self.N, self.T = d, N, T
        self.Q = N + 2 if Q is None else Q
        self.precision = precision
        h = ctypes.c_void_p(0)
        flags = (SETUP_KEEP_M if keep_M else 0) | (SETUP_PROFILE if profile else 0) | (SETUP_AUTOTUNE if autotune else 0) \
            | (SETUP_CONST_PRECOND if const_precond else 0) | (SETUP_SHARED_GPU if shared_gpu else 0)
        if isinstance(a, (list, tuple)) or ta is not None or tb is not None:
            alist = list(a) if isinstance(a, (list, tuple)) else [a] * d
            ta = [[T] * d for _ in range(d)] if ta is None else ta
            tb = [T] * d if tb is None else tb
            pr = LsgProblem()
            pr.d, pr.N, pr.Q, pr.precision, pr.flags = d, N, self.Q, precision, flags
            for j in range(3):
                pr.a[j] = _ptr(alist[j]).value if j < len(alist) else None
                pr.tb[j] = int(tb[j]) if j < d else 0
                for i in range(3):
                    pr.ta[j][i] = int(ta[j][i]) if (j < d and i < d) else 0
            pr.b = _ptr(b).value
            self._keep = (alist, b)
            st = L.lsg_setup_problem(ctypes.byref(h), ctypes.byref(pr), _stream(stream))
        else:
            st = L.lsg_setup_ex(ctypes.byref(h), d, N, T, self.Q, _ptr(a), _ptr(b), precision, flags, _stream(stream))
        self.status = st
        self._h = h
        if st != OK and not (allow_breakdown and st == ERR_ILU_BREAKDOWN and h.value):
            if h.value:
                L.lsg_destroy(h)
                self._h = ctypes.c_void_p(0)
            raise LsgError(st, "lsg_setup")
        self.n = int(L.lsg_query(h, Q_UNKNOWNS))
        self.nq = int(L.lsg_query(h, Q_GRID))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            self._L.lsg_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_A(self, x, y=None, stream=None):
        y = _like(x, self.n) if y is None else y
        _check(self._L.lsg_apply_A(self._h, _ptr(x), _ptr(y), _stream(stream)), "lsg_apply_A")
        return y

    def apply_A_lowp(self, x, y=None, stream=None):
        """y = K x with the tensor-core transforms of a mixed context (float32 CUDA tensors)."""
        if y is None:
            y = torch.empty(self.n, dtype=torch.float32, device=x.device)
        if x.dtype != torch.float32 or y.dtype != torch.float32 or not (x.is_contiguous() and y.is_contiguous()):
            raise ValueError("expected contiguous float32 tensors")
        _check(self._L.lsg_apply_A_lowp(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        _stream(stream)), "lsg_apply_A_lowp")
        return y

    def apply_Minv(self, r, z=None, stream=None):
        z = _like(r, self.n) if z is None else z
        _check(self._L.lsg_apply_Minv(self._h, _ptr(r), _ptr(z), _stream(stream)), "lsg_apply_Minv")
        return z

    def load_vector(self, f, F=None, stream=None):
        F = _like(f, self.n) if F is None else F
        _check(self._L.lsg_load_vector(self._h, _ptr(f), _ptr(F), _stream(stream)), "lsg_load_vector")
        return F

    def eval(self, u, vals=None, stream=None):
        vals = _like(u, self.nq) if vals is None else vals
        _check(self._L.lsg_eval(self._h, _ptr(u), _ptr(vals), _stream(stream)), "lsg_eval")
        return vals

    def pcg_solve(self, F, u=None, rtol=1e-12, kmax=10000, stream=None, check=True):
        if u is None:
            u = _like(F, self.n)
            u[...] = 0.0
        info = LsgInfo()
        st = self._L.lsg_pcg_solve(self._h, _ptr(F), _ptr(u), float(rtol), int(kmax), ctypes.byref(info),
                                   _stream(stream))
        if check:
            _check(st, "lsg_pcg_solve")
        d = info.as_dict()
        d["status"] = st
        return u, d

    def export(self, item):
        cnt = int(self._L.lsg_export_count(self._h, item))
        if cnt <= 0:
            raise LsgError(ERR_ARG, f"lsg_export({item})")
        out = np.zeros(cnt)
        _check(self._L.lsg_export(self._h, item, _ptr(out)), "lsg_export")
        return out

    def query(self, item):
        return int(self._L.lsg_query(self._h, item))

    def autotune_transforms(self, reps=5):
        """Time the tile shapes of K x's contractions and keep the fastest; returns the choice."""
        out = (ctypes.c_int * 6)()
        _check(self._L.lsg_autotune_transforms(self._h, int(reps), out), "lsg_autotune_transforms")
        return list(out)

    def transform_tiles(self):
        out = (ctypes.c_int * 6)()
        _check(self._L.lsg_transform_tiles(self._h, out), "lsg_transform_tiles")
        return list(out)

    def set_transform_tiles(self, choice):
        arr = (ctypes.c_int * 6)(*[int(v) for v in choice])
        _check(self._L.lsg_set_transform_tiles(self._h, arr), "lsg_set_transform_tiles")

    def set_wait_budget(self, cycles):
        """Budget (SM clock cycles) of the sweeps' dependency waits; 0 = default."""
        _check(self._L.lsg_set_wait_budget(self._h, int(cycles)), "lsg_set_wait_budget")


def batch_solve(ctxs, Fs, us, rtol=1e-12, kmax=10000, stream=None):
    L = load()
    n = len(ctxs)
    H = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    Fp = (ctypes.c_void_p * n)(*[_ptr(F).value for F in Fs])
    Up = (ctypes.c_void_p * n)(*[_ptr(u).value for u in us])
    infos = (LsgInfo * n)()
    st = L.lsg_batch_solve(n, H, Fp, Up, float(rtol), int(kmax), infos, _stream(stream))
    return st, [i.as_dict() for i in infos]


class Server:
    """Continuous batching of solve requests (lsg_server_*): requests are admitted as
    worker slots and HBM budget free up, and run on their own streams."""

    def __init__(self, hbm_budget, max_inflight=4, aging_ms=None):
        L = load()
        self._L = L
        h = ctypes.c_void_p(0)
        _check(L.lsg_server_create(ctypes.byref(h), int(hbm_budget), int(max_inflight)), "lsg_server_create")
        self._h = h
        if aging_ms is not None:
            _check(L.lsg_server_set_aging(h, float(aging_ms)), "lsg_server_set_aging")

    def submit(self, rid, d, N, T, a, b, f, Q=None, precision=FP64, rtol=1e-10, kmax=10000):
        """Queue one request; a, b, f are host float64 arrays of Q^d samples (copied)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        req = LsgRequest(id=int(rid), d=d, N=N, T=T, Q=(N + 2 if Q is None else Q), precision=precision,
                         rtol=float(rtol), kmax=int(kmax), a=a.ctypes.data, b=b.ctypes.data, f=f.ctypes.data)
        return self._L.lsg_server_submit(self._h, ctypes.byref(req))

    def poll(self, max_results=64):
        """Finished results: dicts with id, info, latency_ms and the solution (numpy copy)."""
        out = (LsgResult * max_results)()
        cnt = ctypes.c_int(0)
        _check(self._L.lsg_server_poll(self._h, out, max_results, ctypes.byref(cnt)), "lsg_server_poll")
        res = []
        for k in range(cnt.value):
            r = out[k]
            u = np.ctypeslib.as_array(r.u, shape=(r.n,)).copy() if r.n > 0 and r.u else None
            res.append(dict(id=r.id, info=r.info.as_dict(), latency_ms=r.latency_ms, u=u))
            self._L.lsg_server_release(self._h, ctypes.byref(out[k]))
        return res

    def drain(self):
        _check(self._L.lsg_server_drain(self._h), "lsg_server_drain")

    def close(self):
        if self._h is not None and self._h.value:
            self._L.lsg_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
