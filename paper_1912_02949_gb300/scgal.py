"""ctypes binding of libscgal (include/scgal.h).

Argument marshalling only: every computation runs in the CUDA library.  Array
arguments may be numpy arrays (host memory) or torch tensors (host or CUDA);
the binding passes their data pointers.  Functions keep the C names; errors
raise ScgalError, except SCGAL_ENOTDONE which solve() returns.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int8, c_int32, c_int64, c_uint32, c_uint64, c_void_p, c_size_t

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libscgal.so")

SCGAL_OK = 0
SCGAL_ENOTDONE = 1
SCGAL_EINVAL = -1
SCGAL_ENOMEM = -2
SCGAL_ECUDA = -3
SCGAL_ENUMERIC = -4
SCGAL_ETIMEOUT = -5
SCGAL_EBUSY = -6
SCGAL_ESTATE = -7
SCGAL_LMO_EQ, SCGAL_LMO_LEQ, SCGAL_LMO_DEFAULT = 0, 1, -1
SCGAL_OMEGA_STORED, SCGAL_OMEGA_REGEN = 0, 1
SCGAL_K_EQ, SCGAL_K_LEQ = 0, 1
SCGAL_SPMV_AUTO, SCGAL_SPMV_GATHER, SCGAL_SPMV_TILED = 0, 1, 2
SCGAL_FFT_AUTO, SCGAL_FFT_PASSES, SCGAL_FFT_CLUSTER = 0, 1, 2
SCGAL_ADMIT_FIFO, SCGAL_ADMIT_SHORTEST_PREDICTED = 0, 1


class ScgalError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status} ({strerror(status)})")


class scgal_params(Structure):
    _fields_ = [("R", c_int32), ("T_max", c_int32), ("tol", c_double), ("beta0", c_double), ("K", c_double),
                ("lmo", c_int32), ("scale", c_int32), ("trace_correct", c_int32), ("precision", c_int32),
                ("seed", c_uint64), ("instance", c_uint32), ("check_every", c_int32), ("device", c_int32),
                ("omega", c_int32), ("kset", c_int32), ("tune", c_int32), ("spmv", c_int32), ("fft", c_int32),
                ("keep_state", c_int32), ("warm_from", c_int64)]


class scgal_stats(Structure):
    _fields_ = [("t", c_int64), ("q", c_int32), ("k", c_int32), ("xi", c_double), ("p", c_double),
                ("relgap", c_double), ("infeas", c_double), ("gamma", c_double), ("converged", c_int32),
                ("reserved", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class scgal_info(Structure):
    _fields_ = [("n", c_int32), ("d", c_int32), ("R", c_int32), ("precision", c_int32), ("is_complex", c_int32),
                ("lmo", c_int32), ("trace_correct", c_int32), ("scale", c_int32), ("nnz", c_int64),
                ("weight_kind", c_int32), ("qmax", c_int32), ("t", c_int64), ("alpha", c_double),
                ("normC", c_double), ("normA", c_double), ("device_bytes", c_int64), ("spmv_group", c_int32),
                ("spmv_grid", c_int32), ("spmv_kind", c_int32), ("tiled_slots", c_int64),
                ("fft_cluster", c_int32)]


class scgal_result(Structure):
    _fields_ = [("status", c_int32), ("n", c_int32), ("iterations", c_int64), ("relgap", c_double),
                ("infeas", c_double), ("objective", c_double), ("best_cut", c_int64), ("lambda_max", c_double),
                ("queue_ms", c_double), ("latency_ms", c_double), ("first_t", c_int64),
                ("predicted_iterations", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class scgal_server_stats(Structure):
    _fields_ = [("submitted", c_int64), ("admitted", c_int64), ("completed", c_int64), ("rejected", c_int64),
                ("active", c_int32), ("queued", c_int32), ("device_bytes_in_use", c_int64),
                ("device_bytes_peak", c_int64), ("rounds", c_int64), ("wait_ms", c_double),
                ("admit_ms", c_double), ("retire_ms", c_double)]


# name -> (restype, argtypes), exactly the declarations of include/scgal.h
_PROTOS = {
    "scgal_params_default": (None, [POINTER(scgal_params)]),
    "scgal_create_maxcut": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_double,
                                    POINTER(scgal_params), POINTER(c_void_p)]),
    "scgal_create_phase": (c_int, [c_void_p, c_int32, c_int32, c_void_p, c_double, POINTER(scgal_params),
                                   POINTER(c_void_p)]),
    "scgal_create_ptycho": (c_int, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_double, POINTER(scgal_params),
                                    POINTER(c_void_p)]),
    "scgal_step": (c_int, [c_void_p, POINTER(scgal_stats)]),
    "scgal_solve": (c_int, [c_void_p, c_int64, POINTER(scgal_stats)]),
    "scgal_reconstruct": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int64)]),
    "scgal_cut_value": (c_int, [c_void_p, c_void_p, POINTER(c_int64)]),
    "scgal_apply_D": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scgal_lanczos": (c_int, [c_void_p, c_void_p, c_int64, c_int32, POINTER(c_double), POINTER(c_int32), c_void_p]),
    "scgal_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scgal_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scgal_history": (c_int, [c_void_p, c_int64, c_int64, POINTER(scgal_stats)]),
    "scgal_get_info": (c_int, [c_void_p, POINTER(scgal_info)]),
    "scgal_time_kernel": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_double)]),
    "scgal_set_stream": (c_int, [c_void_p, c_void_p]),
    "scgal_dmatvec_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_int32, c_int64, c_void_p,
                                      c_void_p, c_void_p, c_void_p]),
    "scgal_destroy": (c_int, [c_void_p]),
    "scgal_strerror": (c_char_p, [c_int]),
    "scgal_server_create": (c_int, [c_size_t, c_int32, POINTER(c_void_p)]),
    "scgal_server_set_admission": (c_int, [c_void_p, c_int32]),
    "scgal_submit": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int64, POINTER(scgal_params),
                             POINTER(c_uint64)]),
    "scgal_submit_phase": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, POINTER(scgal_params),
                                   POINTER(c_uint64)]),
    "scgal_poll": (c_int, [c_void_p, c_uint64, POINTER(scgal_result), c_int32]),
    "scgal_server_get_stats": (c_int, [c_void_p, POINTER(scgal_server_stats)]),
    "scgal_server_destroy": (c_int, [c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libscgal.so (fails loudly if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libscgal.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load().scgal_strerror(status).decode()
    except Exception:  # library not loadable: still format the number
        return "unknown"


def _check(rc: int, where: str, allow=(SCGAL_OK,)):
    if rc not in allow:
        raise ScgalError(rc, where)
    return rc


def _ptr(x, dtype=None):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):          # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    a = np.asarray(x)
    if dtype is not None and a.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {a.dtype}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def scgal_params_default(**overrides) -> scgal_params:
    p = scgal_params()
    load().scgal_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Handle:
    """An SDP instance of libscgal (wraps scgal_t)."""

    def __init__(self, raw: c_void_p, n: int, d: int, R: int, is_complex: bool):
        self.raw = raw
        self.n, self.d, self.R, self.is_complex = n, d, R, is_complex

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "raw", None) is not None and self.raw.value:
            load().scgal_destroy(self.raw)
            self.raw = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def scgal_create_maxcut(row_ptr, col, w, n: int, nnz: int, alpha: float = 0.0, params: scgal_params | None = None) -> Handle:
    params = params or scgal_params_default()
    h = c_void_p()
    rc = load().scgal_create_maxcut(_ptr(row_ptr), _ptr(col), _ptr(w), int(n), int(nnz), float(alpha),
                                    ctypes.byref(params), ctypes.byref(h))
    _check(rc, "scgal_create_maxcut")
    return Handle(h, int(n), int(n), params.R, False)


def scgal_create_phase(masks, L: int, n: int, b, alpha: float = 0.0, params: scgal_params | None = None) -> Handle:
    """masks: complex128[L, n] (or float64[L, n, 2]); b: float64[L * n]."""
    params = params or scgal_params_default()
    m = masks
    if isinstance(m, np.ndarray) and np.iscomplexobj(m):
        m = np.ascontiguousarray(m.astype(np.complex128)).view(np.float64)
    h = c_void_p()
    rc = load().scgal_create_phase(_ptr(m), int(L), int(n), _ptr(b), float(alpha), ctypes.byref(params), ctypes.byref(h))
    _check(rc, "scgal_create_phase")
    return Handle(h, int(n), int(L) * int(n), params.R, True)


def scgal_create_ptycho(pupil, M: int, N: int, s: int, b, alpha: float = 0.0,
                        params: scgal_params | None = None) -> Handle:
    """pupil: complex128[M * M] (or float64[M * M, 2]); b: float64[(N / s)^2 * M * M]."""
    params = params or scgal_params_default()
    pp = pupil
    if isinstance(pp, np.ndarray) and np.iscomplexobj(pp):
        pp = np.ascontiguousarray(pp.astype(np.complex128)).view(np.float64)
    h = c_void_p()
    rc = load().scgal_create_ptycho(_ptr(pp), int(M), int(N), int(s), _ptr(b), float(alpha), ctypes.byref(params),
                                    ctypes.byref(h))
    _check(rc, "scgal_create_ptycho")
    K = int(N) // int(s)
    return Handle(h, int(N) * int(N), K * K * int(M) * int(M), params.R, True)


def scgal_step(h: Handle) -> dict:
    st = scgal_stats()
    _check(load().scgal_step(h.raw, ctypes.byref(st)), "scgal_step")
    return st.as_dict()


def scgal_solve(h: Handle, T: int):
    """Returns (status, last record); status is SCGAL_OK (converged) or SCGAL_ENOTDONE."""
    st = scgal_stats()
    rc = _check(load().scgal_solve(h.raw, int(T), ctypes.byref(st)), "scgal_solve", (SCGAL_OK, SCGAL_ENOTDONE))
    return rc, st.as_dict()


def scgal_reconstruct(h: Handle, U=None, want_cut: bool = True):
    """Returns (U, lambda, err, best_cut).  U is a new array (column-major n x R
    as a numpy (R, n) array, complex for phase retrieval) unless given."""
    lam = np.zeros(h.R)
    err = np.zeros(h.R)
    if U is None:
        U = np.zeros((h.R, h.n), dtype=np.complex128 if h.is_complex else np.float64)
    cut = c_int64(0)
    rc = load().scgal_reconstruct(h.raw, _ptr(U), _ptr(lam), _ptr(err), ctypes.byref(cut) if want_cut else None)
    _check(rc, "scgal_reconstruct")
    return U, lam, err, (int(cut.value) if want_cut and not h.is_complex else None)


def scgal_cut_value(h: Handle, chi) -> int:
    chi = np.ascontiguousarray(np.asarray(chi), dtype=np.int8) if not hasattr(chi, "data_ptr") else chi
    cut = c_int64(0)
    _check(load().scgal_cut_value(h.raw, _ptr(chi), ctypes.byref(cut)), "scgal_cut_value")
    return int(cut.value)


def _as_real_view(x):
    a = np.ascontiguousarray(x)
    if np.iscomplexobj(a):
        return a.astype(np.complex128).view(np.float64)
    return a.astype(np.float64)


def scgal_apply_D(h: Handle, x, w=None):
    xr = _as_real_view(x)
    out = np.zeros_like(xr)
    wr = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    _check(load().scgal_apply_D(h.raw, _ptr(wr), _ptr(xr), _ptr(out)), "scgal_apply_D")
    return out.view(np.complex128) if h.is_complex else out


def scgal_lanczos(h: Handle, t: int, q: int, w=None):
    xi = c_double(0)
    k = c_int32(0)
    v = np.zeros(2 * h.n if h.is_complex else h.n)
    wr = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    _check(load().scgal_lanczos(h.raw, _ptr(wr), int(t), int(q), ctypes.byref(xi), ctypes.byref(k), _ptr(v)),
           "scgal_lanczos")
    return xi.value, k.value, (v.view(np.complex128) if h.is_complex else v)


def scgal_get_state(h: Handle):
    z = np.zeros(h.d)
    y = np.zeros(h.d)
    S = np.zeros(h.n * h.R * (2 if h.is_complex else 1))
    sc = np.zeros(4)
    _check(load().scgal_get_state(h.raw, _ptr(z), _ptr(y), _ptr(S), _ptr(sc)), "scgal_get_state")
    S = S.view(np.complex128).reshape(h.n, h.R) if h.is_complex else S.reshape(h.n, h.R)
    return dict(z=z, y=y, S=S, p=sc[0], tau=sc[1], t=int(sc[2]), converged=bool(sc[3]))


def scgal_set_state(h: Handle, z=None, y=None, S=None, p=None, tau=None, t=None):
    zr = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
    yr = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
    Sr = None if S is None else _as_real_view(S)
    sc = None
    if p is not None or tau is not None or t is not None:
        cur = scgal_get_state(h)
        sc = np.array([cur["p"] if p is None else p, cur["tau"] if tau is None else tau,
                       cur["t"] if t is None else t, 0.0])
    _check(load().scgal_set_state(h.raw, _ptr(zr), _ptr(yr), _ptr(Sr), _ptr(sc)), "scgal_set_state")


def scgal_history(h: Handle, first: int, count: int):
    arr = (scgal_stats * count)()
    _check(load().scgal_history(h.raw, int(first), int(count), arr), "scgal_history")
    return [r.as_dict() for r in arr]


def scgal_get_info(h: Handle) -> dict:
    inf = scgal_info()
    _check(load().scgal_get_info(h.raw, ctypes.byref(inf)), "scgal_get_info")
    return {f: getattr(inf, f) for f, _ in inf._fields_ if f != "reserved"}


def scgal_time_kernel(h: Handle, kernel: int, reps: int) -> float:
    """Mean milliseconds per launch of iteration kernel `kernel` (0 D-matvec step,
    1 Lanczos update, 2 Ritz vector, 3 tridiagonal solve)."""
    ms = c_double(0)
    _check(load().scgal_time_kernel(h.raw, int(kernel), int(reps), ctypes.byref(ms)), "scgal_time_kernel")
    return ms.value


def scgal_set_stream(h: Handle, stream_ptr: int):
    _check(load().scgal_set_stream(h.raw, c_void_p(stream_ptr)), "scgal_set_stream")


def scgal_destroy(h: Handle):
    h.close()


def scgal_dmatvec_noalloc(row_ptr, col, val, diag, coff: float, n: int, nnz: int, x, y, dot, stream: int = 0):
    """y = diag .* x + coff * (W x) and dot = <x, y> without any device allocation
    (all arguments are caller-owned CUDA tensors; see include/scgal.h)."""
    _check(load().scgal_dmatvec_noalloc(_ptr(row_ptr), _ptr(col), _ptr(val), _ptr(diag), float(coff), int(n),
                                        int(nnz), _ptr(x), _ptr(y), _ptr(dot), c_void_p(stream)),
           "scgal_dmatvec_noalloc")


# --- serving -----------------------------------------------------------------
class Server:
    def __init__(self, raw: c_void_p):
        self.raw = raw

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "raw", None) is not None and self.raw.value:
            load().scgal_server_destroy(self.raw)
            self.raw = None


def scgal_server_create(hbm_budget: int, max_slots: int) -> Server:
    s = c_void_p()
    _check(load().scgal_server_create(int(hbm_budget), int(max_slots), ctypes.byref(s)), "scgal_server_create")
    return Server(s)


def scgal_server_set_admission(s: Server, policy: int) -> None:
    _check(load().scgal_server_set_admission(s.raw, int(policy)), "scgal_server_set_admission")


def scgal_submit(s: Server, row_ptr, col, w, n: int, nnz: int, params: scgal_params) -> int:
    ticket = c_uint64(0)
    _check(load().scgal_submit(s.raw, _ptr(row_ptr), _ptr(col), _ptr(w), int(n), int(nnz), ctypes.byref(params),
                               ctypes.byref(ticket)), "scgal_submit")
    return int(ticket.value)


def scgal_submit_phase(s: Server, masks, L: int, n: int, b, params: scgal_params) -> int:
    """masks: complex128[L, n] (or float64[L, n, 2]); b: float64[L * n]."""
    m = masks
    if isinstance(m, np.ndarray) and np.iscomplexobj(m):
        m = np.ascontiguousarray(m.astype(np.complex128)).view(np.float64)
    ticket = c_uint64(0)
    _check(load().scgal_submit_phase(s.raw, _ptr(m), int(L), int(n), _ptr(b), ctypes.byref(params),
                                     ctypes.byref(ticket)), "scgal_submit_phase")
    return int(ticket.value)


def scgal_poll(s: Server, ticket: int, timeout_ms: int = 0):
    """Returns the result dict, or None if not ready within timeout_ms."""
    r = scgal_result()
    rc = load().scgal_poll(s.raw, c_uint64(ticket), ctypes.byref(r), int(timeout_ms))
    if rc == SCGAL_ETIMEOUT:
        return None
    _check(rc, "scgal_poll")
    return r.as_dict()


def scgal_server_get_stats(s: Server) -> dict:
    st = scgal_server_stats()
    _check(load().scgal_server_get_stats(s.raw, ctypes.byref(st)), "scgal_server_get_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def scgal_server_destroy(s: Server):
    s.close()
