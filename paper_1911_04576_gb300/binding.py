"""Thin ctypes binding of libemsurf (argument marshalling only).

Every function keeps the name of the C entry point it calls.  Host arrays
are NumPy; device vectors are torch CUDA tensors (complex128, contiguous),
passed as raw pointers with the current torch stream.  There is no fallback:
if the compiled library is missing, importing a function raises.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libemsurf.so")

EMSURF_OK, EMSURF_EINVAL, EMSURF_ENOMEM, EMSURF_ECUDA, EMSURF_ENOTCONV = 0, 1, 2, 3, 4
EMSURF_EAGAIN, EMSURF_ETIMEDOUT, EMSURF_EBUSY = 5, 6, 7
FP64, FP32, MIXED = 0, 1, 2


class EmsurfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("emsurf status %d: %s" % (status, msg))
        self.status = status


class C128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("n_edges", C.c_int32), ("n_types", C.c_int32),
        ("n_unique", C.c_int32), ("max_rhs", C.c_int32),
        ("type_map", C.c_void_p), ("macromodels", C.c_void_p),
        ("offset_L", C.c_void_p), ("offset_K", C.c_void_p),
        ("coef", C128 * 4),
        ("uo_index", C.c_void_p), ("uo_sign", C.c_void_p),
        ("grid_px", C.c_int32), ("grid_py", C.c_int32),
        ("precision", C.c_int32), ("tables_on_device", C.c_int32),
        ("device_mem_budget", C.c_int64), ("device", C.c_int32),
    ]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int32), ("max_iters", C.c_int32),
                ("max_refine", C.c_int32), ("inner_rtol", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("n_matvec", C.c_int32),
                ("converged", C.c_int32), ("rel_residual", C.c_double), ("ms_total", C.c_double)]


_lib = None


def lib():
    """Load libemsurf.so (built by paper_1911_04576_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libemsurf.so not built: run paper_1911_04576_gb300/build.py "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32 = C.c_void_p, C.c_int32
        L.emsurf_create.argtypes = [C.POINTER(Problem), C.POINTER(vp)]
        L.emsurf_matvec.argtypes = [vp, vp, vp, i32, i32, vp]
        L.emsurf_solve.argtypes = [vp, vp, vp, i32, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
        L.emsurf_query.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_int64)]
        L.emsurf_destroy.argtypes = [vp]
        L.emsurf_destroy.restype = None
        L.emsurf_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def emsurf_last_error():
    return lib().emsurf_last_error().decode()


def _check(status, ok=(EMSURF_OK,)):
    if status not in ok:
        raise EmsurfError(status, emsurf_last_error())
    return status


def _ptr(a):
    """Raw pointer of a contiguous NumPy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


class Handle:
    """Owns an emsurf_handle; destroyed with emsurf_destroy."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            lib().emsurf_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def emsurf_create(nx, ny, n_edges, n_unique, type_map, macromodels, offset_L, offset_K, coef,
                  uo_index, uo_sign, precision=FP64, max_rhs=1, grid=(0, 0),
                  tables_on_device=False, device_mem_budget=0, device=0):
    """emsurf_create: host NumPy inputs (or torch CUDA tensors for the tables
    and macromodels when tables_on_device=True); returns a Handle."""
    type_map = np.ascontiguousarray(type_map, dtype=np.int32)
    uo_index = np.ascontiguousarray(uo_index, dtype=np.int32)
    uo_sign = np.ascontiguousarray(uo_sign, dtype=np.int8)
    if not tables_on_device:
        macromodels = np.ascontiguousarray(macromodels, dtype=np.complex128)
        offset_L = np.ascontiguousarray(offset_L, dtype=np.complex128)
        offset_K = np.ascontiguousarray(offset_K, dtype=np.complex128)
    n_types = int(macromodels.shape[0])
    p = Problem()
    p.nx, p.ny, p.n_edges, p.n_types, p.n_unique, p.max_rhs = nx, ny, n_edges, n_types, n_unique, max_rhs
    p.type_map, p.macromodels = _ptr(type_map), _ptr(macromodels)
    p.offset_L, p.offset_K = _ptr(offset_L), _ptr(offset_K)
    for i, c in enumerate(coef):
        p.coef[i] = C128(complex(c).real, complex(c).imag)
    p.uo_index, p.uo_sign = _ptr(uo_index), _ptr(uo_sign)
    p.grid_px, p.grid_py = grid
    p.precision = precision
    p.tables_on_device = 1 if tables_on_device else 0
    p.device_mem_budget = device_mem_budget
    p.device = device
    out = C.c_void_p()
    _check(lib().emsurf_create(C.byref(p), C.byref(out)))
    return Handle(out.value, (type_map, uo_index, uo_sign))


def emsurf_matvec(h, x, y, precision=FP64, stream=None):
    """emsurf_matvec: x, y torch complex128 CUDA tensors [nrhs, n_unique]."""
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().emsurf_matvec(h.ptr, _ptr(x), _ptr(y), nrhs, precision, _stream(stream)))


def emsurf_solve(h, b, x, rtol=1e-8, restart=30, max_iters=5000, max_refine=10, inner_rtol=0.0,
                 stream=None):
    """emsurf_solve: returns (status, [info dict per rhs]); ENOTCONV is not raised."""
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    o = SolveOpts(rtol, restart, max_iters, max_refine, inner_rtol)
    info = (SolveInfo * nrhs)()
    st = _check(lib().emsurf_solve(h.ptr, _ptr(b), _ptr(x), nrhs, C.byref(o), info, _stream(stream)),
                ok=(EMSURF_OK, EMSURF_ENOTCONV))
    return st, [{f: getattr(i, f) for f, _ in SolveInfo._fields_} for i in info]


def emsurf_query(h):
    px, py, nb = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib().emsurf_query(h.ptr, C.byref(px), C.byref(py), C.byref(nb)))
    return px.value, py.value, nb.value
