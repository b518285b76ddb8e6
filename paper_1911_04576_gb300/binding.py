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
EMSURF_EAGAIN, EMSURF_ETIMEDOUT, EMSURF_EBUSY, EMSURF_ECANCELED = 5, 6, 7, 8
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
        ("device_mem_budget", C.c_int64), ("device", C.c_int32), ("stream", C.c_void_p),
        ("unknown_xy", C.c_void_p), ("cell_a", C.c_double), ("cell_b", C.c_double),
        ("precond_overlap", C.c_double), ("tensor_cores", C.c_int32),
        ("sym_mask", C.c_int32), ("sym_perm", C.c_void_p), ("sym_sign", C.c_void_p),
        ("precond_int8", C.c_int32),
    ]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int32), ("max_iters", C.c_int32),
                ("max_refine", C.c_int32), ("inner_rtol", C.c_double), ("solver", C.c_int32),
                ("precond", C.c_int32), ("max_ms", C.c_double)]


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
        L.emsurf_create_like.argtypes = [C.POINTER(Problem), vp, C.POINTER(vp)]
        L.emsurf_matvec.argtypes = [vp, vp, vp, i32, i32, vp]
        L.emsurf_solve.argtypes = [vp, vp, vp, i32, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
        L.emsurf_query.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_int64)]
        L.emsurf_destroy.argtypes = [vp]
        L.emsurf_destroy.restype = None
        L.emsurf_last_error.restype = C.c_char_p
        ip = C.POINTER(C.c_int32)
        L.emsurf_setup_box_counts.argtypes = [i32, ip, ip, ip]
        L.emsurf_setup_patch_counts.argtypes = [i32, ip, ip, ip]
        L.emsurf_setup_box_mesh.argtypes = [C.c_double, C.c_double, C.c_double, i32, vp] + [vp] * 7
        L.emsurf_setup_patch_mesh.argtypes = [C.c_double, C.c_double, i32] + [vp] * 7
        L.emsurf_setup_box_mirrors.argtypes = [C.c_double, C.c_double, i32, vp, vp, ip]
        L.emsurf_setup_mirror_orbits.argtypes = [i32, i32, i32, ip, vp, vp, vp]
        L.emsurf_setup_mirror_group.argtypes = [i32, i32, vp, vp, vp]
        L.emsurf_setup_overlap.argtypes = [i32, i32, i32, vp, vp, ip]
        L.emsurf_precond_apply.argtypes = [vp, vp, vp, i32, vp]
        L.emsurf_selftest_wait.argtypes = [vp, C.c_int64, vp]
        L.emsurf_operator_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.emsurf_operator_layout.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.emsurf_tc_tuning.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), vp]
        L.emsurf_precond_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                          C.POINTER(i32)]
        L.emsurf_setup_unknown_xy.argtypes = [C.c_double, C.c_double, C.c_double, i32, i32, i32,
                                              vp, i32, vp]
        d = C.c_double
        L.emsurf_profile.argtypes = [vp, i32]
        L.emsurf_profile_phases.argtypes = [vp, C.c_uint32]
        L.emsurf_profile_read.argtypes = [vp, i32, C.POINTER(d), C.POINTER(C.c_int64)]
        L.emsurf_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.emsurf_check.argtypes = [vp]
        L.emsurf_tabulate.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, i32, i32, vp, vp,
                                      i32, d, vp, vp, vp]
        L.emsurf_tabulate_noalloc.argtypes = L.emsurf_tabulate.argtypes
        L.emsurf_tabulate_offsets.argtypes = [d, d, d, i32, vp, i32, i32, d, vp, vp, vp]
        L.emsurf_macromodel_pec_patch.argtypes = [d, d, d, i32, i32, vp, d, i32, d, vp, vp]
        L.emsurf_macromodel_slab_patch.argtypes = [d, d, d, i32, vp, i32, vp, i32, i32, C128, d,
                                                   vp, vp]
        L.emsurf_excitation.argtypes = [vp, d, d, d, i32, vp, d, i32, vp, vp, vp, vp]
        L.emsurf_far_field.argtypes = [vp, d, d, d, i32, vp, d, vp, i32, i32, vp, vp, vp, vp]
        L.emsurf_setup_slab_zlevels.argtypes = [d, i32, d, vp]
        L.emsurf_setup_slab_cell_counts.argtypes = [d, d, d, i32, vp, d, i32, i32, ip, vp]
        L.emsurf_setup_slab_top_counts.argtypes = [d, d, i32, d, i32, i32, ip, ip, ip]
        L.emsurf_setup_slab_top_mesh.argtypes = [d, d, d, i32, d, i32, i32] + [vp] * 8
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
                  tables_on_device=False, device_mem_budget=0, device=0, unknown_xy=None,
                  cell=(0.0, 0.0), precond_overlap=0.0, tensor_cores=False, share=None, mirrors=None,
                  precond_int8=False):
    """emsurf_create: host NumPy inputs (or torch CUDA tensors for the tables
    and macromodels when tables_on_device=True); returns a Handle.  With
    unknown_xy ([n_unique, 2] from emsurf_setup_unknown_xy), cell = (a, b) and
    precond_overlap > 0 the near-field preconditioner is built.  With share
    (a Handle of the same lattice) it calls emsurf_create_like: the tables are
    not read (may be None) and the new handle reads share's spectra.
    mirrors: (perm, sign, mask) from emsurf_setup_box_mirrors, or None;
    precond_int8: 8-bit preconditioner rows (one or two rhs)."""
    type_map = np.ascontiguousarray(type_map, dtype=np.int32)
    uo_index = np.ascontiguousarray(uo_index, dtype=np.int32)
    uo_sign = np.ascontiguousarray(uo_sign, dtype=np.int8)
    if not tables_on_device:
        macromodels = np.ascontiguousarray(macromodels, dtype=np.complex128)
        if offset_L is not None:
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
    p.stream = None
    if unknown_xy is not None:
        unknown_xy = np.ascontiguousarray(unknown_xy, dtype=np.float64)
        p.unknown_xy = _ptr(unknown_xy)
    p.cell_a, p.cell_b = cell
    p.precond_overlap = precond_overlap
    p.tensor_cores = 1 if tensor_cores else 0
    p.precond_int8 = 1 if precond_int8 else 0
    keep = [type_map, uo_index, uo_sign]
    if mirrors is not None:
        perm = np.ascontiguousarray(mirrors[0], dtype=np.int32)
        sign = np.ascontiguousarray(mirrors[1], dtype=np.int8)
        p.sym_mask, p.sym_perm, p.sym_sign = int(mirrors[2]), _ptr(perm), _ptr(sign)
        keep += [perm, sign]
    out = C.c_void_p()
    if share is not None:
        _check(lib().emsurf_create_like(C.byref(p), share.ptr, C.byref(out)))
        return Handle(out.value, tuple(keep + [share]))
    _check(lib().emsurf_create(C.byref(p), C.byref(out)))
    return Handle(out.value, tuple(keep))


def emsurf_matvec(h, x, y, precision=FP64, stream=None):
    """emsurf_matvec: x, y torch complex128 CUDA tensors [nrhs, n_unique]."""
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().emsurf_matvec(h.ptr, _ptr(x), _ptr(y), nrhs, precision, _stream(stream)))


def emsurf_precond_apply(h, r, y, stream=None):
    """emsurf_precond_apply: r, y torch complex128 CUDA tensors [nrhs, n_unique]."""
    nrhs = 1 if r.dim() == 1 else r.shape[0]
    _check(lib().emsurf_precond_apply(h.ptr, _ptr(r), _ptr(y), nrhs, _stream(stream)))


def emsurf_selftest_wait(h, limit=1000, stream=None):
    """emsurf_selftest_wait: a bounded device wait that always expires."""
    _check(lib().emsurf_selftest_wait(h.ptr, limit, _stream(stream)))


def emsurf_operator_info(h):
    """(stored spectrum bins of the FP32 operator, tensor-core planes built)."""
    nb, tc = C.c_int32(), C.c_int32()
    _check(lib().emsurf_operator_info(h.ptr, C.byref(nb), C.byref(tc)))
    return nb.value, bool(tc.value)


def emsurf_operator_layout(h):
    """(form: 0 full, 1 (k, -k) pairs, 2 mirror orbits; bins one stored bin serves)."""
    f, g = C.c_int32(), C.c_int32()
    _check(lib().emsurf_operator_layout(h.ptr, C.byref(f), C.byref(g)))
    return f.value, g.value


def emsurf_tc_tuning(h):
    """(sources per stage, stages, [ms of the 32 x 5 and 64 x 2 shapes]) of the
    tensor-core bin multiply's autotuned ring."""
    kc, ns = C.c_int32(), C.c_int32()
    ms = np.zeros(2)
    _check(lib().emsurf_tc_tuning(h.ptr, C.byref(kc), C.byref(ns), _ptr(ms)))
    return kc.value, ns.value, ms.tolist()


def emsurf_precond_info(h):
    """(factor entries sum n_m^2, sum n_m, max n_m) of the handle's preconditioner."""
    fe, st, mx = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().emsurf_precond_info(h.ptr, C.byref(fe), C.byref(st), C.byref(mx)))
    return fe.value, st.value, mx.value


SOLVER_DEFAULT, SOLVER_FP64, SOLVER_FP32, SOLVER_MIXED = 0, 1, 2, 3


def emsurf_solve(h, b, x, rtol=1e-8, restart=30, max_iters=5000, max_refine=10, inner_rtol=0.0,
                 solver=SOLVER_DEFAULT, stream=None, precond=0, max_ms=0.0):
    """emsurf_solve: returns (status, [info dict per rhs]); ENOTCONV is not raised.
    precond = -1 ignores the handle's near-field preconditioner; max_ms > 0
    stops the solve at the first restart past that wall time."""
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    o = SolveOpts(rtol, restart, max_iters, max_refine, inner_rtol, solver, precond, max_ms)
    info = (SolveInfo * nrhs)()
    st = _check(lib().emsurf_solve(h.ptr, _ptr(b), _ptr(x), nrhs, C.byref(o), info, _stream(stream)),
                ok=(EMSURF_OK, EMSURF_ENOTCONV))
    return st, [{f: getattr(i, f) for f, _ in SolveInfo._fields_} for i in info]


def emsurf_query(h):
    px, py, nb = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib().emsurf_query(h.ptr, C.byref(px), C.byref(py), C.byref(nb)))
    return px.value, py.value, nb.value


def _mesh_arrays(V, T, E):
    return dict(verts=np.zeros((V, 3)), tris=np.zeros((T, 3), np.int32),
                edges=np.zeros((E, 2), np.int32), tplus=np.zeros(E, np.int32),
                tminus=np.zeros(E, np.int32), slot_rwg=np.zeros((T, 3), np.int32),
                slot_sgn=np.zeros((T, 3), np.int8))


def _counts(fn, n):
    V, T, E = C.c_int32(), C.c_int32(), C.c_int32()
    _check(fn(n, C.byref(V), C.byref(T), C.byref(E)))
    return V.value, T.value, E.value


_MESH_KEYS = ("verts", "tris", "edges", "tplus", "tminus", "slot_rwg", "slot_sgn")


def emsurf_setup_box_mesh(a, b, h, n, zlevels=None):
    """emsurf_setup_box_mesh: returns dict of the canonical box mesh arrays."""
    out = _mesh_arrays(*_counts(lib().emsurf_setup_box_counts, n))
    z = None if zlevels is None else np.ascontiguousarray(zlevels, dtype=np.float64)
    _check(lib().emsurf_setup_box_mesh(a, b, h, n, _ptr(z), *[_ptr(out[k]) for k in _MESH_KEYS]))
    return out


def emsurf_setup_box_mirrors(a, b, n):
    """emsurf_setup_box_mirrors: (perm [3, E] int32, sign [3, E] int8, mask)."""
    E = 18 * n * n
    perm = np.zeros((3, E), np.int32)
    sign = np.zeros((3, E), np.int8)
    mask = C.c_int32(0)
    _check(lib().emsurf_setup_box_mirrors(C.c_double(a), C.c_double(b), n, _ptr(perm), _ptr(sign),
                                          C.byref(mask)))
    return perm, sign, mask.value


def emsurf_setup_mirror_orbits(px, py, n_elem):
    """emsurf_setup_mirror_orbits: (rep [S], slot_bin [S, n_elem], slot_elem [S, n_elem])."""
    ns = C.c_int32()
    rep = np.zeros(px * py, np.int32)
    sb = np.zeros(px * py * n_elem, np.int32)
    se = np.zeros(px * py * n_elem, np.int32)
    _check(lib().emsurf_setup_mirror_orbits(px, py, n_elem, C.byref(ns), _ptr(rep), _ptr(sb), _ptr(se)))
    S = ns.value
    return rep[:S], sb[:S * n_elem].reshape(S, n_elem), se[:S * n_elem].reshape(S, n_elem)


def emsurf_setup_mirror_group(perm, sign, n_elem):
    """emsurf_setup_mirror_group: (index [n_elem, 2E], sign [n_elem, 2E]) of T_e."""
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    E = perm.shape[1]
    t = np.zeros((n_elem, 2 * E), np.uint32)
    _check(lib().emsurf_setup_mirror_group(E, n_elem, _ptr(perm), _ptr(sign), _ptr(t)))
    return (t & 0x7FFFFFFF).astype(np.int64), np.where(t >> 31, -1, 1)


def emsurf_setup_patch_mesh(side, z, n):
    """emsurf_setup_patch_mesh: returns dict of the patch mesh arrays."""
    out = _mesh_arrays(*_counts(lib().emsurf_setup_patch_counts, n))
    _check(lib().emsurf_setup_patch_mesh(side, z, n, *[_ptr(out[k]) for k in _MESH_KEYS]))
    return out


def emsurf_setup_unknown_xy(a, b, h, n, nx, ny, uo_index, n_unique):
    """emsurf_setup_unknown_xy: [n_unique, 2] edge-midpoint (x, y) per unknown."""
    idx = np.ascontiguousarray(uo_index, dtype=np.int32)
    xy = np.zeros((n_unique, 2), np.float64)
    _check(lib().emsurf_setup_unknown_xy(a, b, h, n, nx, ny, _ptr(idx), n_unique, _ptr(xy)))
    return xy


def emsurf_setup_overlap(n, nx, ny):
    """emsurf_setup_overlap: returns (uo_index int32, uo_sign int8, n_unique)."""
    K = 36 * n * n
    idx = np.zeros(nx * ny * K, np.int32)
    sgn = np.zeros(nx * ny * K, np.int8)
    nu = C.c_int32()
    _check(lib().emsurf_setup_overlap(n, nx, ny, _ptr(idx), _ptr(sgn), C.byref(nu)))
    return idx, sgn, nu.value


def emsurf_tabulate(test, src, shifts, singular, k, L, K, stream=None):
    """emsurf_tabulate: test/src mesh dicts (setup helpers); L, K torch CUDA
    complex128 tensors [nb, test_E, src_E]."""
    shifts = np.ascontiguousarray(shifts, dtype=np.float64)
    singular = np.ascontiguousarray(singular, dtype=np.int8)
    m = [test[x] for x in ("verts", "tris", "slot_rwg", "slot_sgn")]
    s = [src[x] for x in ("verts", "tris", "slot_rwg", "slot_sgn")]
    _check(lib().emsurf_tabulate(*[_ptr(v) for v in m], len(test["tris"]), len(test["tplus"]),
                                 *[_ptr(v) for v in s], len(src["tris"]), len(src["tplus"]),
                                 _ptr(shifts), _ptr(singular), len(singular), k, _ptr(L), _ptr(K),
                                 _stream(stream)))


def emsurf_tabulate_noalloc(test, src, shifts, singular, k, L, K, stream=None):
    """emsurf_tabulate_noalloc: as emsurf_tabulate, for callers that cannot
    allocate device memory; its scratch is the library's static per-GPU array."""
    shifts = np.ascontiguousarray(shifts, dtype=np.float64)
    singular = np.ascontiguousarray(singular, dtype=np.int8)
    m = [test[x] for x in ("verts", "tris", "slot_rwg", "slot_sgn")]
    s = [src[x] for x in ("verts", "tris", "slot_rwg", "slot_sgn")]
    _check(lib().emsurf_tabulate_noalloc(*[_ptr(v) for v in m], len(test["tris"]),
                                         len(test["tplus"]), *[_ptr(v) for v in s],
                                         len(src["tris"]), len(src["tplus"]), _ptr(shifts),
                                         _ptr(singular), len(singular), k, _ptr(L), _ptr(K),
                                         _stream(stream)))


def _z(zlevels):
    return None if zlevels is None else np.ascontiguousarray(zlevels, dtype=np.float64)


def emsurf_tabulate_offsets(a, b, h, n, nx, ny, k, L, K, stream=None, zlevels=None):
    """emsurf_tabulate_offsets: L, K torch CUDA complex128 [2ny-1, 2nx-1, E, E];
    zlevels: box row heights [n+1] (None: uniform)."""
    z = _z(zlevels)
    _check(lib().emsurf_tabulate_offsets(a, b, h, n, _ptr(z), nx, ny, k, _ptr(L), _ptr(K),
                                         _stream(stream)))


def emsurf_setup_slab_zlevels(h, n, slab_t):
    """emsurf_setup_slab_zlevels: box row heights [n+1] of a slab cell."""
    z = np.zeros(n + 1)
    _check(lib().emsurf_setup_slab_zlevels(h, n, slab_t, _ptr(z)))
    return z


def emsurf_setup_slab_cell_counts(a, b, h, n, zlevels, side, patch_n, ring_layers=3):
    """emsurf_setup_slab_cell_counts: (interior unknowns, (air RWGs, slab RWGs))."""
    z = _z(zlevels)
    ni = C.c_int32()
    re = np.zeros(2, np.int32)
    _check(lib().emsurf_setup_slab_cell_counts(a, b, h, n, _ptr(z), side, patch_n, ring_layers,
                                               C.byref(ni), _ptr(re)))
    return ni.value, (int(re[0]), int(re[1]))


def emsurf_setup_slab_top_mesh(a, b, z, n, side, patch_n, ring_layers=3):
    """emsurf_setup_slab_top_mesh: dict of the slab-top mesh arrays plus on_patch."""
    V, T, E = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().emsurf_setup_slab_top_counts(a, b, n, side, patch_n, ring_layers, C.byref(V),
                                              C.byref(T), C.byref(E)))
    out = _mesh_arrays(V.value, T.value, E.value)
    out["on_patch"] = np.zeros(T.value, np.int8)
    _check(lib().emsurf_setup_slab_top_mesh(a, b, z, n, side, patch_n, ring_layers,
                                            *[_ptr(out[k]) for k in _MESH_KEYS + ("on_patch",)]))
    return out


def emsurf_macromodel_slab_patch(a, b, h, n, zlevels, sides, patch_n, ring_layers, eps_slab, k0, Z,
                                 stream=None):
    """emsurf_macromodel_slab_patch: Z torch CUDA complex128 [T, K, K]."""
    sides = np.ascontiguousarray(sides, dtype=np.float64)
    z = _z(zlevels)
    e = complex(eps_slab)
    _check(lib().emsurf_macromodel_slab_patch(a, b, h, n, _ptr(z), len(sides), _ptr(sides), patch_n,
                                              ring_layers, C128(e.real, e.imag), k0, _ptr(Z),
                                              _stream(stream)))


def emsurf_macromodel_pec_patch(a, b, h, n, sides, patch_z, patch_n, k, Z, stream=None):
    """emsurf_macromodel_pec_patch: Z torch CUDA complex128 [T, K, K]."""
    sides = np.ascontiguousarray(sides, dtype=np.float64)
    _check(lib().emsurf_macromodel_pec_patch(a, b, h, n, len(sides), _ptr(sides), patch_z, patch_n,
                                             k, _ptr(Z), _stream(stream)))


def emsurf_excitation(hd, a, b, h, n, k, khat, ehat, V, stream=None, zlevels=None):
    """emsurf_excitation: khat, ehat host [nrhs, 3]; V torch CUDA [nrhs, n_unique]."""
    khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    ehat = np.ascontiguousarray(np.atleast_2d(ehat), dtype=np.float64)
    z = _z(zlevels)
    _check(lib().emsurf_excitation(hd.ptr, a, b, h, n, _ptr(z), k, len(khat), _ptr(khat), _ptr(ehat),
                                   _ptr(V), _stream(stream)))


def emsurf_far_field(hd, a, b, h, n, k, Y, rhat, F, rcs=None, stream=None, zlevels=None):
    """emsurf_far_field: Y torch CUDA [nrhs, n_unique]; rhat host [ndir, 3];
    F torch CUDA complex128 [nrhs, ndir, 3]; rcs torch CUDA float64 [nrhs, ndir]."""
    rhat = np.ascontiguousarray(rhat, dtype=np.float64)
    nrhs = 1 if Y.dim() == 1 else Y.shape[0]
    z = _z(zlevels)
    _check(lib().emsurf_far_field(hd.ptr, a, b, h, n, _ptr(z), k, _ptr(Y), nrhs, len(rhat), _ptr(rhat),
                                  _ptr(F), _ptr(rcs), _stream(stream)))


PHASES = {"binmul32": 0, "binmul64": 1, "mm32": 2, "mm64": 3, "fft32": 4, "fft64": 5,
          "arnoldi": 6, "scatter": 7, "precond": 8}


def emsurf_profile(h, enable):
    _check(lib().emsurf_profile(h.ptr, 1 if enable else 0))


def emsurf_profile_phases(h, phases):
    """emsurf_profile_phases: record only the named phases (empty: stop)."""
    mask = 0
    for p in phases:
        mask |= 1 << PHASES[p]
    _check(lib().emsurf_profile_phases(h.ptr, mask))


def emsurf_profile_read(h, phase):
    """Returns (total_ms, intervals) of a phase name from PHASES."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().emsurf_profile_read(h.ptr, PHASES[phase], C.byref(ms), C.byref(n)))
    return ms.value, n.value


def emsurf_launch_count(h):
    n = C.c_int64()
    _check(lib().emsurf_launch_count(h.ptr, C.byref(n)))
    return n.value


def emsurf_check(h):
    """emsurf_check: raises EmsurfError(ETIMEDOUT) if a bounded device wait expired."""
    _check(lib().emsurf_check(h.ptr))


# ------------------------------------------------------------------ serving
class ServerOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("device_mem_budget", C.c_int64), ("max_active", C.c_int32),
                ("no_cache", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("h", C.c_double), ("n", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32), ("k0", C.c_double), ("n_types", C.c_int32),
                ("patch_sides", C.c_void_p), ("patch_z", C.c_double), ("patch_n", C.c_int32),
                ("type_map", C.c_void_p), ("nrhs", C.c_int32), ("khat", C.c_void_p),
                ("ehat", C.c_void_p), ("precision", C.c_int32), ("opts", SolveOpts),
                ("x_out", C.c_void_p), ("precond_overlap", C.c_double), ("slab_t", C.c_double),
                ("slab_eps", C128), ("ring_layers", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_unique", C.c_int32), ("nrhs", C.c_int32),
                ("info", SolveInfo), ("queue_ms", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("latency_ms", C.c_double), ("est_bytes", C.c_int64),
                ("handle_bytes", C.c_int64), ("cache_hit", C.c_int32)]


def _serve_lib():
    L = lib()
    if not getattr(L, "_serve_ready", False):
        vp = C.c_void_p
        L.emsurf_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(vp)]
        L.emsurf_request_bytes.argtypes = [C.POINTER(Request), C.POINTER(C.c_int64)]
        L.emsurf_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.emsurf_poll.argtypes = [vp, C.c_uint64, C.POINTER(Result)]
        L.emsurf_wait.argtypes = [vp, C.c_uint64, C.c_int64, C.POINTER(Result)]
        L.emsurf_cancel.argtypes = [vp, C.c_uint64]
        L.emsurf_request_phase.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int32)]
        L.emsurf_server_destroy.argtypes = [vp]
        L.emsurf_server_destroy.restype = None
        L.emsurf_server_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
        L._serve_ready = True
    return L


class Server:
    """Owns an emsurf_server; keeps each request's arrays alive until collected."""

    def __init__(self, ptr):
        self.ptr = ptr
        self.keep = {}

    def close(self):
        if self.ptr:
            _serve_lib().emsurf_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def emsurf_server_create(device=0, device_mem_budget=0, max_active=2, cache=True):
    o = ServerOpts(device, device_mem_budget, max_active, 0 if cache else 1)
    out = C.c_void_p()
    _check(_serve_lib().emsurf_server_create(C.byref(o), C.byref(out)))
    return Server(out.value)


def make_request(a, b, h, n, nx, ny, k0, patch_sides, patch_z, patch_n, type_map, khat, ehat,
                 precision=MIXED, rtol=1e-6, restart=30, max_iters=20000, max_refine=20,
                 inner_rtol=0.0, solver=0, x_out=None, precond_overlap=0.0, slab_t=0.0,
                 slab_eps=1.0, ring_layers=0, max_ms=0.0):
    """Build an emsurf_request; returns (Request, arrays that must stay alive).
    slab_t > 0: patch-on-slab cells (eps slab_eps, patch on the slab top);
    max_ms > 0: wall-time limit of the solve."""
    sides = np.ascontiguousarray(patch_sides, dtype=np.float64)
    tmap = np.ascontiguousarray(type_map, dtype=np.int32)
    kh = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    eh = np.ascontiguousarray(np.atleast_2d(ehat), dtype=np.float64)
    q = Request(a, b, h, n, nx, ny, k0, len(sides), _ptr(sides), patch_z, patch_n, _ptr(tmap),
                len(kh), _ptr(kh), _ptr(eh), precision,
                SolveOpts(rtol, restart, max_iters, max_refine, inner_rtol, solver, 0, max_ms), _ptr(x_out),
                precond_overlap, slab_t, C128(complex(slab_eps).real, complex(slab_eps).imag),
                ring_layers)
    return q, (sides, tmap, kh, eh, x_out)


def emsurf_request_bytes(req):
    nb = C.c_int64()
    _check(_serve_lib().emsurf_request_bytes(C.byref(req), C.byref(nb)))
    return nb.value


def emsurf_submit(server, req, keep=()):
    """emsurf_submit: returns the ticket; EmsurfError(EBUSY) if never admissible."""
    t = C.c_uint64()
    _check(_serve_lib().emsurf_submit(server.ptr, C.byref(req), C.byref(t)))
    server.keep[t.value] = keep
    return t.value


def _result(r):
    d = {f: getattr(r, f) for f, _ in Result._fields_ if f != "info"}
    d["info"] = {f: getattr(r.info, f) for f, _ in SolveInfo._fields_}
    return d


def emsurf_poll(server, ticket):
    """emsurf_poll: None while pending, else the result dict."""
    r = Result()
    st = _check(_serve_lib().emsurf_poll(server.ptr, ticket, C.byref(r)), ok=(EMSURF_OK, EMSURF_EAGAIN))
    if st == EMSURF_EAGAIN:
        return None
    server.keep.pop(ticket, None)
    return _result(r)


def emsurf_wait(server, ticket, timeout_ms=600000):
    """emsurf_wait: the result dict; EmsurfError(ETIMEDOUT) if not done in time."""
    r = Result()
    _check(_serve_lib().emsurf_wait(server.ptr, ticket, int(timeout_ms), C.byref(r)))
    server.keep.pop(ticket, None)
    return _result(r)


def emsurf_cancel(server, ticket):
    """emsurf_cancel: True if the queued request was withdrawn, False if it
    already runs or ran (its result is then collected as usual)."""
    st = _check(_serve_lib().emsurf_cancel(server.ptr, ticket), ok=(EMSURF_OK, EMSURF_EBUSY))
    return st == EMSURF_OK


REQUEST_PHASES = ("queued", "admitted", "library", "wait_library", "wait_operator", "operator", "solve", "done")


def emsurf_request_phase(server, ticket):
    """emsurf_request_phase: the request's phase as a name (REQUEST_PHASES)."""
    ph = C.c_int32()
    _check(_serve_lib().emsurf_request_phase(server.ptr, ticket, C.byref(ph)))
    return REQUEST_PHASES[ph.value]


def emsurf_server_stats(server):
    """(cached bytes, cached operators, cached libraries, evictions)."""
    b, o, l, e = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
    _check(_serve_lib().emsurf_server_stats(server.ptr, C.byref(b), C.byref(o), C.byref(l), C.byref(e)))
    return b.value, o.value, l.value, e.value
