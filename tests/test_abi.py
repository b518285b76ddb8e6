"""The C-ABI library loads and exports every entry point include/emsurf.h
declares; host-side validation rejects bad problems with EINVAL before any
device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_04576_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.lib()


def declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"EMSURF_API\s+[\w\s\*]+?\b(emsurf_\w+)\s*\(", txt)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert {"emsurf_create", "emsurf_matvec", "emsurf_solve", "emsurf_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_problem_rejected_without_device(lib):
    from paper_1911_04576_gb300 import binding as B
    E, nu = 18, 36
    Z = np.zeros((1, 36, 36), complex)
    L = np.zeros((1, 1, E, E), complex)
    idx = np.arange(36)
    sg = np.ones(36)
    cases = [
        dict(nx=0, ny=1),                                   # empty lattice
        dict(nx=1, ny=1, uo_index=idx + 1),                 # index out of range
        dict(nx=1, ny=1, uo_sign=np.zeros(36)),             # sign not +-1
        dict(nx=1, ny=1, type_map=[3]),                     # type out of range
        dict(nx=1, ny=1, max_rhs=0),
        dict(nx=1, ny=1, max_rhs=65),
        dict(nx=1, ny=1, precision=7),
        dict(nx=2, ny=2, grid=(2, 3), type_map=[0] * 4, uo_index=np.tile(idx, 4),
             uo_sign=np.ones(144)),                         # grid below 2N-1
        dict(nx=1, ny=1, macromodels=_with(Z, (0, 3, 5), np.nan)),       # NaN in a macromodel
        dict(nx=1, ny=1, offset_L=_with(L, (0, 0, 2, 2), np.inf)),       # infinity in a table
        dict(nx=1, ny=1, offset_K=_with(L, (0, 0, 1, 7), 1j * np.nan)),
        dict(nx=1, ny=1, coef=(1, np.nan, -1, 1)),                        # coefficient
    ]
    finite_cases = cases[-4:]
    for c in cases:
        args = dict(nx=1, ny=1, n_edges=E, n_unique=nu, type_map=[0], macromodels=Z, offset_L=L,
                    offset_K=L, coef=(1, 1, -1, 1), uo_index=idx, uo_sign=sg)
        args.update(c)
        with pytest.raises(B.EmsurfError) as e:
            B.emsurf_create(**args)
        assert e.value.status == B.EMSURF_EINVAL, c
        assert B.emsurf_last_error()
        if any(c is f for f in finite_cases):
            assert "not finite" in str(e.value), str(e.value)


def _with(a, at, v):
    b = np.array(a, dtype=complex)
    b[at] = v
    return b


def test_finite_valid_problem_passes_validation(lib):
    """The same inputs without the planted values pass the host checks
    (without a GPU the device selection that follows them refuses)."""
    from paper_1911_04576_gb300 import binding as B
    E, nu = 18, 36
    Z = np.eye(36, dtype=complex)[None]
    L = np.ones((1, 1, E, E), complex)
    try:
        h = B.emsurf_create(1, 1, E, nu, [0], Z, L, L, (1, 1, -1, 1), np.arange(36), np.ones(36))
    except B.EmsurfError as e:
        # no GPU here: the first device call refuses (device selection)
        assert "not finite" not in str(e) and "device" in str(e), str(e)
    else:
        h.close()


def test_null_handle_calls_rejected(lib):
    from paper_1911_04576_gb300 import binding as B
    assert lib.emsurf_matvec(None, None, None, 1, 0, None) == B.EMSURF_EINVAL
    assert lib.emsurf_solve(None, None, None, 1, None, None, None) == B.EMSURF_EINVAL
    assert lib.emsurf_query(None, None, None, None) == B.EMSURF_EINVAL
    lib.emsurf_destroy(None)


def test_noalloc_entry_point_calls_no_allocator():
    """The allocation-free tabulation and its scratch-address helper name no
    allocating call (source scan of their bodies)."""
    import re
    src = open(os.path.join(ROOT, "paper_1911_04576_gb300", "csrc", "tabulate.cu")).read()
    forbidden = re.compile(r"cudaMalloc|cudaMallocAsync|cudaMallocHost|cudaHostAlloc|cudaMallocManaged|"
                           r"cudaFree|dev_alloc|\bnew\b|malloc\(")
    for name in ("int scratch_address(", "int tabulate_blocks_noalloc(", "CtxGetCurrentFn ctx_get_current("):
        start = src.index(name)
        depth, i = 0, src.index("{", start)
        while True:
            depth += {"{": 1, "}": -1}.get(src[i], 0)
            if depth == 0:
                break
            i += 1
        body = src[start:i]
        assert not forbidden.search(body), (name, forbidden.search(body).group(0))
