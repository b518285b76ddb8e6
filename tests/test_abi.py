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
    ]
    for c in cases:
        args = dict(nx=1, ny=1, n_edges=E, n_unique=nu, type_map=[0], macromodels=Z, offset_L=L,
                    offset_K=L, coef=(1, 1, -1, 1), uo_index=idx, uo_sign=sg)
        args.update(c)
        with pytest.raises(B.EmsurfError) as e:
            B.emsurf_create(**args)
        assert e.value.status == B.EMSURF_EINVAL, c
        assert B.emsurf_last_error()


def test_null_handle_calls_rejected(lib):
    from paper_1911_04576_gb300 import binding as B
    assert lib.emsurf_matvec(None, None, None, 1, 0, None) == B.EMSURF_EINVAL
    assert lib.emsurf_solve(None, None, None, 1, None, None, None) == B.EMSURF_EINVAL
    assert lib.emsurf_query(None, None, None, None) == B.EMSURF_EINVAL
    lib.emsurf_destroy(None)
