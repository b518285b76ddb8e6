"""Host-side admission estimate of the server (no GPU): emsurf_request_bytes
counts every resident array a request's handle creates, so it must grow
with the lattice, the mesh and the rhs count, and a MIXED request (FP64
operator, its FP32 hi/lo planes, the FP32 copy) must need more than an FP32
one and at least the FP64 spectrum plus its planes."""
import os

import numpy as np
import pytest

from paper_1911_04576_gb300 import binding as B
from paper_1911_04576_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1911_04576_gb300 import build
    if not os.path.exists(B.LIB_PATH):
        build.build()
    return B.lib()


def _bytes(n=3, nx=4, ny=4, rhs=1, precision=B.MIXED, overlap=0.0):
    sides = np.full(2, 0.6 * W.PERIOD)
    khat = np.tile([[0.0, 0.0, -1.0]], (rhs, 1))
    ehat = np.tile([[1.0, 0.0, 0.0]], (rhs, 1))
    q, keep = B.make_request(W.PERIOD, W.PERIOD, W.BOX_H, n, nx, ny, W.K0, sides, W.PATCH_Z, 2,
                             np.zeros(nx * ny, np.int32), khat, ehat, precision=precision,
                             precond_overlap=overlap)
    return B.emsurf_request_bytes(q)


def test_estimate_grows_with_the_problem():
    base = _bytes()
    assert _bytes(nx=8, ny=8) > base
    assert _bytes(n=4) > base
    assert _bytes(rhs=8) > base
    assert _bytes(overlap=0.6 * W.PERIOD / 3) > base


def test_estimate_counts_the_fp64_operator_and_its_planes():
    n, nx, ny = 3, 4, 4
    E = 18 * n * n
    px = py = 8                    # smallest 2,3,5-smooth size >= 2 * 4 - 1
    b64 = 2 * E * E * px * py * 16
    mixed, fp32 = _bytes(n, nx, ny, precision=B.MIXED), _bytes(n, nx, ny, precision=B.FP32)
    assert mixed > fp32
    assert _bytes(n, nx, ny, precision=B.FP64) >= 2 * b64
