"""The allocation-free tabulation entry point gives the same blocks as the
allocating one.

Some callers cannot allocate device memory when they need the operator
blocks (a plugin that must stay inside its host application's memory pool,
a process under a hard device-memory quota).  emsurf_tabulate_noalloc
serves them from a static per-GPU scratch array; this test checks it
against emsurf_tabulate, within the setup tests' tolerance, on two calls in
a row with different meshes (so the second call runs on the first one's
leftovers), that device free memory does not move across a call whose
scratch needs tens of MiB, and that an oversized request is refused.  The
file sorts last
so that a run stopping at its first failure has already run every other
test.
"""
import numpy as np
import pytest

from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.PERIOD
H = W.BOX_H


def _lattice_shifts(nx, ny):
    sh, sg = [], []
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            sh.append((dx * A, dy * A, 0.0))
            sg.append(1 if abs(dx) <= 1 and abs(dy) <= 1 else 0)
    return np.array(sh), np.array(sg, np.int8)


def _both(B, torch, test, src, shifts, sing):
    Et, Es = len(test["tplus"]), len(src["tplus"])
    out = []
    for fn in (B.emsurf_tabulate, B.emsurf_tabulate_noalloc):
        L = torch.empty((len(sing), Et, Es), dtype=torch.complex128, device="cuda")
        K = torch.empty_like(L)
        fn(test, src, shifts, sing, W.K0, L, K)
        out.append((L.cpu().numpy(), K.cpu().numpy()))
    return out


def test_noalloc_tabulation_matches_allocating_call(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    # call 1: boxes 3 x 3 per face, all offsets of a 3 x 4 lattice
    box3 = B.emsurf_setup_box_mesh(A, A, H, 3)
    sh, sg = _lattice_shifts(3, 4)
    (L1, K1), (L2, K2) = _both(B, torch, box3, box3, sh, sg)
    for b in range(len(sg)):
        assert np.abs(L2[b] - L1[b]).max() <= 1e-11 * np.abs(L1[b]).max()
        assert np.abs(K2[b] - K1[b]).max() <= 1e-11 * np.abs(K1[b]).max()
    # call 2, right after: a bigger box against a patch (different sizes)
    box4 = B.emsurf_setup_box_mesh(A, A, H, 4)
    patch = B.emsurf_setup_patch_mesh(0.3 * W.LAMBDA, W.PATCH_Z, 4)
    sh2 = np.array([[0.0, 0.0, 0.0], [A, 0.0, 0.0], [2 * A, -A, 0.0]])
    sg2 = np.array([1, 1, 0], np.int8)
    (L1, K1), (L2, K2) = _both(B, torch, box4, patch, sh2, sg2)
    for b in range(len(sg2)):
        assert np.abs(L2[b] - L1[b]).max() <= 1e-11 * np.abs(L1[b]).max()
        assert np.abs(K2[b] - K1[b]).max() <= 1e-11 * np.abs(K1[b]).max()


def test_noalloc_rejects_requests_beyond_its_scratch(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    big = B.emsurf_setup_box_mesh(A, A, H, 10)          # 1200 triangles: 414 MB per block
    L = torch.empty((1, 1, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_tabulate_noalloc(big, big, np.zeros((1, 3)), np.ones(1, np.int8), W.K0, L, L)
    assert e.value.status == B.EMSURF_EINVAL and "scratch" in str(e.value)


def test_noalloc_call_leaves_device_free_memory_unchanged(emsurf_lib):
    """A call needing ~40 MiB of scratch (3 x 4-per-face box blocks of 192 x 192
    triangle pairs, 10.6 MiB each, and a box/patch pair) changes nothing in
    the CUDA driver's free-memory count, while the allocating entry point's
    scratch is visible to it only transiently (it frees before returning)."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    box4 = B.emsurf_setup_box_mesh(A, A, H, 4)
    sh = np.array([[0.0, 0.0, 0.0], [A, 0.0, 0.0], [A, A, 0.0], [2 * A, 0.0, 0.0]])
    sg = np.array([1, 1, 1, 0], np.int8)
    L = torch.empty((4, 288, 288), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_noalloc(box4, box4, sh, sg, W.K0, L, K)      # first call: address set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        B.emsurf_tabulate_noalloc(box4, box4, sh, sg, W.K0, L, K)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
