"""Pins for oracle/mesh.py: counts and symmetries fixed by Sec. II-A."""
import numpy as np
import pytest

from oracle.mesh import box_mesh, patch_mesh, sphere_mesh
from oracle.operators import _slot_coef
from oracle.quadrature import tri_area


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_box_counts_closed_surface(n):
    box = box_mesh(0.015, 0.015, 0.0075, n)
    assert len(box.tris) == 12 * n * n
    assert box.n_rwg == 18 * n * n                     # E = 3F/2 on a closed surface
    assert np.all(box.slot_rwg >= 0)                   # every edge carries an RWG
    assert len(box.verts) == (n + 1) ** 3 - max(n - 1, 0) ** 3


@pytest.mark.parametrize("n", [2, 3])
def test_opposite_faces_are_translates(n):
    a, b, h = 0.015, 0.012, 0.0075
    box = box_mesh(a, b, h, n)
    F = 2 * n * n
    tri = box.tri_coords()
    for f, shift in ((0, [a, 0, 0]), (2, [0, b, 0]), (4, [0, 0, h])):
        lo = tri[f * F:(f + 1) * F] + np.array(shift)
        hi = tri[(f + 1) * F:(f + 2) * F]
        assert np.allclose(lo, hi, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3])
def test_rwg_zero_net_charge_and_continuity(n):
    box = box_mesh(0.015, 0.015, 0.0075, n)
    c, A = _slot_coef(box, box.tri_coords())
    charge = np.zeros(box.n_rwg)
    for t in range(len(box.tris)):
        for i in range(3):
            charge[box.slot_rwg[t, i]] += 2 * c[t, i] * A[t]    # div * area
    assert np.abs(charge).max() < 1e-12
    # normal component across the edge is continuous: |c| * h_perp = 1 on both sides
    L = box.slot_len()
    for e in range(box.n_rwg):
        for t in (box.tplus[e], box.tminus[e]):
            i = list(box.slot_rwg[t]).index(e)
            hperp = 2 * tri_area(box.tri_coords()[t]) / L[t, i]
            assert abs(abs(c[t, i]) * hperp - 1.0) < 1e-12


def test_patch_interior_edges_only():
    p = patch_mesh(0.009, 0.00076, 4)
    assert len(p.tris) == 32 and p.n_rwg == 3 * 16 - 2 * 4
    assert np.all(p.verts[:, 2] == 0.00076)


@pytest.mark.parametrize("s", [0, 1, 2])
def test_sphere_closed_surface(s):
    r, c = 3e-3, np.array([0.0, 0.0, 3.75e-3])
    m = sphere_mesh(r, c, s)
    T = 20 * 4 ** s
    assert len(m.tris) == T
    assert m.n_rwg == 3 * T // 2                  # closed: every edge shared by two triangles
    assert len(m.verts) - m.n_rwg + T == 2        # Euler characteristic of a sphere
    assert np.allclose(np.linalg.norm(m.verts - c, axis=1), r)
    # the facets approach the sphere's area from below as the mesh is refined
    area = tri_area(m.tri_coords()).sum()
    assert area < 4 * np.pi * r ** 2 and area > (0.76, 0.92, 0.98)[s] * 4 * np.pi * r ** 2
    # RWG zero net charge: the +/- halves carry equal and opposite charge l
    L = m.slot_len()
    for e in range(0, m.n_rwg, 7):
        tp, tm = m.tplus[e], m.tminus[e]
        lp = L[tp][m.slot_rwg[tp] == e][0]
        lm = L[tm][m.slot_rwg[tm] == e][0]
        assert abs(lp - lm) <= 1e-15 * r
