"""Pins for the box mirror symmetries (oracle/mesh.py box_mirrors) and the
mirror relations they give the lattice offset tables (Eqs. out, blockZo):

  L(g d) = P_g L(d) P_g^T,   K(g d) = det(g) P_g K(d) P_g^T,

P_g the signed permutation of the RWG functions under mirror g.  L pairs
two vector fields through the scalar G and their divergences, both
invariant under any rotation or reflection; K pairs them through
grad G x f, a cross product, which changes sign under a reflection
(det g = -1).  A wrong sign rule, a transposed permutation or a mirrored
triangle with the wrong orientation fails these at O(1).
"""
import numpy as np
import pytest

from oracle.lattice import offset_tables
from oracle.mesh import MIRRORS, box_mesh, box_mirrors
from oracle.operators import _slot_coef


def _signed_perm(pi, sign):
    E = len(pi)
    P = np.zeros((E, E))
    P[pi, np.arange(E)] = sign               # P e_n = sign_n e_pi(n)
    return P


@pytest.mark.parametrize("n", [2, 4])
def test_even_boxes_have_all_mirrors(n):
    assert sorted(box_mirrors(box_mesh(0.015, 0.015, 0.0075, n), 0.015, 0.015)) == ["d", "x", "y"]
    assert sorted(box_mirrors(box_mesh(0.015, 0.012, 0.0075, n), 0.015, 0.012)) == ["x", "y"]
    z = [0.0, 0.00076, 0.004, 0.0075, 0.01][: n + 1]
    if n == 4:
        assert sorted(box_mirrors(box_mesh(0.015, 0.015, 0.01, n, z), 0.015, 0.015)) == ["d", "x", "y"]


def test_odd_boxes_have_no_axis_mirror():
    # the middle row of quads lies on the mirror plane: one diagonal cannot be symmetric
    assert "x" not in box_mirrors(box_mesh(0.015, 0.015, 0.0075, 3), 0.015, 0.015)
    assert "y" not in box_mirrors(box_mesh(0.015, 0.015, 0.0075, 3), 0.015, 0.015)


@pytest.mark.parametrize("n", [2, 4])
def test_mirrors_are_involutions(n):
    for name, (pi, sign) in box_mirrors(box_mesh(0.015, 0.015, 0.0075, n), 0.015, 0.015).items():
        assert sorted(pi) == list(range(len(pi)))
        P = _signed_perm(pi, sign)
        assert np.array_equal(P @ P, np.eye(len(pi))), name


@pytest.mark.parametrize("n", [2, 4])
def test_mirrored_rwg_functions_pointwise(n):
    """g f_n(r) = sign_n f_pi(n)(g r) at the centroid of each support triangle."""
    a = b = 0.015
    box = box_mesh(a, b, 0.0075, n)
    tri = box.tri_coords()
    c, _ = _slot_coef(box, tri)
    cen = tri.mean(axis=1)
    owner = {}
    for t in range(len(box.tris)):
        for i in range(3):
            owner.setdefault(box.slot_rwg[t, i], []).append((t, i))

    def f(m, r):
        for t, i in owner[m]:
            lam = np.linalg.solve(np.c_[tri[t, 1] - tri[t, 0], tri[t, 2] - tri[t, 0],
                                        np.cross(tri[t, 1] - tri[t, 0], tri[t, 2] - tri[t, 0])],
                                  r - tri[t, 0])
            if lam[0] >= -1e-9 and lam[1] >= -1e-9 and lam[0] + lam[1] <= 1 + 1e-9 and abs(lam[2]) < 1e-9:
                return c[t, i] * (r - tri[t, i])
        return np.zeros(3)

    for name, (pi, sign) in box_mirrors(box, a, b).items():
        g = MIRRORS[name]
        for m in range(0, box.n_rwg, 7):
            for t, i in owner[m]:
                lhs = g @ (c[t, i] * (cen[t] - tri[t, i]))
                rhs = sign[m] * f(pi[m], g @ cen[t])
                assert np.allclose(lhs, rhs, atol=1e-9 * np.abs(lhs).max()), (name, m)


def test_offset_tables_mirror_relations():
    a = b = 0.015
    n, nx, ny = 2, 3, 3
    k = 2 * np.pi / 0.03
    box = box_mesh(a, b, 0.0075, n)
    Lt, Kt = offset_tables(box, nx, ny, a, b, k)
    scale = max(np.abs(Lt).max(), np.abs(Kt).max())
    for name, (pi, sign) in box_mirrors(box, a, b).items():
        g = MIRRORS[name]
        det = round(np.linalg.det(g))
        P = _signed_perm(pi, sign)
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                gx, gy = (g[:2, :2] @ np.array([dx, dy])).astype(int)
                L, K = Lt[dy + ny - 1, dx + nx - 1], Kt[dy + ny - 1, dx + nx - 1]
                L2, K2 = Lt[gy + ny - 1, gx + nx - 1], Kt[gy + ny - 1, gx + nx - 1]
                assert np.abs(L2 - P @ L @ P.T).max() <= 1e-12 * scale, (name, dx, dy)
                assert np.abs(K2 - det * P @ K @ P.T).max() <= 1e-12 * scale, (name, dx, dy)
                # the opposite sign rule is wrong at O(1) wherever K is not negligible
                if np.abs(K).max() > 1e-3 * scale:
                    assert np.abs(K2 + det * P @ K @ P.T).max() > 1e-3 * scale
