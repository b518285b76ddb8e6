"""Pins for oracle/operators.py: reciprocity and structural zeros."""
import numpy as np

from oracle.mesh import box_mesh
from oracle.operators import galerkin_LK
from oracle.lattice import cell_shift

LAM = 0.03
K0 = 2 * np.pi / LAM
A = B = 0.5 * LAM
H = 0.25 * LAM
ORIGIN = (0.0, 0.0, 0.0)


def test_far_offsets_reciprocal_exactly():
    # with the same symmetric rule on both triangles, L(-d) = L(d)^T and
    # K(-d) = K(d)^T hold to rounding (Galerkin symmetry of both kernels)
    box = box_mesh(A, B, H, 2)
    for d in [(2, 0), (3, -1), (0, 2)]:
        Lp, Kp = galerkin_LK(box, cell_shift(*d, A, B), box, ORIGIN, K0, False)
        Lm, Km = galerkin_LK(box, cell_shift(-d[0], -d[1], A, B), box, ORIGIN, K0, False)
        assert np.abs(Lm - Lp.T).max() <= 1e-13 * np.abs(Lp).max()
        assert np.abs(Km - Kp.T).max() <= 1e-13 * np.abs(Kp).max()


def test_near_offsets_reciprocal_to_quadrature_accuracy():
    # one-sided closed-form integration at touching boxes: the asymmetry is
    # the 7-point test rule's error on the near-singular kernels (a few
    # percent of the largest entry for K at a corner-touching offset, about
    # 0.2 at an edge-touching one), which is why the tables take the
    # reciprocal part
    box = box_mesh(A, B, H, 3)
    Lp, Kp = galerkin_LK(box, cell_shift(1, 1, A, B), box, ORIGIN, K0, True)
    Lm, Km = galerkin_LK(box, cell_shift(-1, -1, A, B), box, ORIGIN, K0, True)
    assert np.abs(Lm - Lp.T).max() <= 2e-2 * np.abs(Lp).max()
    assert np.abs(Km - Kp.T).max() <= 1e-1 * np.abs(Kp).max()


def test_singular_extraction_agrees_with_plain_quadrature_far_away():
    box = box_mesh(A, B, H, 2)
    sh = (3 * LAM, 0.5 * LAM, 0.1 * LAM)
    L1, K1 = galerkin_LK(box, sh, box, ORIGIN, K0, True)
    L2, K2 = galerkin_LK(box, sh, box, ORIGIN, K0, False)
    assert np.abs(L1 - L2).max() < 1e-7 * np.abs(L2).max()
    assert np.abs(K1 - K2).max() < 1e-7 * np.abs(K2).max()


def test_coplanar_K_vanishes():
    # Lam_m . (grad G x Lam_n) = 0 when both RWGs lie in one plane (top faces)
    n = 2
    box = box_mesh(A, B, H, n)
    top = np.where(np.all(np.isclose(box.verts[box.edges][:, :, 2], H), axis=1))[0]
    tops = [e for e in top if box.tplus[e] >= 10 * n * n and box.tminus[e] >= 10 * n * n]
    for sh, sing in ((cell_shift(1, 0, A, B), True), (cell_shift(3, 2, A, B), False)):
        _, K = galerkin_LK(box, sh, box, ORIGIN, K0, sing)
        assert np.abs(K[np.ix_(tops, tops)]).max() < 1e-12 * np.abs(K).max()
    _, K = galerkin_LK(box, ORIGIN, box, ORIGIN, K0, True)
    assert np.abs(K[np.ix_(tops, tops)]).max() < 1e-12 * np.abs(K).max()
