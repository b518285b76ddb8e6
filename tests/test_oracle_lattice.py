"""Pins for oracle/lattice.py: U_o structure, translation invariance, the
1-D circulant example of Sec. IV-B and the direct product of Eq. MVP."""
import os

import numpy as np
import pytest

from oracle import lattice, macromodel
from oracle.mesh import box_mesh

LAM = 0.03
K0 = 2 * np.pi / LAM
A = B = 0.5 * LAM
H = 0.25 * LAM
COEF = (1j * K0, 1.0, -1.0, 1j * K0)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_circulant_layout_is_first_column_generator():
    """The printed 5x5 circulant L'_aa (Eq. LJV3) has entry (i,j) equal to the
    block at offset d = test - source with d = (i - j) mod 5: the circulant's
    FIRST COLUMN is c[d mod P] = L(d).  (Eq. LJV5 transforms the first row,
    which equals the first column only for symmetric blocks.)"""
    rows = [l.split() for l in open(os.path.join(GOLD, "circulant_1d_example.txt"))
            if l.strip() and not l.startswith("#")]
    box_of = {1: 0, 3: 1, 5: 2}
    assert len(rows) == 5
    for i, row in enumerate(rows):
        for j, ent in enumerate(row):
            m, n = (int(v) for v in ent.split(","))
            d = box_of[m] - box_of[n]
            assert d % 5 == (i - j) % 5


def test_first_column_circulant_reproduces_toeplitz_product():
    rng = np.random.default_rng(7)
    N, P = 3, 5
    Ld = {d: rng.standard_normal() + 1j * rng.standard_normal() for d in range(-N + 1, N)}
    T = np.array([[Ld[i - j] for j in range(N)] for i in range(N)])
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c = np.zeros(P, complex)
    for d, v in Ld.items():
        c[d % P] = v
    xp = np.concatenate([x, np.zeros(P - N)])
    y = np.fft.ifft(np.fft.fft(c) * np.fft.fft(xp))[:N]
    assert np.allclose(y, T @ x, atol=1e-14)
    r = np.array([c[(-j) % P] for j in range(P)])     # first row
    y_row = np.fft.ifft(np.fft.fft(r) * np.fft.fft(xp))[:N]
    assert not np.allclose(y_row, T @ x, atol=1e-6)   # wrong for L^{ab} != (L^{ab})^T


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (1, 3), (2, 2), (3, 3)])
def test_overlap_map_structure(nx, ny):
    n = 2
    box = box_mesh(A, B, H, n)
    E = box.n_rwg
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, B)
    M = nx * ny
    assert idx.shape == (M * 2 * E,) and set(np.unique(sgn)) <= {-1, 1}
    assert idx.min() == 0 and idx.max() == nu - 1
    counts = np.bincount(idx, minlength=nu)
    assert set(np.unique(counts)) <= {1, 2, 4}
    # at least the face-interior RWGs of every shared face are merged
    shared = (nx - 1) * ny + nx * (ny - 1)
    assert nu <= M * 2 * E - 2 * (3 * n * n - 2 * n) * shared
    if M == 1:
        assert nu == 2 * E and np.array_equal(idx, np.arange(2 * E)) and np.all(sgn == 1)
    # first appearance numbering: ids increase along the scan
    first = np.full(nu, -1)
    for p, u in enumerate(idx):
        if first[u] < 0:
            first[u] = p
    assert np.all(np.diff(first) > 0)
    # J and M halves carry the same merge pattern
    blk = idx.reshape(M, 2, E)
    sg = sgn.reshape(M, 2, E)
    assert np.array_equal(sg[:, 0], sg[:, 1])
    assert np.array_equal(np.bincount(blk[:, 0].ravel())[np.unique(blk[:, 0])],
                          np.bincount(blk[:, 1].ravel())[np.unique(blk[:, 1])])


def test_direct_product_equals_box_pair_assembly():
    """Offset-table product (translation invariance, Sec. IV-A) equals the
    matrix built by tabulating every box pair directly."""
    n, nx, ny = 2, 2, 2
    box = box_mesh(A, B, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, B)
    rng = np.random.default_rng(3)
    Kl = 2 * box.n_rwg
    Zt = rng.standard_normal((2, Kl, Kl)) + 1j * rng.standard_normal((2, Kl, Kl))
    tmap = np.array([0, 1, 1, 0])
    Lt, Kt = lattice.offset_tables(box, nx, ny, A, B, K0)
    Ad = lattice.assemble_dense(box, nx, ny, A, B, K0, COEF, Zt, tmap, idx, sgn, nu)
    x = rng.standard_normal((2, nu)) + 1j * rng.standard_normal((2, nu))
    y = lattice.matvec_direct(x, Lt, Kt, COEF, Zt, tmap, idx, sgn, nu, nx, ny)
    assert np.abs(y - x @ Ad.T).max() <= 1e-13 * np.abs(y).max()


def test_sampled_rows_equal_full_direct_product():
    n, nx, ny = 2, 3, 2
    box = box_mesh(A, B, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, B)
    rng = np.random.default_rng(5)
    E = box.n_rwg
    Lt = rng.standard_normal((2 * ny - 1, 2 * nx - 1, E, E)) + 1j * rng.standard_normal((2 * ny - 1, 2 * nx - 1, E, E))
    Kt = rng.standard_normal(Lt.shape) + 1j * rng.standard_normal(Lt.shape)
    Zt = rng.standard_normal((3, 2 * E, 2 * E)) + 0j
    tmap = np.array([0, 1, 2, 2, 1, 0])
    x = rng.standard_normal(nu) + 1j * rng.standard_normal(nu)
    y = lattice.matvec_direct(x, Lt, Kt, COEF, Zt, tmap, idx, sgn, nu, nx, ny)
    rows = [0, 7, nu // 2, nu - 1]
    yr = lattice.matvec_direct_rows(x, rows, Lt, Kt, COEF, Zt, tmap, idx, sgn, nx, ny)
    assert np.abs(yr - y[rows]).max() <= 1e-12 * np.abs(y).max()
    Ad = lattice.assemble_from_tables(Lt, Kt, COEF, Zt, tmap, idx, sgn, nu, nx, ny)
    assert np.abs(Ad @ x - y).max() <= 1e-12 * np.abs(y).max()


def test_offset_tables_reciprocal_exactly():
    """The tables are the reciprocal part of the one-sided blocks: L(-d) =
    L(d)^T and K(-d) = K(d)^T to rounding at every offset, touching ones
    included, and at far offsets (where the one-sided blocks are already
    reciprocal) they equal the one-sided blocks."""
    from oracle.operators import galerkin_LK
    box = box_mesh(A, B, H, 2)
    nx, ny = 3, 3
    Lt, Kt = lattice.offset_tables(box, nx, ny, A, B, K0)
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            Lp, Kp = Lt[dy + ny - 1, dx + nx - 1], Kt[dy + ny - 1, dx + nx - 1]
            Lm, Km = Lt[-dy + ny - 1, -dx + nx - 1], Kt[-dy + ny - 1, -dx + nx - 1]
            assert np.abs(Lm - Lp.T).max() <= 1e-15 * np.abs(Lp).max()
            assert np.abs(Km - Kp.T).max() <= 1e-15 * np.abs(Kp).max() + 1e-300
    L1, K1 = galerkin_LK(box, lattice.cell_shift(2, 1, A, B), box, (0.0, 0.0, 0.0), K0, False)
    assert np.abs(Lt[1 + ny - 1, 2 + nx - 1] - L1).max() <= 1e-13 * np.abs(L1).max()
    assert np.abs(Kt[1 + ny - 1, 2 + nx - 1] - K1).max() <= 1e-13 * np.abs(K1).max()
    # the explicit-offset form gives the same blocks
    d = lattice.offset_tables(box, nx, ny, A, B, K0, offsets=[(1, 0), (0, 0)])
    assert np.array_equal(d[(1, 0)][0], Lt[ny - 1, 1 + nx - 1])
    assert np.array_equal(d[(0, 0)][1], Kt[ny - 1, nx - 1])
