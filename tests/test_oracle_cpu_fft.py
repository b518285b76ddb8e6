"""The CPU FFT product (the timed CPU FFT baseline) equals the oracle's
FFT-free direct product (Eq. MVP) to rounding, on non-symmetric random
blocks (so a row instead of a column generator, a transposed block or a
wrong sign of d fails) and for any grid >= 2N - 1 (Sec. IV-B embedding)."""
import numpy as np
import pytest

from oracle import cpu_fft, lattice
from oracle.mesh import box_mesh
from paper_1911_04576_gb300 import workloads as W


@pytest.mark.parametrize("n,nx,ny,grid", [(1, 3, 2, (5, 3)), (1, 4, 4, (8, 7)), (2, 2, 3, (3, 6)), (1, 1, 1, (1, 1))])
def test_cpu_fft_product_equals_direct(n, nx, ny, grid):
    a = 0.015
    box = box_mesh(a, a, 0.0075, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, a, a)
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, 31 + nx)
    Z = W.random_macromodels(3, 2 * E, 32)
    tmap = np.random.default_rng(33).integers(0, 3, nx * ny)
    coef = (0.3 + 1.1j, -0.7, 1.3 + 0.2j, 0.5j)
    x = W.random_vectors(1, nu, 34)[0]
    px, py = grid
    Lh, Kh = cpu_fft.spectrum(Lt, Kt, px, py, workers=2)
    y = cpu_fft.matvec(x, Lh, Kh, coef, Z, tmap, idx, sgn, nu, nx, ny, workers=2)
    ref = lattice.matvec_direct(x, Lt, Kt, coef, Z, tmap, idx, sgn, nu, nx, ny)
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
