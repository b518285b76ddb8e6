"""CPU FFT-accelerated product of Eq. final: a timing baseline only.

Test and timing infrastructure, like the rest of oracle/: the product path
never imports it.  It computes the same y = U_o^T [Z_eq + Z_o] U_o x as
lattice.matvec_direct (Eq. MVP), but the way Sec. IV-B does on a CPU:

1. the offset blocks embedded in a circulant over a px x py grid (first
   column generator: block B(d) at grid point (dx mod px, dy mod py),
   d = test - source) and transformed by a 2-D FFT over the lattice for
   every block entry -- the spectrum, built once;
2. per product: x1 = U_o x zero-padded onto the grid and transformed,
   the per-bin block product y^(k) = B^(k) x^(k) (L/K form:
   y_J = a L^ x_J + b K^ x_M, y_M = g K^ x_J + d L^ x_M), the inverse
   transform (1/P) cropped to the lattice, plus the block-diagonal
   macromodel product, then U_o^T.

complex128 throughout, numpy/scipy with every host core (scipy.fft
workers; BLAS threads for the batched per-bin products).  Pin: equal to
lattice.matvec_direct to rounding (tests/test_oracle_cpu_fft.py).
"""
import numpy as np
import scipy.fft as sfft

from .lattice import gather, scatter


def spectrum(Lt, Kt, px, py, workers=-1):
    """L^, K^ of shape (py, px, E, E): the circulant first columns transformed."""
    ny, nx = (Lt.shape[0] + 1) // 2, (Lt.shape[1] + 1) // 2
    if px < 2 * nx - 1 or py < 2 * ny - 1:
        raise ValueError("grid smaller than 2N - 1")
    out = []
    for T in (Lt, Kt):
        G = np.zeros((py, px) + T.shape[2:], dtype=complex)
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                G[dy % py, dx % px] = T[dy + ny - 1, dx + nx - 1]
        out.append(sfft.fft2(G, axes=(0, 1), workers=workers, overwrite_x=True))
    return out[0], out[1]


def matvec(x, Lh, Kh, coef, macromodels, type_map, index, sign, n_unique, nx, ny, workers=-1):
    """y = A x for x of shape (n_unique,) with the spectrum of spectrum()."""
    py, px, E, _ = Lh.shape
    Kl = 2 * E
    M = nx * ny
    x1 = gather(np.asarray(x), index, sign, M, Kl)                 # (M, K)
    Xg = np.zeros((py, px, Kl), dtype=complex)
    Xg[:ny, :nx] = x1.reshape(ny, nx, Kl)
    Xh = sfft.fft2(Xg, axes=(0, 1), workers=workers, overwrite_x=True)
    al, be, ga, de = coef
    XJ, XM = Xh[..., :E, None], Xh[..., E:, None]
    Yh = np.empty_like(Xh)
    Yh[..., :E] = (al * np.matmul(Lh, XJ) + be * np.matmul(Kh, XM))[..., 0]
    Yh[..., E:] = (ga * np.matmul(Kh, XJ) + de * np.matmul(Lh, XM))[..., 0]
    Yg = sfft.ifft2(Yh, axes=(0, 1), workers=workers, overwrite_x=True)
    y1 = Yg[:ny, :nx].reshape(M, Kl)
    y1 = y1 + np.einsum("mkl,ml->mk", macromodels[type_map], x1)
    return scatter(y1.reshape(-1), index, sign, n_unique)
