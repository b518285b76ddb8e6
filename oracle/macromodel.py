"""Per-cell macromodels (oracle), Sec. II-B..D.

Follows the paper's steps for a cell whose interior is one homogeneous region
(free space) bounded by S_eq and containing PEC sheets:

1. per-region Galerkin blocks [L^E K^E; K^H L^H] over all surfaces of the
   region (Eq. ch5_macromodel_composite_SIE_Block), with the scaled form
   [[j k0 L, K], [-K, j k0 L]] (see operators.py) -- a PEC sheet carries J
   only, so it adds EFIE rows and J columns only (Sec. II-A);
2. U collects the S_eq unknowns first and the interior ones after
   (Eq. incidence1); for one interior region U is a permutation, so
   U^T Z U (Eq. mmm_mult) is the reordered block matrix;
3. the Schur complement Z~ = Z_ee - Z_ei Z_ii^{-1} Z_ie (Eq. Zmacromodel),
   solved with LU.

Reading: the configurations' eps_r = 3 slab is not modelled; the patch sits
in free space at the slab-top height.

Pins: empty box reproduces the incident-field currents (physics test);
PEC patch obeys the optical theorem (lossless) and reciprocity
Z~^T = S Z~ S, S = diag(I, -I); the Schur step equals solving the
unreduced system (brute force).
"""
import numpy as np
import scipy.linalg as sla

from .operators import galerkin_LK

ORIGIN = (0.0, 0.0, 0.0)


def region_block(L, K, k0, eps_r=1.0):
    return np.block([[1j * k0 * L, K], [-K, 1j * k0 * eps_r * L]])


def empty_box(box, k0):
    """Macromodel of an empty box: the interior free-space operator on S_eq."""
    L, K = galerkin_LK(box, ORIGIN, box, ORIGIN, k0, True)
    return region_block(L, K, k0)


def pec_sheet_system(box, sheet, k0):
    """Unreduced interior system of a box holding a PEC sheet.

    Unknown order: [J_eq (E), M_eq (E) | J_sheet (P)]; rows: EFIE on S_eq,
    MFIE on S_eq | EFIE on the sheet.  Returns (Z, n_eq)."""
    Lee, Kee = galerkin_LK(box, ORIGIN, box, ORIGIN, k0, True)
    Lep, Kep = galerkin_LK(box, ORIGIN, sheet, ORIGIN, k0, True)
    Lpe, Kpe = galerkin_LK(sheet, ORIGIN, box, ORIGIN, k0, True)
    Lpp, _ = galerkin_LK(sheet, ORIGIN, sheet, ORIGIN, k0, True)
    jk = 1j * k0
    Z = np.block([
        [jk * Lee, Kee, jk * Lep],
        [-Kee, jk * Lee, -Kep],
        [jk * Lpe, Kpe, jk * Lpp],
    ])
    return Z, 2 * box.n_rwg


def schur(Z, n_eq):
    """Z~ = Z_ee - Z_ei Z_ii^{-1} Z_ie (Eq. Zmacromodel)."""
    Zee, Zei = Z[:n_eq, :n_eq], Z[:n_eq, n_eq:]
    Zie, Zii = Z[n_eq:, :n_eq], Z[n_eq:, n_eq:]
    if Zii.shape[0] == 0:
        return Zee.copy()
    lu = sla.lu_factor(Zii)
    return Zee - Zei @ sla.lu_solve(lu, Zie)


def pec_patch(box, sheet, k0):
    Z, n_eq = pec_sheet_system(box, sheet, k0)
    return schur(Z, n_eq)
