"""Near-field preconditioner by cell subdomains (oracle; test infrastructure only).

Sec. IV-A preconditions Eq. final on the right with the near-field part of
the system (Eq. final_precond: entries between basis functions closer than a
threshold).  The preconditioner checked here groups that near field by cell
and applies it as restricted additive Schwarz (Cai & Sarkis 1999):

* position of a unique unknown: the midpoint of its RWG edge in the first
  cell that references it (all copies merged by U_o share that edge, so any
  copy gives the same point);
* owner of a unique unknown: the first cell that references it (cells
  scanned m = iy*Nx + ix, local unknowns in order);
* subdomain S_m: every unique unknown whose position lies in cell m's
  footprint [-a/2, a/2] x [-b/2, b/2] (centred on the cell's shift) grown by
  the margin delta on each side;
* M^{-1} r = sum_m Rt_m^T A[S_m, S_m]^{-1} r[S_m], where Rt_m keeps only the
  entries of S_m owned by m.

A is the dense matrix of Eq. final (assemble_from_tables).  Everything is
complex128 with dense solves, so this is the exact-arithmetic definition that
the device's FP32 factorisation is compared with.  For lattices too large for
a dense A, subdomain_matrix forms one block A[S, S] from the same definition
restricted to the cells that hold a copy of an unknown in S.
"""
import numpy as np

from .lattice import _block, cell_shift


def unknown_positions(box, index, nx, ny, a, b):
    """(xy [n_unique, 2], owner [n_unique]) from the first referencing copy."""
    E = box.n_rwg
    Kl = 2 * E
    n_unique = int(index.max()) + 1
    mid = 0.5 * (box.verts[box.edges[:, 0]] + box.verts[box.edges[:, 1]])
    xy = np.zeros((n_unique, 2))
    owner = -np.ones(n_unique, dtype=np.int64)
    for m in range(nx * ny):
        shift = cell_shift(m % nx, m // nx, a, b)
        for k in range(Kl):
            u = index[m * Kl + k]
            if owner[u] < 0:
                owner[u] = m
                xy[u] = (mid[k % E] + shift)[:2]
    return xy, owner


def subdomains(xy, owner, nx, ny, a, b, delta, eps=1e-12):
    """[(S_m sorted unique ids, owned mask)] for every cell m."""
    out = []
    for m in range(nx * ny):
        c = cell_shift(m % nx, m // nx, a, b)
        inside = (np.abs(xy[:, 0] - c[0]) <= 0.5 * a + delta + eps) & \
                 (np.abs(xy[:, 1] - c[1]) <= 0.5 * b + delta + eps)
        S = np.nonzero(inside)[0]
        out.append((S, owner[S] == m))
    return out


def ras_apply(A, subs, r):
    """M^{-1} r for one vector r (complex128)."""
    y = np.zeros(A.shape[0], dtype=np.complex128)
    for S, own in subs:
        z = np.linalg.solve(A[np.ix_(S, S)], r[S])
        y[S[own]] += z[own]
    return y


def subdomain_matrix(S, Lt, Kt, coef, macromodels, type_map, index, sign, nx, ny):
    """A[S, S] of A = U_o^T [Z_eq + Z_o] U_o (Eq. final) for unique unknowns S.
    Column u of U_o is zero outside the local slots that copy u, so only the
    cells holding such a copy enter: Z_eq + Z_o is formed over those cells
    (offset blocks plus the macromodel on the diagonal, Eqs. out, blockZo,
    Zmacromodel_Array) and reduced with the matching rows of U_o."""
    E = Lt.shape[-1]
    Kl = 2 * E
    S = np.asarray(S)
    col = -np.ones(int(index.max()) + 1, dtype=np.int64)
    col[S] = np.arange(len(S))
    locs = np.nonzero(col[index] >= 0)[0]
    cells = np.unique(locs // Kl)
    pos = {int(m): a for a, m in enumerate(cells)}
    nc = len(cells)
    Z = np.zeros((nc * Kl, nc * Kl), dtype=complex)
    for a, m in enumerate(cells):
        ix, iy = m % nx, m // nx
        for b, ms in enumerate(cells):
            jx, jy = ms % nx, ms // nx
            Z[a * Kl:(a + 1) * Kl, b * Kl:(b + 1) * Kl] = _block(Lt, Kt, coef, ix - jx, iy - jy, nx, ny)
        Z[a * Kl:(a + 1) * Kl, a * Kl:(a + 1) * Kl] += macromodels[type_map[m]]
    U = np.zeros((nc * Kl, len(S)))
    rows = np.array([pos[int(l // Kl)] * Kl + int(l % Kl) for l in locs], dtype=np.int64)
    U[rows, col[index[locs]]] = sign[locs]
    return U.T @ Z @ U
