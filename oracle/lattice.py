"""Lattice-level objects of Sec. III and the direct matrix-vector product (oracle).

* offset_tables: L(d), K(d) for every lattice offset d = test cell - source
  cell (Eqs. out, blockZo); blocks depend only on d because all boxes are
  translates of one mesh and G is translation invariant (Sec. IV-A).  The
  continuous operators are reciprocal (L(-d) = L(d)^T, K(-d) = K(d)^T by
  the symmetry of G and of the Galerkin pairing); the closed-form singular
  parts integrate the source triangle exactly and the test triangle by
  quadrature, which breaks that symmetry at touching offsets.  The tables
  are therefore the reciprocal part of the one-sided blocks,
  L(d) = (L1(d) + L1(-d)^T) / 2 (same for K): the average of the two
  one-sided quadratures, exactly reciprocal.
* overlap_map: the sparse +-1 matrix U_o of Eq. connections_IUI, built
  geometrically: two RWG functions of different boxes are merged when their
  edges coincide and one of their triangles coincides (rule 1, "surface
  common to two equivalent surfaces", with the limit Delta -> 0 of
  Fig. connections).  The signs make the coincident halves cancel, which
  states J^(m) = -J^(m') for vector fields on the shared face (outward
  normals are opposite).  Unique unknowns are numbered by first appearance
  scanning cells m = iy*Nx+ix, then local unknowns k (J_1..J_E, M_1..M_E).
* matvec_direct: y = U_o^T [Z_eq + Z_o] U_o x (Eq. MVP) as the plain sum
  y1^(m) = sum_m' B(c_m - c_m') x1^(m') + Z~^{t(m)} x1^(m); no FFT.
* assemble_dense: the full matrix of Eq. final with every box pair
  tabulated directly (not through the offset table).
"""
import numpy as np

from .operators import galerkin_LK


def cell_shift(ix, iy, a, b):
    return np.array([ix * a, iy * b, 0.0])


def coupling_block(L, K, coef):
    al, be, ga, de = coef
    return np.block([[al * L, be * K], [ga * K, de * L]])


def offset_tables(box, nx, ny, a, b, k, offsets=None):
    """L(d), K(d) for d in [-(nx-1), nx-1] x [-(ny-1), ny-1].

    Returns arrays (2ny-1, 2nx-1, E, E) indexed [dy+ny-1, dx+nx-1], or, when
    ``offsets`` (list of (dx,dy)) is given, a dict {(dx,dy): (L, K)}.
    Closed-form singular parts are used for touching boxes (|dx|,|dy| <= 1).
    """
    def one(dx, dy):
        sing = abs(dx) <= 1 and abs(dy) <= 1
        return galerkin_LK(box, cell_shift(dx, dy, a, b), box, (0.0, 0.0, 0.0), k, sing)

    def sym(dx, dy):
        Lp, Kp = one(dx, dy)
        Lm, Km = one(-dx, -dy)
        return 0.5 * (Lp + Lm.T), 0.5 * (Kp + Km.T)
    if offsets is not None:
        return {d: sym(*d) for d in offsets}
    E = box.n_rwg
    L1 = np.zeros((2 * ny - 1, 2 * nx - 1, E, E), dtype=complex)
    K1 = np.zeros_like(L1)
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            L1[dy + ny - 1, dx + nx - 1], K1[dy + ny - 1, dx + nx - 1] = one(dx, dy)
    # entry -d of the flipped table, transposed
    Lt = 0.5 * (L1 + np.swapaxes(L1[::-1, ::-1], 2, 3))
    Kt = 0.5 * (K1 + np.swapaxes(K1[::-1, ::-1], 2, 3))
    return Lt, Kt


def _key(p, scale):
    return tuple(int(round(c / scale)) for c in p)


def overlap_map(box, nx, ny, a, b):
    """U_o as (index (M*K,), sign (M*K,), n_unique); geometric construction."""
    E = box.n_rwg
    M = nx * ny
    scale = 1e-9 * max(a, b)
    edge_members = {}
    for iy in range(ny):
        for ix in range(nx):
            m = iy * nx + ix
            sh = cell_shift(ix, iy, a, b)
            V = box.verts + sh
            for e in range(E):
                ek = tuple(sorted((_key(V[box.edges[e, 0]], scale), _key(V[box.edges[e, 1]], scale))))
                tk = []
                for t in (box.tplus[e], box.tminus[e]):
                    tk.append(tuple(sorted(_key(V[v], scale) for v in box.tris[t])))
                edge_members.setdefault(ek, []).append((m, e, tk))
    parent = list(range(M * E))
    parity = [1] * (M * E)          # sign relative to parent

    def find(x):
        if parent[x] == x:
            return x, 1
        r, p = find(parent[x])
        parent[x] = r
        parity[x] *= p
        return r, parity[x]

    def union(x, y, s):             # enforce sigma_y = s * sigma_x
        rx, px = find(x)
        ry, py = find(y)
        if rx == ry:
            if px * py != s:
                raise ValueError("inconsistent U_o signs")
            return
        parent[ry] = rx
        parity[ry] = s * px * py

    for members in edge_members.values():
        for i in range(len(members)):
            for j in range(i + 1, len(members)):
                (m1, e1, t1), (m2, e2, t2) = members[i], members[j]
                if m1 == m2:
                    continue
                for r1, k1 in enumerate(t1):
                    for r2, k2 in enumerate(t2):
                        if k1 == k2:
                            s1 = 1 if r1 == 0 else -1
                            s2 = 1 if r2 == 0 else -1
                            union(m1 * E + e1, m2 * E + e2, -s1 * s2)
    uid = {}
    first_par = {}
    Kl = 2 * E
    index = np.zeros(M * Kl, dtype=np.int64)
    sign = np.zeros(M * Kl, dtype=np.int64)
    nxt = 0
    for m in range(M):
        for kk in range(Kl):
            part, e = divmod(kk, E)
            r, p = find(m * E + e)
            key = (r, part)
            if key not in uid:
                uid[key] = nxt
                first_par[key] = p
                nxt += 1
            index[m * Kl + kk] = uid[key]
            sign[m * Kl + kk] = p * first_par[key]
    return index, sign, nxt


def gather(x, index, sign, M, Kl):
    """x1 = U_o x, returned as (M, K)."""
    return (sign * x[index]).reshape(M, Kl)


def scatter(y1, index, sign, n_unique):
    """y = U_o^T y1."""
    y = np.zeros(n_unique, dtype=complex)
    np.add.at(y, index, sign * y1.reshape(-1))
    return y


def matvec_direct(x, Lt, Kt, coef, macromodels, type_map, index, sign, n_unique, nx, ny):
    """y = U_o^T [Z_eq + Z_o] U_o x (Eq. MVP), plain offset sum, no FFT.

    Lt, Kt: (2ny-1, 2nx-1, E, E) offset tables; macromodels (T, K, K);
    type_map (ny*nx,) cell -> type; x: (n_unique,) or (R, n_unique).
    """
    x = np.asarray(x)
    if x.ndim == 2:
        return np.stack([matvec_direct(xi, Lt, Kt, coef, macromodels, type_map, index,
                                       sign, n_unique, nx, ny) for xi in x])
    E = Lt.shape[-1]
    Kl = 2 * E
    M = nx * ny
    x1 = gather(x, index, sign, M, Kl)
    y1 = np.zeros((M, Kl), dtype=complex)
    for m in range(M):
        y1[m] += macromodels[type_map[m]] @ x1[m]
    for dy in range(-(ny - 1), ny):
        for dx in range(-(nx - 1), nx):
            B = coupling_block(Lt[dy + ny - 1, dx + nx - 1], Kt[dy + ny - 1, dx + nx - 1], coef)
            for iy in range(max(0, dy), min(ny, ny + dy)):
                for ix in range(max(0, dx), min(nx, nx + dx)):
                    m, ms = iy * nx + ix, (iy - dy) * nx + (ix - dx)
                    y1[m] += B @ x1[ms]
    return scatter(y1, index, sign, n_unique)


def assemble_dense(box, nx, ny, a, b, k, coef, macromodels, type_map, index, sign, n_unique):
    """Dense A = U_o^T [Z_eq + Z_o] U_o (Eq. final) with every box pair
    (m, m') tabulated directly by quadrature (reciprocal part of the
    one-sided blocks, as in offset_tables)."""
    E = box.n_rwg
    Kl = 2 * E
    M = nx * ny
    Z = np.zeros((M * Kl, M * Kl), dtype=complex)
    for m in range(M):
        ix, iy = m % nx, m // nx
        for ms in range(M):
            jx, jy = ms % nx, ms // nx
            sing = abs(ix - jx) <= 1 and abs(iy - jy) <= 1
            Lp, Kp = galerkin_LK(box, cell_shift(ix, iy, a, b), box, cell_shift(jx, jy, a, b),
                                 k, sing)
            Lm, Km = galerkin_LK(box, cell_shift(jx, jy, a, b), box, cell_shift(ix, iy, a, b),
                                 k, sing)
            L, K = 0.5 * (Lp + Lm.T), 0.5 * (Kp + Km.T)
            Z[m * Kl:(m + 1) * Kl, ms * Kl:(ms + 1) * Kl] = coupling_block(L, K, coef)
        Z[m * Kl:(m + 1) * Kl, m * Kl:(m + 1) * Kl] += macromodels[type_map[m]]
    U = np.zeros((M * Kl, n_unique))
    U[np.arange(M * Kl), index] = sign
    return U.T @ Z @ U


def _block(Lt, Kt, coef, dx, dy, nx, ny):
    return coupling_block(Lt[dy + ny - 1, dx + nx - 1], Kt[dy + ny - 1, dx + nx - 1], coef)


def matvec_direct_rows(x, rows, Lt, Kt, coef, macromodels, type_map, index, sign, nx, ny):
    """Entries ``rows`` of y = U_o^T [Z_eq + Z_o] U_o x, one at a time:
    y[u] = sum over local unknowns (m,k) of u of sign * (row k of
    sum_m' B(c_m - c_m') x1^(m') + Z~^{t(m)} x1^(m))."""
    E = Lt.shape[-1]
    Kl = 2 * E
    M = nx * ny
    x1 = gather(np.asarray(x), index, sign, M, Kl)
    out = np.zeros(len(rows), dtype=complex)
    for q, u in enumerate(rows):
        for loc in np.nonzero(index == u)[0]:
            m, k = divmod(int(loc), Kl)
            ix, iy = m % nx, m // nx
            acc = macromodels[type_map[m]][k] @ x1[m]
            for ms in range(M):
                jx, jy = ms % nx, ms // nx
                dx, dy = ix - jx, iy - jy
                half, kk = divmod(k, E)
                Lr = Lt[dy + ny - 1, dx + nx - 1][kk]
                Kr = Kt[dy + ny - 1, dx + nx - 1][kk]
                al, be, ga, de = coef
                if half == 0:
                    acc += al * (Lr @ x1[ms, :E]) + be * (Kr @ x1[ms, E:])
                else:
                    acc += ga * (Kr @ x1[ms, :E]) + de * (Lr @ x1[ms, E:])
            out[q] += sign[loc] * acc
    return out


def assemble_from_tables(Lt, Kt, coef, macromodels, type_map, index, sign, n_unique, nx, ny):
    """Dense U_o^T [Z_eq + Z_o] U_o built block by block from the offset tables."""
    E = Lt.shape[-1]
    Kl = 2 * E
    M = nx * ny
    Z = np.zeros((M * Kl, M * Kl), dtype=complex)
    for m in range(M):
        ix, iy = m % nx, m // nx
        for ms in range(M):
            jx, jy = ms % nx, ms // nx
            Z[m * Kl:(m + 1) * Kl, ms * Kl:(ms + 1) * Kl] = _block(Lt, Kt, coef, ix - jx, iy - jy, nx, ny)
        Z[m * Kl:(m + 1) * Kl, m * Kl:(m + 1) * Kl] += macromodels[type_map[m]]
    U = np.zeros((M * Kl, n_unique))
    U[np.arange(M * Kl), index] = sign
    return U.T @ Z @ U
