"""Per-cell macromodels (oracle), Sec. II-B..D.

Follows the paper's steps for a cell bounded by S_eq:

1. per-region Galerkin blocks [L^E K^E; K^H L^H] over all surfaces of the
   region (Eq. ch5_macromodel_composite_SIE_Block), with the scaled form
   [[j k0 L_v, K_v], [-K_v, j k0 eps_v L_v]], k_v = k0 sqrt(eps_v) (see
   operators.py) -- an RWG touching a PEC carries J only, so it adds EFIE
   rows and J columns only (Sec. II-A);
2. Z = the block diagonal of the regions (Eq. discretized_SIE);
3. U collects the S_eq unknowns first and the interior ones after and
   enforces the boundary conditions of Sec. II-C (Eq. incidence1): rules
   1-3 inside the cell and the junction of an interface with S_eq;
4. U^T Z U (Eq. mmm_mult);
5. the Schur complement Z~ = Z_ee - Z_ei Z_ii^{-1} Z_ie (Eq. Zmacromodel),
   solved with LU.

Cells: empty_box (one free-space region), pec_patch (a PEC sheet inside a
free-space box: one region, U a permutation), slab_patch (the
configurations' cell: a lossy dielectric slab filling the bottom of the box,
a PEC patch on the slab top, air above -- two regions, composite_system).

Readings: the slab top is a mesh surface of its own, conforming to the box
row boundary at the slab height (the junction of Fig. composite) and to the
patch; its ring around the patch is refined toward the patch edge (see
mesh.slab_top_mesh).  Interior Galerkin blocks are one-sided (closed-form
singular integration over the source triangle), so reciprocity holds to
quadrature accuracy.

Pins: empty box reproduces the incident-field currents (physics test);
PEC patch obeys the optical theorem (lossless) and reciprocity
Z~^T = S Z~ S, S = diag(I, -I); the Schur step equals solving the
unreduced system (brute force); a transparent slab scatters nothing and a
patch on it approaches the free-space patch; a lossy dielectric sphere
matches the Mie series; lossless slab cells obey the optical theorem and
lossy ones absorb (tests/test_oracle_slab.py).
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


def _tri_edge(mesh, t1, t2):
    """Vertex pair of the edge shared by triangles t1 and t2 of a mesh."""
    common = set(mesh.tris[t1].tolist()) & set(mesh.tris[t2].tolist())
    if len(common) != 2:
        raise ValueError("triangles do not share an edge")
    return common


def _rwg_of(mesh, t_key_a, t_key_b):
    """RWG of `mesh` whose triangles are (t_key_a, t_key_b) in either order."""
    for e in range(mesh.n_rwg):
        if {int(mesh.tplus[e]), int(mesh.tminus[e])} == {t_key_a, t_key_b}:
            return e
    raise ValueError("no RWG on triangles %d, %d" % (t_key_a, t_key_b))


def _rwg_sign(mesh_a, ra, ta, mesh_b, rb, tb):
    """+1 if RWG ra of mesh_a on its triangle ta is the same vector field as
    RWG rb of mesh_b on its triangle tb (the same physical triangle), else -1.
    Both are +-(r - free vertex) l / (2A), the free vertex being the one off
    the common edge, so only the slot signs differ."""
    sa = mesh_a.slot_sgn[ta][mesh_a.slot_rwg[ta] == ra][0]
    sb = mesh_b.slot_sgn[tb][mesh_b.slot_rwg[tb] == rb][0]
    return int(sa * sb)


def composite_system(box, regions, surfaces, k0):
    """Interior system U^T Z U of a cell with several homogeneous regions
    (Secs. II-B, II-C) and its split into S_eq and interior unknowns.

    box: the S_eq mesh; its RWGs carry the unknowns J_eq, M_eq (ordered
    J_1..J_E, M_1..M_E, first in X~).
    surfaces: {name: (mesh, pec (T,) bool, (v_plus, v_minus))} interior
    surfaces; an interface between two regions lists both (v_minus None
    for a PEC sheet inside one region).
    regions: list of (mesh, keys, eps_r): the closed surface S_v of region
    v, keys[t] = ('eq', box triangle) or (surface name, surface triangle).

    Step 1 (Eq. ch5_macromodel_composite_SIE_Block): per region, with
    k_v = k0 sqrt(eps_v), the tested EFIE/MFIE block
    [[j k0 L_v, K_v], [-K_v, j k0 eps_v L_v]] over the RWGs of S_v; an RWG
    touching a PEC triangle carries J only (M = 0 on a PEC, Sec. II-A), so
    its M column and its MFIE row are dropped.
    Step 2 (Eq. discretized_SIE): Z = block diagonal of the regions.
    Step 3 (Eq. incidence1): U maps X~ to the region unknowns X by the
    rules of Sec. II-C:
      * S_eq RWG (both triangles on S_eq) and the junction of an interface
        with S_eq (one triangle on S_eq, the other on the interface, label 2
        of Fig. composite): the region RWG equals the S_eq RWG of that edge;
      * interface between two dielectrics (rule 1): one J and one M unknown
        shared by the two regions, with opposite signs (the fields
        n_v x H and -n_v x E flip with the normal);
      * PEC-dielectric junction (rule 3, one triangle on the patch): one
        shared J unknown as in rule 1, no M;
      * PEC at an interface (rule 2, both triangles on the PEC): one J
        unknown per side.
    Every region copy of an S_eq unknown takes the same sign, so the sign
    convention between n_v and the outward normal of S_eq cancels in the
    Schur complement.
    Step 4 (Eq. mmm_mult): U^T Z U.  Returns (Zt, n_eq)."""
    E = box.n_rwg
    box_edge = {tuple(sorted(map(int, box.edges[e]))): e for e in range(E)}
    cols = {}            # X~ unknown key -> column
    for e in range(E):
        cols[("J", "eq", e)] = e
        cols[("M", "eq", e)] = E + e
    blocks, rowmaps = [], []
    for v, (mesh, keys, eps) in enumerate(regions):
        kv = k0 * np.sqrt(complex(eps))
        L, Kop = galerkin_LK(mesh, ORIGIN, mesh, ORIGIN, kv, True)
        Zv = np.block([[1j * k0 * L, Kop], [-Kop, 1j * k0 * eps * L]])
        Ev = mesh.n_rwg
        keep, rmap = [], []
        for r in range(Ev):
            tp, tm = int(mesh.tplus[r]), int(mesh.tminus[r])
            kp, km = keys[tp], keys[tm]
            if kp[0] == "eq" or km[0] == "eq":
                t_eq, t_loc = (kp[1], tp) if kp[0] == "eq" else (km[1], tm)
                if kp[0] != "eq" and surfaces[kp[0]][1][kp[1]] or km[0] != "eq" and surfaces[km[0]][1][km[1]]:
                    raise ValueError("PEC touching S_eq is not modelled")
                ed = box_edge[tuple(sorted(int(mesh_v) for mesh_v in _box_vertex_pair(mesh, tp, tm, box)))]
                s = _rwg_sign(mesh, r, t_loc, box, ed, t_eq)
                entries = [("J", "eq", ed, s), ("M", "eq", ed, s)]
            else:
                if kp[0] != km[0]:
                    raise ValueError("RWG across two interior surfaces")
                name = kp[0]
                smesh, pec, (vp, vm) = surfaces[name]
                sr = _rwg_of(smesh, kp[1], km[1])
                s = _rwg_sign(mesh, r, tp, smesh, sr, kp[1])
                side = 1 if v == vp else -1
                npec = int(pec[kp[1]]) + int(pec[km[1]])
                if npec == 2:                                   # rule 2
                    entries = [("J", ("pec", v), (name, sr), s)]
                elif npec == 1:                                 # rule 3
                    entries = [("J", "int", (name, sr), side * s)]
                else:                                           # rule 1
                    entries = [("J", "int", (name, sr), side * s), ("M", "int", (name, sr), side * s)]
            has_m = any(en[0] == "M" for en in entries)
            keep.append(r)
            rmap.append(entries[0])
            if has_m:
                keep.append(Ev + r)
                rmap.append(entries[1])
        blocks.append(Zv[np.ix_(keep, keep)])
        rowmaps.append(rmap)
        for kind, cls, key, _ in rmap:
            ck = (kind, cls, key)
            if ck not in cols:
                cols[ck] = len(cols)
    nx_ = sum(len(rm) for rm in rowmaps)
    U = np.zeros((nx_, len(cols)))
    Zbd = np.zeros((nx_, nx_), dtype=complex)
    o = 0
    for Zv, rmap in zip(blocks, rowmaps):
        n_v = len(rmap)
        Zbd[o:o + n_v, o:o + n_v] = Zv
        for i, (kind, cls, key, s) in enumerate(rmap):
            U[o + i, cols[(kind, cls, key)]] = s
        o += n_v
    return U.T @ Zbd @ U, 2 * E


def _box_vertex_pair(mesh, tp, tm, box):
    """The common edge of region triangles tp, tm as box vertex indices
    (region meshes list the box vertices first, unchanged)."""
    pair = _tri_edge(mesh, tp, tm)
    if max(pair) >= len(box.verts):
        raise ValueError("edge on S_eq not made of box vertices")
    return pair


def slab_patch(box, n, side, patch_n, eps_r, k0, slab_t, ring_layers=3):
    """Macromodel Z~ (Eq. Zmacromodel) of the configurations' cell: a
    dielectric slab of relative permittivity eps_r (lossy: Im eps_r < 0
    under e^{jwt}) filling the bottom slab_t of the box, a flat PEC square
    patch of the given side on the slab top (side <= 0: slab only), air
    above.  box: box_mesh(a, b, h, n, slab_zlevels(h, n, slab_t)).  Regions
    (air: eps 1, slab: eps_r) and U follow composite_system; the Schur
    complement eliminates the slab-top and patch unknowns."""
    from .mesh import slab_region_meshes, slab_top_mesh
    a = box.verts[:, 0].max() - box.verts[:, 0].min()
    b = box.verts[:, 1].max() - box.verts[:, 1].min()
    if side > 0:
        top, pec = slab_top_mesh(a, b, slab_t, n, side, patch_n, ring_layers)
    else:
        top, pec = _bare_top(a, b, slab_t, n)
    (air, kair), (slab, kslab) = slab_region_meshes(box, n, top)
    surfaces = {"top": (top, pec, (1, 0))}
    Z, n_eq = composite_system(box, [(air, kair, 1.0), (slab, kslab, eps_r)], surfaces, k0)
    return schur(Z, n_eq)


def _bare_top(a, b, z, n):
    """Slab top without a patch: the footprint grid of the box rows, n x n
    quads split like the box faces, vertices ordered so the boundary ones
    come last in _perimeter order (as slab_top_mesh)."""
    from .mesh import Mesh, _perimeter
    xs = -0.5 * a + a * np.arange(n + 1) / n
    ys = -0.5 * b + b * np.arange(n + 1) / n
    per = _perimeter(n)
    inner = [(i, j) for i in range(1, n) for j in range(1, n)]
    order = inner + per
    index = {q: m for m, q in enumerate(order)}
    verts = np.array([[xs[i], ys[j], z] for i, j in order])
    tris = []
    for v in range(n):
        for u in range(n):
            c00, c10, c01, c11 = index[(u, v)], index[(u + 1, v)], index[(u, v + 1)], index[(u + 1, v + 1)]
            tris.append((c00, c10, c11))
            tris.append((c00, c11, c01))
    return Mesh(verts, tris), np.zeros(len(tris), dtype=bool)
