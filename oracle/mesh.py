"""Box-surface and patch meshes with RWG bases (oracle).

Follows Sec. II-A: each unit cell is enclosed by a rectangular prism S_eq
with the cell footprint; opposite side faces are meshed identically so that
coincident faces of neighbouring boxes carry identical triangles and every
box is a translate of box 0.  Currents are expanded in RWG functions
(Eqs. Hdiscretebox, Ediscretebox).

Canonical numbering (the product's setup library implements the same
convention independently; tests compare the two arrays exactly):

* box for cell (0,0): x in [-a/2, a/2], y in [-b/2, b/2], z in [0, h];
  surface grid points (i,j,k) in {0..n}^3 with at least one index in {0,n},
  numbered in lexicographic (i,j,k) order;
* faces in the order x-, x+, y-, y+, z-, z+; in-plane axes (u,v) are (j,k),
  (i,k), (i,j) for x, y, z faces; quad (u,v) has index v*n+u; for even n
  it is cut along the diagonal that points at the face centre (a
  union-jack pattern): when (2u+1 < n) == (2v+1 < n) its two triangles
  are (c00,c10,c11) then (c00,c11,c01), else (c00,c10,c01) then
  (c10,c11,c01); for odd n every quad is cut the first way;
  triangle index = face*2n^2 + 2*(v*n+u) + {0,1};
* RWG edges are the distinct vertex pairs (lo,hi), sorted lexicographically;
  T+ is the lower-numbered of the two triangles sharing the edge;
* slot i of a triangle is the edge opposite its vertex i (free vertex i).

The union-jack cut makes the box mesh invariant under the mirrors
x -> -x and y -> -y (and x <-> y when a = b), so each mirror maps
every RWG function onto +-1 times another (box_mirrors); the lattice
operator then inherits the mirror symmetries of the continuous problem
exactly, and the blocks of mirrored lattice offsets are signed
permutations of one another.  For odd n the middle quads of a face lie on
a mirror plane and no cut of them is symmetric; those boxes keep the
uniform cut (which is also more accurate than the union jack on coarse
boxes: RCS of a dielectric sphere within 0.83 dB of the Mie series at
n = 3 against 1.0 dB).

Pins: E = 18 n^2 edges on a closed box, each shared by two triangles,
opposite faces are exact translates, and every RWG has zero net charge.
"""
import numpy as np

FACES = (("x", 0), ("x", 1), ("y", 0), ("y", 1), ("z", 0), ("z", 1))


def _face_triple(axis, fixed, u, v):
    if axis == "x":
        return (fixed, u, v)
    if axis == "y":
        return (u, fixed, v)
    return (u, v, fixed)


class Mesh:
    """Triangle mesh with RWG functions on its interior edges.

    verts (V,3) float, tris (T,3) int, edges (E,2) int, tplus/tminus (E,),
    slot_rwg (T,3) RWG index of the edge opposite vertex i (-1: no RWG),
    slot_sgn (T,3) +1 if the triangle is T+ of that RWG, -1 if T-.
    """

    def __init__(self, verts, tris):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        T = len(self.tris)
        owners = {}
        for t in range(T):
            for i in range(3):
                p, q = self.tris[t, (i + 1) % 3], self.tris[t, (i + 2) % 3]
                key = (min(p, q), max(p, q))
                owners.setdefault(key, []).append((t, i))
        keys = sorted(k for k, o in owners.items() if len(o) == 2)
        for k, o in owners.items():
            if len(o) > 2:
                raise ValueError("non-manifold edge %r" % (k,))
        self.edges = np.array(keys, dtype=np.int64).reshape(-1, 2)
        self.slot_rwg = -np.ones((T, 3), dtype=np.int64)
        self.slot_sgn = np.zeros((T, 3), dtype=np.int64)
        self.tplus = np.zeros(len(keys), dtype=np.int64)
        self.tminus = np.zeros(len(keys), dtype=np.int64)
        for e, k in enumerate(keys):
            (t1, i1), (t2, i2) = sorted(owners[k])
            self.tplus[e], self.tminus[e] = t1, t2
            self.slot_rwg[t1, i1], self.slot_sgn[t1, i1] = e, 1
            self.slot_rwg[t2, i2], self.slot_sgn[t2, i2] = e, -1

    @property
    def n_rwg(self):
        return len(self.edges)

    def tri_coords(self, shift=(0.0, 0.0, 0.0)):
        return self.verts[self.tris] + np.asarray(shift, dtype=np.float64)

    def slot_len(self):
        """Length of the edge opposite each vertex, (T,3)."""
        c = self.verts[self.tris]
        return np.stack([np.linalg.norm(c[:, (i + 2) % 3] - c[:, (i + 1) % 3], axis=-1)
                         for i in range(3)], axis=-1)


def box_grid_points(n):
    """Integer surface grid points of the box, lexicographic (i,j,k)."""
    pts = [(i, j, k) for i in range(n + 1) for j in range(n + 1) for k in range(n + 1)
           if i in (0, n) or j in (0, n) or k in (0, n)]
    return pts


def box_mesh(a, b, h, n, zlevels=None):
    """Closed box surface, n x n quads per face (Sec. II-A).

    zlevels: optional (n+1,) increasing z coordinates of the grid rows,
    default uniform in [0, h].
    """
    pts = box_grid_points(n)
    index = {p: m for m, p in enumerate(pts)}
    xs = -0.5 * a + a * np.arange(n + 1) / n
    ys = -0.5 * b + b * np.arange(n + 1) / n
    zs = h * np.arange(n + 1) / n if zlevels is None else np.asarray(zlevels, float)
    verts = np.array([[xs[i], ys[j], zs[k]] for (i, j, k) in pts])
    tris = []
    for axis, side in FACES:
        fixed = n * side
        for v in range(n):
            for u in range(n):
                c00 = index[_face_triple(axis, fixed, u, v)]
                c10 = index[_face_triple(axis, fixed, u + 1, v)]
                c01 = index[_face_triple(axis, fixed, u, v + 1)]
                c11 = index[_face_triple(axis, fixed, u + 1, v + 1)]
                if n % 2 == 1 or (2 * u + 1 < n) == (2 * v + 1 < n):
                    tris.append((c00, c10, c11))
                    tris.append((c00, c11, c01))
                else:
                    tris.append((c00, c10, c01))
                    tris.append((c10, c11, c01))
    return Mesh(verts, tris)


# the mirrors of the box about its axis: x -> -x, y -> -y, x <-> y
MIRRORS = {"x": np.diag([-1.0, 1.0, 1.0]), "y": np.diag([1.0, -1.0, 1.0]),
           "d": np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])}


def box_mirrors(box, a, b):
    """Signed permutations of the RWG functions under the box's mirrors.

    For each mirror g in MIRRORS that maps the mesh onto itself (every
    vertex onto a vertex, every triangle onto a triangle; "d" only when
    a == b), the RWG function f_n mirrored, (g f_n)(r) = g f_n(g r), is
    sign[n] * f_pi[n]: its edge is the image of edge n and its T+ is the
    image of n's T+ (sign +1) or of n's T- (sign -1).  Returns
    {name: (pi, sign)} for the mirrors that apply.
    """
    out = {}
    V = box.verts
    scale = max(np.abs(V).max(), 1e-300)
    key = {tuple(np.round(v / scale, 9)): i for i, v in enumerate(V)}
    ekey = {tuple(e): i for i, e in enumerate(box.edges)}
    tkey = {tuple(sorted(t)): i for i, t in enumerate(box.tris)}
    for name, g in MIRRORS.items():
        if name == "d" and a != b:
            continue
        vmap = []
        for v in V @ g.T:
            vmap.append(key.get(tuple(np.round(v / scale, 9)), -1))
        vmap = np.array(vmap)
        if (vmap < 0).any():
            continue
        pi = np.zeros(box.n_rwg, dtype=np.int64)
        sign = np.zeros(box.n_rwg, dtype=np.int64)
        ok = True
        for n, (p, q) in enumerate(box.edges):
            m = ekey.get(tuple(sorted((vmap[p], vmap[q]))), -1)
            tp = tkey.get(tuple(sorted(vmap[box.tris[box.tplus[n]]])), -1)
            if m < 0 or tp not in (box.tplus[m], box.tminus[m]):
                ok = False
                break
            pi[n] = m
            sign[n] = 1 if tp == box.tplus[m] else -1
        if ok:
            out[name] = (pi, sign)
    return out

def patch_mesh(side, z, n):
    """Flat square PEC patch of the given side centred on the cell axis at
    height z, n x n quads each cut along its (c00, c11) diagonal; RWGs on
    interior edges."""
    xs = -0.5 * side + side * np.arange(n + 1) / n
    verts = np.array([[xs[i], xs[j], z] for i in range(n + 1) for j in range(n + 1)])
    idx = lambda i, j: i * (n + 1) + j
    tris = []
    for v in range(n):
        for u in range(n):
            c00, c10, c01, c11 = idx(u, v), idx(u + 1, v), idx(u, v + 1), idx(u + 1, v + 1)
            tris.append((c00, c10, c11))
            tris.append((c00, c11, c01))
    return Mesh(verts, tris)


def sphere_mesh(radius, center, subdivisions):
    """Closed sphere surface: the regular icosahedron with every triangle
    split into four `subdivisions` times, vertices projected onto the
    sphere (20 * 4^s triangles).  A PEC object for pinning the macromodel
    chain against the Mie series; RWGs on all edges."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.asarray(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    tris = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
            (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
            (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdivisions):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]

        split = []
        for a, b, c in tris:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            split += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = split
    return Mesh(np.array(verts) * radius + np.asarray(center, dtype=np.float64), tris)


def slab_zlevels(h, n, t):
    """z of the box grid rows when a slab of thickness t fills the bottom of
    the cell (reading of the configurations' cell: the side faces' first row
    ends at the slab top so the interface meets S_eq on mesh edges, the
    junction of Fig. composite; the other rows are uniform)."""
    if n < 2 or not 0.0 < t < h:
        raise ValueError("slab needs n >= 2 and 0 < t < h")
    return np.concatenate([[0.0], t + (h - t) * np.arange(n) / (n - 1)])


def _perimeter(m):
    """Grid indices (i, j) of the boundary of an m x m quad grid, walked
    counter-clockwise from (0, 0): m points per side, 4m in all."""
    out = [(i, 0) for i in range(m)]
    out += [(m, j) for j in range(m)]
    out += [(m - i, m) for i in range(m)]
    out += [(0, m - j) for j in range(m)]
    return out


def slab_top_mesh(a, b, z, n, side, patch_n, ring_layers=3):
    """Dielectric interface at height z over the whole cell footprint
    (the slab top, an interior surface of Sec. II-A), holding a centred
    square PEC patch of the given side.

    Vertices: the patch grid (patch_n + 1)^2 at index i*(patch_n+1)+j (as
    patch_mesh); then ring_layers - 1 rings of 4 patch_n points (in the
    order of _perimeter(patch_n)), ring k on the rectangle of half-widths
    side/2 + (a/2 - side/2) (k/ring_layers)^2 (and likewise in y), graded
    toward the patch edge where the interface fields are singular; then
    the footprint boundary points in the order of _perimeter(n) -- they
    coincide with the box vertices of grid row 1.
    Triangles: the patch quads split as patch_mesh; each ring band in quads
    (c00 = inner q, c10 = outer q, c11 = outer q+1, c01 = inner q+1) split
    as (c00, c10, c11), (c00, c11, c01); then the last band joins the
    outermost ring (patch_n segments per side) to the footprint boundary
    (n segments per side) side by side, zipped from the corner: the next
    triangle advances the outer polyline while its next parameter
    (j+1)/n <= (i+1)/patch_n, else the inner one.

    Returns (mesh, on_patch (T,) bool)."""
    p, m = patch_n, ring_layers
    if not 0.0 < side < min(a, b) or m < 1:
        raise ValueError("patch must fit strictly inside the footprint; ring_layers >= 1")
    xs = -0.5 * side + side * np.arange(p + 1) / p
    verts = [[xs[i], xs[j], z] for i in range(p + 1) for j in range(p + 1)]
    pidx = lambda i, j: i * (p + 1) + j
    tris = []
    for v in range(p):
        for u in range(p):
            c00, c10, c01, c11 = pidx(u, v), pidx(u + 1, v), pidx(u, v + 1), pidx(u + 1, v + 1)
            tris.append((c00, c10, c11))
            tris.append((c00, c11, c01))
    npatch = len(tris)
    per = _perimeter(p)
    inner = [pidx(i, j) for i, j in per]
    for k in range(1, m):
        f = (k / m) ** 2
        hx, hy = 0.5 * side + (0.5 * a - 0.5 * side) * f, 0.5 * side + (0.5 * b - 0.5 * side) * f
        base = len(verts)
        verts += [[-hx + 2 * hx * i / p, -hy + 2 * hy * j / p, z] for i, j in per]
        ring = [base + q for q in range(4 * p)]
        for q in range(4 * p):
            c00, c01 = inner[q], inner[(q + 1) % (4 * p)]
            c10, c11 = ring[q], ring[(q + 1) % (4 * p)]
            tris.append((c00, c10, c11))
            tris.append((c00, c11, c01))
        inner = ring
    nin = len(verts)
    ox = -0.5 * a + a * np.arange(n + 1) / n
    oy = -0.5 * b + b * np.arange(n + 1) / n
    verts += [[ox[i], oy[j], z] for i, j in _perimeter(n)]
    for s in range(4):
        I = [inner[(s * p + i) % (4 * p)] for i in range(p + 1)]
        O = [nin + (s * n + j) % (4 * n) for j in range(n + 1)]
        i = j = 0
        while i < p or j < n:
            if j < n and (i == p or (j + 1) * p <= (i + 1) * n):
                tris.append((I[i], O[j], O[j + 1]))
                j += 1
            else:
                tris.append((I[i], O[j], I[i + 1]))
                i += 1
    on_patch = np.zeros(len(tris), dtype=bool)
    on_patch[:npatch] = True
    return Mesh(np.array(verts), tris), on_patch


def slab_region_meshes(box, n, top):
    """The closed surfaces S_v of the two interior regions of a slab cell
    (Sec. II-A, V = 2): the air above the slab is bounded by the box
    triangles above grid row 1 and the slab top, the slab by the box
    triangles of row 0, the bottom face and the slab top.

    box: box_mesh with slab_zlevels; top: slab_top_mesh.  The slab top's
    footprint boundary vertices are identified with the box vertices of
    grid row 1.  Returns [(mesh, keys)] for (air, slab), keys[t] = ('eq', tb)
    or ('top', tt) naming where region triangle t comes from."""
    pts = box_grid_points(n)
    index = {q: m for m, q in enumerate(pts)}
    row = np.array([max(pts[v][2] for v in tri) for tri in box.tris])   # highest grid row per triangle
    nin = len(top.verts) - 4 * n
    remap = np.arange(len(top.verts)) + len(box.verts)
    for s, (i, j) in enumerate(_perimeter(n)):
        remap[nin + s] = index[(i, j, 1)]
    verts = np.concatenate([box.verts, top.verts])
    out = []
    for sel in (row >= 2, row <= 1):
        tb = np.nonzero(sel)[0]
        tris = np.concatenate([box.tris[tb], remap[top.tris]])
        keys = [("eq", int(t)) for t in tb] + [("top", t) for t in range(len(top.tris))]
        out.append((Mesh(verts, tris), keys))
    return out
