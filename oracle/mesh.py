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
  (i,k), (i,j) for x, y, z faces; quad (u,v) has index v*n+u; its two
  triangles are (c00,c10,c11) then (c00,c11,c01); triangle index
  = face*2n^2 + 2*(v*n+u) + {0,1};
* RWG edges are the distinct vertex pairs (lo,hi), sorted lexicographically;
  T+ is the lower-numbered of the two triangles sharing the edge;
* slot i of a triangle is the edge opposite its vertex i (free vertex i).

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
                tris.append((c00, c10, c11))
                tris.append((c00, c11, c01))
    return Mesh(verts, tris)


def patch_mesh(side, z, n):
    """Flat square PEC patch of the given side centred on the cell axis at
    height z, n x n quads split like the box faces; RWGs on interior edges."""
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
