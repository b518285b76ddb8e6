// Host-side setup: canonical meshes of S_eq and the patch, and the overlap
// map U_o, all by integer index arithmetic.
//
// Sec. II-A: every cell's box S_eq is the prism of the cell footprint, with
// opposite faces meshed identically so that all boxes are translates.  On the
// lattice every box grid point (i,j,k) of cell (ix,iy) sits at the global
// integer point (ix*n + i, iy*n + j, k); coincident edges and triangles of
// neighbouring boxes are recognised by equal global integer keys, which is
// exact.  U_o (Eq. connections_IUI, Sec. III-D rule 1) merges two RWG
// functions of different boxes whose edges coincide and that share a
// coincident triangle, with the sign that cancels the coincident halves.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <numeric>
#include <unordered_map>
#include <utility>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

struct MeshOut {
    std::vector<double> verts;          // [V][3]
    std::vector<int32_t> tris;          // [T][3]
    std::vector<int32_t> edges;         // [E][2]
    std::vector<int32_t> tplus, tminus; // [E]
    std::vector<int32_t> slot_rwg;      // [T][3]
    std::vector<int8_t> slot_sgn;       // [T][3]
};

// RWGs on the edges shared by two triangles; T+ = lower triangle index;
// slot i of a triangle = edge opposite vertex i.
int finish_mesh(MeshOut& m, bool closed) {
    const int T = (int)m.tris.size() / 3;
    struct Own { int64_t lo, hi; int t, slot; };
    std::vector<Own> own;
    own.reserve(3 * T);
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < 3; ++i) {
            const int p = m.tris[3 * t + (i + 1) % 3], q = m.tris[3 * t + (i + 2) % 3];
            own.push_back({std::min(p, q), std::max(p, q), t, i});
        }
    std::sort(own.begin(), own.end(), [](const Own& a, const Own& b) {
        if (a.lo != b.lo) return a.lo < b.lo;
        if (a.hi != b.hi) return a.hi < b.hi;
        return a.t < b.t;
    });
    m.slot_rwg.assign(3 * T, -1);
    m.slot_sgn.assign(3 * T, 0);
    size_t s = 0;
    while (s < own.size()) {
        size_t e = s;
        while (e < own.size() && own[e].lo == own[s].lo && own[e].hi == own[s].hi) ++e;
        const size_t cnt = e - s;
        if (cnt > 2) { set_error("non-manifold edge"); return EMSURF_EINVAL; }
        if (cnt == 1 && closed) { set_error("open edge on a closed box"); return EMSURF_EINVAL; }
        if (cnt == 2) {
            const int r = (int)m.tplus.size();
            m.edges.push_back((int32_t)own[s].lo);
            m.edges.push_back((int32_t)own[s].hi);
            m.tplus.push_back(own[s].t);
            m.tminus.push_back(own[s + 1].t);
            m.slot_rwg[3 * own[s].t + own[s].slot] = r;
            m.slot_sgn[3 * own[s].t + own[s].slot] = 1;
            m.slot_rwg[3 * own[s + 1].t + own[s + 1].slot] = r;
            m.slot_sgn[3 * own[s + 1].t + own[s + 1].slot] = -1;
        }
        s = e;
    }
    return EMSURF_OK;
}

// Box surface grid: point (i,j,k) -> vertex index (lexicographic), -1 inside.
std::vector<int32_t> box_index(int n) {
    std::vector<int32_t> idx((size_t)(n + 1) * (n + 1) * (n + 1), -1);
    int c = 0;
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j)
            for (int k = 0; k <= n; ++k)
                if (i == 0 || i == n || j == 0 || j == n || k == 0 || k == n)
                    idx[((size_t)i * (n + 1) + j) * (n + 1) + k] = c++;
    return idx;
}

// grid point of face f (x-,x+,y-,y+,z-,z+) at in-plane (u,v)
inline void face_point(int f, int n, int u, int v, int& i, int& j, int& k) {
    const int fixed = (f % 2) ? n : 0;
    switch (f / 2) {
        case 0: i = fixed; j = u; k = v; break;
        case 1: i = u; j = fixed; k = v; break;
        default: i = u; j = v; k = fixed; break;
    }
}

int build_box(double a, double b, double h, int n, const double* zlevels, MeshOut& m,
              std::vector<int32_t>* grid_of_vertex) {
    if (n < 1 || !(a > 0) || !(b > 0) || !(h > 0)) {
        set_error("box mesh needs n >= 1 and positive sides");
        return EMSURF_EINVAL;
    }
    const std::vector<int32_t> idx = box_index(n);
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j)
            for (int k = 0; k <= n; ++k)
                if (idx[((size_t)i * (n + 1) + j) * (n + 1) + k] >= 0) {
                    m.verts.push_back(-0.5 * a + a * i / n);
                    m.verts.push_back(-0.5 * b + b * j / n);
                    m.verts.push_back(zlevels ? zlevels[k] : h * k / n);
                    if (grid_of_vertex) {
                        grid_of_vertex->push_back(i);
                        grid_of_vertex->push_back(j);
                        grid_of_vertex->push_back(k);
                    }
                }
    auto at = [&](int f, int u, int v) {
        int i, j, k;
        face_point(f, n, u, v, i, j, k);
        return idx[((size_t)i * (n + 1) + j) * (n + 1) + k];
    };
    // for even n each quad is cut along the diagonal pointing at the face
    // centre (a union-jack pattern), which makes the mesh invariant under the
    // mirrors x -> -x, y -> -y (and x <-> y on a square footprint); odd n,
    // whose middle quads no cut makes symmetric, keeps one diagonal throughout
    for (int f = 0; f < 6; ++f)
        for (int v = 0; v < n; ++v)
            for (int u = 0; u < n; ++u) {
                const int c00 = at(f, u, v), c10 = at(f, u + 1, v);
                const int c01 = at(f, u, v + 1), c11 = at(f, u + 1, v + 1);
                if ((n & 1) || (2 * u + 1 < n) == (2 * v + 1 < n)) {
                    const int t0[3] = {c00, c10, c11}, t1[3] = {c00, c11, c01};
                    m.tris.insert(m.tris.end(), t0, t0 + 3);
                    m.tris.insert(m.tris.end(), t1, t1 + 3);
                } else {
                    const int t0[3] = {c00, c10, c01}, t1[3] = {c10, c11, c01};
                    m.tris.insert(m.tris.end(), t0, t0 + 3);
                    m.tris.insert(m.tris.end(), t1, t1 + 3);
                }
            }
    return finish_mesh(m, true);
}

// Mirrors of the box about its axis (0: x -> -x, 1: y -> -y, 2: x <-> y) as
// signed permutations of its RWG functions: mirrored f_e = sign[e] f_perm[e]
// (the image of edge e, with sign +1 when the image of e's T+ is the T+ of
// the image edge).  Exact, on the integer grid points.  Bit g of the returned
// mask is set when mirror g maps the mesh onto itself.
int box_mirror_perms(int n, bool square, const MeshOut& m, const std::vector<int32_t>& grid,
                     std::vector<int32_t>& perm, std::vector<int8_t>& sign) {
    const std::vector<int32_t> idx = box_index(n);
    const int E = (int)m.tplus.size(), T = (int)m.tris.size() / 3;
    std::map<std::pair<int, int>, int> edge_of;
    for (int e = 0; e < E; ++e) edge_of[{m.edges[2 * e], m.edges[2 * e + 1]}] = e;
    std::map<std::vector<int>, int> tri_of;
    for (int t = 0; t < T; ++t) {
        std::vector<int> key(m.tris.begin() + 3 * t, m.tris.begin() + 3 * t + 3);
        std::sort(key.begin(), key.end());
        tri_of[key] = t;
    }
    const int V = (int)grid.size() / 3;
    perm.assign((size_t)3 * E, 0);
    sign.assign((size_t)3 * E, 0);
    int mask = 0;
    for (int g = 0; g < 3; ++g) {
        if (g == 2 && !square) continue;
        std::vector<int> vmap(V);
        for (int q = 0; q < V; ++q) {
            int i = grid[3 * q], j = grid[3 * q + 1];
            const int k = grid[3 * q + 2];
            if (g == 0) i = n - i;
            else if (g == 1) j = n - j;
            else std::swap(i, j);
            vmap[q] = idx[((size_t)i * (n + 1) + j) * (n + 1) + k];
        }
        bool ok = true;
        for (int e = 0; e < E && ok; ++e) {
            const int p = vmap[m.edges[2 * e]], q = vmap[m.edges[2 * e + 1]];
            auto it = edge_of.find({std::min(p, q), std::max(p, q)});
            std::vector<int> key(3);
            for (int c = 0; c < 3; ++c) key[c] = vmap[m.tris[3 * m.tplus[e] + c]];
            std::sort(key.begin(), key.end());
            auto tt = tri_of.find(key);
            if (it == edge_of.end() || tt == tri_of.end()) {
                ok = false;
                break;
            }
            const int img = it->second;
            if (tt->second != m.tplus[img] && tt->second != m.tminus[img]) {
                ok = false;
                break;
            }
            perm[(size_t)g * E + e] = img;
            sign[(size_t)g * E + e] = tt->second == m.tplus[img] ? 1 : -1;
        }
        if (ok) mask |= 1 << g;
    }
    return mask;
}

int build_patch(double side, double z, int n, MeshOut& m) {
    if (n < 1 || !(side > 0)) {
        set_error("patch mesh needs n >= 1 and a positive side");
        return EMSURF_EINVAL;
    }
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j) {
            m.verts.push_back(-0.5 * side + side * i / n);
            m.verts.push_back(-0.5 * side + side * j / n);
            m.verts.push_back(z);
        }
    auto id = [n](int i, int j) { return i * (n + 1) + j; };
    for (int v = 0; v < n; ++v)
        for (int u = 0; u < n; ++u) {
            const int t0[3] = {id(u, v), id(u + 1, v), id(u + 1, v + 1)};
            const int t1[3] = {id(u, v), id(u + 1, v + 1), id(u, v + 1)};
            m.tris.insert(m.tris.end(), t0, t0 + 3);
            m.tris.insert(m.tris.end(), t1, t1 + 3);
        }
    return finish_mesh(m, false);
}

void copy_mesh(const MeshOut& m, double* verts, int32_t* tris, int32_t* edges, int32_t* tplus,
               int32_t* tminus, int32_t* slot_rwg, int8_t* slot_sgn) {
    if (verts) std::copy(m.verts.begin(), m.verts.end(), verts);
    if (tris) std::copy(m.tris.begin(), m.tris.end(), tris);
    if (edges) std::copy(m.edges.begin(), m.edges.end(), edges);
    if (tplus) std::copy(m.tplus.begin(), m.tplus.end(), tplus);
    if (tminus) std::copy(m.tminus.begin(), m.tminus.end(), tminus);
    if (slot_rwg) std::copy(m.slot_rwg.begin(), m.slot_rwg.end(), slot_rwg);
    if (slot_sgn) std::copy(m.slot_sgn.begin(), m.slot_sgn.end(), slot_sgn);
}

// union-find with parity: sigma(x) = par(x) * sigma(root)
struct ParityDSU {
    std::vector<int32_t> parent;
    std::vector<int8_t> par;
    explicit ParityDSU(size_t n) : parent(n), par(n, 1) { std::iota(parent.begin(), parent.end(), 0); }
    std::pair<int32_t, int> find(int32_t x) {
        int p = 1;
        int32_t r = x;
        while (parent[r] != r) { p *= par[r]; r = parent[r]; }
        // compress
        int acc = p;
        int32_t y = x;
        while (parent[y] != y) {
            const int32_t nxt = parent[y];
            const int py = par[y];
            parent[y] = r;
            par[y] = (int8_t)acc;
            acc *= py;
            y = nxt;
        }
        return {r, p};
    }
    // enforce sigma(y) = s * sigma(x); false on a contradiction
    bool unite(int32_t x, int32_t y, int s) {
        auto [rx, px] = find(x);
        auto [ry, py] = find(y);
        if (rx == ry) return px * py == s;
        parent[ry] = rx;
        par[ry] = (int8_t)(s * px * py);
        return true;
    }
};

// ---------------------------------------------------------------------------
// The configurations' cell (Secs. II-A..C): a dielectric slab fills the
// bottom of the box up to the first row boundary zlevels[1] of the side
// faces; its top is an interface surface that meets S_eq on the box edges
// of grid row 1 (the junction of Fig. composite) and carries a centred PEC
// square patch.

// boundary of an m x m quad grid, counter-clockwise from (0, 0), m points a side
std::vector<std::pair<int, int>> grid_perimeter(int m) {
    std::vector<std::pair<int, int>> out;
    for (int i = 0; i < m; ++i) out.push_back({i, 0});
    for (int j = 0; j < m; ++j) out.push_back({m, j});
    for (int i = 0; i < m; ++i) out.push_back({m - i, m});
    for (int j = 0; j < m; ++j) out.push_back({0, m - j});
    return out;
}

void push_tri(MeshOut& m, int a, int b, int c) {
    m.tris.push_back(a);
    m.tris.push_back(b);
    m.tris.push_back(c);
}

void push_vert(MeshOut& m, double x, double y, double z) {
    m.verts.push_back(x);
    m.verts.push_back(y);
    m.verts.push_back(z);
}

// Slab top with a patch: patch grid, ring_layers - 1 graded rings of
// 4 patch_n points, then the 4n footprint boundary points; patch quads,
// ring bands, and a zipped last band to the footprint boundary.
int build_slab_top(double a, double b, double z, int n, double side, int p, int layers,
                   MeshOut& m, std::vector<int8_t>& pec) {
    if (n < 2 || p < 1 || layers < 1 || !(side > 0.0) || !(side < std::min(a, b))) {
        set_error("slab top needs n >= 2, patch_n >= 1, ring_layers >= 1 and 0 < side < min(a, b)");
        return EMSURF_EINVAL;
    }
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j)
            push_vert(m, -0.5 * side + side * i / p, -0.5 * side + side * j / p, z);
    auto pidx = [p](int i, int j) { return i * (p + 1) + j; };
    for (int v = 0; v < p; ++v)
        for (int u = 0; u < p; ++u) {
            push_tri(m, pidx(u, v), pidx(u + 1, v), pidx(u + 1, v + 1));
            push_tri(m, pidx(u, v), pidx(u + 1, v + 1), pidx(u, v + 1));
        }
    const int npatch = (int)m.tris.size() / 3;
    const auto per = grid_perimeter(p);
    std::vector<int> inner;
    for (auto& q : per) inner.push_back(pidx(q.first, q.second));
    for (int k = 1; k < layers; ++k) {
        const double f = ((double)k / layers) * ((double)k / layers);
        const double hx = 0.5 * side + (0.5 * a - 0.5 * side) * f;
        const double hy = 0.5 * side + (0.5 * b - 0.5 * side) * f;
        const int base = (int)m.verts.size() / 3;
        for (auto& q : per) push_vert(m, -hx + 2.0 * hx * q.first / p, -hy + 2.0 * hy * q.second / p, z);
        std::vector<int> ring(4 * p);
        for (int q = 0; q < 4 * p; ++q) ring[q] = base + q;
        for (int q = 0; q < 4 * p; ++q) {
            const int c00 = inner[q], c01 = inner[(q + 1) % (4 * p)];
            const int c10 = ring[q], c11 = ring[(q + 1) % (4 * p)];
            push_tri(m, c00, c10, c11);
            push_tri(m, c00, c11, c01);
        }
        inner = ring;
    }
    const int nin = (int)m.verts.size() / 3;
    for (auto& q : grid_perimeter(n)) push_vert(m, -0.5 * a + a * q.first / n, -0.5 * b + b * q.second / n, z);
    for (int s = 0; s < 4; ++s) {
        int i = 0, j = 0;
        auto I = [&](int x) { return inner[(s * p + x) % (4 * p)]; };
        auto O = [&](int x) { return nin + (s * n + x) % (4 * n); };
        while (i < p || j < n) {
            if (j < n && (i == p || (j + 1) * p <= (i + 1) * n)) {
                push_tri(m, I(i), O(j), O(j + 1));
                ++j;
            } else {
                push_tri(m, I(i), O(j), I(i + 1));
                ++i;
            }
        }
    }
    pec.assign(m.tris.size() / 3, 0);
    std::fill(pec.begin(), pec.begin() + npatch, 1);
    return finish_mesh(m, false);
}

// Slab top without a patch: the n x n footprint grid, inner points first
// (i-major), then the boundary in grid_perimeter order; quads split as the
// box faces.
int build_bare_top(double a, double b, double z, int n, MeshOut& m, std::vector<int8_t>& pec) {
    if (n < 2) { set_error("slab top needs n >= 2"); return EMSURF_EINVAL; }
    std::vector<int> id((n + 1) * (n + 1), -1);
    int c = 0;
    for (int i = 1; i < n; ++i)
        for (int j = 1; j < n; ++j) {
            id[i * (n + 1) + j] = c++;
            push_vert(m, -0.5 * a + a * i / n, -0.5 * b + b * j / n, z);
        }
    for (auto& q : grid_perimeter(n)) {
        id[q.first * (n + 1) + q.second] = c++;
        push_vert(m, -0.5 * a + a * q.first / n, -0.5 * b + b * q.second / n, z);
    }
    auto at = [&](int i, int j) { return id[i * (n + 1) + j]; };
    for (int v = 0; v < n; ++v)
        for (int u = 0; u < n; ++u) {
            push_tri(m, at(u, v), at(u + 1, v), at(u + 1, v + 1));
            push_tri(m, at(u, v), at(u + 1, v + 1), at(u, v + 1));
        }
    pec.assign(m.tris.size() / 3, 0);
    return finish_mesh(m, false);
}

int slot_sign(const MeshOut& m, int rwg, int t) {
    for (int i = 0; i < 3; ++i)
        if (m.slot_rwg[3 * t + i] == rwg) return m.slot_sgn[3 * t + i];
    return 0;
}

}  // namespace

int slab_top(double a, double b, double z, int n, double side, int patch_n, int ring_layers,
             std::vector<double>& verts, std::vector<int32_t>& tris, std::vector<int32_t>& edges,
             std::vector<int32_t>& tplus, std::vector<int32_t>& tminus,
             std::vector<int32_t>& slot_rwg, std::vector<int8_t>& slot_sgn,
             std::vector<int8_t>& on_patch) {
    MeshOut m;
    if (side > 0.0) EMS_TRY(build_slab_top(a, b, z, n, side, patch_n, ring_layers, m, on_patch));
    else EMS_TRY(build_bare_top(a, b, z, n, m, on_patch));
    verts = m.verts;
    tris = m.tris;
    edges = m.edges;
    tplus = m.tplus;
    tminus = m.tminus;
    slot_rwg = m.slot_rwg;
    slot_sgn = m.slot_sgn;
    return EMSURF_OK;
}

int slab_cell_plan(double a, double b, double h, int n, const double* zlevels, double side,
                   int patch_n, int ring_layers, SlabPlan& out) {
    if (!zlevels || n < 2) { set_error("slab cell needs n >= 2 and the box row heights"); return EMSURF_EINVAL; }
    for (int k = 0; k < n; ++k)
        if (!(zlevels[k + 1] > zlevels[k])) { set_error("zlevels must increase"); return EMSURF_EINVAL; }
    if (zlevels[0] != 0.0 || zlevels[n] != h) { set_error("zlevels must run from 0 to h"); return EMSURF_EINVAL; }
    MeshOut box, top;
    std::vector<int32_t> gv;
    EMS_TRY(build_box(a, b, h, n, zlevels, box, &gv));
    std::vector<int8_t> pec;
    const double zt = zlevels[1];
    if (side > 0.0) EMS_TRY(build_slab_top(a, b, zt, n, side, patch_n, ring_layers, top, pec));
    else EMS_TRY(build_bare_top(a, b, zt, n, top, pec));
    const int Vb = (int)box.verts.size() / 3, Tb = (int)box.tris.size() / 3, E = (int)box.tplus.size();
    const int Vt = (int)top.verts.size() / 3, Tt = (int)top.tris.size() / 3;
    // top vertex -> region vertex: interior ones after the box's, boundary
    // ones onto the box vertices of grid row 1
    const std::vector<int32_t> bidx = box_index(n);
    std::vector<int32_t> remap(Vt);
    for (int v = 0; v < Vt; ++v) remap[v] = Vb + v;
    const auto per = grid_perimeter(n);
    for (int s = 0; s < 4 * n; ++s)
        remap[Vt - 4 * n + s] = bidx[((size_t)per[s].first * (n + 1) + per[s].second) * (n + 1) + 1];
    std::map<std::pair<int, int>, int> box_edge, top_rwg;
    for (int e = 0; e < E; ++e) box_edge[{box.edges[2 * e], box.edges[2 * e + 1]}] = e;
    for (int r = 0; r < (int)top.tplus.size(); ++r)
        top_rwg[{std::min(top.tplus[r], top.tminus[r]), std::max(top.tplus[r], top.tminus[r])}] = r;
    // region triangles: box triangles by their highest grid row, then the whole top
    std::vector<std::vector<int>> key(2);      // >= 0: box triangle; < 0: -(top triangle) - 1
    MeshOut reg[2];
    for (int v = 0; v < 2; ++v) {
        reg[v].verts = box.verts;
        reg[v].verts.insert(reg[v].verts.end(), top.verts.begin(), top.verts.end());
        for (int t = 0; t < Tb; ++t) {
            int row = 0;
            for (int c = 0; c < 3; ++c) row = std::max(row, gv[3 * box.tris[3 * t + c] + 2]);
            if ((v == 0) != (row >= 2)) continue;
            push_tri(reg[v], box.tris[3 * t], box.tris[3 * t + 1], box.tris[3 * t + 2]);
            key[v].push_back(t);
        }
        for (int t = 0; t < Tt; ++t) {
            push_tri(reg[v], remap[top.tris[3 * t]], remap[top.tris[3 * t + 1]], remap[top.tris[3 * t + 2]]);
            key[v].push_back(-t - 1);
        }
        EMS_TRY(finish_mesh(reg[v], true));
    }
    // U (Eq. incidence1): region unknown -> X~ column, interior columns by
    // first appearance, S_eq columns after them (coded -1 - k until then)
    const int nrt = (int)top.tplus.size();
    std::vector<int> shJ(nrt, -1), shM(nrt, -1);
    int nint = 0;
    struct Ent { int col, local, sgn; };
    std::vector<Ent> ents[2];
    for (int v = 0; v < 2; ++v) {
        const MeshOut& m = reg[v];
        const int Ev = (int)m.tplus.size();
        const int side_v = v == 1 ? 1 : -1;
        for (int r = 0; r < Ev; ++r) {
            const int tp = m.tplus[r], tm = m.tminus[r];
            const int kp = key[v][tp], km = key[v][tm];
            if (kp >= 0 || km >= 0) {
                const int te = kp >= 0 ? tp : tm, tb = kp >= 0 ? kp : km;
                const int other = kp >= 0 ? km : kp;
                if (other < 0 && pec[-other - 1]) { set_error("PEC touching S_eq is not modelled"); return EMSURF_EINVAL; }
                const int p0 = m.edges[2 * r], p1 = m.edges[2 * r + 1];
                auto it = box_edge.find({p0, p1});
                if (p1 >= Vb || it == box_edge.end()) { set_error("slab cell: S_eq edge not found"); return EMSURF_EINVAL; }
                const int e = it->second;
                const int s = slot_sign(m, r, te) * slot_sign(box, e, tb);
                ents[v].push_back({-1 - e, r, s});
                ents[v].push_back({-1 - (E + e), Ev + r, s});
                continue;
            }
            const int a0 = -kp - 1, b0 = -km - 1;
            auto it = top_rwg.find({std::min(a0, b0), std::max(a0, b0)});
            if (it == top_rwg.end()) { set_error("slab cell: interface RWG not found"); return EMSURF_EINVAL; }
            const int sr = it->second;
            const int s = slot_sign(m, r, tp) * slot_sign(top, sr, a0);
            const int npec = pec[a0] + pec[b0];
            if (npec == 2) {                                   // rule 2: one current per side
                ents[v].push_back({nint++, r, s});
            } else {                                           // rules 1 and 3: shared, opposite sides
                if (shJ[sr] < 0) shJ[sr] = nint++;
                ents[v].push_back({shJ[sr], r, side_v * s});
                if (npec == 0) {                               // rule 1 also shares M
                    if (shM[sr] < 0) shM[sr] = nint++;
                    ents[v].push_back({shM[sr], Ev + r, side_v * s});
                }
            }
        }
    }
    out.n_int = nint;
    out.N = nint + 2 * E;
    out.E = E;
    for (int v = 0; v < 2; ++v) {
        out.copy[v].assign(out.N, -1);
        out.sgn[v].assign(out.N, 0);
        for (const Ent& en : ents[v]) {
            const int col = en.col >= 0 ? en.col : nint + (-en.col - 1);
            if (out.copy[v][col] >= 0) { set_error("slab cell: two copies of one unknown in a region"); return EMSURF_EINVAL; }
            if (en.sgn == 0) { set_error("slab cell: orientation lookup failed"); return EMSURF_EINVAL; }
            out.copy[v][col] = en.local;
            out.sgn[v][col] = (int8_t)en.sgn;
        }
        SlabRegionMesh& rm = out.region[v];
        rm.verts = reg[v].verts;
        rm.tris = reg[v].tris;
        rm.slot_rwg = reg[v].slot_rwg;
        rm.slot_sgn = reg[v].slot_sgn;
        rm.T = (int)reg[v].tris.size() / 3;
        rm.E = (int)reg[v].tplus.size();
    }
    return EMSURF_OK;
}

int orbit_image(int e, int kx, int ky, int px, int py) {
    if (e & 4) std::swap(kx, ky);
    if (e & 2) ky = (py - ky) % py;
    if (e & 1) kx = (px - kx) % px;
    return ky * px + kx;
}

// T_e = diag(P_e, det(e) P_e) with P_e = Px^a Py^b Pd^c (bits a, b, c of e),
// P e_n = sign_n e_perm[n]; products composed as (P_A P_B) e_n =
// sign_B[n] sign_A[perm_B[n]] e_perm_A[perm_B[n]]
void mirror_group_perms(int E, int G, const int32_t* perm, const int8_t* sign, std::vector<uint32_t>& tperm) {
    const int E2 = 2 * E;
    tperm.assign((size_t)G * E2, 0u);
    for (int e = 0; e < G; ++e) {
        std::vector<int32_t> pi(E);
        std::vector<int8_t> sg(E, 1);
        for (int n = 0; n < E; ++n) pi[n] = n;
        int det = 1;
        for (int g = 0; g < 3; ++g) {
            if (!(e & (1 << g))) continue;
            std::vector<int32_t> npi(E);
            std::vector<int8_t> nsg(E);
            for (int n = 0; n < E; ++n) {     // P <- P P_g
                const int m = perm[(size_t)g * E + n];
                npi[n] = pi[m];
                nsg[n] = (int8_t)(sign[(size_t)g * E + n] * sg[m]);
            }
            pi.swap(npi);
            sg.swap(nsg);
            det = -det;
        }
        for (int n = 0; n < E; ++n) {
            tperm[(size_t)e * E2 + n] = (uint32_t)pi[n] | (sg[n] < 0 ? 0x80000000u : 0u);
            tperm[(size_t)e * E2 + E + n] = (uint32_t)(E + pi[n]) | (sg[n] * det < 0 ? 0x80000000u : 0u);
        }
    }
}

// the smallest bin index represents each orbit; its slots are the distinct
// images in the order of the group elements
void mirror_orbits(int px, int py, int G, std::vector<int32_t>& rep, std::vector<int32_t>& obin,
                   std::vector<int32_t>& oelem) {
    rep.clear();
    obin.clear();
    oelem.clear();
    for (int ky = 0; ky < py; ++ky)
        for (int kx = 0; kx < px; ++kx) {
            const int b = ky * px + kx;
            int imgs[8];
            int r = b;
            for (int e = 0; e < G; ++e) {
                imgs[e] = orbit_image(e, kx, ky, px, py);
                r = std::min(r, imgs[e]);
            }
            if (r != b) continue;
            rep.push_back(b);
            int nslot = 0;
            for (int e = 0; e < G; ++e) {
                bool seen = false;
                for (int u = 0; u < nslot; ++u) seen = seen || obin[obin.size() - nslot + u] == imgs[e];
                if (seen) continue;
                obin.push_back(imgs[e]);
                oelem.push_back(e);
                ++nslot;
            }
            for (; nslot < G; ++nslot) {
                obin.push_back(-1);
                oelem.push_back(0);
            }
        }
}

namespace {
}  // namespace
}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API int emsurf_setup_box_counts(int32_t n, int32_t* n_verts, int32_t* n_tris,
                                       int32_t* n_edges) {
    if (n < 1) { set_error("n must be >= 1"); return EMSURF_EINVAL; }
    if (n_verts) *n_verts = (n + 1) * (n + 1) * (n + 1) - (n - 1) * (n - 1) * (n - 1);
    if (n_tris) *n_tris = 12 * n * n;
    if (n_edges) *n_edges = 18 * n * n;
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_box_mesh(double a, double b, double h, int32_t n,
                                     const double* zlevels, double* verts, int32_t* tris,
                                     int32_t* edges, int32_t* tplus, int32_t* tminus,
                                     int32_t* slot_rwg, int8_t* slot_sgn) {
    MeshOut m;
    EMS_TRY(build_box(a, b, h, n, zlevels, m, nullptr));
    copy_mesh(m, verts, tris, edges, tplus, tminus, slot_rwg, slot_sgn);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_box_mirrors(double a, double b, int32_t n, int32_t* perm, int8_t* sign,
                                        int32_t* mask) {
    if (!perm || !sign || !mask) { set_error("box mirrors: null output"); return EMSURF_EINVAL; }
    MeshOut m;
    std::vector<int32_t> grid;
    EMS_TRY(build_box(a, b, 1.0, n, nullptr, m, &grid));
    std::vector<int32_t> p;
    std::vector<int8_t> sg;
    const bool square = std::fabs(a - b) <= 1e-12 * std::max(a, b);
    *mask = box_mirror_perms(n, square, m, grid, p, sg);
    std::copy(p.begin(), p.end(), perm);
    std::copy(sg.begin(), sg.end(), sign);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_mirror_orbits(int32_t px, int32_t py, int32_t n_elem, int32_t* n_stored,
                                          int32_t* rep, int32_t* slot_bin, int32_t* slot_elem) {
    if (px < 1 || py < 1 || (n_elem != 4 && n_elem != 8) || (n_elem == 8 && px != py) || !n_stored) {
        set_error("mirror orbits: grid >= 1, 4 or 8 group elements (8 on a square grid)");
        return EMSURF_EINVAL;
    }
    std::vector<int32_t> r, ob, oe;
    mirror_orbits(px, py, n_elem, r, ob, oe);
    *n_stored = (int32_t)r.size();
    if (rep) std::copy(r.begin(), r.end(), rep);
    if (slot_bin) std::copy(ob.begin(), ob.end(), slot_bin);
    if (slot_elem) std::copy(oe.begin(), oe.end(), slot_elem);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_mirror_group(int32_t n_edges, int32_t n_elem, const int32_t* perm, const int8_t* sign,
                                         uint32_t* tperm) {
    if (n_edges < 1 || (n_elem != 4 && n_elem != 8) || !perm || !sign || !tperm) {
        set_error("mirror group: bad arguments");
        return EMSURF_EINVAL;
    }
    std::vector<uint32_t> t;
    mirror_group_perms(n_edges, n_elem, perm, sign, t);
    std::copy(t.begin(), t.end(), tperm);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_patch_counts(int32_t n, int32_t* n_verts, int32_t* n_tris,
                                         int32_t* n_edges) {
    if (n < 1) { set_error("n must be >= 1"); return EMSURF_EINVAL; }
    if (n_verts) *n_verts = (n + 1) * (n + 1);
    if (n_tris) *n_tris = 2 * n * n;
    if (n_edges) *n_edges = 3 * n * n - 2 * n;
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_patch_mesh(double side, double z, int32_t n, double* verts,
                                       int32_t* tris, int32_t* edges, int32_t* tplus,
                                       int32_t* tminus, int32_t* slot_rwg, int8_t* slot_sgn) {
    MeshOut m;
    EMS_TRY(build_patch(side, z, n, m));
    copy_mesh(m, verts, tris, edges, tplus, tminus, slot_rwg, slot_sgn);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_unknown_xy(double a, double b, double h, int32_t n, int32_t nx,
                                       int32_t ny, const int32_t* uo_index, int32_t n_unique,
                                       double* xy) {
    if (n < 1 || nx < 1 || ny < 1 || !uo_index || !xy || n_unique < 1) {
        set_error("emsurf_setup_unknown_xy: bad arguments");
        return EMSURF_EINVAL;
    }
    MeshOut m;
    EMS_TRY(build_box(a, b, h, n, nullptr, m, nullptr));
    const int E = (int)m.tplus.size(), K = 2 * E;
    std::vector<char> set(n_unique, 0);
    for (int c = 0; c < nx * ny; ++c)
        for (int k = 0; k < K; ++k) {
            const int u = uo_index[(size_t)c * K + k];
            if (u < 0 || u >= n_unique) {
                set_error("emsurf_setup_unknown_xy: uo_index out of range");
                return EMSURF_EINVAL;
            }
            if (set[u]) continue;
            set[u] = 1;
            const int e = k % E, p = m.edges[2 * e], q = m.edges[2 * e + 1];
            xy[2 * u] = 0.5 * (m.verts[3 * p] + m.verts[3 * q]) + (c % nx) * a;
            xy[2 * u + 1] = 0.5 * (m.verts[3 * p + 1] + m.verts[3 * q + 1]) + (c / nx) * b;
        }
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_overlap(int32_t n, int32_t nx, int32_t ny, int32_t* uo_index,
                                    int8_t* uo_sign, int32_t* n_unique) {
    if (n < 1 || nx < 1 || ny < 1 || !uo_index || !uo_sign || !n_unique) {
        set_error("overlap map needs n, nx, ny >= 1 and output arrays");
        return EMSURF_EINVAL;
    }
    MeshOut m;
    std::vector<int32_t> gv;
    EMS_TRY(build_box(1.0, 1.0, 1.0, n, nullptr, m, &gv));
    const int E = (int)m.tplus.size(), K = 2 * E;
    const int64_t M = (int64_t)nx * ny;
    if (M * K > INT32_MAX) { set_error("lattice too large"); return EMSURF_EINVAL; }
    const int64_t GX = (int64_t)nx * n + 1, GY = (int64_t)ny * n + 1, GZ = n + 1;
    auto gkey = [&](int cell, int v) -> int64_t {
        const int ix = cell % nx, iy = cell / nx;
        const int64_t X = (int64_t)ix * n + gv[3 * v], Y = (int64_t)iy * n + gv[3 * v + 1];
        return (X * GY + Y) * GZ + gv[3 * v + 2];
    };
    (void)GX;
    // triangle key: sorted global vertex keys
    struct TriKey { int64_t a, b, c; bool operator==(const TriKey& o) const { return a == o.a && b == o.b && c == o.c; } };
    auto tkey = [&](int cell, int t) {
        int64_t k[3] = {gkey(cell, m.tris[3 * t]), gkey(cell, m.tris[3 * t + 1]), gkey(cell, m.tris[3 * t + 2])};
        std::sort(k, k + 3);
        return TriKey{k[0], k[1], k[2]};
    };
    // only edges on the side walls can coincide with a neighbour's
    std::map<std::pair<int64_t, int64_t>, std::vector<int64_t>> by_edge;
    const int nn = n;
    auto on_side = [&](int v) {
        const int i = gv[3 * v], j = gv[3 * v + 1];
        return i == 0 || i == nn || j == 0 || j == nn;
    };
    for (int64_t c = 0; c < M; ++c)
        for (int e = 0; e < E; ++e) {
            const int p = m.edges[2 * e], q = m.edges[2 * e + 1];
            if (!on_side(p) || !on_side(q)) continue;
            int64_t a = gkey((int)c, p), b = gkey((int)c, q);
            if (a > b) std::swap(a, b);
            by_edge[{a, b}].push_back(c * E + e);
        }
    ParityDSU dsu((size_t)M * E);
    for (auto& kv : by_edge) {
        const auto& mem = kv.second;
        for (size_t x = 0; x < mem.size(); ++x)
            for (size_t y = x + 1; y < mem.size(); ++y) {
                const int c1 = (int)(mem[x] / E), e1 = (int)(mem[x] % E);
                const int c2 = (int)(mem[y] / E), e2 = (int)(mem[y] % E);
                if (c1 == c2) continue;
                const int t1[2] = {m.tplus[e1], m.tminus[e1]};
                const int t2[2] = {m.tplus[e2], m.tminus[e2]};
                for (int r1 = 0; r1 < 2; ++r1)
                    for (int r2 = 0; r2 < 2; ++r2)
                        if (tkey(c1, t1[r1]) == tkey(c2, t2[r2])) {
                            const int s1 = r1 == 0 ? 1 : -1, s2 = r2 == 0 ? 1 : -1;
                            if (!dsu.unite((int32_t)mem[x], (int32_t)mem[y], -s1 * s2)) {
                                set_error("inconsistent overlap signs");
                                return EMSURF_EINVAL;
                            }
                        }
            }
    }
    // number unique unknowns by first appearance over (cell, k)
    std::unordered_map<int64_t, std::pair<int32_t, int>> uid;   // (root, part) -> (id, parity of first)
    uid.reserve((size_t)M * K);
    int32_t next = 0;
    for (int64_t c = 0; c < M; ++c)
        for (int k = 0; k < K; ++k) {
            const int part = k / E, e = k % E;
            auto [root, p] = dsu.find((int32_t)(c * E + e));
            const int64_t key = (int64_t)root * 2 + part;
            auto it = uid.find(key);
            if (it == uid.end()) it = uid.emplace(key, std::make_pair(next++, p)).first;
            uo_index[c * K + k] = it->second.first;
            uo_sign[c * K + k] = (int8_t)(p * it->second.second);
        }
    *n_unique = next;
    return EMSURF_OK;
}


EMSURF_API int emsurf_setup_slab_zlevels(double h, int32_t n, double slab_t, double* zlevels) {
    if (n < 2 || !(slab_t > 0.0) || !(slab_t < h) || !zlevels) {
        set_error("emsurf_setup_slab_zlevels needs n >= 2 and 0 < slab_t < h");
        return EMSURF_EINVAL;
    }
    zlevels[0] = 0.0;
    for (int k = 1; k <= n; ++k) zlevels[k] = slab_t + (h - slab_t) * (k - 1) / (n - 1);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_slab_top_counts(double a, double b, int32_t n, double side,
                                            int32_t patch_n, int32_t ring_layers,
                                            int32_t* n_verts, int32_t* n_tris, int32_t* n_edges) {
    std::vector<double> v;
    std::vector<int32_t> t, e, tp, tm, sr;
    std::vector<int8_t> ss, pc;
    EMS_TRY(slab_top(a, b, 0.0, n, side, patch_n, ring_layers, v, t, e, tp, tm, sr, ss, pc));
    if (n_verts) *n_verts = (int32_t)(v.size() / 3);
    if (n_tris) *n_tris = (int32_t)(t.size() / 3);
    if (n_edges) *n_edges = (int32_t)tp.size();
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_slab_top_mesh(double a, double b, double z, int32_t n, double side,
                                          int32_t patch_n, int32_t ring_layers, double* verts,
                                          int32_t* tris, int32_t* edges, int32_t* tplus,
                                          int32_t* tminus, int32_t* slot_rwg, int8_t* slot_sgn,
                                          int8_t* on_patch) {
    MeshOut m;
    std::vector<int8_t> pc;
    EMS_TRY(slab_top(a, b, z, n, side, patch_n, ring_layers, m.verts, m.tris, m.edges, m.tplus,
                     m.tminus, m.slot_rwg, m.slot_sgn, pc));
    copy_mesh(m, verts, tris, edges, tplus, tminus, slot_rwg, slot_sgn);
    if (on_patch) std::copy(pc.begin(), pc.end(), on_patch);
    return EMSURF_OK;
}

EMSURF_API int emsurf_setup_slab_cell_counts(double a, double b, double h, int32_t n,
                                             const double* zlevels, double side, int32_t patch_n,
                                             int32_t ring_layers, int32_t* n_interior,
                                             int32_t* region_edges) {
    SlabPlan pl;
    EMS_TRY(slab_cell_plan(a, b, h, n, zlevels, side, patch_n, ring_layers, pl));
    if (n_interior) *n_interior = pl.n_int;
    if (region_edges) {
        region_edges[0] = pl.region[0].E;
        region_edges[1] = pl.region[1].E;
    }
    return EMSURF_OK;
}

}  // extern "C"
