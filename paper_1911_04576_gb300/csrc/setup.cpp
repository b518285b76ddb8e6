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
    for (int f = 0; f < 6; ++f)
        for (int v = 0; v < n; ++v)
            for (int u = 0; u < n; ++u) {
                const int c00 = at(f, u, v), c10 = at(f, u + 1, v);
                const int c01 = at(f, u, v + 1), c11 = at(f, u + 1, v + 1);
                const int t0[3] = {c00, c10, c11}, t1[3] = {c00, c11, c01};
                m.tris.insert(m.tris.end(), t0, t0 + 3);
                m.tris.insert(m.tris.end(), t1, t1 + 3);
            }
    return finish_mesh(m, true);
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

}  // extern "C"
