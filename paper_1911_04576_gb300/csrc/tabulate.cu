// Tabulation of the Galerkin L and K blocks (Eqs. SIE_LOperator1,
// SIE_KOperator1 tested with RWG functions, Eq. blockZo) on the GPU.
//
//   L[m,n] = int int [Lam_m . Lam_n - (div Lam_m)(div' Lam_n)/k^2] G dS' dS
//   K[m,n] = int int Lam_m(r) . [grad_r G(r,r') x Lam_n(r')] dS' dS   (p.v.)
//   G = e^{-jkR} / (4 pi R)
//
// Quadrature (the paper names none): 7-point degree-5 Radon rule on both
// triangles; for blocks flagged singular (touching boxes, one cell) the 1/R
// and grad(1/R) parts are integrated over the source triangle in closed form
// (Wilton et al. 1984; Graglia 1993) and the remainder G - 1/(4 pi R) by the
// same rule.  Points within 1e-9 (relative) of the source plane take the
// principal value; point pairs within 1e-9 (relative) of each other are
// coincident (remainder at its R -> 0 limit, no gradient term).
//
// Stage 1: one thread per (block, test triangle, source triangle) computes
//          the 3x3 slot integrals of both operators into a scratch buffer.
// Stage 2: one thread per (block, test RWG, source RWG) sums the 2 x 2
//          triangle combinations of the two RWGs with their amplitudes.
// Blocks are processed in chunks so the scratch stays below 256 MB.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;
constexpr size_t kScratchBytes = 256ull << 20;

struct TriGeo {
    double v[9];     // vertices
    double q[21];    // quadrature points
    double area;
    double n[3];     // unit normal (v1-v0) x (v2-v0)
    double scale;    // max(|v1-v0|, |v2-v0|)
};

struct RwgSlots {    // the two (triangle, slot) pairs of an RWG with amplitude sgn*len/(2A)
    int t[2];
    int s[2];
    double c[2];
};

__constant__ double c_w[7];

struct Vec3 {
    double x, y, z;
};
__device__ __forceinline__ Vec3 v3(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Vec3 operator*(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ Vec3 cross(Vec3 a, Vec3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm3(Vec3 a) { return sqrt(dot(a, a)); }

// G and grad_r G = (r - r') * gfac, far form
__device__ __forceinline__ void green_far(double R, double k, double2& G, double2& gfac) {
    double s, c;
    sincos(k * R, &s, &c);
    const double2 e = make_double2(c, -s);                       // e^{-jkR}
    G = make_double2(e.x / (kFourPi * R), e.y / (kFourPi * R));
    const double2 a = make_double2(1.0, k * R);                  // 1 + jkR
    const double2 ae = cmul(a, e);
    const double d = -1.0 / (kFourPi * R * R * R);
    gfac = make_double2(ae.x * d, ae.y * d);
}

// remainder after removing 1/(4 pi R): series for kR < 0.1, closed form otherwise
__device__ __forceinline__ void green_smooth(double R, double k, double2& Gs, double2& gfac) {
    const double kR = k * R;
    if (kR < 0.1) {
        // (e^{-jkR}-1)/R = sum_{n>=1} c_n R^{n-1},  d/dR = sum_{n>=2} c_n (n-1) R^{n-2},
        // c_n = (-jk)^n / n!
        double2 c = make_double2(1.0, 0.0);
        double2 g = make_double2(0.0, 0.0), h = make_double2(0.0, 0.0);
        double Rp_n1 = 1.0;    // R^{n-1}
        double Rp_n2 = 0.0;    // R^{n-2}
        for (int n = 1; n < 12; ++n) {
            c = cmul(c, make_double2(0.0, -k / (double)n));
            g.x += c.x * Rp_n1;
            g.y += c.y * Rp_n1;
            if (n >= 2) {
                h.x += c.x * (double)(n - 1) * Rp_n2;
                h.y += c.y * (double)(n - 1) * Rp_n2;
            }
            Rp_n2 = Rp_n1;
            Rp_n1 *= R;
        }
        Gs = make_double2(g.x / kFourPi, g.y / kFourPi);
        if (R > 0.0) gfac = make_double2(h.x / (kFourPi * R), h.y / (kFourPi * R));
        else gfac = make_double2(0.0, 0.0);
        return;
    }
    double s, cc;
    sincos(kR, &s, &cc);
    const double2 e = make_double2(cc, -s);
    Gs = make_double2((e.x - 1.0) / (kFourPi * R), e.y / (kFourPi * R));
    const double2 ae = cmul(make_double2(1.0, kR), e);           // (1 + jkR) e
    const double R2 = R * R;
    const double2 hh = make_double2((1.0 - ae.x) / R2, -ae.y / R2);
    gfac = make_double2(hh.x / (kFourPi * R), hh.y / (kFourPi * R));
}

// Lossy region (Sec. II-B, k_v = w sqrt(mu0 eps_v) with complex eps_v): the
// same two functions for k = kr + j ki, e^{-jkR} = e^{ki R} e^{-j kr R}.
__device__ __forceinline__ double2 exp_mjkR(double R, double kr, double ki) {
    double s, c;
    sincos(kr * R, &s, &c);
    const double m = exp(ki * R);
    return make_double2(m * c, -m * s);
}

__device__ __forceinline__ void green_far_cx(double R, double kr, double ki, double2& G, double2& gfac) {
    const double2 e = exp_mjkR(R, kr, ki);
    G = make_double2(e.x / (kFourPi * R), e.y / (kFourPi * R));
    const double2 ae = cmul(make_double2(1.0 - ki * R, kr * R), e);     // (1 + jkR) e
    const double d = -1.0 / (kFourPi * R * R * R);
    gfac = make_double2(ae.x * d, ae.y * d);
}

__device__ __forceinline__ void green_smooth_cx(double R, double kr, double ki, double2& Gs, double2& gfac) {
    if (hypot(kr, ki) * R < 0.1) {
        double2 c = make_double2(1.0, 0.0);
        double2 g = make_double2(0.0, 0.0), h = make_double2(0.0, 0.0);
        double Rp_n1 = 1.0, Rp_n2 = 0.0;
        for (int n = 1; n < 12; ++n) {
            c = cmul(c, make_double2(ki / (double)n, -kr / (double)n));   // (-jk)^n / n!
            g.x += c.x * Rp_n1;
            g.y += c.y * Rp_n1;
            if (n >= 2) {
                h.x += c.x * (double)(n - 1) * Rp_n2;
                h.y += c.y * (double)(n - 1) * Rp_n2;
            }
            Rp_n2 = Rp_n1;
            Rp_n1 *= R;
        }
        Gs = make_double2(g.x / kFourPi, g.y / kFourPi);
        if (R > 0.0) gfac = make_double2(h.x / (kFourPi * R), h.y / (kFourPi * R));
        else gfac = make_double2(0.0, 0.0);
        return;
    }
    const double2 e = exp_mjkR(R, kr, ki);
    Gs = make_double2((e.x - 1.0) / (kFourPi * R), e.y / (kFourPi * R));
    const double2 ae = cmul(make_double2(1.0 - ki * R, kr * R), e);
    const double R2 = R * R;
    const double2 hh = make_double2((1.0 - ae.x) / R2, -ae.y / R2);
    gfac = make_double2(hh.x / (kFourPi * R), hh.y / (kFourPi * R));
}

__device__ __forceinline__ double edge_log(double lp, double lm, double Rp, double Rm, double R02) {
    if (lm >= 0.0) return log((Rp + lp) / (Rm + lm));
    if (lp <= 0.0) return log((Rm - lm) / (Rp - lp));
    return log((Rp + lp) * (Rm - lm) / R02);
}

// closed-form int 1/R, int (rho'-rho)/R, int grad_r(1/R) over source triangle;
// also returns rho (projection of r on the plane, after the in-plane snap)
__device__ void potentials(Vec3 r, const TriGeo& T, double& I0, Vec3& I1, Vec3& Ig, Vec3& rho) {
    const Vec3 v0 = v3(T.v), n = v3(T.n);
    double d = dot(n, r - v0);
    if (fabs(d) <= 1e-9 * T.scale) d = 0.0;
    rho = r - d * n;
    const double ad = fabs(d);
    I0 = 0.0;
    I1 = {0.0, 0.0, 0.0};
    Vec3 fu = {0.0, 0.0, 0.0};
    double bsum = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const Vec3 a = v3(T.v + 3 * i), b = v3(T.v + 3 * ((i + 1) % 3));
        const Vec3 ba = b - a;
        const double le = norm3(ba);
        const Vec3 lh = (1.0 / le) * ba;
        const Vec3 u = cross(lh, n);
        const double lp = dot(b - rho, lh), lm = dot(a - rho, lh);
        const double t = dot(a - rho, u);
        const double R02 = t * t + d * d;
        const double Rp = sqrt(R02 + lp * lp), Rm = sqrt(R02 + lm * lm);
        const double f = edge_log(lp, lm, Rp, Rm, R02);
        const double beta = atan2(t * lp, R02 + ad * Rp) - atan2(t * lm, R02 + ad * Rm);
        I0 += t * f - ad * beta;
        I1 = I1 + (0.5 * (R02 * f + lp * Rp - lm * Rm)) * u;
        fu = fu + f * u;
        bsum += beta;
    }
    const double sg = (d > 0.0) - (d < 0.0);
    Ig = (-sg * bsum) * n - fu;
}

// out[((b*Tt + t)*Ts + s)*18 + {0..8: L(i,j), 9..17: K(i,j)}]; CX: complex
// wavenumber k + j ki (lossy region), else ki is ignored
template <bool CX>
__global__ void __launch_bounds__(128)
tri_pairs_kernel(const TriGeo* __restrict__ tg, int Tt, const TriGeo* __restrict__ sg, int Ts,
                 const double* __restrict__ shifts, const int8_t* __restrict__ sing, int b0,
                 double k, double ki, double2* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    const int bl = blockIdx.z;
    if (s >= Ts) return;
    const int b = b0 + bl;
    const TriGeo& A = tg[t];
    const TriGeo& S = sg[s];
    const Vec3 sh = v3(shifts + 3 * b);
    const bool singular = sing[b] != 0;
    double2 ik2c;                                   // 4 / k^2
    if constexpr (CX) {
        const double2 k2 = make_double2(k * k - ki * ki, 2.0 * k * ki);
        const double d = 4.0 / (k2.x * k2.x + k2.y * k2.y);
        ik2c = make_double2(k2.x * d, -k2.y * d);
    } else {
        ik2c = make_double2(4.0 / (k * k), 0.0);
    }
    const double ik2 = ik2c.x;
    double2 CL[9], CK[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) CL[q] = CK[q] = make_double2(0.0, 0.0);
    const Vec3 tv[3] = {v3(A.v) + sh, v3(A.v + 3) + sh, v3(A.v + 6) + sh};
    const Vec3 sv[3] = {v3(S.v), v3(S.v + 3), v3(S.v + 6)};
    double2 sumWG = make_double2(0.0, 0.0);
    for (int q = 0; q < 7; ++q) {
        const Vec3 r = v3(A.q + 3 * q) + sh;
        const double wq = c_w[q] * A.area;
        const Vec3 a[3] = {r - tv[0], r - tv[1], r - tv[2]};
        for (int p = 0; p < 7; ++p) {
            const Vec3 rp = v3(S.q + 3 * p);
            const double W = wq * c_w[p] * S.area;
            const Vec3 diff = r - rp;
            double R = norm3(diff);
            double2 G, gf;
            // coincident points (up to rounding) take the R -> 0 limit of the
            // remainder: -jk/(4 pi) and no gradient term
            if (singular && R <= 1e-9 * S.scale) R = 0.0;
            if constexpr (CX) {
                if (singular) green_smooth_cx(R, k, ki, G, gf);
                else green_far_cx(R, k, ki, G, gf);
            } else {
                if (singular) green_smooth(R, k, G, gf);
                else green_far(R, k, G, gf);
            }
            const double2 WG = make_double2(W * G.x, W * G.y);
            sumWG.x += WG.x;
            sumWG.y += WG.y;
            const double2 Wg = make_double2(W * gf.x, W * gf.y);
            const Vec3 bj[3] = {rp - sv[0], rp - sv[1], rp - sv[2]};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const Vec3 dxb = cross(diff, bj[j]);     // (r-r') x b_j
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double ab = dot(a[i], bj[j]);
                    CL[3 * i + j].x += WG.x * ab;
                    CL[3 * i + j].y += WG.y * ab;
                    const double trip = dot(a[i], dxb);    // a . ((r-r') x b)
                    CK[3 * i + j].x += Wg.x * trip;
                    CK[3 * i + j].y += Wg.y * trip;
                }
            }
        }
        if (singular) {
            double I0;
            Vec3 I1, Ig, rho;
            potentials(r, S, I0, I1, Ig, rho);
            const double f = wq / kFourPi;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const Vec3 vecL = I1 + I0 * (rho - sv[j]);
                const Vec3 cr = cross(Ig, r - sv[j]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    CL[3 * i + j].x += f * (dot(a[i], vecL) - ik2 * I0);
                    if constexpr (CX) CL[3 * i + j].y -= f * ik2c.y * I0;
                    CK[3 * i + j].x += f * dot(a[i], cr);
                }
            }
        }
    }
    double2* o = out + (((size_t)bl * Tt + t) * Ts + s) * 18;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        if constexpr (CX) {
            const double2 t = cmul(ik2c, sumWG);
            o[q] = make_double2(CL[q].x - t.x, CL[q].y - t.y);
        } else {
            o[q] = make_double2(CL[q].x - ik2 * sumWG.x, CL[q].y - ik2 * sumWG.y);
        }
        o[9 + q] = CK[q];
    }
}

// L[b][m][n], K[b][m][n] from the slot integrals of one chunk
__global__ void rwg_gather_kernel(const double2* __restrict__ S, const RwgSlots* __restrict__ tr,
                                  int Et, const RwgSlots* __restrict__ sr, int Es, int Tt, int Ts,
                                  int b0, int nb, double2* __restrict__ L, double2* __restrict__ K) {
    const size_t total = (size_t)nb * Et * Es;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(e % Es);
        const size_t t2 = e / Es;
        const int m = (int)(t2 % Et);
        const int bl = (int)(t2 / Et);
        const RwgSlots A = tr[m], B = sr[n];
        double2 l = make_double2(0.0, 0.0), kk = make_double2(0.0, 0.0);
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                const double c = A.c[x] * B.c[y];
                const double2* p = S + (((size_t)bl * Tt + A.t[x]) * Ts + B.t[y]) * 18;
                const int ij = 3 * A.s[x] + B.s[y];
                l.x += c * p[ij].x;
                l.y += c * p[ij].y;
                kk.x += c * p[9 + ij].x;
                kk.y += c * p[9 + ij].y;
            }
        const size_t o = ((size_t)(b0 + bl) * Et + m) * Es + n;
        L[o] = l;
        K[o] = kk;
    }
}

// ---------------------------------------------------------------- host side
void radon7(double bary[7][3], double w[7]) {
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
    const double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    for (int q = 0; q < 7; ++q) {
        w[q] = W[q];
        for (int v = 0; v < 3; ++v) bary[q][v] = B[q][v];
    }
}

int prepare_mesh(const double* verts, const int32_t* tris, const int32_t* slot_rwg,
                 const int8_t* slot_sgn, int T, int E, std::vector<TriGeo>& geo,
                 std::vector<RwgSlots>& rw) {
    double bary[7][3], w[7];
    radon7(bary, w);
    geo.resize(T);
    rw.assign(E, RwgSlots{{-1, -1}, {0, 0}, {0.0, 0.0}});
    std::vector<int> seen(E, 0);
    for (int t = 0; t < T; ++t) {
        TriGeo& g = geo[t];
        double V[3][3];
        for (int v = 0; v < 3; ++v)
            for (int x = 0; x < 3; ++x) V[v][x] = g.v[3 * v + x] = verts[3 * tris[3 * t + v] + x];
        for (int q = 0; q < 7; ++q)
            for (int x = 0; x < 3; ++x)
                g.q[3 * q + x] = bary[q][0] * V[0][x] + bary[q][1] * V[1][x] + bary[q][2] * V[2][x];
        const double e1[3] = {V[1][0] - V[0][0], V[1][1] - V[0][1], V[1][2] - V[0][2]};
        const double e2[3] = {V[2][0] - V[0][0], V[2][1] - V[0][1], V[2][2] - V[0][2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(cn > 0.0)) { set_error("degenerate triangle %d", t); return EMSURF_EINVAL; }
        g.area = 0.5 * cn;
        for (int x = 0; x < 3; ++x) g.n[x] = c[x] / cn;
        g.scale = std::max(std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]),
                           std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
        for (int i = 0; i < 3; ++i) {
            const int m = slot_rwg[3 * t + i];
            if (m < 0) continue;
            if (m >= E || seen[m] >= 2) { set_error("bad RWG slot map"); return EMSURF_EINVAL; }
            const double* p = V[(i + 1) % 3];
            const double* q = V[(i + 2) % 3];
            const double len = std::sqrt((p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) +
                                         (p[2] - q[2]) * (p[2] - q[2]));
            RwgSlots& r = rw[m];
            const int x = seen[m]++;
            r.t[x] = t;
            r.s[x] = i;
            r.c[x] = (double)slot_sgn[3 * t + i] * len / (2.0 * g.area);
        }
    }
    for (int m = 0; m < E; ++m)
        if (seen[m] != 2) { set_error("RWG %d has %d triangles", m, seen[m]); return EMSURF_EINVAL; }
    return EMSURF_OK;
}

}  // namespace


// L, K: device [nb][Et][Es]; wavenumber k + j ki (ki = 0: lossless)
int tabulate_blocks_cx(const MeshView& test, const MeshView& src, const double* shifts,
                       const int8_t* singular, int nb, double k, double ki, double2* L, double2* K,
                       cudaStream_t st) {
    if (!(k > 0.0) || !(ki <= 0.0) || nb < 1) {
        set_error("tabulate needs Re k > 0, Im k <= 0 and >= 1 block");
        return EMSURF_EINVAL;
    }
    std::vector<TriGeo> tg, sgeo;
    std::vector<RwgSlots> tr, sr;
    EMS_TRY(prepare_mesh(test.verts, test.tris, test.slot_rwg, test.slot_sgn, test.T, test.E, tg, tr));
    EMS_TRY(prepare_mesh(src.verts, src.tris, src.slot_rwg, src.slot_sgn, src.T, src.E, sgeo, sr));
    double bary[7][3], w[7];
    radon7(bary, w);
    EMS_CUDA(cudaMemcpyToSymbolAsync(c_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st));
    const size_t per_block = (size_t)test.T * src.T * 18 * sizeof(double2);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(nb, kScratchBytes / per_block));
    TriGeo *dtg = nullptr, *dsg = nullptr;
    RwgSlots *dtr = nullptr, *dsr = nullptr;
    double* dsh = nullptr;
    int8_t* dsi = nullptr;
    double2* scratch = nullptr;
    int status = EMSURF_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        set_error("tabulate: %s: %s", what, cudaGetErrorString(e));
        status = EMSURF_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&dtg, sizeof(TriGeo) * tg.size())) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&dsg, sizeof(TriGeo) * sgeo.size())) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&dtr, sizeof(RwgSlots) * tr.size())) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&dsr, sizeof(RwgSlots) * sr.size())) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&dsh, sizeof(double) * 3 * nb)) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&dsi, nb)) != cudaSuccess) fail(e, "alloc");
    if (!status && (e = cudaMalloc(&scratch, per_block * chunk)) != cudaSuccess) fail(e, "scratch alloc");
    if (!status) {
        cudaMemcpyAsync(dtg, tg.data(), sizeof(TriGeo) * tg.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dsg, sgeo.data(), sizeof(TriGeo) * sgeo.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dtr, tr.data(), sizeof(RwgSlots) * tr.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dsr, sr.data(), sizeof(RwgSlots) * sr.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dsh, shifts, sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dsi, singular, nb, cudaMemcpyHostToDevice, st);
        for (int b0 = 0; b0 < nb && !status; b0 += chunk) {
            const int nc = std::min(chunk, nb - b0);
            dim3 g1((src.T + 127) / 128, test.T, nc);
            if (ki != 0.0)
                tri_pairs_kernel<true><<<g1, 128, 0, st>>>(dtg, test.T, dsg, src.T, dsh, dsi, b0, k, ki, scratch);
            else
                tri_pairs_kernel<false><<<g1, 128, 0, st>>>(dtg, test.T, dsg, src.T, dsh, dsi, b0, k, 0.0, scratch);
            if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "tri_pairs_kernel"); break; }
            const size_t tot = (size_t)nc * test.E * src.E;
            const int g2 = (int)std::min<size_t>((tot + 255) / 256, 152 * 64);
            rwg_gather_kernel<<<g2, 256, 0, st>>>(scratch, dtr, test.E, dsr, src.E, test.T, src.T, b0,
                                                  nc, L, K);
            if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "rwg_gather_kernel"); break; }
        }
        if (!status && (e = cudaStreamSynchronize(st)) != cudaSuccess) fail(e, "synchronize");
    }
    cudaFree(dtg);
    cudaFree(dsg);
    cudaFree(dtr);
    cudaFree(dsr);
    cudaFree(dsh);
    cudaFree(dsi);
    cudaFree(scratch);
    return status;
}

int tabulate_blocks(const MeshView& test, const MeshView& src, const double* shifts,
                    const int8_t* singular, int nb, double k, double2* L, double2* K,
                    cudaStream_t st) {
    return tabulate_blocks_cx(test, src, shifts, singular, nb, k, 0.0, L, K, st);
}

// ---------------------------------------------------------------------------
// Allocation-free tabulation.  Scratch lives in one file-scope device array
// that every GPU loading this library holds until the process exits.  Host
// code must not use the array's name as a device address (it is a host-side
// stand-in); the device address comes from cudaGetSymbolAddress, taken once
// per device with that device current and cached.
namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;   // 64 MiB per device
static __device__ __align__(256) unsigned char g_tab_scratch[kNoAllocBytes];

std::mutex g_tab_scratch_mu;
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    void* ctx = nullptr;     // context the address was taken in
    void* addr = nullptr;
};
ScratchAddr g_tab_scratch_addr[kMaxDevices];

// cuCtxGetCurrent through the runtime's driver entry point (no link to the
// driver library); a context created after a device reset gets a new handle,
// so the cached address is taken again in it
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

int scratch_address(void** out) {
    int dev = -1;
    EMS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d outside [0, %d)", dev, kMaxDevices);
        return EMSURF_EINVAL;
    }
    const CtxGetCurrentFn fn = ctx_get_current();
    void* ctx = nullptr;
    if (fn) fn(&ctx);
    std::lock_guard<std::mutex> lock(g_tab_scratch_mu);
    ScratchAddr& c = g_tab_scratch_addr[dev];
    if (!c.addr || !ctx || c.ctx != ctx) {
        void* p = nullptr;
        // binds the device's primary context if none is current yet
        const cudaError_t e = cudaGetSymbolAddress(&p, g_tab_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return EMSURF_ECUDA;
        }
        if (fn && !ctx) fn(&ctx);
        c.ctx = ctx;
        c.addr = p;
    }
    *out = c.addr;
    return EMSURF_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int tabulate_blocks_noalloc(const MeshView& test, const MeshView& src, const double* shifts,
                            const int8_t* singular, int nb, double k, double2* L, double2* K,
                            cudaStream_t st) {
    if (!(k > 0.0) || nb < 1) { set_error("tabulate needs k > 0 and >= 1 block"); return EMSURF_EINVAL; }
    std::vector<TriGeo> tg, sgeo;
    std::vector<RwgSlots> tr, sr;
    EMS_TRY(prepare_mesh(test.verts, test.tris, test.slot_rwg, test.slot_sgn, test.T, test.E, tg, tr));
    EMS_TRY(prepare_mesh(src.verts, src.tris, src.slot_rwg, src.slot_sgn, src.T, src.E, sgeo, sr));
    // carve the static array: geometry, then the per-chunk pair integrals
    const size_t o_tg = 0;
    const size_t o_sg = o_tg + align256(sizeof(TriGeo) * tg.size());
    const size_t o_tr = o_sg + align256(sizeof(TriGeo) * sgeo.size());
    const size_t o_sr = o_tr + align256(sizeof(RwgSlots) * tr.size());
    const size_t o_sh = o_sr + align256(sizeof(RwgSlots) * sr.size());
    const size_t o_si = o_sh + align256(sizeof(double) * 3 * (size_t)nb);
    const size_t o_pairs = o_si + align256((size_t)nb);
    const size_t per_block = (size_t)test.T * src.T * 18 * sizeof(double2);
    if (o_pairs + per_block > kNoAllocBytes) {
        set_error("emsurf_tabulate_noalloc needs %zu bytes of scratch for these meshes and %d "
                  "blocks; its static scratch holds %zu bytes",
                  o_pairs + per_block, nb, kNoAllocBytes);
        return EMSURF_EINVAL;
    }
    void* base = nullptr;
    EMS_TRY(scratch_address(&base));
    unsigned char* b = static_cast<unsigned char*>(base);
    TriGeo* dtg = reinterpret_cast<TriGeo*>(b + o_tg);
    TriGeo* dsg = reinterpret_cast<TriGeo*>(b + o_sg);
    RwgSlots* dtr = reinterpret_cast<RwgSlots*>(b + o_tr);
    RwgSlots* dsr = reinterpret_cast<RwgSlots*>(b + o_sr);
    double* dsh = reinterpret_cast<double*>(b + o_sh);
    int8_t* dsi = reinterpret_cast<int8_t*>(b + o_si);
    double2* pairs = reinterpret_cast<double2*>(b + o_pairs);
    const int chunk = (int)std::min<size_t>(nb, (kNoAllocBytes - o_pairs) / per_block);
    double bary[7][3], w[7];
    radon7(bary, w);
    // from the first queued copy on, every return goes through the stream
    // synchronisation below, so no queued work outlives the call
    int status = EMSURF_OK;
    auto step = [&](cudaError_t e, const char* what) {
        if (status == EMSURF_OK && e != cudaSuccess) {
            set_error("emsurf_tabulate_noalloc: %s: %s", what, cudaGetErrorString(e));
            status = EMSURF_ECUDA;
        }
    };
    step(cudaMemcpyToSymbolAsync(c_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st), "copy weights");
    if (!status) step(cudaMemcpyAsync(dtg, tg.data(), sizeof(TriGeo) * tg.size(), cudaMemcpyHostToDevice, st), "copy");
    if (!status) step(cudaMemcpyAsync(dsg, sgeo.data(), sizeof(TriGeo) * sgeo.size(), cudaMemcpyHostToDevice, st), "copy");
    if (!status) step(cudaMemcpyAsync(dtr, tr.data(), sizeof(RwgSlots) * tr.size(), cudaMemcpyHostToDevice, st), "copy");
    if (!status) step(cudaMemcpyAsync(dsr, sr.data(), sizeof(RwgSlots) * sr.size(), cudaMemcpyHostToDevice, st), "copy");
    if (!status) step(cudaMemcpyAsync(dsh, shifts, sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, st), "copy");
    if (!status) step(cudaMemcpyAsync(dsi, singular, nb, cudaMemcpyHostToDevice, st), "copy");
    // every pair integral is written before it is read, so nothing needs clearing
    for (int b0 = 0; b0 < nb && !status; b0 += chunk) {
        const int nc = std::min(chunk, nb - b0);
        dim3 g1((src.T + 127) / 128, test.T, nc);
        tri_pairs_kernel<false><<<g1, 128, 0, st>>>(dtg, test.T, dsg, src.T, dsh, dsi, b0, k, 0.0, pairs);
        step(cudaGetLastError(), "tri_pairs_kernel");
        if (status) break;
        const size_t tot = (size_t)nc * test.E * src.E;
        const int g2 = (int)std::min<size_t>((tot + 255) / 256, 152 * 64);
        rwg_gather_kernel<<<g2, 256, 0, st>>>(pairs, dtr, test.E, dsr, src.E, test.T, src.T, b0, nc,
                                              L, K);
        step(cudaGetLastError(), "rwg_gather_kernel");
    }
    step(cudaStreamSynchronize(st), "synchronize");
    return status;
}

}  // namespace

}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API int emsurf_tabulate_noalloc(const double* test_verts, const int32_t* test_tris,
                                       const int32_t* test_slot_rwg, const int8_t* test_slot_sgn,
                                       int32_t test_T, int32_t test_E, const double* src_verts,
                                       const int32_t* src_tris, const int32_t* src_slot_rwg,
                                       const int8_t* src_slot_sgn, int32_t src_T, int32_t src_E,
                                       const double* shifts, const int8_t* singular,
                                       int32_t n_blocks, double k, emsurf_c128* L, emsurf_c128* K,
                                       void* stream) {
    if (!test_verts || !test_tris || !test_slot_rwg || !test_slot_sgn || !src_verts || !src_tris ||
        !src_slot_rwg || !src_slot_sgn || !shifts || !singular || !L || !K || test_T < 1 ||
        src_T < 1 || test_E < 1 || src_E < 1) {
        set_error("emsurf_tabulate_noalloc: NULL pointer or empty mesh");
        return EMSURF_EINVAL;
    }
    MeshView t{test_verts, test_tris, test_slot_rwg, test_slot_sgn, test_T, test_E};
    MeshView s{src_verts, src_tris, src_slot_rwg, src_slot_sgn, src_T, src_E};
    return tabulate_blocks_noalloc(t, s, shifts, singular, n_blocks, k, reinterpret_cast<double2*>(L),
                                   reinterpret_cast<double2*>(K), reinterpret_cast<cudaStream_t>(stream));
}

EMSURF_API int emsurf_tabulate(const double* test_verts, const int32_t* test_tris,
                               const int32_t* test_slot_rwg, const int8_t* test_slot_sgn,
                               int32_t test_T, int32_t test_E, const double* src_verts,
                               const int32_t* src_tris, const int32_t* src_slot_rwg,
                               const int8_t* src_slot_sgn, int32_t src_T, int32_t src_E,
                               const double* shifts, const int8_t* singular, int32_t n_blocks,
                               double k, emsurf_c128* L, emsurf_c128* K, void* stream) {
    if (!test_verts || !test_tris || !test_slot_rwg || !test_slot_sgn || !src_verts || !src_tris ||
        !src_slot_rwg || !src_slot_sgn || !shifts || !singular || !L || !K || test_T < 1 ||
        src_T < 1 || test_E < 1 || src_E < 1) {
        set_error("emsurf_tabulate: NULL pointer or empty mesh");
        return EMSURF_EINVAL;
    }
    MeshView t{test_verts, test_tris, test_slot_rwg, test_slot_sgn, test_T, test_E};
    MeshView s{src_verts, src_tris, src_slot_rwg, src_slot_sgn, src_T, src_E};
    return tabulate_blocks(t, s, shifts, singular, n_blocks, k, reinterpret_cast<double2*>(L),
                           reinterpret_cast<double2*>(K), reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace emsurf {
namespace {
// T(d) <- (T(d) + T(-d)^T) / 2 for both tables in place: offset o and its
// mirror nof - 1 - o form one pair, handled by one thread per entry pair.
__global__ void reciprocal_part_kernel(double2* __restrict__ L, double2* __restrict__ K, int nof, int E) {
    const size_t EE = (size_t)E * E, total = (size_t)nof * EE;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / EE), om = nof - 1 - o;
        const int i = (int)((e % EE) / E), j = (int)(e % E);
        if (o > om || (o == om && i >= j)) continue;
        const size_t p = e, q = (size_t)om * EE + (size_t)j * E + i;
        double2 t[2] = {L[p], K[p]};
        double2 u[2] = {L[q], K[q]};
        const double2 sl = make_double2((t[0].x + u[0].x) * 0.5, (t[0].y + u[0].y) * 0.5);
        const double2 sk = make_double2((t[1].x + u[1].x) * 0.5, (t[1].y + u[1].y) * 0.5);
        L[p] = sl;
        L[q] = sl;
        K[p] = sk;
        K[q] = sk;
    }
}
}  // namespace
}  // namespace emsurf

extern "C" {

EMSURF_API int emsurf_tabulate_offsets(double a, double b, double h, int32_t n,
                                       const double* zlevels, int32_t nx, int32_t ny, double k,
                                       emsurf_c128* L, emsurf_c128* K, void* stream) {
    if (n < 1 || nx < 1 || ny < 1 || !L || !K) {
        set_error("emsurf_tabulate_offsets: bad sizes or NULL output");
        return EMSURF_EINVAL;
    }
    int32_t V, T, E;
    EMS_TRY(emsurf_setup_box_counts(n, &V, &T, &E));
    std::vector<double> verts(3 * V);
    std::vector<int32_t> tris(3 * T), edges(2 * E), tp(E), tm(E), srw(3 * T);
    std::vector<int8_t> ssg(3 * T);
    EMS_TRY(emsurf_setup_box_mesh(a, b, h, n, zlevels, verts.data(), tris.data(), edges.data(),
                                  tp.data(), tm.data(), srw.data(), ssg.data()));
    const int nox = 2 * nx - 1, noy = 2 * ny - 1;
    std::vector<double> shifts(3 * (size_t)nox * noy);
    std::vector<int8_t> sing((size_t)nox * noy);
    for (int dyi = 0; dyi < noy; ++dyi)
        for (int dxi = 0; dxi < nox; ++dxi) {
            const int dx = dxi - (nx - 1), dy = dyi - (ny - 1);
            const size_t o = (size_t)dyi * nox + dxi;
            shifts[3 * o] = dx * a;
            shifts[3 * o + 1] = dy * b;
            shifts[3 * o + 2] = 0.0;
            sing[o] = (std::abs(dx) <= 1 && std::abs(dy) <= 1) ? 1 : 0;
        }
    MeshView mv{verts.data(), tris.data(), srw.data(), ssg.data(), T, E};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    EMS_TRY(tabulate_blocks(mv, mv, shifts.data(), sing.data(), nox * noy, k, reinterpret_cast<double2*>(L),
                            reinterpret_cast<double2*>(K), st));
    // reciprocal part of the one-sided blocks (exactly reciprocal tables)
    const size_t total = (size_t)nox * noy * E * E;
    reciprocal_part_kernel<<<(int)std::min<size_t>((total + 255) / 256, 152 * 64), 256, 0, st>>>(
        reinterpret_cast<double2*>(L), reinterpret_cast<double2*>(K), nox * noy, E);
    EMS_CUDA(cudaGetLastError());
    EMS_CUDA(cudaStreamSynchronize(st));
    return EMSURF_OK;
}

}  // extern "C"
