// Excitation vector (Eq. out) and far field / RCS (Sec. III-D: fields
// radiated by the solved box currents through the free-space operators).
//
// Plane wave E_inc = e^{-jk khat.r} ehat, |E_inc| = 1 V/m, eta0 H_inc =
// (khat x ehat) e^{-jk khat.r}.  V^(m) tests E_inc (rows J) and eta0 H_inc
// (rows M) with the RWGs of box m; since box m is box 0 translated by c_m,
// V^(m) = e^{-jk khat.c_m} V^(0) exactly.  V~ = U_o^T V (Eq. final).
//
// Far field, E ~ F e^{-jkr}/r:  F = -(jk/4pi) [N_perp - rhat x L_M] with
// N = sum_m e^{jk rhat.c_m} sum_e x_J[m,e] R_e(rhat),
// L_M = same with x_M, R_e(rhat) = int Lam_e e^{jk rhat.r'} dS' on box 0,
// x = U_o Y~.  Bistatic RCS sigma = 4 pi |F|^2 / |E_inc|^2.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;

// per RWG: 14 quadrature points (7 on T+, 7 on T-), weight w*A*sgn*len/(2A),
// free vertex of the point's triangle
struct RwgQuad {
    double r[14][3];
    double w[14];
    double p[14][3];
};

__device__ __forceinline__ double2 cexpj(double phase) {   // e^{j phase}
    double s, c;
    sincos(phase, &s, &c);
    return make_double2(c, s);
}

// V0[r][e] = <Lam_e, ehat e^{-jk khat.r}>, V0[r][E+e] = <Lam_e, (khat x ehat) e^{..}>
__global__ void excitation_box_kernel(const RwgQuad* __restrict__ q, int E, int R,
                                      const double* __restrict__ khat, const double* __restrict__ ehat,
                                      double k, double2* __restrict__ V0) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (e >= E) return;
    const double* kh = khat + 3 * r;
    const double* eh = ehat + 3 * r;
    const double hv[3] = {kh[1] * eh[2] - kh[2] * eh[1], kh[2] * eh[0] - kh[0] * eh[2],
                          kh[0] * eh[1] - kh[1] * eh[0]};
    double2 vE = make_double2(0.0, 0.0), vH = make_double2(0.0, 0.0);
    const RwgQuad& Q = q[e];
    for (int i = 0; i < 14; ++i) {
        const double a[3] = {Q.r[i][0] - Q.p[i][0], Q.r[i][1] - Q.p[i][1], Q.r[i][2] - Q.p[i][2]};
        const double2 ph = cexpj(-k * (kh[0] * Q.r[i][0] + kh[1] * Q.r[i][1] + kh[2] * Q.r[i][2]));
        const double pe = Q.w[i] * (a[0] * eh[0] + a[1] * eh[1] + a[2] * eh[2]);
        const double phh = Q.w[i] * (a[0] * hv[0] + a[1] * hv[1] + a[2] * hv[2]);
        vE.x += pe * ph.x;
        vE.y += pe * ph.y;
        vH.x += phh * ph.x;
        vH.y += phh * ph.y;
    }
    V0[(size_t)r * 2 * E + e] = vE;
    V0[(size_t)r * 2 * E + E + e] = vH;
}

// V~[r][u] = sum over (m,k) of u: sign * e^{-jk khat.c_m} V0[r][k]
__global__ void excitation_scatter_kernel(const double2* __restrict__ V0, const int32_t* __restrict__ ptr,
                                          const int32_t* __restrict__ ent, const int8_t* __restrict__ esg,
                                          int nx, double a, double b, const double* __restrict__ khat,
                                          double k, int K, int n_unique, int R,
                                          double2* __restrict__ V) {
    const size_t total = (size_t)R * n_unique;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(e % n_unique), r = (int)(e / n_unique);
        const double* kh = khat + 3 * r;
        double2 acc = make_double2(0.0, 0.0);
        for (int q = ptr[u]; q < ptr[u + 1]; ++q) {
            const int loc = ent[q];
            const int m = loc / K, kk = loc % K;
            const double cx = (m % nx) * a, cy = (m / nx) * b;
            const double2 ph = cexpj(-k * (kh[0] * cx + kh[1] * cy));
            const double2 v = cmul(ph, V0[(size_t)r * K + kk]);
            const double s = (double)esg[q];
            acc.x += s * v.x;
            acc.y += s * v.y;
        }
        V[e] = acc;
    }
}

// Rv[d][e][3] = int Lam_e e^{jk rhat_d . r'}
__global__ void radiation_kernel(const RwgQuad* __restrict__ q, int E, const double* __restrict__ rhat,
                                 int D, double k, double2* __restrict__ Rv) {
    const size_t total = (size_t)D * E;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(x % E);
        const int d = (int)(x / E);
        const double* rh = rhat + 3 * d;
        const RwgQuad& Q = q[e];
        double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        for (int i = 0; i < 14; ++i) {
            const double2 ph = cexpj(k * (rh[0] * Q.r[i][0] + rh[1] * Q.r[i][1] + rh[2] * Q.r[i][2]));
            for (int c = 0; c < 3; ++c) {
                const double a = Q.w[i] * (Q.r[i][c] - Q.p[i][c]);
                acc[c].x += a * ph.x;
                acc[c].y += a * ph.y;
            }
        }
        for (int c = 0; c < 3; ++c) Rv[x * 3 + c] = acc[c];
    }
}

// S[r][d][k] = sum_m e^{jk rhat_d . c_m} sign * Y[r][idx[m*K + k]]
__global__ void lattice_sum_kernel(const double2* __restrict__ Y, const int32_t* __restrict__ idx,
                                   const int8_t* __restrict__ sgn, int nx, int M, int K, int n_unique,
                                   double a, double b, const double* __restrict__ rhat, int D,
                                   int R, double k, double2* __restrict__ S) {
    const size_t total = (size_t)R * D * K;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(x % K);
        const int d = (int)((x / K) % D);
        const int r = (int)(x / ((size_t)K * D));
        const double* rh = rhat + 3 * d;
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) {
            const size_t loc = (size_t)m * K + kk;
            const double2 y = Y[(size_t)r * n_unique + idx[loc]];
            const double s = (double)sgn[loc];
            const double2 ph = cexpj(k * (rh[0] * (m % nx) * a + rh[1] * (m / nx) * b));
            acc.x += s * (ph.x * y.x - ph.y * y.y);
            acc.y += s * (ph.x * y.y + ph.y * y.x);
        }
        S[x] = acc;
    }
}

__global__ void far_field_kernel(const double2* __restrict__ S, const double2* __restrict__ Rv,
                                 const double* __restrict__ rhat, int D, int E, int R, double k,
                                 double2* __restrict__ F, double* __restrict__ rcs) {
    const size_t total = (size_t)R * D;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int d = (int)(x % D);
        const double* rh = rhat + 3 * d;
        const double2* s = S + x * 2 * E;
        const double2* rv = Rv + (size_t)d * E * 3;
        double2 N[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        double2 L[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        for (int e = 0; e < E; ++e)
            for (int c = 0; c < 3; ++c) {
                cfma(N[c], s[e], rv[3 * e + c]);
                cfma(L[c], s[E + e], rv[3 * e + c]);
            }
        double2 rn = make_double2(0, 0);
        for (int c = 0; c < 3; ++c) {
            rn.x += rh[c] * N[c].x;
            rn.y += rh[c] * N[c].y;
        }
        double2 v[3];
        for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            // N_perp - rhat x L
            const double2 rxl = make_double2(rh[c1] * L[c2].x - rh[c2] * L[c1].x,
                                             rh[c1] * L[c2].y - rh[c2] * L[c1].y);
            v[c] = make_double2(N[c].x - rn.x * rh[c] - rxl.x, N[c].y - rn.y * rh[c] - rxl.y);
        }
        double mag = 0.0;
        for (int c = 0; c < 3; ++c) {
            // -(jk / 4pi) v
            const double2 f = make_double2(k * v[c].y / kFourPi, -k * v[c].x / kFourPi);
            F[x * 3 + c] = f;
            mag += f.x * f.x + f.y * f.y;
        }
        if (rcs) rcs[x] = kFourPi * mag;
    }
}

int box_quadrature(double a, double b, double h, int n, const double* zlevels, int E_expected,
                   std::vector<RwgQuad>& out) {
    int32_t V, T, E;
    EMS_TRY(emsurf_setup_box_counts(n, &V, &T, &E));
    if (E != E_expected) {
        set_error("box mesh n=%d has %d RWGs, the handle has %d", n, E, E_expected);
        return EMSURF_EINVAL;
    }
    std::vector<double> verts(3 * V);
    std::vector<int32_t> tris(3 * T), edges(2 * E), tp(E), tm(E), srw(3 * T);
    std::vector<int8_t> ssg(3 * T);
    EMS_TRY(emsurf_setup_box_mesh(a, b, h, n, zlevels, verts.data(), tris.data(), edges.data(),
                                  tp.data(), tm.data(), srw.data(), ssg.data()));
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
    const double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    out.assign(E, RwgQuad{});
    std::vector<int> seen(E, 0);
    for (int t = 0; t < T; ++t) {
        double P[3][3];
        for (int v = 0; v < 3; ++v)
            for (int x = 0; x < 3; ++x) P[v][x] = verts[3 * tris[3 * t + v] + x];
        const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double A = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int i = 0; i < 3; ++i) {
            const int m = srw[3 * t + i];
            const double* p = P[(i + 1) % 3];
            const double* qv = P[(i + 2) % 3];
            const double len = std::sqrt((p[0] - qv[0]) * (p[0] - qv[0]) + (p[1] - qv[1]) * (p[1] - qv[1]) +
                                         (p[2] - qv[2]) * (p[2] - qv[2]));
            const double amp = ssg[3 * t + i] * len / (2.0 * A);
            const int base = 7 * seen[m]++;
            for (int q = 0; q < 7; ++q) {
                for (int x = 0; x < 3; ++x) {
                    out[m].r[base + q][x] = B[q][0] * P[0][x] + B[q][1] * P[1][x] + B[q][2] * P[2][x];
                    out[m].p[base + q][x] = P[i][x];
                }
                out[m].w[base + q] = W[q] * A * amp;
            }
        }
    }
    return EMSURF_OK;
}

template <typename T>
int to_device(T** d, const T* h, size_t n, cudaStream_t st) {
    EMS_CUDA(cudaMalloc(d, sizeof(T) * std::max<size_t>(n, 1)));
    EMS_CUDA(cudaMemcpyAsync(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice, st));
    return EMSURF_OK;
}

struct Scoped {
    std::vector<void*> p;
    ~Scoped() {
        for (void* x : p) cudaFree(x);
    }
};

}  // namespace
}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API int emsurf_excitation(emsurf_handle* h, double a, double b, double hgt, int32_t n,
                                 const double* zlevels, double k, int32_t nrhs, const double* khat, const double* ehat,
                                 emsurf_c128* V, void* stream) {
    if (!h || !khat || !ehat || !V || nrhs < 1 || !(k > 0.0)) {
        set_error("emsurf_excitation: bad arguments");
        return EMSURF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<RwgQuad> q;
    EMS_TRY(box_quadrature(a, b, hgt, n, zlevels, h->E, q));
    Scoped sc;
    RwgQuad* dq;
    double *dk, *de;
    double2* V0;
    EMS_TRY(to_device(&dq, q.data(), q.size(), st));
    sc.p.push_back(dq);
    EMS_TRY(to_device(&dk, khat, 3 * (size_t)nrhs, st));
    sc.p.push_back(dk);
    EMS_TRY(to_device(&de, ehat, 3 * (size_t)nrhs, st));
    sc.p.push_back(de);
    EMS_CUDA(cudaMalloc(&V0, sizeof(double2) * nrhs * h->K));
    sc.p.push_back(V0);
    excitation_box_kernel<<<dim3((h->E + 127) / 128, nrhs), 128, 0, st>>>(dq, h->E, nrhs, dk, de, k, V0);
    EMS_CUDA(cudaGetLastError());
    const size_t tot = (size_t)nrhs * h->n_unique;
    excitation_scatter_kernel<<<(int)std::min<size_t>((tot + 255) / 256, 152 * 32), 256, 0, st>>>(
        V0, h->d_inv_ptr, h->d_inv_ent, h->d_inv_sgn, h->nx, a, b, dk, k, h->K, h->n_unique, nrhs,
        reinterpret_cast<double2*>(V));
    EMS_CUDA(cudaGetLastError());
    EMS_CUDA(cudaStreamSynchronize(st));
    return EMSURF_OK;
}

EMSURF_API int emsurf_far_field(emsurf_handle* h, double a, double b, double hgt, int32_t n,
                                const double* zlevels, double k,
                                const emsurf_c128* Y, int32_t nrhs, int32_t ndir, const double* rhat,
                                emsurf_c128* F, double* rcs, void* stream) {
    if (!h || !Y || !rhat || !F || nrhs < 1 || ndir < 1 || !(k > 0.0)) {
        set_error("emsurf_far_field: bad arguments");
        return EMSURF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<RwgQuad> q;
    EMS_TRY(box_quadrature(a, b, hgt, n, zlevels, h->E, q));
    const int E = h->E, K = h->K;
    // directions in chunks so the per-chunk work arrays stay under ~512 MB
    const size_t per_dir = (size_t)E * 3 * sizeof(double2) + (size_t)nrhs * K * sizeof(double2);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(ndir, (512ull << 20) / per_dir));
    Scoped sc;
    RwgQuad* dq;
    double* dr;
    double2 *Rv, *S;
    EMS_TRY(to_device(&dq, q.data(), q.size(), st));
    sc.p.push_back(dq);
    EMS_TRY(to_device(&dr, rhat, 3 * (size_t)ndir, st));
    sc.p.push_back(dr);
    EMS_CUDA(cudaMalloc(&Rv, sizeof(double2) * (size_t)chunk * E * 3));
    sc.p.push_back(Rv);
    EMS_CUDA(cudaMalloc(&S, sizeof(double2) * (size_t)chunk * nrhs * K));
    sc.p.push_back(S);
    double2* Fo = reinterpret_cast<double2*>(F);
    std::vector<double2> hbuf;
    for (int d0 = 0; d0 < ndir; d0 += chunk) {
        const int nd = std::min(chunk, ndir - d0);
        const size_t t1 = (size_t)nd * E;
        radiation_kernel<<<(int)std::min<size_t>((t1 + 127) / 128, 152 * 32), 128, 0, st>>>(
            dq, E, dr + 3 * (size_t)d0, nd, k, Rv);
        EMS_CUDA(cudaGetLastError());
        const size_t t2 = (size_t)nrhs * nd * K;
        lattice_sum_kernel<<<(int)std::min<size_t>((t2 + 255) / 256, 152 * 32), 256, 0, st>>>(
            reinterpret_cast<const double2*>(Y), h->d_uo_index, h->d_uo_sign, h->nx, h->M, K,
            h->n_unique, a, b, dr + 3 * (size_t)d0, nd, nrhs, k, S);
        EMS_CUDA(cudaGetLastError());
        // F chunk is written per rhs into [nrhs][ndir][3]
        for (int r = 0; r < nrhs; ++r) {
            const size_t t3 = (size_t)nd;
            far_field_kernel<<<(int)std::min<size_t>((t3 + 127) / 128, 152 * 32), 128, 0, st>>>(
                S + (size_t)r * nd * K, Rv, dr + 3 * (size_t)d0, nd, E, 1, k,
                Fo + ((size_t)r * ndir + d0) * 3, rcs ? rcs + (size_t)r * ndir + d0 : nullptr);
            EMS_CUDA(cudaGetLastError());
        }
    }
    EMS_CUDA(cudaStreamSynchronize(st));
    return EMSURF_OK;
}

}  // extern "C"
