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

// X1[m][r K + k] = sign * Y[r][idx[m K + k]]: every cell's box currents
template <typename C>
__global__ void gather_cells_kernel(const double2* __restrict__ Y, const int32_t* __restrict__ idx,
                                    const int8_t* __restrict__ sgn, int M, int K, int R, int n_unique,
                                    C* __restrict__ X1) {
    const size_t N = (size_t)R * K, total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t m = e / N, rem = e - m * N;
        const int r = (int)(rem / K), kk = (int)(rem - (size_t)r * K);
        const size_t loc = m * K + kk;
        const double s = (double)sgn[loc];
        const double2 y = Y[(size_t)r * n_unique + idx[loc]];
        C v;
        v.x = s * y.x;
        v.y = s * y.y;
        X1[e] = v;
    }
}

// The array factor of every column: S[d][n] = sum_m e^{jk rhat_d . c_m}
// X1[m][n], c_m = (ix a, iy b, 0).  A block computes kLsD directions x kLsN
// columns; the phase of cell m factors into per-direction tables
// e^{jk rx a ix} e^{jk ry b iy} (one sincos per direction and row or column of
// the lattice instead of one per term), X1 is staged kLsM cells at a time.
// Each thread holds 2 directions x 4 columns (columns tn + 16 c, so a
// warp's shared-memory reads are consecutive).  T: arithmetic type (double
// for FP64 handles; float, with float accumulation over the cells, for
// FP32 / MIXED handles).
constexpr int kLsD = 32, kLsN = 64, kLsM = 16, kLsThreads = 256;

template <typename T, typename C>
__global__ void __launch_bounds__(kLsThreads)
lattice_sum_tiled_kernel(const C* __restrict__ X1, int M, int N, int nx, int ny, double a, double b,
                         const double* __restrict__ rhat, int nd, double k, C* __restrict__ S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* px = reinterpret_cast<C*>(smem_raw);            // [kLsD][nx]
    C* py = px + kLsD * nx;                            // [kLsD][ny]
    C* xs = py + kLsD * ny;                            // [kLsM][kLsN]
    const int d0 = blockIdx.y * kLsD, n0 = blockIdx.x * kLsN;
    for (int e = threadIdx.x; e < kLsD * nx; e += blockDim.x) {
        const int dd = e / nx, ix = e - dd * nx, d = d0 + dd;
        double sn = 0.0, cs = 1.0;
        if (d < nd) sincos(k * a * rhat[3 * d] * ix, &sn, &cs);
        px[e].x = (T)cs;
        px[e].y = (T)sn;
    }
    for (int e = threadIdx.x; e < kLsD * ny; e += blockDim.x) {
        const int dd = e / ny, iy = e - dd * ny, d = d0 + dd;
        double sn = 0.0, cs = 1.0;
        if (d < nd) sincos(k * b * rhat[3 * d + 1] * iy, &sn, &cs);
        py[e].x = (T)cs;
        py[e].y = (T)sn;
    }
    const int tn = threadIdx.x & 15, td = threadIdx.x >> 4;     // 16 column groups x 16 direction pairs
    C acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c].x = acc[i][c].y = (T)0;
    const C* pxa = px + (2 * td) * nx;
    const C* pxb = pxa + nx;
    const C* pya = py + (2 * td) * ny;
    const C* pyb = pya + ny;
    for (int m0 = 0; m0 < M; m0 += kLsM) {
        __syncthreads();
        for (int e = threadIdx.x; e < kLsM * kLsN; e += blockDim.x) {
            const int mm = e / kLsN, c = e - mm * kLsN;
            C v;
            v.x = v.y = (T)0;
            if (m0 + mm < M && n0 + c < N) v = X1[(size_t)(m0 + mm) * N + n0 + c];
            xs[e] = v;
        }
        __syncthreads();
        const int mend = min(kLsM, M - m0);
        for (int mm = 0; mm < mend; ++mm) {
            const int m = m0 + mm, iy = m / nx, ix = m - iy * nx;
            C pa, pb;
            pa.x = pxa[ix].x * pya[iy].x - pxa[ix].y * pya[iy].y;
            pa.y = pxa[ix].x * pya[iy].y + pxa[ix].y * pya[iy].x;
            pb.x = pxb[ix].x * pyb[iy].x - pxb[ix].y * pyb[iy].y;
            pb.y = pxb[ix].x * pyb[iy].y + pxb[ix].y * pyb[iy].x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const C x = xs[mm * kLsN + tn + 16 * c];
                acc[0][c].x += pa.x * x.x - pa.y * x.y;
                acc[0][c].y += pa.x * x.y + pa.y * x.x;
                acc[1][c].x += pb.x * x.x - pb.y * x.y;
                acc[1][c].y += pb.x * x.y + pb.y * x.x;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int d = d0 + 2 * td + i;
        if (d >= nd) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = n0 + tn + 16 * c;
            if (n < N) S[(size_t)d * N + n] = acc[i][c];
        }
    }
}

// F[r][d] = -(jk/4pi) [N_perp - rhat x L_M] of the column sums S[d][r K + e]
template <typename C>
__global__ void far_field_kernel(const C* __restrict__ S, const double2* __restrict__ Rv,
                                 const double* __restrict__ rhat, int D, int E, int R, double k,
                                 double2* __restrict__ F, double* __restrict__ rcs, int ndir_all) {
    const size_t total = (size_t)R * D;
    const int K = 2 * E;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int d = (int)(x % D), r = (int)(x / D);
        const double* rh = rhat + 3 * d;
        const C* s = S + (size_t)d * R * K + (size_t)r * K;
        const double2* rv = Rv + (size_t)d * E * 3;
        double2 N[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        double2 L[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        for (int e = 0; e < E; ++e) {
            const double2 sj = make_double2((double)s[e].x, (double)s[e].y);
            const double2 sm = make_double2((double)s[E + e].x, (double)s[E + e].y);
            for (int c = 0; c < 3; ++c) {
                cfma(N[c], sj, rv[3 * e + c]);
                cfma(L[c], sm, rv[3 * e + c]);
            }
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
        double2* f = F + ((size_t)r * ndir_all + d) * 3;
        for (int c = 0; c < 3; ++c) {
            // -(jk / 4pi) v
            const double2 fc = make_double2(k * v[c].y / kFourPi, -k * v[c].x / kFourPi);
            f[c] = fc;
            mag += fc.x * fc.x + fc.y * fc.y;
        }
        if (rcs) rcs[(size_t)r * ndir_all + d] = kFourPi * mag;
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

template <typename T, typename C>
int far_field_run(emsurf_handle* h, const std::vector<RwgQuad>& q, double a, double b, double k,
                  const emsurf_c128* Y, int nrhs, int ndir, const double* rhat, emsurf_c128* F, double* rcs,
                  cudaStream_t st) {
    const int E = h->E, K = h->K, M = h->M, N = nrhs * K;
    // directions in chunks so the per-chunk arrays stay under ~512 MB
    const size_t per_dir = (size_t)E * 3 * sizeof(double2) + (size_t)N * sizeof(C);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(ndir, (512ull << 20) / per_dir));
    Scoped sc;
    RwgQuad* dq;
    double* dr;
    double2* Rv;
    C *S, *X1;
    EMS_TRY(to_device(&dq, q.data(), q.size(), st));
    sc.p.push_back(dq);
    EMS_TRY(to_device(&dr, rhat, 3 * (size_t)ndir, st));
    sc.p.push_back(dr);
    EMS_CUDA(cudaMalloc(&Rv, sizeof(double2) * (size_t)chunk * E * 3));
    sc.p.push_back(Rv);
    EMS_CUDA(cudaMalloc(&S, sizeof(C) * (size_t)chunk * N));
    sc.p.push_back(S);
    EMS_CUDA(cudaMalloc(&X1, sizeof(C) * (size_t)M * N));
    sc.p.push_back(X1);
    gather_cells_kernel<C><<<(int)std::min<size_t>(((size_t)M * N + 255) / 256, 152 * 32), 256, 0, st>>>(
        reinterpret_cast<const double2*>(Y), h->d_uo_index, h->d_uo_sign, M, K, nrhs, h->n_unique, X1);
    EMS_CUDA(cudaGetLastError());
    const size_t lsm = ((size_t)kLsD * (h->nx + h->ny) + (size_t)kLsM * kLsN) * sizeof(C);
    if (lsm > 227 * 1024) {
        set_error("emsurf_far_field: lattice %d x %d too large for the phase tables", h->nx, h->ny);
        return EMSURF_EINVAL;
    }
    EMS_TRY(set_smem_once(lattice_sum_tiled_kernel<T, C>, lsm));
    double2* Fo = reinterpret_cast<double2*>(F);
    for (int d0 = 0; d0 < ndir; d0 += chunk) {
        const int nd = std::min(chunk, ndir - d0);
        const size_t t1 = (size_t)nd * E;
        radiation_kernel<<<(int)std::min<size_t>((t1 + 127) / 128, 152 * 32), 128, 0, st>>>(
            dq, E, dr + 3 * (size_t)d0, nd, k, Rv);
        EMS_CUDA(cudaGetLastError());
        const dim3 g2((unsigned)((N + kLsN - 1) / kLsN), (unsigned)((nd + kLsD - 1) / kLsD));
        lattice_sum_tiled_kernel<T, C><<<g2, kLsThreads, lsm, st>>>(X1, M, N, h->nx, h->ny, a, b,
                                                                     dr + 3 * (size_t)d0, nd, k, S);
        EMS_CUDA(cudaGetLastError());
        const size_t t3 = (size_t)nrhs * nd;
        far_field_kernel<C><<<(int)std::min<size_t>((t3 + 127) / 128, 152 * 32), 128, 0, st>>>(
            S, Rv, dr + 3 * (size_t)d0, nd, E, nrhs, k, Fo + (size_t)d0 * 3, rcs ? rcs + d0 : nullptr, ndir);
        EMS_CUDA(cudaGetLastError());
    }
    EMS_CUDA(cudaStreamSynchronize(st));
    return EMSURF_OK;
}

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
    if (h->precision == EMSURF_FP64) return far_field_run<double, double2>(h, q, a, b, k, Y, nrhs, ndir, rhat, F, rcs, st);
    return far_field_run<float, float2>(h, q, a, b, k, Y, nrhs, ndir, rhat, F, rcs, st);
}

}  // extern "C"
