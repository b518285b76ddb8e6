// Restarted GMRES on the device for Eq. final (Sec. IV-A).
//
// The paper solves Eq. final with GMRES (PETSc); restart length, initial
// guess and orthogonalisation are not given.  Here: zero initial guess,
// GMRES(m) with classical Gram-Schmidt and a second pass when the DGKS test
// asks for it (Daniel, Gragg, Kaufman, Stewart 1976: ||w'|| < eta ||w||, here
// eta = 1/sqrt(10); PETSc's GMRES, which the paper uses, refines never by
// default), Givens rotations and the upper-triangular solve on the device,
// all FP64.  H[j+1][j] comes from the same sums: ||w - V h||^2 = ||w||^2 -
// ||h||^2 for orthonormal V, which the test bounds below by ||w||^2 / 10 when
// no second pass is taken, so its relative error is at most ~10 times that
// of the sums (after a second pass the identity is applied to w' and h2).
// Right-hand sides are independent systems that share every operator
// application.
//
// With the near-field preconditioner M (Sec. IV-A applies it on the right)
// the Arnoldi process runs on A M^{-1} in its flexible form (Saad 1993):
// Z_j = M^{-1} V_j is kept and the update is x += Z y, so the FP32
// factorisation inside M^{-1} does not limit the accuracy of x.
//
// MIXED precision: iterative refinement with FP64 residuals
//   r = b - A64 x;  solve A32 d = r with FP32-operator GMRES to inner_rtol;
//   x += d;  until ||r|| / ||b|| <= rtol.
// The inner GMRES keeps its Krylov vectors in FP32 and forms products and
// updates in FP32 (FP64 arithmetic is ~60x slower on this part); sums across
// lanes and blocks, the Hessenberg matrix, the rotations and the least
// squares stay FP64.  The vector kernels are templates over the vector type
// VT (double2 for the FP64 solver, float2 for the inner solve).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace emsurf {

namespace {

constexpr int kRedBlocks = 152;     // one per SM of GB300
constexpr int kRedThreads = 256;
constexpr double kDgks = 0.1;       // second pass when ||w'||^2 < kDgks ||w||^2
constexpr int kArnThreads = 1024;   // 32 warps: one per Krylov vector in the dot phase
constexpr int kArnChunkMax = 4096;  // vector elements per block (64 KB of shared w)

struct Gm {
    std::chrono::steady_clock::time_point deadline{};   // wall-time limit of the current solve
    bool has_deadline = false;
    int m = 0, R = 0;
    size_t n = 0;
    double2* V = nullptr;      // [(m+1)][R][n]
    double2* Z = nullptr;      // [m][R][n] preconditioned directions (with M)
    // FP32 Krylov state of the inner solve of MIXED
    float2* V32 = nullptr;     // [(m+1)][R][n]
    float2* Z32 = nullptr;     // [m][R][n] (with M)
    float2* w32 = nullptr;     // [R][n]
    float2* r032 = nullptr;    // [R][n]
    float2* d32 = nullptr;     // [R][n] right-hand side of the inner solve
    float2* c32 = nullptr;     // [R][n] its solution
    double2* w = nullptr;      // [R][n]
    double2* r0 = nullptr;     // [R][n]
    double2* d = nullptr;      // [R][n] FP64 residual of the refinement (mixed)
    double2* c = nullptr;      // [R][n] correction of the refinement (mixed)
    double2* H = nullptr;      // [R][m][m+1]  column j at H[r][j][0..j+1]
    double2* cs = nullptr;     // [R][m]
    double2* sn = nullptr;     // [R][m]
    double2* g = nullptr;      // [R][m+1]
    double2* hv = nullptr;     // [R][m+1] projections of one CGS pass
    double2* hv2 = nullptr;    // [R][m+1] projections of the second CGS pass
    int nblk = 0, chunk = 0;       // Arnoldi blocks and elements per block
    int* reorth = nullptr;         // [R] second Gram-Schmidt pass needed (DGKS test)
    double2* part = nullptr;   // [R][m+1][max(nblk, kRedBlocks)] block partials
    double2* part2 = nullptr;  // [R][m+1][nblk] partials of the second Gram-Schmidt pass
    double* nrm = nullptr;     // [R]
    double* bnorm = nullptr;   // [R]
    double* res = nullptr;     // [R] estimated relative residual
    int* active = nullptr;     // [R]
    int* jend = nullptr;       // [R]
    double* h_res = nullptr;   // pinned host mirror [R]
    int* h_act = nullptr;      // pinned host mirror [R]
    int* h_ring = nullptr;     // pinned [2][R] convergence flags of the last two steps
    cudaEvent_t ev[2] = {nullptr, nullptr};   // their copies done
    int64_t launches = 0;      // kernels launched by the solver itself
    // single-rhs cooperative Arnoldi step ([0] FP32, [1] FP64 vectors): blocks
    // (chunks + the bookkeeping block, all resident) and elements per chunk;
    // 0 blocks = not available (the three-kernel step is used)
    int coop_blocks[2] = {0, 0};
    int coop_chunk[2] = {0, 0};
};

template <typename VT> struct VScalar;
template <> struct VScalar<double2> { using T = double; };
template <> struct VScalar<float2> { using T = float; };

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
template <typename VT> __device__ __forceinline__ VT from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}

template <typename VT>
__device__ __forceinline__ VT conj_mul(VT a, VT b) {   // conj(a) * b
    VT r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// part[r][i][blk] = sum over this block's slice of conj(V_i[r]) . w[r]
template <typename VT>
__global__ void dot_partial_kernel(const VT* __restrict__ V, int nvec, size_t vstride,
                                   const VT* __restrict__ w, size_t n, int R,
                                   double2* __restrict__ part, int ldv) {
    __shared__ double2 red[kRedThreads / 32];
    const int i = blockIdx.y, r = blockIdx.z;
    const VT* a = V + (size_t)i * vstride + (size_t)r * n;
    const VT* b = w + (size_t)r * n;
    VT accv;
    accv.x = 0;
    accv.y = 0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x) {
        const VT p = conj_mul(a[e], b[e]);
        accv.x += p.x;
        accv.y += p.y;
    }
    double2 acc = warp_sum(to_d2(accv));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double2 v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : make_double2(0.0, 0.0);
        v = warp_sum(v);
        if (threadIdx.x == 0) part[((size_t)r * ldv + i) * gridDim.x + blockIdx.x] = v;
    }
    (void)nvec;
}

// hv[r][i] = sum_blk part[r][i][blk]; mode 0: H col = hv, 1: H col += hv,
// 2: nrm[r] = sqrt(Re hv[r][0])
__global__ void dot_final_kernel(const double2* __restrict__ part, int nblk, int nvec, int ldv,
                                 double2* __restrict__ hv, double2* __restrict__ H, int m, int j,
                                 double* __restrict__ nrm, int mode) {
    const int i = blockIdx.x, r = blockIdx.y;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblk; b += 32) {
        const double2 v = part[((size_t)r * ldv + i) * nblk + b];
        acc.x += v.x;
        acc.y += v.y;
    }
    acc = warp_sum(acc);
    if (threadIdx.x == 0) {
        hv[(size_t)r * ldv + i] = acc;
        double2* col = H + ((size_t)r * m + j) * (m + 1);
        if (mode == 0) col[i] = acc;
        else if (mode == 1) col[i] = make_double2(col[i].x + acc.x, col[i].y + acc.y);
        else nrm[r] = sqrt(fmax(acc.x, 0.0));
    }
    (void)nvec;
}

// dst[r] = src[r] / nrm[r] (0 if nrm == 0); optionally H[j+1][j] = nrm
template <typename VT>
__global__ void normalize_kernel(VT* __restrict__ dst, const VT* __restrict__ src,
                                 const double* __restrict__ nrm, size_t n, int R,
                                 double2* __restrict__ H, int m, int j) {
    using S = typename VScalar<VT>::T;
    __shared__ S sinv[64];
    for (int r = threadIdx.x; r < R; r += blockDim.x) sinv[r] = (S)(nrm[r] > 0.0 ? 1.0 / nrm[r] : 0.0);
    __syncthreads();
    const size_t total = (size_t)R * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const S s = sinv[(int)(e / n)];
        const VT v = src[e];
        VT o;
        o.x = v.x * s;
        o.y = v.y * s;
        dst[e] = o;
    }
    if (H != nullptr && blockIdx.x == 0 && threadIdx.x < R) {
        const int r = threadIdx.x;
        H[((size_t)r * m + j) * (m + 1) + j + 1] = make_double2(nrm[r], 0.0);
    }
}

// r0 = b - w
template <typename VT>
__global__ void residual_kernel(VT* __restrict__ r0, const VT* __restrict__ b,
                                const VT* __restrict__ w, size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        VT o;
        o.x = b[e].x - w[e].x;
        o.y = b[e].y - w[e].y;
        r0[e] = o;
    }
}

// o = (float) i
__global__ void to_f32_kernel(float2* __restrict__ o, const double2* __restrict__ i, size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        o[e] = make_float2((float)i[e].x, (float)i[e].y);
}

// ---------------------------------------------------------------- fused step
// w -= sum_i c_i V_i on one element (c from shared memory), 16 (FP32) or 8
// (FP64) loads in flight
template <typename VT>
__device__ __forceinline__ VT update_one(const VT* __restrict__ V, int nvec, size_t vstride,
                                         size_t off, VT acc, const VT* __restrict__ cs) {
    constexpr int G = sizeof(VT) == sizeof(float2) ? 16 : 8;   // loads in flight
    for (int i0 = 0; i0 < nvec; i0 += G) {
        VT v[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            if (i0 + c < nvec) {
                v[c] = V[(size_t)(i0 + c) * vstride + off];
            } else {
                v[c].x = 0;
                v[c].y = 0;
            }
        }
#pragma unroll
        for (int c = 0; c < G; ++c) {
            if (i0 + c < nvec) {
                const VT q = cs[i0 + c];
                acc.x -= q.x * v[c].x - q.y * v[c].y;
                acc.y -= q.x * v[c].y + q.y * v[c].x;
            }
        }
    }
    return acc;
}

__device__ void givens_update(int r, double2* __restrict__ col, double2* __restrict__ c,
                              double2* __restrict__ s, double2* __restrict__ gg,
                              const double* __restrict__ bnorm, double* __restrict__ res,
                              int* __restrict__ active, int* __restrict__ jend, int m, int j,
                              double rtol);

// State of one Arnoldi step shared by its kernels.
struct ArnStep {
    double2* H;            // [R][m][m+1]
    double2* cs;           // [R][m]
    double2* sn;           // [R][m]
    double2* g;            // [R][m+1]
    const double* bnorm;   // [R]
    double* res;           // [R]
    int* active;           // [R]
    int* jend;             // [R]
    double* nrm;           // [R] H[j+1][j] of the step
    int* reorth;           // [R] second Gram-Schmidt pass taken
    double2* part1;        // [R][ldv][nch] chunk partials of the first pass
    double2* part2;        // [R][ldv][nch] chunk partials of the second pass
    int m, j, ldv, nch;
    double rtol;
};

// H[j+1][j] = nu and the Givens update of column j (column, rotations and g
// staged in shared memory; one thread rotates).  Whole block.
__device__ void finish_column(const ArnStep& a, int r, double nu) {
    __shared__ double2 scol[66], sc[65], ssn[65], sg[66];
    const int j = a.j, m = a.m;
    double2* col = a.H + ((size_t)r * m + j) * (m + 1);
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) scol[i] = col[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        sc[i] = a.cs[(size_t)r * m + i];
        ssn[i] = a.sn[(size_t)r * m + i];
    }
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) sg[i] = a.g[(size_t)r * (m + 1) + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        a.nrm[r] = nu;
        scol[j + 1] = make_double2(nu, 0.0);
        givens_update(r, scol, sc, ssn, sg, a.bnorm, a.res, a.active, a.jend, m, j, a.rtol);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) {
        col[i] = scol[i];
        a.g[(size_t)r * (m + 1) + i] = sg[i];
    }
    if (threadIdx.x == 0) {
        a.cs[(size_t)r * m + j] = sc[j];
        a.sn[(size_t)r * m + j] = ssn[j];
    }
}

// Dot products of the staged chunk ws with V_0..V_{nvec-1} and with itself
// (value nvec): one warp per vector, eight independent loads per lane in
// flight, lane sums in VT's precision (fixed order), the warp sum in FP64,
// chunk partials to part[r][i][c].
template <typename VT>
__device__ __forceinline__ void chunk_dots(const VT* __restrict__ V, int nvec, size_t vstride, const VT* ws,
                                           int ne, size_t off, double2* part, int ldv, int nch, int r, int c) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i <= nvec; i += nw) {
        const VT* a = i < nvec ? V + (size_t)i * vstride + off : ws;
        VT accv;
        accv.x = 0;
        accv.y = 0;
        for (int q0 = 0; q0 < ne; q0 += 256) {
            VT av[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + 32 * u + lane;
                if (q < ne) {
                    av[u] = a[q];
                } else {
                    av[u].x = 0;
                    av[u].y = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + 32 * u + lane;
                if (q < ne) {
                    const VT p = conj_mul(av[u], ws[q]);
                    accv.x += p.x;
                    accv.y += p.y;
                }
            }
        }
        const double2 acc = warp_sum(to_d2(accv));
        if (lane == 0) part[((size_t)r * ldv + i) * nch + c] = acc;
    }
}

// sh[i] = sum over chunks of part[r][i][.] for i < nv (fixed order, so every
// block that calls this gets bit-identical values), then sh[nv] holds nothing
// new; returns sum_{i < nv - 1} |sh[i]|^2 in every thread.
__device__ __forceinline__ double reduce_partials(const double2* __restrict__ part, int nv, int nch, int ldv,
                                                  int r, double2* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < nv; i += nw) {
        const double2* p = part + ((size_t)r * ldv + i) * nch;
        double2 acc = make_double2(0.0, 0.0);
        for (int b0 = 0; b0 < nch; b0 += 256) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = b0 + 32 * u + lane;
                v[u] = b < nch ? __ldcg(p + b) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                acc.x += v[u].x;
                acc.y += v[u].y;
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) sh[i] = acc;
    }
    __syncthreads();
    __shared__ double hh;
    if (wid == 0) {
        double t = 0.0;
        for (int i = lane; i < nv - 1; i += 32) t += sh[i].x * sh[i].x + sh[i].y * sh[i].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) hh = t;
    }
    __syncthreads();
    return hh;
}

// First classical Gram-Schmidt pass of Arnoldi step j (nvec = j + 1): each
// block owns chunk c of the vector, stages it in shared memory and writes its
// partials of h = V^H w and of ||w||^2.
template <typename VT>
__global__ void __launch_bounds__(kArnThreads)
arn_dots_kernel(const VT* __restrict__ V, size_t vstride, const VT* __restrict__ w, size_t n, int chunk,
                ArnStep a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* ws = reinterpret_cast<VT*>(smem_raw);   // [chunk]
    const int r = blockIdx.y, c = blockIdx.x, nvec = a.j + 1;
    const size_t e0 = (size_t)c * chunk;
    const int ne = (int)(e0 < n ? min((size_t)chunk, n - e0) : 0);
    const VT* wr = w + (size_t)r * n + e0;
    for (int q = threadIdx.x; q < ne; q += blockDim.x) ws[q] = wr[q];
    __syncthreads();
    chunk_dots(V, nvec, vstride, ws, ne, (size_t)r * n + e0, a.part1, a.ldv, a.nch, r, c);
}

// Second kernel of step j (grid nch + 1).  Every block sums the first pass's
// partials (identically) and takes the DGKS decision: with ||w - V h||^2 =
// ||w||^2 - ||h||^2 >= ||w||^2 / 2 no second pass is needed and that
// difference is H[j+1][j] = nu, so chunk blocks write V_{j+1} = (w - V h) / nu.
// Otherwise they store w' = w - V h and the partials of h2 = V^H w' and
// ||w'||^2.  Block 0 writes column j of H (and, without a second pass,
// H[j+1][j] and the Givens update).
template <typename VT>
__global__ void __launch_bounds__(kArnThreads)
arn_update_kernel(const VT* __restrict__ V, size_t vstride, VT* __restrict__ w, VT* __restrict__ vnext,
                  size_t n, int chunk, ArnStep a) {
    using S = typename VScalar<VT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* ws = reinterpret_cast<VT*>(smem_raw);   // [chunk]
    __shared__ double2 sh[66];
    __shared__ VT cs[65];
    const int r = blockIdx.y, nvec = a.j + 1;
    const double hh = reduce_partials(a.part1, nvec + 1, a.nch, a.ldv, r, sh);
    const double ww = sh[nvec].x;
    const bool second = ww - hh < kDgks * ww;
    const double nu = sqrt(fmax(ww - hh, 0.0));
    if (blockIdx.x == 0) {
        double2* col = a.H + ((size_t)r * a.m + a.j) * (a.m + 1);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) col[i] = sh[i];
        if (threadIdx.x == 0) a.reorth[r] = second ? 1 : 0;
        if (!second) finish_column(a, r, nu);
        return;
    }
    const int c = blockIdx.x - 1;
    const size_t e0 = (size_t)c * chunk;
    const int ne = (int)(e0 < n ? min((size_t)chunk, n - e0) : 0);
    const size_t off = (size_t)r * n + e0;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = from_d2<VT>(sh[i]);
    __syncthreads();
    if (!second) {
        const S sinv = (S)(nu > 0.0 ? 1.0 / nu : 0.0);
        for (int q = threadIdx.x; q < ne; q += blockDim.x) {
            VT v = update_one(V, nvec, vstride, off + q, w[off + q], cs);
            v.x *= sinv;
            v.y *= sinv;
            vnext[off + q] = v;
        }
        return;
    }
    for (int q = threadIdx.x; q < ne; q += blockDim.x) {
        const VT v = update_one(V, nvec, vstride, off + q, w[off + q], cs);
        w[off + q] = v;
        ws[q] = v;
    }
    __syncthreads();
    chunk_dots(V, nvec, vstride, ws, ne, off, a.part2, a.ldv, a.nch, r, c);
}

// Third kernel of step j, only after a second pass (grid nch + 1): every
// block sums the second pass's partials; H[j+1][j] = nu = sqrt(||w'||^2 -
// ||h2||^2); chunk blocks write V_{j+1} = (w' - V h2) / nu; block 0 adds h2
// to column j of H and does the Givens update.
template <typename VT>
__global__ void __launch_bounds__(kArnThreads)
arn_reorth_kernel(const VT* __restrict__ V, size_t vstride, const VT* __restrict__ w, VT* __restrict__ vnext,
                  size_t n, int chunk, ArnStep a) {
    using S = typename VScalar<VT>::T;
    const int r = blockIdx.y, nvec = a.j + 1;
    if (!a.reorth[r]) return;
    __shared__ double2 sh[66];
    __shared__ VT cs[65];
    const double hh = reduce_partials(a.part2, nvec + 1, a.nch, a.ldv, r, sh);
    const double nu = sqrt(fmax(sh[nvec].x - hh, 0.0));
    if (blockIdx.x == 0) {
        double2* col = a.H + ((size_t)r * a.m + a.j) * (a.m + 1);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) col[i] = make_double2(col[i].x + sh[i].x, col[i].y + sh[i].y);
        finish_column(a, r, nu);
        return;
    }
    const int c = blockIdx.x - 1;
    const size_t e0 = (size_t)c * chunk;
    const int ne = (int)(e0 < n ? min((size_t)chunk, n - e0) : 0);
    const size_t off = (size_t)r * n + e0;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = from_d2<VT>(sh[i]);
    __syncthreads();
    const S sinv = (S)(nu > 0.0 ? 1.0 / nu : 0.0);
    for (int q = threadIdx.x; q < ne; q += blockDim.x) {
        VT v = update_one(V, nvec, vstride, off + q, w[off + q], cs);
        v.x *= sinv;
        v.y *= sinv;
        vnext[off + q] = v;
    }
}

// ---------------------------------------------------------------- one-launch step
// Grid barrier of a cooperative launch (all blocks co-resident): arrival
// count bar[0], generation bar[1].  Thread 0 arrives; the last arrival resets
// the count and advances the generation, the others poll it (bounded: on
// expiry *err = 4 and false is returned, and the caller's block leaves).
constexpr long long kBarLimit = 1LL << 22;

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err,
                                             long long limit = kBarLimit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
            ok = 1;
        } else {
            ok = 0;
            for (long long it = 0; it < limit; ++it) {
                if (*gen != g0) {
                    ok = 1;
                    break;
                }
                __nanosleep(64);
            }
            if (!ok) atomicExch(err, 4);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Arnoldi step j for one rhs as a single cooperative launch: blocks
// 0 .. gridDim.x - 2 own chunks of the vector, the last block keeps H and the
// Givens rotations.  Phases, separated by grid barriers: partials of h = V^H w
// and ||w||^2; every block sums them (same order, same decision) and either
// writes V_{j+1} = (w - V h) / sqrt(||w||^2 - ||h||^2) or, when the DGKS
// test asks for a second pass, stores w' = w - V h with the partials of
// h2 = V^H w' and ||w'||^2; after the second barrier V_{j+1} = (w' - V h2) /
// sqrt(||w'||^2 - ||h2||^2).  The same arithmetic as arn_dots/update/reorth.
template <typename VT>
__global__ void __launch_bounds__(kArnThreads)
arn_step_coop_kernel(const VT* __restrict__ V, size_t vstride, VT* __restrict__ w, VT* __restrict__ vnext,
                     size_t n, int chunk, ArnStep a, unsigned* __restrict__ bar, int* __restrict__ err) {
    using S = typename VScalar<VT>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* ws = reinterpret_cast<VT*>(smem_raw);   // [chunk]
    __shared__ double2 sh[66];
    __shared__ VT cs[65];
    const int nvec = a.j + 1, nch = gridDim.x - 1;
    const bool book = (int)blockIdx.x == nch;
    const int c = blockIdx.x;
    const size_t e0 = (size_t)c * chunk;
    const int ne = (!book && e0 < n) ? (int)min((size_t)chunk, n - e0) : 0;
    if (!book) {
        for (int q = threadIdx.x; q < ne; q += blockDim.x) ws[q] = w[e0 + q];
        __syncthreads();
        chunk_dots(V, nvec, vstride, ws, ne, e0, a.part1, a.ldv, nch, 0, c);
    }
    if (!grid_barrier(bar, gridDim.x, err)) return;
    const double hh = reduce_partials(a.part1, nvec + 1, nch, a.ldv, 0, sh);
    const double ww = sh[nvec].x;
    const bool second = ww - hh < kDgks * ww;
    const double nu = sqrt(fmax(ww - hh, 0.0));
    if (book) {
        double2* col = a.H + (size_t)a.j * (a.m + 1);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) col[i] = sh[i];
        if (threadIdx.x == 0) a.reorth[0] = second ? 1 : 0;
        if (!second) {
            finish_column(a, 0, nu);
            return;
        }
    } else {
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = from_d2<VT>(sh[i]);
        __syncthreads();
        if (!second) {
            const S sinv = (S)(nu > 0.0 ? 1.0 / nu : 0.0);
            for (int q = threadIdx.x; q < ne; q += blockDim.x) {
                VT v = update_one(V, nvec, vstride, e0 + q, w[e0 + q], cs);
                v.x *= sinv;
                v.y *= sinv;
                vnext[e0 + q] = v;
            }
            return;
        }
        for (int q = threadIdx.x; q < ne; q += blockDim.x) {
            const VT v = update_one(V, nvec, vstride, e0 + q, w[e0 + q], cs);
            w[e0 + q] = v;
            ws[q] = v;
        }
        __syncthreads();
        chunk_dots(V, nvec, vstride, ws, ne, e0, a.part2, a.ldv, nch, 0, c);
    }
    // a second pass (the decision is the same in every block)
    if (!grid_barrier(bar, gridDim.x, err)) return;
    const double hh2 = reduce_partials(a.part2, nvec + 1, nch, a.ldv, 0, sh);
    const double nu2 = sqrt(fmax(sh[nvec].x - hh2, 0.0));
    if (book) {
        double2* col = a.H + (size_t)a.j * (a.m + 1);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) col[i] = make_double2(col[i].x + sh[i].x, col[i].y + sh[i].y);
        finish_column(a, 0, nu2);
        return;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = from_d2<VT>(sh[i]);
    __syncthreads();
    const S sinv = (S)(nu2 > 0.0 ? 1.0 / nu2 : 0.0);
    for (int q = threadIdx.x; q < ne; q += blockDim.x) {
        VT v = update_one(V, nvec, vstride, e0 + q, w[e0 + q], cs);
        v.x *= sinv;
        v.y *= sinv;
        vnext[e0 + q] = v;
    }
}

// Exercises the expiry path of grid_barrier: one block waits for a second
// block that is never launched, at most `limit` polls.
__global__ void grid_barrier_selftest_kernel(unsigned* bar, int* err, long long limit) {
    grid_barrier(bar, 2u, err, limit);
}

// start of a cycle: g = [beta, 0...], res = beta/bnorm, active = res > rtol
__global__ void cycle_start_kernel(const double* __restrict__ nrm, const double* __restrict__ bnorm,
                                   double2* __restrict__ g, double* __restrict__ res,
                                   int* __restrict__ active, int* __restrict__ jend, int m, int R,
                                   double rtol) {
    const int r = threadIdx.x;
    if (r >= R) return;
    const double bn = bnorm[r] > 0.0 ? bnorm[r] : 1.0;
    res[r] = nrm[r] / bn;
    active[r] = res[r] > rtol ? 1 : 0;
    jend[r] = 0;
    for (int i = 0; i <= m; ++i) g[(size_t)r * (m + 1) + i] = make_double2(0.0, 0.0);
    g[(size_t)r * (m + 1)] = make_double2(nrm[r], 0.0);
}

// Givens update of column j of right-hand side r (if still active): col =
// column j of its Hessenberg matrix, c/s its rotations, gg its g vector.
__device__ void givens_update(int r, double2* __restrict__ col, double2* __restrict__ c,
                              double2* __restrict__ s, double2* __restrict__ gg,
                              const double* __restrict__ bnorm, double* __restrict__ res,
                              int* __restrict__ active, int* __restrict__ jend, int m, int j,
                              double rtol) {
    if (!active[r]) return;
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        // [conj(c) conj(s); -s c] [a; b]
        const double2 t = make_double2(c[i].x * a.x + c[i].y * a.y + s[i].x * b.x + s[i].y * b.y,
                                       c[i].x * a.y - c[i].y * a.x + s[i].x * b.y - s[i].y * b.x);
        col[i + 1] = make_double2(-(s[i].x * a.x - s[i].y * a.y) + (c[i].x * b.x - c[i].y * b.y),
                                  -(s[i].x * a.y + s[i].y * a.x) + (c[i].x * b.y + c[i].y * b.x));
        col[i] = t;
    }
    const double2 a = col[j], b = col[j + 1];
    const double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    double2 cj, sj;
    if (den > 0.0) {
        cj = make_double2(a.x / den, a.y / den);
        sj = make_double2(b.x / den, b.y / den);
    } else {
        cj = make_double2(1.0, 0.0);
        sj = make_double2(0.0, 0.0);
    }
    c[j] = cj;
    s[j] = sj;
    col[j] = make_double2(den, 0.0);
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = gg[j];
    gg[j + 1] = make_double2(-(sj.x * gj.x - sj.y * gj.y), -(sj.x * gj.y + sj.y * gj.x));
    gg[j] = make_double2(cj.x * gj.x + cj.y * gj.y, cj.x * gj.y - cj.y * gj.x);
    const double bn = bnorm[r] > 0.0 ? bnorm[r] : 1.0;
    res[r] = sqrt(gg[j + 1].x * gg[j + 1].x + gg[j + 1].y * gg[j + 1].y) / bn;
    jend[r] = j + 1;
    if (res[r] <= rtol || den == 0.0) active[r] = 0;
}

// y = H[0:jend,0:jend]^{-1} g[0:jend] by back substitution, column by column:
// one block per rhs stages its triangle in shared memory, then one warp runs
// k = n-1 .. 0: the lane holding g_k forms y_k = g_k / H[k][k] and
// broadcasts it, and every lane updates its g_i -= H[i][k] y_k (i < k; lanes
// hold i and i + 32), so each step is one division, one shuffle and one
// independent complex multiply-add per lane.
__global__ void trisolve_kernel(const double2* __restrict__ H, const double2* __restrict__ g,
                                double2* __restrict__ y, const int* __restrict__ jend, int m, int R) {
    __shared__ double2 sH[64 * 65 / 2];   // column k rows 0..k at k (k + 1) / 2
    const int r = blockIdx.x;
    if (r >= R) return;
    const int n = jend[r];
    const double2* Hr = H + (size_t)r * m * (m + 1);
    for (int e = threadIdx.x; e < n * (m + 1); e += blockDim.x) {
        const int k = e / (m + 1), i = e % (m + 1);
        if (i <= k) sH[k * (k + 1) / 2 + i] = Hr[e];
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double2 ga = lane < n ? g[(size_t)r * (m + 1) + lane] : make_double2(0.0, 0.0);
    double2 gb = lane + 32 < n ? g[(size_t)r * (m + 1) + lane + 32] : make_double2(0.0, 0.0);
    double2* yr = y + (size_t)r * (m + 1);
    for (int k = n - 1; k >= 0; --k) {
        const int owner = k & 31;
        double2 yk = make_double2(0.0, 0.0);
        if (lane == owner) {
            const double2 gk = k < 32 ? ga : gb;
            const double2 d = sH[k * (k + 1) / 2 + k];
            const double dd = d.x * d.x + d.y * d.y;
            if (dd > 0.0) yk = make_double2((gk.x * d.x + gk.y * d.y) / dd, (gk.y * d.x - gk.x * d.y) / dd);
            yr[k] = yk;
        }
        yk.x = __shfl_sync(0xffffffffu, yk.x, owner);
        yk.y = __shfl_sync(0xffffffffu, yk.y, owner);
        const double2* col = sH + k * (k + 1) / 2;
        if (lane < k) {
            const double2 h = col[lane];
            ga.x -= h.x * yk.x - h.y * yk.y;
            ga.y -= h.x * yk.y + h.y * yk.x;
        }
        if (lane + 32 < k) {
            const double2 h = col[lane + 32];
            gb.x -= h.x * yk.x - h.y * yk.y;
            gb.y -= h.x * yk.y + h.y * yk.x;
        }
    }
}

// x[r] += sum_{i<jend[r]} y[r][i] V_i[r]  (y staged in VT precision)
template <typename VT>
__global__ void xupdate_kernel(VT* __restrict__ x, const VT* __restrict__ V,
                               size_t vstride, const double2* __restrict__ y,
                               const int* __restrict__ jend, int m, size_t n, int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT* ys = reinterpret_cast<VT*>(smem_raw);   // [R][m+1]
    for (int q = threadIdx.x; q < R * (m + 1); q += blockDim.x) ys[q] = from_d2<VT>(y[q]);
    __syncthreads();
    const size_t total = (size_t)R * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n);
        VT acc = x[e];
        for (int i = 0; i < jend[r]; ++i) {
            const VT c = ys[(size_t)r * (m + 1) + i];
            const VT v = V[(size_t)i * vstride + e];
            acc.x += c.x * v.x - c.y * v.y;
            acc.y += c.x * v.y + c.y * v.x;
        }
        x[e] = acc;
    }
}

// x += d (x FP64, d of either precision)
template <typename VT>
__global__ void axpy_kernel(double2* __restrict__ x, const VT* __restrict__ d, size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = to_d2(d[e]);
        x[e] = make_double2(x[e].x + v.x, x[e].y + v.y);
    }
}

int blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 16));
}

int gm_alloc(emsurf_handle* h, Gm*& gm, int m, int R) {
    if (h->gm) {
        Gm* old = static_cast<Gm*>(h->gm);
        if (old->m >= m && old->R >= R) {
            gm = old;
            return EMSURF_OK;
        }
    }
    // grow: keep the largest shape seen
    Gm* g = new Gm();
    const int mm = std::max(m, h->gm ? static_cast<Gm*>(h->gm)->m : 0);
    const int RR = std::max(R, h->gm ? static_cast<Gm*>(h->gm)->R : 0);
    g->m = mm;
    g->R = RR;
    g->n = (size_t)h->n_unique;
    const size_t vec = (size_t)RR * g->n * sizeof(double2);
    EMS_TRY(dev_alloc(h, (void**)&g->V, vec * (mm + 1)));
    if (h->have_pc) EMS_TRY(dev_alloc(h, (void**)&g->Z, vec * mm));
    EMS_TRY(dev_alloc(h, (void**)&g->w, vec));
    EMS_TRY(dev_alloc(h, (void**)&g->r0, vec));
    EMS_TRY(dev_alloc(h, (void**)&g->d, vec));
    EMS_TRY(dev_alloc(h, (void**)&g->c, vec));
    if (h->have32) {
        const size_t vec32 = (size_t)RR * g->n * sizeof(float2);
        EMS_TRY(dev_alloc(h, (void**)&g->V32, vec32 * (mm + 1)));
        if (h->have_pc) EMS_TRY(dev_alloc(h, (void**)&g->Z32, vec32 * mm));
        EMS_TRY(dev_alloc(h, (void**)&g->w32, vec32));
        EMS_TRY(dev_alloc(h, (void**)&g->r032, vec32));
        EMS_TRY(dev_alloc(h, (void**)&g->d32, vec32));
        EMS_TRY(dev_alloc(h, (void**)&g->c32, vec32));
    }
    EMS_TRY(dev_alloc(h, (void**)&g->H, sizeof(double2) * RR * mm * (mm + 1)));
    EMS_TRY(dev_alloc(h, (void**)&g->cs, sizeof(double2) * RR * mm));
    EMS_TRY(dev_alloc(h, (void**)&g->sn, sizeof(double2) * RR * mm));
    EMS_TRY(dev_alloc(h, (void**)&g->g, sizeof(double2) * RR * (mm + 1)));
    EMS_TRY(dev_alloc(h, (void**)&g->hv, sizeof(double2) * RR * (mm + 1)));
    EMS_TRY(dev_alloc(h, (void**)&g->hv2, sizeof(double2) * RR * (mm + 1)));
    EMS_TRY(dev_alloc(h, (void**)&g->reorth, sizeof(int) * RR));
    g->nblk = (int)std::max<size_t>(std::max(1, h->num_sms), (g->n + kArnChunkMax - 1) / kArnChunkMax);
    g->chunk = (int)((g->n + g->nblk - 1) / g->nblk);
    EMS_TRY(dev_alloc(h, (void**)&g->part,
                      sizeof(double2) * RR * (mm + 1) * std::max<size_t>(g->nblk, kRedBlocks)));
    EMS_TRY(dev_alloc(h, (void**)&g->part2, sizeof(double2) * RR * (mm + 1) * g->nblk));
    {
        // one chunk block per SM but one, plus the bookkeeping block; used only
        // when the device runs cooperative launches and all blocks fit at once
        int coop = 0;
        EMS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
        const int blocks = std::max(2, h->num_sms);
        const size_t chunk = (g->n + blocks - 2) / (blocks - 1);
        for (int t = 0; t < 2 && coop; ++t) {
            const size_t wsm = chunk * (t ? sizeof(double2) : sizeof(float2));
            if (wsm > 200 * 1024) continue;
            int occ = 0;
            if (t) {
                EMS_TRY(set_smem_once(arn_step_coop_kernel<double2>, wsm));
                EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, arn_step_coop_kernel<double2>,
                                                                       kArnThreads, wsm));
            } else {
                EMS_TRY(set_smem_once(arn_step_coop_kernel<float2>, wsm));
                EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, arn_step_coop_kernel<float2>,
                                                                       kArnThreads, wsm));
            }
            if (occ * h->num_sms >= blocks) {
                g->coop_blocks[t] = blocks;
                g->coop_chunk[t] = (int)chunk;
            }
        }
    }
    EMS_TRY(dev_alloc(h, (void**)&g->nrm, sizeof(double) * RR));
    EMS_TRY(dev_alloc(h, (void**)&g->bnorm, sizeof(double) * RR));
    EMS_TRY(dev_alloc(h, (void**)&g->res, sizeof(double) * RR));
    EMS_TRY(dev_alloc(h, (void**)&g->active, sizeof(int) * RR));
    EMS_TRY(dev_alloc(h, (void**)&g->jend, sizeof(int) * RR));
    EMS_CUDA(cudaMallocHost(&g->h_res, sizeof(double) * RR));
    EMS_CUDA(cudaMallocHost(&g->h_act, sizeof(int) * RR));
    EMS_CUDA(cudaMallocHost(&g->h_ring, 2 * sizeof(int) * RR));
    for (int i = 0; i < 2; ++i) EMS_CUDA(cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming));
    if (h->gm) {
        Gm* old = static_cast<Gm*>(h->gm);
        cudaFreeHost(old->h_res);
        cudaFreeHost(old->h_act);
        cudaFreeHost(old->h_ring);
        for (int i = 0; i < 2; ++i) cudaEventDestroy(old->ev[i]);
        delete old;   // device buffers stay in h->allocations until destroy
    }
    h->gm = g;
    gm = g;
    return EMSURF_OK;
}

// nrm[r] = ||v[r]||
template <typename VT>
int norms(Gm* g, const VT* v, int R, cudaStream_t st) {
    dim3 grid(kRedBlocks, 1, R);
    dot_partial_kernel<VT><<<grid, kRedThreads, 0, st>>>(v, 1, 0, v, g->n, R, g->part, g->m + 1);
    EMS_CUDA(cudaGetLastError());
    ++g->launches;
    dot_final_kernel<<<dim3(1, R), 32, 0, st>>>(g->part, kRedBlocks, 1, g->m + 1, g->hv, g->H,
                                                g->m, 0, g->nrm, 2);
    EMS_CUDA(cudaGetLastError());
    ++g->launches;
    return EMSURF_OK;
}

// The operator and the preconditioner on vectors of type VT: FP64 vectors
// take the FP64 or the FP32 operator, FP32 vectors the FP32 one.
template <typename VT>
struct Apply {
    emsurf_handle* h;
    int prec;   // operator used inside GMRES (EMSURF_FP64 / EMSURF_FP32)
    int count = 0;
    int operator()(const VT* x, VT* y, int R, cudaStream_t st) {
        ++count;
        if constexpr (std::is_same<VT, float2>::value) {
            return apply_operator_f32(h, x, y, R, st);
        } else {
            if (prec == EMSURF_FP32) return apply_operator<float2>(h, h->op32, x, y, R, st);
            return apply_operator<double2>(h, h->op64, x, y, R, st);
        }
    }
    int precond(const VT* r, VT* y, int R, cudaStream_t st) {
        if constexpr (std::is_same<VT, float2>::value) return pc_apply_f32(h, r, y, R, st);
        else return pc_apply(h, r, y, R, st);
    }
};

// The Krylov buffers of one vector type.
template <typename VT>
struct Kv {
    VT *V, *Z, *w, *r0;
};
template <typename VT> Kv<VT> kv(Gm* g);
template <> Kv<double2> kv<double2>(Gm* g) { return {g->V, g->Z, g->w, g->r0}; }
template <> Kv<float2> kv<float2>(Gm* g) { return {g->V32, g->Z32, g->w32, g->r032}; }

bool past_deadline(const Gm* g) {
    return g->has_deadline && std::chrono::steady_clock::now() >= g->deadline;
}

// GMRES(m) from x (used as the initial guess), until every rhs reaches rtol
// or the iteration budget (or the wall-time limit, checked per restart) runs
// out.  Returns the number of Arnoldi steps.
// stop_on_stall (the inner solves of the mixed refinement): also stop once
// the worst relative residual of the active rhs has fallen by less than 1 %
// over each of kStallCycles consecutive restarts.  A perturbed operator in
// FP32 arithmetic cannot push the residual below about its own error times
// the condition number; past that level more restarts gain nothing, and the
// FP64 residual of the next refinement step is the way forward.
constexpr int kStallCycles = 3;
constexpr double kStallRatio = 0.99;

template <typename VT>
int gmres_core(emsurf_handle* h, Gm* g, Apply<VT>& A, const VT* b, VT* x, int R, int m,
               double rtol, int max_iters, bool x_is_zero, bool pc, cudaStream_t st, int* iters_out,
               bool stop_on_stall = false) {
    const size_t n = g->n, nv = (size_t)R * n;
    const size_t vstride = nv;
    const int nb = blocks_for(nv);
    const Kv<VT> K = kv<VT>(g);
    int it = 0;
    // ||b||
    EMS_TRY(norms<VT>(g, b, R, st));
    EMS_CUDA(cudaMemcpyAsync(g->bnorm, g->nrm, sizeof(double) * R, cudaMemcpyDeviceToDevice, st));
    bool first = true;
    double prev_worst = 0.0;
    int stalls = 0;
    while (true) {
        if (first && x_is_zero) {
            EMS_CUDA(cudaMemcpyAsync(K.r0, b, nv * sizeof(VT), cudaMemcpyDeviceToDevice, st));
        } else {
            EMS_TRY(A(x, K.w, R, st));
            residual_kernel<VT><<<nb, 256, 0, st>>>(K.r0, b, K.w, nv);
            EMS_CUDA(cudaGetLastError());
            ++g->launches;
        }
        first = false;
        EMS_TRY(norms<VT>(g, K.r0, R, st));
        cycle_start_kernel<<<1, 64, 0, st>>>(g->nrm, g->bnorm, g->g, g->res, g->active, g->jend,
                                              m, R, rtol);
        EMS_CUDA(cudaGetLastError());
        ++g->launches;
        normalize_kernel<VT><<<nb, 256, 0, st>>>(K.V, K.r0, g->nrm, n, R, nullptr, m, 0);
        EMS_CUDA(cudaGetLastError());
        ++g->launches;
        EMS_CUDA(cudaMemcpyAsync(g->h_act, g->active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        if (stop_on_stall) EMS_CUDA(cudaMemcpyAsync(g->h_res, g->res, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        EMS_CUDA(cudaStreamSynchronize(st));
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || g->h_act[r];
        if (!any || it >= max_iters || past_deadline(g)) break;
        if (stop_on_stall) {
            double worst = 0.0;
            for (int r = 0; r < R; ++r)
                if (g->h_act[r]) worst = std::max(worst, g->h_res[r]);
            stalls = (prev_worst > 0.0 && worst > kStallRatio * prev_worst) ? stalls + 1 : 0;
            prev_worst = worst;
            if (stalls >= kStallCycles) break;
        }
        for (int j = 0; j < m; ++j) {
            VT* Vj = K.V + (size_t)j * vstride;
            if (pc) {
                VT* Zj = K.Z + (size_t)j * vstride;
                prof_mark(h, EMS_PH_PRECOND, true, st);
                EMS_TRY(A.precond(Vj, Zj, R, st));
                prof_mark(h, EMS_PH_PRECOND, false, st);
                EMS_TRY(A(Zj, K.w, R, st));
            } else {
                EMS_TRY(A(Vj, K.w, R, st));
            }
            // classical Gram-Schmidt with the DGKS second pass, H[j+1][j] and
            // the Givens update: one cooperative launch for a single rhs (all
            // blocks resident), else 2 kernels and a third after a second pass
            const ArnStep as{g->H, g->cs, g->sn, g->g, g->bnorm, g->res, g->active, g->jend, g->nrm,
                             g->reorth, g->part, g->part2, m, j, m + 1, g->nblk, rtol};
            VT* vnext = K.V + (size_t)(j + 1) * vstride;
            prof_mark(h, EMS_PH_ARNOLDI, true, st);
            constexpr int ti = sizeof(VT) == sizeof(double2) ? 1 : 0;
            if (R == 1 && h->coop_ok && g->coop_blocks[ti] > 0) {
                ArnStep ac = as;
                ac.nch = g->coop_blocks[ti] - 1;
                const VT* Vc = K.V;
                VT* wc = K.w;
                size_t nn = n;
                int ch = g->coop_chunk[ti];
                unsigned* bar = h->d_grid_bar;
                int* err = h->d_err;
                void* args[] = {(void*)&Vc, (void*)&vstride, (void*)&wc, (void*)&vnext, (void*)&nn, (void*)&ch,
                                (void*)&ac, (void*)&bar, (void*)&err};
                EMS_CUDA(cudaLaunchCooperativeKernel((const void*)arn_step_coop_kernel<VT>, dim3(g->coop_blocks[ti], 1),
                                                     dim3(kArnThreads), args, (size_t)ch * sizeof(VT), st));
                g->launches += 1;
            } else {
                const size_t wsm = (size_t)g->chunk * sizeof(VT);
                EMS_TRY(set_smem_once(arn_dots_kernel<VT>, wsm));
                EMS_TRY(set_smem_once(arn_update_kernel<VT>, wsm));
                arn_dots_kernel<VT><<<dim3(g->nblk, R), kArnThreads, wsm, st>>>(K.V, vstride, K.w, n, g->chunk, as);
                EMS_CUDA(cudaGetLastError());
                arn_update_kernel<VT><<<dim3(g->nblk + 1, R), kArnThreads, wsm, st>>>(K.V, vstride, K.w, vnext, n,
                                                                                     g->chunk, as);
                EMS_CUDA(cudaGetLastError());
                arn_reorth_kernel<VT><<<dim3(g->nblk + 1, R), kArnThreads, 0, st>>>(K.V, vstride, K.w, vnext, n,
                                                                                   g->chunk, as);
                EMS_CUDA(cudaGetLastError());
                g->launches += 3;
            }
            prof_mark(h, EMS_PH_ARNOLDI, false, st);
            ++it;
            // the convergence flags of step j are copied to pinned memory behind
            // its kernels; the host reads those of step j - 1 while step j runs,
            // so the GPU does not wait for the host and at most one step is
            // computed after every rhs converged (such a step leaves the
            // solution untouched: the update uses the steps before jend)
            int* hr = g->h_ring + (size_t)(j & 1) * R;
            EMS_CUDA(cudaMemcpyAsync(hr, g->active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
            EMS_CUDA(cudaEventRecord(g->ev[j & 1], st));
            if (it >= max_iters) break;
            if (j >= 1) {
                EMS_CUDA(cudaEventSynchronize(g->ev[(j - 1) & 1]));
                const int* hp = g->h_ring + (size_t)((j - 1) & 1) * R;
                bool act = false;
                for (int r = 0; r < R; ++r) act = act || hp[r];
                if (!act) break;
            }
        }
        trisolve_kernel<<<R, 256, 0, st>>>(g->H, g->g, g->hv, g->jend, m, R);
        EMS_CUDA(cudaGetLastError());
        ++g->launches;
        xupdate_kernel<VT><<<nb, 256, (size_t)R * (m + 1) * sizeof(VT), st>>>(
            x, pc ? K.Z : K.V, vstride, g->hv, g->jend, m, n, R);
        EMS_CUDA(cudaGetLastError());
        ++g->launches;
    }
    *iters_out = it;
    return EMSURF_OK;
}

// true relative residual per rhs with the given FP64-vector operator, into host res[]
int true_residual(emsurf_handle* h, Gm* g, Apply<double2>& A, const double2* b, const double2* x, int R,
                  cudaStream_t st, double* res) {
    const size_t nv = (size_t)R * g->n;
    EMS_TRY(A(x, g->w, R, st));
    residual_kernel<double2><<<blocks_for(nv), 256, 0, st>>>(g->r0, b, g->w, nv);
    EMS_CUDA(cudaGetLastError());
    ++g->launches;
    EMS_TRY(norms<double2>(g, g->r0, R, st));
    std::vector<double> rn(R), bn(R);
    EMS_CUDA(cudaMemcpyAsync(rn.data(), g->nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    EMS_TRY(norms<double2>(g, b, R, st));
    EMS_CUDA(cudaMemcpyAsync(bn.data(), g->nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    EMS_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) res[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
    return EMSURF_OK;
}

}  // namespace

int grid_barrier_selftest(emsurf_handle* h, long long limit, cudaStream_t st) {
    grid_barrier_selftest_kernel<<<1, 32, 0, st>>>(h->d_grid_bar, h->d_err, limit);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}

int gmres_solve(emsurf_handle* h, const double2* b, double2* x, int R, const emsurf_solve_opts* o,
                emsurf_solve_info* info, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const int m = o->restart;
    Gm* g = nullptr;
    EMS_TRY(gm_alloc(h, g, m, R));
    g->has_deadline = o->max_ms > 0.0;
    if (g->has_deadline)
        g->deadline = t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                std::chrono::duration<double, std::milli>(o->max_ms));
    const size_t nv = (size_t)R * g->n;
    EMS_CUDA(cudaMemsetAsync(x, 0, nv * sizeof(double2), st));
    const int64_t launches0 = g->launches;
    int iters = 0, refines = 0, nmv = 0;
    std::vector<double> res(R, 0.0);
    Apply<double2> A64{h, EMSURF_FP64};
    Apply<double2> A32{h, EMSURF_FP32};
    Apply<float2> A32f{h, EMSURF_FP32};
    const bool pc = h->have_pc && o->precond >= 0;
    int mode = o->solver;
    if (mode == 0) mode = h->precision == EMSURF_MIXED ? 3 : (h->precision == EMSURF_FP32 ? 2 : 1);
    if (mode == 3) {
        // inner tolerance: the part of the remaining reduction that is still
        // needed (half of it), but not below what an FP32 operator can
        // resolve (~1e-7 relative; the default floor 1e-6 keeps a margin),
        // so that one inner solve usually reaches rtol and the FP64 residual
        // only confirms it
        // (the BF16x3 tensor-core operator resolves ~3e-5, the FP32 one ~1e-7)
        const double inner = o->inner_rtol > 0 ? o->inner_rtol : (h->have_tc && R >= kTcMinRhs ? 3e-5 : 1e-6);
        bool zero = true;
        while (true) {
            // FP64 residual r = b - A64 x (x = 0 on the first pass)
            if (zero) {
                EMS_CUDA(cudaMemcpyAsync(g->d, b, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
                EMS_TRY(norms<double2>(g, b, R, st));
                std::vector<double> bn(R);
                EMS_CUDA(cudaMemcpyAsync(bn.data(), g->nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
                EMS_CUDA(cudaStreamSynchronize(st));
                for (int r = 0; r < R; ++r) res[r] = bn[r] > 0 ? 1.0 : 0.0;
            } else {
                EMS_TRY(true_residual(h, g, A64, b, x, R, st, res.data()));
                EMS_CUDA(cudaMemcpyAsync(g->d, g->r0, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            }
            double worst = 0.0;
            for (int r = 0; r < R; ++r) worst = std::max(worst, res[r]);
            if (worst <= o->rtol || refines >= o->max_refine || iters >= o->max_iters || past_deadline(g)) break;
            // inner solve A32 c = d with FP32-operator GMRES on FP32 vectors
            to_f32_kernel<<<blocks_for(nv), 256, 0, st>>>(g->d32, g->d, nv);
            EMS_CUDA(cudaGetLastError());
            ++g->launches;
            EMS_CUDA(cudaMemsetAsync(g->c32, 0, nv * sizeof(float2), st));
            const double tol = std::max(inner, 0.5 * o->rtol / std::max(worst, 1e-300));
            int it = 0;
            EMS_TRY(gmres_core<float2>(h, g, A32f, g->d32, g->c32, R, m, std::min(tol, 0.5),
                                       o->max_iters - iters, true, pc, st, &it, true));
            iters += it;
            axpy_kernel<float2><<<blocks_for(nv), 256, 0, st>>>(x, g->c32, nv);
            EMS_CUDA(cudaGetLastError());
    ++g->launches;
            ++refines;
            zero = false;
        }
        nmv = A64.count + A32f.count;
    } else {
        Apply<double2>& A = (mode == 2) ? A32 : A64;
        EMS_TRY(gmres_core<double2>(h, g, A, b, x, R, m, o->rtol, o->max_iters, true, pc, st, &iters));
        EMS_TRY(true_residual(h, g, A, b, x, R, st, res.data()));
        nmv = A.count;
    }
    EMS_CUDA(cudaStreamSynchronize(st));
    h->launches += g->launches - launches0;
    {
        int flag = 0;
        EMS_CUDA(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            EMS_TRY(clear_wait_error(h));
            set_error("a bounded device wait expired during the solve");
            return EMSURF_ETIMEDOUT;
        }
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int r = 0; r < R; ++r) {
        const bool ok = res[r] <= o->rtol;
        all = all && ok;
        if (info) {
            info[r].iters = iters;
            info[r].refinements = refines;
            info[r].n_matvec = nmv;
            info[r].converged = ok ? 1 : 0;
            info[r].rel_residual = res[r];
            info[r].ms_total = ms;
        }
    }
    return all ? EMSURF_OK : EMSURF_ENOTCONV;
}

}  // namespace emsurf

namespace emsurf {

void gmres_release(emsurf_handle* h) {
    if (!h->gm) return;
    Gm* g = static_cast<Gm*>(h->gm);
    if (g->h_res) cudaFreeHost(g->h_res);
    if (g->h_act) cudaFreeHost(g->h_act);
    if (g->h_ring) cudaFreeHost(g->h_ring);
    for (int i = 0; i < 2; ++i)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    delete g;   // device buffers are released with the handle's allocations
    h->gm = nullptr;
}

}  // namespace emsurf
