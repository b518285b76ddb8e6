// Per-type macromodels on the GPU (Sec. II-B..D, Eq. Zmacromodel).
//
// A cell is a free-space box S_eq holding a flat PEC patch (J only on PEC,
// Sec. II-A).  With the scaled unknowns x_J = eta0 J, x_M = M the interior
// region's tested equations (Eq. ch5_macromodel_composite_SIE_Block, one
// region, so U of Eq. incidence1 is a permutation) are
//
//        [ jk L_ee   K_ee   jk L_ep ] [J_eq]      rows: EFIE on S_eq
//    Z = [ -K_ee   jk L_ee   -K_ep  ] [M_eq]            MFIE on S_eq
//        [ jk L_pe   K_pe   jk L_pp ] [J_p ]            EFIE on the patch
//
// and the macromodel is the Schur complement Z~ = Z_ee - Z_ei Z_ii^{-1} Z_ie
// (Eq. Zmacromodel), solved here with an LU factorisation with partial
// pivoting of the patch block Z_ii, one CTA per type.  A type with side <= 0
// is an empty box: Z~ = Z_ee.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace emsurf {


namespace {

constexpr int kMaxPatchRwg = 100;

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Solve Z_ii W = Z_ie for one type.  Lpp [P][P], Lpe/Kpe [P][E] (global);
// W [P][2E] (global, output).  Z_ii = jk Lpp, Z_ie = [jk Lpe | Kpe].
__global__ void patch_solve_kernel(const double2* __restrict__ Lpp, const double2* __restrict__ Lpe,
                                   const double2* __restrict__ Kpe, double2* __restrict__ W, int P,
                                   int E, double k, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* A = reinterpret_cast<double2*>(smem_raw);       // [P][P]
    int* piv = reinterpret_cast<int*>(A + P * P);             // [P]
    __shared__ int s_p;
    const int t = blockIdx.x;
    const double2* lpp = Lpp + (size_t)t * P * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x)
        A[e] = make_double2(-k * lpp[e].y, k * lpp[e].x);     // jk * Lpp
    __syncthreads();
    // LU with partial pivoting by modulus
    for (int c = 0; c < P; ++c) {
        if (threadIdx.x == 0) {
            int best = c;
            double bm = -1.0;
            for (int r = c; r < P; ++r) {
                const double m = A[r * P + c].x * A[r * P + c].x + A[r * P + c].y * A[r * P + c].y;
                if (m > bm) { bm = m; best = r; }
            }
            piv[c] = best;
            s_p = best;
            if (!(bm > 0.0)) atomicExch(status, 1);
        }
        __syncthreads();
        const int p = s_p;
        if (p != c)
            for (int j = threadIdx.x; j < P; j += blockDim.x) {
                const double2 tmp = A[c * P + j];
                A[c * P + j] = A[p * P + j];
                A[p * P + j] = tmp;
            }
        __syncthreads();
        const double2 d = A[c * P + c];
        for (int r = c + 1 + threadIdx.x; r < P; r += blockDim.x) A[r * P + c] = cdiv(A[r * P + c], d);
        __syncthreads();
        for (int e = threadIdx.x; e < (P - c - 1) * (P - c - 1); e += blockDim.x) {
            const int r = c + 1 + e / (P - c - 1), j = c + 1 + e % (P - c - 1);
            A[r * P + j] = csub(A[r * P + j], cmul(A[r * P + c], A[c * P + j]));
        }
        __syncthreads();
    }
    // columns of the right-hand side
    const int ncol = 2 * E;
    const double2* lpe = Lpe + (size_t)t * P * E;
    const double2* kpe = Kpe + (size_t)t * P * E;
    double2* w = W + (size_t)t * P * ncol;
    for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
        for (int r = 0; r < P; ++r) {
            const double2 v = col < E ? lpe[(size_t)r * E + col] : kpe[(size_t)r * E + col - E];
            w[(size_t)r * ncol + col] = col < E ? make_double2(-k * v.y, k * v.x) : v;
        }
        for (int c = 0; c < P; ++c) {          // apply row swaps in order
            const int p = piv[c];
            if (p != c) {
                const double2 tmp = w[(size_t)c * ncol + col];
                w[(size_t)c * ncol + col] = w[(size_t)p * ncol + col];
                w[(size_t)p * ncol + col] = tmp;
            }
        }
        for (int r = 1; r < P; ++r) {          // L y = b (unit lower)
            double2 acc = w[(size_t)r * ncol + col];
            for (int j = 0; j < r; ++j) acc = csub(acc, cmul(A[r * P + j], w[(size_t)j * ncol + col]));
            w[(size_t)r * ncol + col] = acc;
        }
        for (int r = P - 1; r >= 0; --r) {     // U x = y
            double2 acc = w[(size_t)r * ncol + col];
            for (int j = r + 1; j < P; ++j) acc = csub(acc, cmul(A[r * P + j], w[(size_t)j * ncol + col]));
            w[(size_t)r * ncol + col] = cdiv(acc, A[r * P + r]);
        }
    }
}

// Z~[t][r][c] = Z_ee[r][c] - sum_p Z_ei[t][r][p] W[t][p][c]
// Z_ee = [[jk Lee, Kee], [-Kee, jk Lee]]; Z_ei = [[jk Lep], [-Kep]]
__global__ void schur_kernel(const double2* __restrict__ Lee, const double2* __restrict__ Kee,
                             const double2* __restrict__ Lep, const double2* __restrict__ Kep,
                             const double2* __restrict__ W, const int8_t* __restrict__ has_patch,
                             const int* __restrict__ tidx, int T, int P, int E, double k,
                             double2* __restrict__ Z) {
    const int K = 2 * E;
    const size_t total = (size_t)T * K * K;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % K);
        const int r = (int)((e / K) % K);
        const int t = (int)(e / ((size_t)K * K));
        const int rb = r < E ? 0 : 1, cb = c < E ? 0 : 1;
        const int ri = r - rb * E, ci = c - cb * E;
        double2 z;
        if (rb == cb) {
            const double2 l = Lee[(size_t)ri * E + ci];
            z = make_double2(-k * l.y, k * l.x);
        } else {
            const double2 kv = Kee[(size_t)ri * E + ci];
            z = rb == 0 ? kv : make_double2(-kv.x, -kv.y);
        }
        if (has_patch[t]) {
            const int s = tidx[t];
            const double2* w = W + (size_t)s * P * K;
            double2 acc = make_double2(0.0, 0.0);
            if (rb == 0) {
                const double2* lep = Lep + ((size_t)s * E + ri) * P;
                for (int p = 0; p < P; ++p) cfma(acc, make_double2(-k * lep[p].y, k * lep[p].x), w[(size_t)p * K + c]);
            } else {
                const double2* kep = Kep + ((size_t)s * E + ri) * P;
                for (int p = 0; p < P; ++p) cfma(acc, make_double2(-kep[p].x, -kep[p].y), w[(size_t)p * K + c]);
            }
            z = csub(z, acc);
        }
        Z[e] = z;
    }
}

struct HostMesh {
    std::vector<double> verts;
    std::vector<int32_t> tris, edges, tp, tm, srw;
    std::vector<int8_t> ssg;
    int T = 0, E = 0;
    MeshView view() const { return {verts.data(), tris.data(), srw.data(), ssg.data(), T, E}; }
};

}  // namespace
}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API int emsurf_macromodel_pec_patch(double a, double b, double h, int32_t n,
                                           int32_t n_types, const double* sides, double patch_z,
                                           int32_t patch_n, double k, emsurf_c128* Z,
                                           void* stream) {
    if (n < 1 || n_types < 1 || !sides || patch_n < 1 || !(k > 0.0) || !Z) {
        set_error("emsurf_macromodel_pec_patch: bad arguments");
        return EMSURF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HostMesh box;
    int32_t V;
    EMS_TRY(emsurf_setup_box_counts(n, &V, &box.T, &box.E));
    box.verts.resize(3 * V);
    box.tris.resize(3 * box.T);
    box.edges.resize(2 * box.E);
    box.tp.resize(box.E);
    box.tm.resize(box.E);
    box.srw.resize(3 * box.T);
    box.ssg.resize(3 * box.T);
    EMS_TRY(emsurf_setup_box_mesh(a, b, h, n, nullptr, box.verts.data(), box.tris.data(),
                                  box.edges.data(), box.tp.data(), box.tm.data(), box.srw.data(),
                                  box.ssg.data()));
    const int E = box.E, K = 2 * E;
    int32_t PV, PT, P;
    EMS_TRY(emsurf_setup_patch_counts(patch_n, &PV, &PT, &P));
    if (P > kMaxPatchRwg) {
        set_error("patch mesh has %d RWGs; at most %d supported", P, kMaxPatchRwg);
        return EMSURF_EINVAL;
    }
    std::vector<int8_t> has(n_types);
    std::vector<int> tidx(n_types, 0);
    int npatch = 0;
    for (int t = 0; t < n_types; ++t) {
        has[t] = sides[t] > 0.0 ? 1 : 0;
        if (has[t]) tidx[t] = npatch++;
        if (has[t] && (sides[t] >= std::min(a, b) || patch_z <= 0.0 || patch_z >= h)) {
            set_error("patch %d (side %g, z %g) is not strictly inside the box", t, sides[t], patch_z);
            return EMSURF_EINVAL;
        }
    }
    const double zero3[3] = {0.0, 0.0, 0.0};
    const int8_t one = 1;
    double2 *Lee = nullptr, *Kee = nullptr, *Lep = nullptr, *Kep = nullptr, *Lpe = nullptr,
            *Kpe = nullptr, *Lpp = nullptr, *Kpp = nullptr, *W = nullptr;
    int8_t* dhas = nullptr;
    int* dtidx = nullptr;
    int* dstat = nullptr;
    int status = EMSURF_OK;
    const int np = std::max(npatch, 1);
    auto alloc = [&](void** p, size_t bytes) {
        if (status) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("emsurf_macromodel_pec_patch: device allocation of %zu bytes failed", bytes);
            status = EMSURF_ENOMEM;
        }
    };
    alloc((void**)&Lee, sizeof(double2) * E * E);
    alloc((void**)&Kee, sizeof(double2) * E * E);
    alloc((void**)&Lep, sizeof(double2) * np * E * P);
    alloc((void**)&Kep, sizeof(double2) * np * E * P);
    alloc((void**)&Lpe, sizeof(double2) * np * P * E);
    alloc((void**)&Kpe, sizeof(double2) * np * P * E);
    alloc((void**)&Lpp, sizeof(double2) * np * P * P);
    alloc((void**)&Kpp, sizeof(double2) * np * P * P);
    alloc((void**)&W, sizeof(double2) * np * P * K);
    alloc((void**)&dhas, n_types);
    alloc((void**)&dtidx, sizeof(int) * n_types);
    alloc((void**)&dstat, sizeof(int));
    if (!status) status = tabulate_blocks(box.view(), box.view(), zero3, &one, 1, k, Lee, Kee, st);
    for (int t = 0; t < n_types && !status; ++t) {
        if (!has[t]) continue;
        HostMesh pm;
        pm.T = PT;
        pm.E = P;
        pm.verts.resize(3 * PV);
        pm.tris.resize(3 * PT);
        pm.edges.resize(2 * P);
        pm.tp.resize(P);
        pm.tm.resize(P);
        pm.srw.resize(3 * PT);
        pm.ssg.resize(3 * PT);
        status = emsurf_setup_patch_mesh(sides[t], patch_z, patch_n, pm.verts.data(), pm.tris.data(),
                                         pm.edges.data(), pm.tp.data(), pm.tm.data(), pm.srw.data(),
                                         pm.ssg.data());
        const size_t s = tidx[t];
        if (!status)
            status = tabulate_blocks(box.view(), pm.view(), zero3, &one, 1, k, Lep + s * E * P,
                                     Kep + s * E * P, st);
        if (!status)
            status = tabulate_blocks(pm.view(), box.view(), zero3, &one, 1, k, Lpe + s * P * E,
                                     Kpe + s * P * E, st);
        if (!status)
            status = tabulate_blocks(pm.view(), pm.view(), zero3, &one, 1, k, Lpp + s * P * P,
                                     Kpp + s * P * P, st);
    }
    if (!status) {
        cudaMemcpyAsync(dhas, has.data(), n_types, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dtidx, tidx.data(), sizeof(int) * n_types, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(dstat, 0, sizeof(int), st);
        if (npatch > 0) {
            const size_t smem = sizeof(double2) * P * P + sizeof(int) * P;
            cudaFuncSetAttribute(patch_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            patch_solve_kernel<<<npatch, 256, smem, st>>>(Lpp, Lpe, Kpe, W, P, E, k, dstat);
        }
        const size_t tot = (size_t)n_types * K * K;
        schur_kernel<<<(int)std::min<size_t>((tot + 255) / 256, 152 * 64), 256, 0, st>>>(
            Lee, Kee, Lep, Kep, W, dhas, dtidx, n_types, P, E, k, reinterpret_cast<double2*>(Z));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("emsurf_macromodel_pec_patch: %s", cudaGetErrorString(e));
            status = EMSURF_ECUDA;
        } else {
            int hs = 0;
            cudaMemcpy(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost);
            if (hs) {
                set_error("emsurf_macromodel_pec_patch: singular patch block");
                status = EMSURF_EINVAL;
            }
        }
    }
    for (void* p : {(void*)Lee, (void*)Kee, (void*)Lep, (void*)Kep, (void*)Lpe, (void*)Kpe,
                    (void*)Lpp, (void*)Kpp, (void*)W, (void*)dhas, (void*)dtidx, (void*)dstat})
        cudaFree(p);
    return status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The configurations' cell: lossy dielectric slab under a PEC patch, air
// above (Secs. II-A..D with V = 2 interior regions).  Per type:
//   1. L_v, K_v on the closed surface of each region with k_v = k0 sqrt(eps_v)
//      (Eq. ch5_macromodel_composite_SIE_Block), tabulated on the device;
//   2. U^T Z U (Eqs. discretized_SIE, incidence1, mmm_mult) assembled by a
//      gather: every X~ unknown has at most one copy per region, so
//      M[p][q] = sum_v s_v(p) s_v(q) Z_v[c_v(p)][c_v(q)] with
//      Z_v = [[j k0 L_v, K_v], [-K_v, j k0 eps_v L_v]];
//   3. the Schur complement of Eq. Zmacromodel by Gaussian elimination of
//      the interior unknowns (ordered first), partial pivoting among the
//      interior rows only: after n_int steps the trailing 2E x 2E block is
//      Z~ = Z_ee - Z_ei Z_ii^{-1} Z_ie.  Each step reads one buffer and writes
//      the other, so the CTAs of a type need no synchronisation.
namespace emsurf {
namespace {

struct SlabType {
    long long offL[2];   // region v's L in the table buffer; its K follows at + E_v^2
    int Ev[2];
    int N, nint;
    long long offB;      // this type's N x N matrix in the elimination buffers
    long long offMap;    // this type's copy/sign arrays ([2][N])
};

__global__ void slab_assemble_kernel(const SlabType* __restrict__ ty, const double2* __restrict__ LK,
                                     const int32_t* __restrict__ cpy, const int8_t* __restrict__ sgn,
                                     double k0, double2 eps, double2* __restrict__ B) {
    const SlabType T = ty[blockIdx.y];
    const size_t NN = (size_t)T.N * T.N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < NN; e += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / T.N), q = (int)(e % T.N);
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int cp = cpy[T.offMap + (size_t)v * T.N + p], cq = cpy[T.offMap + (size_t)v * T.N + q];
            if (cp < 0 || cq < 0) continue;
            const int Ev = T.Ev[v];
            const double2* L = LK + T.offL[v];
            const double2* K = L + (size_t)Ev * Ev;
            const bool rm = cp >= Ev, cm = cq >= Ev;
            const size_t o = (size_t)(cp - (rm ? Ev : 0)) * Ev + (cq - (cm ? Ev : 0));
            double2 z;
            if (rm == cm) {
                double2 l = L[o];
                if (rm && v == 1) l = cmul(eps, l);               // j k0 eps_v L_v
                z = make_double2(-k0 * l.y, k0 * l.x);
            } else {
                z = rm ? make_double2(-K[o].x, -K[o].y) : K[o];
            }
            const double s = (double)(sgn[T.offMap + (size_t)v * T.N + p] * sgn[T.offMap + (size_t)v * T.N + q]);
            acc.x += s * z.x;
            acc.y += s * z.y;
        }
        B[T.offB + e] = acc;
    }
}

// one elimination step c for every type: Bout = trailing block of Bin after
// moving the pivot row of column 0 to the top and eliminating column 0
__global__ void __launch_bounds__(256)
slab_eliminate_kernel(const SlabType* __restrict__ ty, int c, const double2* __restrict__ Bin,
                      double2* __restrict__ Bout, int* __restrict__ status) {
    const SlabType T = ty[blockIdx.y];
    const double2* bi = Bin + T.offB;
    double2* bo = Bout + T.offB;
    const int N = T.N;
    if (c >= T.nint) {                 // this type is done: carry its Z~ over
        const int n = N - T.nint;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
            bo[(size_t)(e / n) * N + e % n] = bi[(size_t)(e / n) * N + e % n];
        return;
    }
    __shared__ double s_m[256];
    __shared__ int s_i[256];
    double best = -1.0;
    int bi_row = 0;
    for (int r = threadIdx.x; r < T.nint - c; r += blockDim.x) {
        const double2 v = bi[(size_t)r * N];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi_row = r; }
    }
    s_m[threadIdx.x] = best;
    s_i[threadIdx.x] = bi_row;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double m2 = s_m[threadIdx.x + w];
            const int i2 = s_i[threadIdx.x + w];
            if (m2 > s_m[threadIdx.x] || (m2 == s_m[threadIdx.x] && i2 < s_i[threadIdx.x])) {
                s_m[threadIdx.x] = m2;
                s_i[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const int p = s_i[0];
    if (!(s_m[0] > 0.0)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(status, 1);
        return;
    }
    const double2 piv = bi[(size_t)p * N];
    const double dd = 1.0 / (piv.x * piv.x + piv.y * piv.y);
    const double2 inv = make_double2(piv.x * dd, -piv.y * dd);
    const int no = N - c - 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < no * no; e += gridDim.x * blockDim.x) {
        const int i = e / no, j = e % no;
        const int ro = (i + 1 == p) ? 0 : i + 1;
        const double2 l = cmul(bi[(size_t)ro * N], inv);
        const double2 u = bi[(size_t)p * N + j + 1];
        const double2 a = bi[(size_t)ro * N + j + 1];
        bo[(size_t)i * N + j] = make_double2(a.x - (l.x * u.x - l.y * u.y), a.y - (l.x * u.y + l.y * u.x));
    }
}

__global__ void slab_copy_out_kernel(const SlabType* __restrict__ ty, const double2* __restrict__ B,
                                     int K, double2* __restrict__ Z) {
    const SlabType T = ty[blockIdx.y];
    double2* z = Z + (size_t)blockIdx.y * K * K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x)
        z[e] = B[T.offB + (size_t)(e / K) * T.N + e % K];
}

}  // namespace
}  // namespace emsurf

extern "C" {

EMSURF_API int emsurf_macromodel_slab_patch(double a, double b, double h, int32_t n,
                                            const double* zlevels, int32_t n_types,
                                            const double* sides, int32_t patch_n,
                                            int32_t ring_layers, emsurf_c128 eps_slab, double k0,
                                            emsurf_c128* Z, void* stream) {
    if (n < 2 || !zlevels || n_types < 1 || !sides || patch_n < 1 || ring_layers < 1 || !(k0 > 0.0) ||
        !Z || !(eps_slab.re > 0.0) || !(eps_slab.im <= 0.0)) {
        set_error("emsurf_macromodel_slab_patch: bad arguments (n >= 2, zlevels, Re eps > 0 >= Im eps)");
        return EMSURF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<SlabPlan> plan(n_types);
    std::vector<SlabType> ty(n_types);
    long long nLK = 0, nB = 0, nMap = 0;
    int E = 0, max_nint = 0;
    for (int t = 0; t < n_types; ++t) {
        EMS_TRY(slab_cell_plan(a, b, h, n, zlevels, sides[t], patch_n, ring_layers, plan[t]));
        E = plan[t].E;
        SlabType& T = ty[t];
        for (int v = 0; v < 2; ++v) {
            T.Ev[v] = plan[t].region[v].E;
            T.offL[v] = nLK;
            nLK += 2ll * T.Ev[v] * T.Ev[v];
        }
        T.N = plan[t].N;
        T.nint = plan[t].n_int;
        T.offB = nB;
        nB += (long long)T.N * T.N;
        T.offMap = nMap;
        nMap += 2ll * T.N;
        max_nint = std::max(max_nint, T.nint);
    }
    const int K = 2 * E;
    // region wavenumbers: air k0, slab k0 sqrt(eps) (principal root, Im <= 0)
    const double er = eps_slab.re, ei = eps_slab.im, mod = std::sqrt(er * er + ei * ei);
    const double sr = std::sqrt(0.5 * (mod + er)), si = -std::sqrt(std::max(0.0, 0.5 * (mod - er)));
    const double kv_re[2] = {k0, k0 * sr}, kv_im[2] = {0.0, k0 * si};
    double2 *LK = nullptr, *B0 = nullptr, *B1 = nullptr;
    int32_t* dcpy = nullptr;
    int8_t* dsgn = nullptr;
    SlabType* dty = nullptr;
    int* dstat = nullptr;
    int status = EMSURF_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (status) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("emsurf_macromodel_slab_patch: device allocation of %zu bytes failed", bytes);
            status = EMSURF_ENOMEM;
        }
    };
    alloc((void**)&LK, sizeof(double2) * nLK);
    alloc((void**)&B0, sizeof(double2) * nB);
    alloc((void**)&B1, sizeof(double2) * nB);
    alloc((void**)&dcpy, sizeof(int32_t) * nMap);
    alloc((void**)&dsgn, nMap);
    alloc((void**)&dty, sizeof(SlabType) * n_types);
    alloc((void**)&dstat, sizeof(int));
    const double zero3[3] = {0.0, 0.0, 0.0};
    const int8_t one = 1;
    std::vector<int32_t> hcpy(nMap);
    std::vector<int8_t> hsgn(nMap);
    for (int t = 0; t < n_types && !status; ++t) {
        for (int v = 0; v < 2 && !status; ++v) {
            const SlabRegionMesh& rm = plan[t].region[v];
            const MeshView mv{rm.verts.data(), rm.tris.data(), rm.slot_rwg.data(), rm.slot_sgn.data(), rm.T, rm.E};
            double2* L = LK + ty[t].offL[v];
            status = tabulate_blocks_cx(mv, mv, zero3, &one, 1, kv_re[v], kv_im[v], L,
                                        L + (size_t)rm.E * rm.E, st);
            std::copy(plan[t].copy[v].begin(), plan[t].copy[v].end(), hcpy.begin() + ty[t].offMap + (size_t)v * ty[t].N);
            std::copy(plan[t].sgn[v].begin(), plan[t].sgn[v].end(), hsgn.begin() + ty[t].offMap + (size_t)v * ty[t].N);
        }
    }
    if (!status) {
        cudaError_t e = cudaMemcpyAsync(dcpy, hcpy.data(), sizeof(int32_t) * nMap, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dsgn, hsgn.data(), nMap, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dty, ty.data(), sizeof(SlabType) * n_types, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dstat, 0, sizeof(int), st);
        const int gx = std::max(1, 152 * 8 / n_types);
        if (e == cudaSuccess) {
            slab_assemble_kernel<<<dim3(gx, n_types), 256, 0, st>>>(dty, LK, dcpy, dsgn, k0,
                                                                    make_double2(er, ei), B0);
            e = cudaGetLastError();
        }
        double2 *bin = B0, *bout = B1;
        for (int c = 0; c < max_nint && e == cudaSuccess; ++c) {
            slab_eliminate_kernel<<<dim3(gx, n_types), 256, 0, st>>>(dty, c, bin, bout, dstat);
            e = cudaGetLastError();
            std::swap(bin, bout);
        }
        if (e == cudaSuccess) {
            slab_copy_out_kernel<<<dim3(gx, n_types), 256, 0, st>>>(dty, bin, K, reinterpret_cast<double2*>(Z));
            e = cudaGetLastError();
        }
        const cudaError_t es = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = es;
        if (e != cudaSuccess) {
            set_error("emsurf_macromodel_slab_patch: %s", cudaGetErrorString(e));
            status = EMSURF_ECUDA;
        } else {
            int hs = 0;
            cudaMemcpy(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost);
            if (hs) {
                set_error("emsurf_macromodel_slab_patch: singular interior block");
                status = EMSURF_EINVAL;
            }
        }
    }
    for (void* p : {(void*)LK, (void*)B0, (void*)B1, (void*)dcpy, (void*)dsgn, (void*)dty, (void*)dstat})
        cudaFree(p);
    return status;
}

}  // extern "C"
