// Near-field preconditioner on the GPU: restricted additive Schwarz over the
// cells with an overlap margin.
//
// The paper applies P = U_o^T [Z_eq^NF + Z_o^NF] U_o (Eq. final_precond,
// entries between basis functions closer than Delta_NF) as a right
// preconditioner through a sparse LU (Sec. IV-A).  Here the near field is
// grouped by cell: subdomain m holds every unique unknown whose RWG edge
// midpoint lies inside cell m's footprint grown by an overlap margin delta
// (one mesh layer of the neighbours).  Its exact block A_m = R_m A R_m^T of
// Eq. final is assembled from the offset tables and macromodels, factored
// once (complex FP32 LU with partial pivoting, one CTA per cell), and each
// application computes
//     M^{-1} r = sum_m R~_m^T A_m^{-1} R_m r,
// where R~_m keeps only the unknowns the cell owns (restricted additive
// Schwarz; each unknown is owned by the first cell that references it), so
// every output is written once and the result does not depend on the order
// of the cells.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

constexpr int kLuNB = 16;           // panel width of the blocked LU
constexpr int kLuThreads = 512;
constexpr int kPcMaxN = 1100;       // largest subdomain (panel must fit in shared memory)

__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cdivf(float2 a, float2 b) {
    const float d = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// A_m[a][b] = sum over local copies (c,k) of u = sub[a] and (c',k') of
// v = sub[b] of s s' (B(c - c')[k][k'] + [c == c'] Z~^{t(c)}[k][k']), with
// B(d) = [[al L(d), be K(d)], [ga K(d), de L(d)]] for |dx|, |dy| <= 2.
__global__ void pc_assemble_kernel(float2* __restrict__ mats, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ nsz, const int32_t* __restrict__ sub_ptr,
                                   const int32_t* __restrict__ sub_ids, const int32_t* __restrict__ inv_ptr,
                                   const int32_t* __restrict__ inv_ent, const int8_t* __restrict__ inv_sgn,
                                   const double2* __restrict__ nearL, const double2* __restrict__ nearK,
                                   const double2* __restrict__ Zt, const int32_t* __restrict__ type_map,
                                   int nx, int E, double2 al, double2 be, double2 ga, double2 de) {
    const int m = blockIdx.x;
    const int n = nsz[m];
    const int K = 2 * E;
    const int32_t* sub = sub_ids + sub_ptr[m];
    float2* A = mats + off[m];
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < n * n; e += gridDim.y * blockDim.x) {
        const int a = e / n, b = e % n;
        const int u = sub[a], v = sub[b];
        double2 acc = make_double2(0.0, 0.0);
        for (int p = inv_ptr[u]; p < inv_ptr[u + 1]; ++p) {
            const int lu = inv_ent[p];
            const int c = lu / K, k = lu % K;
            for (int q = inv_ptr[v]; q < inv_ptr[v + 1]; ++q) {
                const int lv = inv_ent[q];
                const int cp = lv / K, kp = lv % K;
                const int dx = c % nx - cp % nx, dy = c / nx - cp / nx;
                const double s = (double)inv_sgn[p] * (double)inv_sgn[q];
                const int hk = k / E, hkp = kp / E, i = k % E, j = kp % E;
                const size_t boff = ((size_t)((dy + 2) * 5 + (dx + 2)) * E + i) * E + j;
                double2 val;
                if (hk == hkp) {
                    const double2 l = nearL[boff];
                    val = cmul(hk == 0 ? al : de, l);
                } else {
                    const double2 kv = nearK[boff];
                    val = cmul(hk == 0 ? be : ga, kv);
                }
                if (c == cp) {
                    const double2 z = Zt[((size_t)type_map[c] * K + kp) * K + k];
                    val.x += z.x;
                    val.y += z.y;
                }
                acc.x += s * val.x;
                acc.y += s * val.y;
            }
        }
        A[(size_t)a * n + b] = make_float2((float)acc.x, (float)acc.y);
    }
}

// In-place blocked LU with partial pivoting of one matrix per CTA (row-major,
// leading dimension n): P A = L U, L unit lower.  perm[a] is the row of A
// that ends in row a.  status[m] = 1 on a zero pivot.
__global__ void __launch_bounds__(kLuThreads)
pc_lu_kernel(float2* __restrict__ mats, const int64_t* __restrict__ off, const int32_t* __restrict__ nsz,
             const int32_t* __restrict__ sub_ptr, int32_t* __restrict__ perm_all, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.x;
    const int n = nsz[m];
    float2* A = mats + off[m];
    int32_t* perm = perm_all + sub_ptr[m];
    float2* P = reinterpret_cast<float2*>(smem_raw);                // [n][kLuNB] panel rows kb..n-1
    __shared__ float red_v[kLuThreads / 32];
    __shared__ int red_i[kLuThreads / 32];
    __shared__ int s_piv;
    __shared__ int pivs[kLuNB];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int a = tid; a < n; a += blockDim.x) perm[a] = a;
    __syncthreads();
    for (int kb = 0; kb < n; kb += kLuNB) {
        const int nb = min(kLuNB, n - kb), rows = n - kb;
        for (int e = tid; e < rows * nb; e += blockDim.x) {
            const int r = e / nb, c = e % nb;
            P[r * kLuNB + c] = A[(size_t)(kb + r) * n + kb + c];
        }
        __syncthreads();
        for (int c = 0; c < nb; ++c) {
            // pivot: largest modulus in column c, rows c..rows-1
            float best = -1.f;
            int bi = c;
            for (int r = c + tid; r < rows; r += blockDim.x) {
                const float2 v = P[r * kLuNB + c];
                const float mg = v.x * v.x + v.y * v.y;
                if (mg > best) { best = mg; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
            __syncthreads();
            if (tid == 0) {
                float b = red_v[0];
                int i = red_i[0];
                for (int w = 1; w < nw; ++w)
                    if (red_v[w] > b || (red_v[w] == b && red_i[w] < i)) { b = red_v[w]; i = red_i[w]; }
                s_piv = i;
                pivs[c] = i;
                if (!(b > 0.f)) status[m] = 1;
            }
            __syncthreads();
            const int p = s_piv;
            if (p != c)
                for (int j = tid; j < nb; j += blockDim.x) {
                    const float2 t = P[c * kLuNB + j];
                    P[c * kLuNB + j] = P[p * kLuNB + j];
                    P[p * kLuNB + j] = t;
                }
            __syncthreads();
            float2 d = P[c * kLuNB + c];
            if (!(d.x * d.x + d.y * d.y > 0.f)) d = make_float2(1.f, 0.f);
            for (int r = c + 1 + tid; r < rows; r += blockDim.x) {
                const float2 l = cdivf(P[r * kLuNB + c], d);
                P[r * kLuNB + c] = l;
                for (int j = c + 1; j < nb; ++j) P[r * kLuNB + j] = csubf(P[r * kLuNB + j], cmul(l, P[c * kLuNB + j]));
            }
            __syncthreads();
        }
        // panel back to A
        for (int e = tid; e < rows * nb; e += blockDim.x) {
            const int r = e / nb, c = e % nb;
            A[(size_t)(kb + r) * n + kb + c] = P[r * kLuNB + c];
        }
        // the panel's row swaps on the columns outside the panel, and in perm
        for (int c = 0; c < nb; ++c) {
            const int p = pivs[c];
            if (p == c) continue;
            const int r0 = kb + c, r1 = kb + p;
            for (int j = tid; j < n; j += blockDim.x) {
                if (j >= kb && j < kb + nb) continue;
                const float2 t = A[(size_t)r0 * n + j];
                A[(size_t)r0 * n + j] = A[(size_t)r1 * n + j];
                A[(size_t)r1 * n + j] = t;
            }
            if (tid == 0) {
                const int t = perm[r0];
                perm[r0] = perm[r1];
                perm[r1] = t;
            }
            __syncthreads();
        }
        __syncthreads();
        // U12 = L11^{-1} A12 (unit lower L11 from the panel)
        const int j0 = kb + nb;
        for (int j = j0 + tid; j < n; j += blockDim.x) {
            float2 x[kLuNB];
            for (int r = 0; r < nb; ++r) {
                float2 acc = A[(size_t)(kb + r) * n + j];
                for (int q = 0; q < r; ++q) acc = csubf(acc, cmul(P[r * kLuNB + q], x[q]));
                x[r] = acc;
                A[(size_t)(kb + r) * n + j] = acc;
            }
        }
        __syncthreads();
        // A22 -= L21 U12, one column per thread
        for (int j = j0 + tid; j < n; j += blockDim.x) {
            float2 u[kLuNB];
            for (int r = 0; r < nb; ++r) u[r] = A[(size_t)(kb + r) * n + j];
            for (int r = nb; r < rows; ++r) {
                float2 acc = A[(size_t)(kb + r) * n + j];
#pragma unroll
                for (int q = 0; q < kLuNB; ++q)
                    if (q < nb) acc = csubf(acc, cmul(P[r * kLuNB + q], u[q]));
                A[(size_t)(kb + r) * n + j] = acc;
            }
        }
        __syncthreads();
    }
}

// y[sub[a]] = (A_m^{-1} R_m r)[a] for the owned a of every cell m: gather
// with the pivot permutation, blocked forward (unit L) and backward (U)
// substitution in shared memory, owned rows written out.  One CTA per cell.
__global__ void __launch_bounds__(256)
pc_apply_kernel(const float2* __restrict__ mats, const int64_t* __restrict__ off,
                const int32_t* __restrict__ nsz, const int32_t* __restrict__ own,
                const int32_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_ids,
                const int32_t* __restrict__ perm_all, const double2* __restrict__ r, double2* __restrict__ y,
                int n_unique) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* b = reinterpret_cast<float2*>(smem_raw);   // [n]
    const int m = blockIdx.x;
    const int rr = blockIdx.y;
    const int n = nsz[m];
    const float2* A = mats + off[m];
    const int32_t* sub = sub_ids + sub_ptr[m];
    const int32_t* perm = perm_all + sub_ptr[m];
    const double2* rv = r + (size_t)rr * n_unique;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const double2 v = rv[sub[perm[a]]];
        b[a] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    __shared__ float2 tile[32][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // forward: L z = b, blocks of 32 rows (diagonal block staged in shared memory)
    for (int s = 0; s < n; s += 32) {
        const int bs = min(32, n - s);
        for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
            const int i = e / bs, j = e % bs;
            tile[i][j] = A[(size_t)(s + i) * n + s + j];
        }
        __syncthreads();
        if (wid == 0) {
            float2 v = lane < bs ? b[s + lane] : make_float2(0.f, 0.f);
            for (int j = 0; j < bs; ++j) {
                const float2 zj = make_float2(__shfl_sync(0xffffffffu, v.x, j), __shfl_sync(0xffffffffu, v.y, j));
                if (lane > j && lane < bs) v = csubf(v, cmul(tile[lane][j], zj));
            }
            if (lane < bs) b[s + lane] = v;
        }
        __syncthreads();
        for (int i = s + bs + threadIdx.x; i < n; i += blockDim.x) {
            float2 acc = b[i];
            const float2* row = A + (size_t)i * n + s;
            for (int j = 0; j < bs; ++j) acc = csubf(acc, cmul(row[j], b[s + j]));
            b[i] = acc;
        }
        __syncthreads();
    }
    // backward: U x = z, blocks of 32 rows from the bottom
    for (int e = n; e > 0; e -= 32) {
        const int s = max(0, e - 32), bs = e - s;
        for (int q = threadIdx.x; q < bs * bs; q += blockDim.x) {
            const int i = q / bs, j = q % bs;
            tile[i][j] = A[(size_t)(s + i) * n + s + j];
        }
        __syncthreads();
        if (wid == 0) {
            float2 v = lane < bs ? b[s + lane] : make_float2(0.f, 0.f);
            for (int j = bs - 1; j >= 0; --j) {
                if (lane == j) v = cdivf(v, tile[j][j]);
                const float2 xj = make_float2(__shfl_sync(0xffffffffu, v.x, j), __shfl_sync(0xffffffffu, v.y, j));
                if (lane < j) v = csubf(v, cmul(tile[lane][j], xj));
            }
            if (lane < bs) b[s + lane] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < s; i += blockDim.x) {
            float2 acc = b[i];
            const float2* row = A + (size_t)i * n + s;
            for (int j = 0; j < bs; ++j) acc = csubf(acc, cmul(row[j], b[s + j]));
            b[i] = acc;
        }
        __syncthreads();
    }
    double2* yv = y + (size_t)rr * n_unique;
    for (int a = threadIdx.x; a < own[m]; a += blockDim.x) yv[sub[a]] = make_double2((double)b[a].x, (double)b[a].y);
}

}  // namespace

int pc_apply(emsurf_handle* h, const double2* r, double2* y, int R, cudaStream_t st) {
    const size_t smem = (size_t)h->pc_nmax * sizeof(float2);
    EMS_TRY(set_smem_once(pc_apply_kernel, smem));
    pc_apply_kernel<<<dim3(h->M, R), 256, smem, st>>>(h->pc_mat, h->pc_off, h->pc_n, h->pc_own, h->pc_sub_ptr,
                                                       h->pc_sub_ids, h->pc_perm, r, y, h->n_unique);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}

// Subdomains, near tables, assembly and factorisation (create time).
int pc_build(emsurf_handle* h, const emsurf_problem* p) {
    const int M = h->M, K = h->K, E = h->E, nx = h->nx, ny = h->ny;
    const double a = p->cell_a, b = p->cell_b, del = p->precond_overlap;
    const double* xy = p->unknown_xy;
    // the subdomain of a cell then reaches only its 3 x 3 neighbours, and
    // any two of its unknowns' copies are at most 2 cells apart
    if (!(del < 0.5 * std::min(a, b))) {
        set_error("precond_overlap must be below half the smaller cell side");
        return EMSURF_EINVAL;
    }
    // owner of each unique unknown: first cell referencing it
    std::vector<int32_t> owner(h->n_unique, -1);
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < K; ++k) {
            const int u = p->uo_index[(size_t)m * K + k];
            if (owner[u] < 0) owner[u] = m;
        }
    std::vector<int32_t> sptr(M + 1, 0), sids, own(M), nsz(M);
    std::vector<int> mark(h->n_unique, -1);
    std::vector<int32_t> cand;
    for (int m = 0; m < M; ++m) {
        const int ix = m % nx, iy = m / nx;
        const double cx = ix * a, cy = iy * b;
        cand.clear();
        for (int jy = std::max(0, iy - 1); jy <= std::min(ny - 1, iy + 1); ++jy)
            for (int jx = std::max(0, ix - 1); jx <= std::min(nx - 1, ix + 1); ++jx) {
                const int c = jy * nx + jx;
                for (int k = 0; k < K; ++k) {
                    const int u = p->uo_index[(size_t)c * K + k];
                    if (mark[u] == m) continue;
                    const double x = xy[2 * u], yy = xy[2 * u + 1];
                    if (std::fabs(x - cx) <= 0.5 * a + del + 1e-12 && std::fabs(yy - cy) <= 0.5 * b + del + 1e-12) {
                        mark[u] = m;
                        cand.push_back(u);
                    }
                }
            }
        std::sort(cand.begin(), cand.end());
        std::stable_partition(cand.begin(), cand.end(), [&](int u) { return owner[u] == m; });
        int no = 0;
        for (int u : cand) no += owner[u] == m;
        own[m] = no;
        nsz[m] = (int)cand.size();
        if (nsz[m] > kPcMaxN) {
            set_error("preconditioner subdomain of %d unknowns exceeds %d; reduce the overlap", nsz[m], kPcMaxN);
            return EMSURF_EINVAL;
        }
        h->pc_nmax = std::max(h->pc_nmax, nsz[m]);
        sids.insert(sids.end(), cand.begin(), cand.end());
        sptr[m + 1] = (int32_t)sids.size();
    }
    // every unknown is owned by exactly one subdomain
    for (int u = 0; u < h->n_unique; ++u) {
        const int m = owner[u];
        bool found = false;
        for (int q = sptr[m]; q < sptr[m] + own[m]; ++q) found = found || sids[q] == u;
        if (!found) {
            set_error("unknown %d is not inside its own cell's subdomain (positions inconsistent)", u);
            return EMSURF_EINVAL;
        }
    }
    std::vector<int64_t> moff(M + 1, 0);
    for (int m = 0; m < M; ++m) moff[m + 1] = moff[m] + (int64_t)nsz[m] * nsz[m];
    cudaStream_t st = h->setup_stream;
    auto up = [&](auto** d, const auto* src, size_t cnt) -> int {
        EMS_TRY(dev_alloc(h, (void**)d, cnt * sizeof(**d)));
        EMS_CUDA(cudaMemcpyAsync(*d, src, cnt * sizeof(**d), cudaMemcpyHostToDevice, st));
        return EMSURF_OK;
    };
    EMS_TRY(up(&h->pc_sub_ptr, sptr.data(), sptr.size()));
    EMS_TRY(up(&h->pc_sub_ids, sids.data(), sids.size()));
    EMS_TRY(up(&h->pc_own, own.data(), own.size()));
    EMS_TRY(up(&h->pc_n, nsz.data(), nsz.size()));
    EMS_TRY(up(&h->pc_off, moff.data(), (size_t)M));
    EMS_TRY(dev_alloc(h, (void**)&h->pc_perm, sids.size() * sizeof(int32_t)));
    EMS_TRY(dev_alloc(h, (void**)&h->pc_mat, (size_t)moff[M] * sizeof(float2)));
    // near offset tables |dx|, |dy| <= 2 -> [5][5][E][E] (zero outside the lattice)
    const size_t EE = (size_t)E * E;
    double2 *nL = nullptr, *nK = nullptr;
    EMS_CUDA(cudaMalloc(&nL, 25 * EE * sizeof(double2)));
    EMS_CUDA(cudaMalloc(&nK, 25 * EE * sizeof(double2)));
    EMS_CUDA(cudaMemsetAsync(nL, 0, 25 * EE * sizeof(double2), st));
    EMS_CUDA(cudaMemsetAsync(nK, 0, 25 * EE * sizeof(double2), st));
    const cudaMemcpyKind kind = p->tables_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            if (std::abs(dx) > nx - 1 || std::abs(dy) > ny - 1) continue;
            const size_t src = ((size_t)(dy + ny - 1) * (2 * nx - 1) + (dx + nx - 1)) * EE;
            const size_t dst = (size_t)((dy + 2) * 5 + (dx + 2)) * EE;
            EMS_CUDA(cudaMemcpyAsync(nL + dst, p->offset_L + src, EE * sizeof(double2), kind, st));
            EMS_CUDA(cudaMemcpyAsync(nK + dst, p->offset_K + src, EE * sizeof(double2), kind, st));
        }
    // macromodels (transposed, FP64) for the assembly
    double2* Zt = nullptr;
    bool own_zt = false;
    if (h->have64) {
        Zt = h->op64.Zt;
    } else {
        own_zt = true;
        EMS_CUDA(cudaMalloc(&Zt, (size_t)h->T * K * K * sizeof(double2)));
        // transpose of the input macromodels
        std::vector<double2> hz((size_t)h->T * K * K);
        std::vector<double2> zin((size_t)h->T * K * K);
        EMS_CUDA(cudaMemcpyAsync(zin.data(), p->macromodels, zin.size() * sizeof(double2),
                                 p->tables_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
        EMS_CUDA(cudaStreamSynchronize(st));
        for (int t = 0; t < h->T; ++t)
            for (int i = 0; i < K; ++i)
                for (int j = 0; j < K; ++j) hz[((size_t)t * K + j) * K + i] = zin[((size_t)t * K + i) * K + j];
        EMS_CUDA(cudaMemcpyAsync(Zt, hz.data(), hz.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        EMS_CUDA(cudaStreamSynchronize(st));
    }
    double2 co[4];
    for (int c = 0; c < 4; ++c) co[c] = make_double2(p->coef[c].re, p->coef[c].im);
    pc_assemble_kernel<<<dim3(M, 64), 256, 0, st>>>(h->pc_mat, h->pc_off, h->pc_n, h->pc_sub_ptr, h->pc_sub_ids,
                                                    h->d_inv_ptr, h->d_inv_ent, h->d_inv_sgn, nL, nK, Zt,
                                                    h->d_type_map, nx, E, co[0], co[1], co[2], co[3]);
    EMS_CUDA(cudaGetLastError());
    int* dstat = nullptr;
    EMS_CUDA(cudaMalloc(&dstat, sizeof(int) * M));
    EMS_CUDA(cudaMemsetAsync(dstat, 0, sizeof(int) * M, st));
    const size_t lsm = (size_t)h->pc_nmax * kLuNB * sizeof(float2);
    EMS_TRY(set_smem_once(pc_lu_kernel, lsm));
    pc_lu_kernel<<<M, kLuThreads, lsm, st>>>(h->pc_mat, h->pc_off, h->pc_n, h->pc_sub_ptr, h->pc_perm, dstat);
    EMS_CUDA(cudaGetLastError());
    std::vector<int> hs(M);
    EMS_CUDA(cudaMemcpyAsync(hs.data(), dstat, sizeof(int) * M, cudaMemcpyDeviceToHost, st));
    EMS_CUDA(cudaStreamSynchronize(st));
    cudaFree(dstat);
    cudaFree(nL);
    cudaFree(nK);
    if (own_zt) cudaFree(Zt);
    for (int m = 0; m < M; ++m)
        if (hs[m]) {
            set_error("preconditioner block of cell %d is singular", m);
            return EMSURF_EINVAL;
        }
    h->pc_elems = moff[M];
    h->pc_sub_total = (int64_t)sids.size();
    h->have_pc = true;
    return EMSURF_OK;
}

}  // namespace emsurf
