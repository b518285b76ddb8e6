// Near-field preconditioner on the GPU: restricted additive Schwarz over the
// cells with an overlap margin.
//
// The paper applies P = U_o^T [Z_eq^NF + Z_o^NF] U_o (Eq. final_precond,
// entries between basis functions closer than Delta_NF) as a right
// preconditioner through a sparse LU (Sec. IV-A).  Here the near field is
// grouped by cell: subdomain m holds every unique unknown whose RWG edge
// midpoint lies inside cell m's footprint grown by an overlap margin delta
// (one mesh layer of the neighbours).  Its exact block A_m = R_m A R_m^T of
// Eq. final is assembled from the offset tables and macromodels and factored
// once (complex FP32 LU with partial pivoting, one CTA per cell).  Each
// application computes
//     M^{-1} r = sum_m R~_m^T A_m^{-1} R_m r,
// where R~_m keeps only the unknowns the cell owns (restricted additive
// Schwarz; each unknown is owned by the first cell that references it), so
// every output is written once and the result does not depend on the order
// of the cells.  Only the owned rows of A_m^{-1} are ever used, so they are
// formed from the factors at create time and the application is a batched
// matrix-vector product over own_m x n_m entries (about half of n_m^2, and
// without the serial steps of a triangular solve); the factors are freed.
// The rows are kept in FP16 with one FP32 scale per row (the preconditioner
// only steers the flexible GMRES, whose accuracy comes from the operator):
// half the bytes of complex64 per application.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

constexpr int kLuNB = 16;           // panel width of the blocked LU
constexpr int kLuThreads = 512;
constexpr int kPcMaxN = 1100;       // largest subdomain (panel must fit in shared memory)
constexpr int kInvNR = 16;          // inverse rows per CTA
constexpr int kInvThreads = 512;
constexpr int kApThreads = 256;
constexpr int kApUnroll = 8;        // 16-byte loads in flight per lane

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

__device__ __forceinline__ float2 crecipf(float2 b) {
    const float d = b.x * b.x + b.y * b.y;
    return make_float2(b.x / d, -b.y / d);
}

// Owned rows of A_m^{-1} from the factors P A = L U:  A^{-1} = U^{-1} L^{-1} P,
// so row i is v^T P with U^T w = e_i (forward) and L^T v = w (backward), and
// row[perm[a]] = v[a].  U^T w = e_i is solved in the scaled form s = D w
// (D = diag U): s[b] -= (U[a][b] / U[a][a]) s[a], then w = D^{-1} s.  Both
// sweeps read one row of the factors per step (coalesced); the kInvNR right-
// hand sides of the CTA live in shared memory as W[q][a].
__global__ void __launch_bounds__(kInvThreads)
pc_invrows_kernel(const float2* __restrict__ lu, const int64_t* __restrict__ luoff,
                  const int32_t* __restrict__ nsz, const int32_t* __restrict__ own,
                  const int32_t* __restrict__ sub_ptr, const int32_t* __restrict__ perm_all,
                  float2* __restrict__ X, const int64_t* __restrict__ xoff, const int32_t* __restrict__ ldx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* W = reinterpret_cast<float2*>(smem_raw);     // [kInvNR][n]
    const int m = blockIdx.y;
    const int n = nsz[m], i0 = blockIdx.x * kInvNR;
    if (i0 >= own[m]) return;
    const int nr = min(kInvNR, own[m] - i0);
    const float2* A = lu + luoff[m];
    const int tid = threadIdx.x;
    for (int e = tid; e < kInvNR * n; e += blockDim.x) {
        const int q = e / n, a = e % n;
        W[e] = make_float2(q < nr && a == i0 + q ? 1.f : 0.f, 0.f);
    }
    // forward: e_i has no entry before i0
    for (int a = i0; a < n - 1; ++a) {
        __syncthreads();
        const float2 rd = crecipf(A[(size_t)a * n + a]);
        for (int b = a + 1 + tid; b < n; b += blockDim.x) {
            const float2 u = cmul(A[(size_t)a * n + b], rd);
            for (int q = 0; q < nr; ++q) W[q * n + b] = csubf(W[q * n + b], cmul(u, W[q * n + a]));
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * n; e += blockDim.x) {
        const int a = e % n;
        W[e] = cmul(W[e], crecipf(A[(size_t)a * n + a]));
    }
    // backward with the unit upper L^T
    for (int a = n - 1; a > 0; --a) {
        __syncthreads();
        for (int b = tid; b < a; b += blockDim.x) {
            const float2 l = A[(size_t)a * n + b];
            for (int q = 0; q < nr; ++q) W[q * n + b] = csubf(W[q * n + b], cmul(l, W[q * n + a]));
        }
    }
    __syncthreads();
    const int32_t* perm = perm_all + sub_ptr[m];
    const int ld = ldx[m];
    float2* Xm = X + xoff[m];
    for (int e = tid; e < nr * n; e += blockDim.x) {
        const int q = e / n, a = e % n;
        Xm[(size_t)(i0 + q) * ld + perm[a]] = W[e];
    }
}

// FP16 copy of the owned inverse rows for the apply: one warp per owned row
// g, scale = (largest |component| of the row) / 2^14, so every entry keeps
// FP16's 11-bit significand unless it is below ~6e-5 of the row maximum
// (then its absolute error is below 2^-24 of that maximum).
__global__ void pc_to_half_kernel(const float2* __restrict__ X, const int64_t* __restrict__ xoff,
                                  const int32_t* __restrict__ ldx, const int32_t* __restrict__ own_ptr, int M,
                                  int n_rows, __half2* __restrict__ H, float* __restrict__ rscale) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_rows; g += warps) {
        int lo = 0, hi = M;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (own_ptr[mid] <= g) lo = mid; else hi = mid;
        }
        const int m = lo, i = g - own_ptr[m], ld = ldx[m];
        const float2* row = X + xoff[m] + (size_t)i * ld;
        float mx = 0.f;
        for (int c = lane; c < ld; c += 32) mx = fmaxf(mx, fmaxf(fabsf(row[c].x), fabsf(row[c].y)));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.f ? mx / 16384.f : 1.f;
        const float inv = 1.f / sc;
        __half2* out = H + xoff[m] + (size_t)i * ld;
        for (int c = lane; c < ld; c += 32) out[c] = __floats2half2_rn(row[c].x * inv, row[c].y * inv);
        if (lane == 0) rscale[g] = sc;
    }
}

// 8-bit copy of the owned inverse rows (handles asking for it, 1-2 rhs): one
// warp per owned row g, scale = (largest |component| of the row) / 127, each
// component rounded to the nearest integer in [-127, 127] and stored offset
// by 128 (so a byte b decodes to b - 128 exactly through its FP32 bit
// pattern 2^23 + b); absolute error <= 2^-1 / 127 of the row's largest
// component per entry.
__global__ void pc_to_int8_kernel(const float2* __restrict__ X, const int64_t* __restrict__ xoff,
                                  const int32_t* __restrict__ ldx, const int32_t* __restrict__ own_ptr, int M,
                                  int n_rows, uchar2* __restrict__ Q, float* __restrict__ rscale) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_rows; g += warps) {
        int lo = 0, hi = M;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (own_ptr[mid] <= g) lo = mid; else hi = mid;
        }
        const int m = lo, i = g - own_ptr[m], ld = ldx[m];
        const float2* row = X + xoff[m] + (size_t)i * ld;
        float mx = 0.f;
        for (int c = lane; c < ld; c += 32) mx = fmaxf(mx, fmaxf(fabsf(row[c].x), fabsf(row[c].y)));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.f ? mx / 127.f : 1.f;
        const float inv = 1.f / sc;
        uchar2* out = Q + xoff[m] + (size_t)i * ld;
        for (int c = lane; c < ld; c += 32) {
            const float qr = fminf(fmaxf(rintf(row[c].x * inv), -127.f), 127.f);
            const float qi = fminf(fmaxf(rintf(row[c].y * inv), -127.f), 127.f);
            out[c] = make_uchar2((unsigned char)((int)qr + 128), (unsigned char)((int)qi + 128));
        }
        if (lane == 0) rscale[g] = sc;
    }
}

// b - 128 for byte k of w (offset-binary 8-bit entries): the float with bit
// pattern 0x4B0000bb is 2^23 + b exactly
__device__ __forceinline__ float pc_q8(uint32_t w, uint32_t k) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7540u | k)) - 8388736.0f;
}

// rs[q][j] = r[q][sub_ids[j]] in FP32 for every subdomain entry j (all cells
// back to back, each cell's segment starting at an even index).
template <typename VT>
__global__ void pc_gather_kernel(const VT* __restrict__ r, const int32_t* __restrict__ sub_ids,
                                 const int32_t* __restrict__ sub_cell, const int32_t* __restrict__ sub_ptr,
                                 const int64_t* __restrict__ rs_off, float2* __restrict__ rs,
                                 int total, int n_unique, int64_t rs_stride, int R) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        const int m = sub_cell[j];
        const int64_t o = rs_off[m] + (j - sub_ptr[m]);
        const int u = sub_ids[j];
        for (int q = 0; q < R; ++q) {
            const VT d = r[(size_t)q * n_unique + u];
            rs[q * rs_stride + o] = make_float2((float)d.x, (float)d.y);
        }
    }
}

// y[sub[i]] = sum_c X_m[i][c] rs_m[c] for the owned rows i of every cell
// (the restricted additive Schwarz sum: each unknown is owned once).  The
// owned rows of all cells form one list; each warp takes whole rows
// (16-byte loads of X, eight in flight per lane; the cell's rs segment is
// reused from L1/L2) and reduces once per row and right-hand side.  Used for
// fewer rhs than the tensor-core path takes.
// The grid is exactly the resident capacity, so the row list is shared out
// in one wave.
template <int RQ, typename VO>
__global__ void __launch_bounds__(kApThreads, RQ >= 2 ? 2 : 4)
pc_apply_kernel(const __half2* __restrict__ X, const float* __restrict__ rscale, const int64_t* __restrict__ xoff,
                const int32_t* __restrict__ ldx, const int32_t* __restrict__ own_ptr,
                const int32_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_ids,
                const int64_t* __restrict__ rs_off, const float2* __restrict__ rs, int64_t rs_stride,
                VO* __restrict__ y, int n_rows, int M, int n_unique, int r0, int nr) {
    const int lane = threadIdx.x & 31;
    // warps take rows in a grid stride: at any time the warps of the whole
    // grid work on one window of consecutive rows (a few cells), whose
    // gathered r segments stay in L1/L2
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_rows; g += warps) {
        // cell of owned row g: own_ptr[m] <= g < own_ptr[m+1]
        int lo = 0, hi = M;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (own_ptr[mid] <= g) lo = mid; else hi = mid;
        }
        const int m = lo;
        const int i = g - own_ptr[m], ld = ldx[m], quarter = ld >> 2;
        const uint4* row = reinterpret_cast<const uint4*>(X + xoff[m] + (size_t)i * ld);   // 4 complex each
        const float4* rv4 = reinterpret_cast<const float4*>(rs + rs_off[m]);
        float2 acc[RQ];
#pragma unroll
        for (int q = 0; q < RQ; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int c0 = lane; c0 < quarter; c0 += 32 * kApUnroll) {
            uint4 xv[kApUnroll];
#pragma unroll
            for (int u = 0; u < kApUnroll; ++u)
                xv[u] = c0 + 32 * u < quarter ? __ldg(row + c0 + 32 * u) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int u = 0; u < kApUnroll; ++u) {
                const int c4 = min(c0 + 32 * u, quarter - 1);
                const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&xv[u].x));
                const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&xv[u].y));
                const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&xv[u].z));
                const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&xv[u].w));
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    if (RQ > 2 && q >= nr) break;   // rhs past the live count (wide kernels only)
                    const float4 ra = __ldg(rv4 + q * (rs_stride >> 1) + 2 * c4);
                    const float4 rb = __ldg(rv4 + q * (rs_stride >> 1) + 2 * c4 + 1);
                    acc[q].x += f0.x * ra.x - f0.y * ra.y + f1.x * ra.z - f1.y * ra.w +
                                f2.x * rb.x - f2.y * rb.y + f3.x * rb.z - f3.y * rb.w;
                    acc[q].y += f0.x * ra.y + f0.y * ra.x + f1.x * ra.w + f1.y * ra.z +
                                f2.x * rb.y + f2.y * rb.x + f3.x * rb.w + f3.y * rb.z;
                }
            }
        }
        {
            const float sc = rscale[g];
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                acc[q].x *= sc;
                acc[q].y *= sc;
            }
        }
#pragma unroll
        for (int q = 0; q < RQ; ++q)
            for (int o = 16; o > 0; o >>= 1) {
                acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
            }
        if (lane == 0) {
            const int u = sub_ids[sub_ptr[m] + i];
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                if (RQ > 2 && q >= nr) break;
                VO o;
                o.x = acc[q].x;
                o.y = acc[q].y;
                y[(size_t)(r0 + q) * n_unique + u] = o;
            }
        }
    }
}

// Single- and two-rhs apply without the gather pass.  The owned rows are cut
// into gridDim.x contiguous ranges of equal length; a block walks its range
// cell by cell: it gathers the cell's r segment straight from r into shared
// memory (FP32, zero past n_m up to ld_m), then each warp takes two rows at a
// time (16-byte loads of the FP16 rows, kApSegLoads per row and lane in
// flight: all of a row of up to 1024 entries in one round) and reduces both
// rows' sums with one reduce-scatter.
constexpr int kApSegThreads = 256;
constexpr int kApSegMaxLd = 1024;   // longest row (complex entries) of this kernel
constexpr int kApSegLoads = 8;      // 16-byte row loads per row and lane in flight (a whole row of up to 1024)

template <typename VT>
__device__ __forceinline__ float2 to_f2(VT v) { return make_float2((float)v.x, (float)v.y); }

template <int RQ, typename VT, bool Q8>
__global__ void __launch_bounds__(kApSegThreads, RQ == 1 ? 3 : 2)
pc_apply_seg_kernel(const void* __restrict__ X, const float* __restrict__ rscale,
                    const int64_t* __restrict__ xoff, const int32_t* __restrict__ ldx,
                    const int32_t* __restrict__ own_ptr, const int32_t* __restrict__ sub_ptr,
                    const int32_t* __restrict__ sub_ids, const VT* __restrict__ r, VT* __restrict__ y,
                    int n_rows, int M, int n_unique) {
    __shared__ __align__(16) float2 rsm[RQ][kApSegMaxLd];
    constexpr int NV = 4 * RQ;            // floats per lane and row pair: [row][q][re, im]
    constexpr int kSpan = 32 / NV;        // lanes per reduced value
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint64_t pol = l2_evict_first();     // the rows are read once per apply
    const int g0 = (int)((long long)blockIdx.x * n_rows / gridDim.x);
    const int g1 = (int)((long long)(blockIdx.x + 1) * n_rows / gridDim.x);
    if (g0 >= g1) return;
    // cell of row g0: the last m with own_ptr[m] <= g0
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (own_ptr[mid] <= g0) lo = mid; else hi = mid;
    }
    int m = lo;
    for (int g = g0; g < g1;) {
        while (own_ptr[m + 1] <= g) ++m;           // cells that own no row
        const int e = min(g1, own_ptr[m + 1]);
        const int ld = ldx[m], n = sub_ptr[m + 1] - sub_ptr[m];
        const int32_t* ids = sub_ids + sub_ptr[m];
        __syncthreads();                           // readers of the previous segment are done
        for (int c = threadIdx.x; c < ld; c += blockDim.x) {
            const int u = c < n ? ids[c] : 0;
#pragma unroll
            for (int q = 0; q < RQ; ++q)
                rsm[q][c] = c < n ? to_f2(r[(size_t)q * n_unique + u]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // 16-byte loads per row: 4 FP16 complex or 8 offset-binary 8-bit ones
        constexpr int kPer = Q8 ? 8 : 4;
        const int quarter = ld / kPer;
        const uint4* Xm = reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(X) +
                                                         (size_t)xoff[m] * (Q8 ? 2 : 4));
        // a load past the row reads as zeros (0x80 bytes in the 8-bit encoding)
        const uint32_t zw = Q8 ? 0x80808080u : 0u;
        const int i0 = g - own_ptr[m], cnt = e - g;
        for (int p = 2 * warp; p < cnt; p += 2 * nw) {
            const int ia = i0 + p, ib = p + 1 < cnt ? ia + 1 : ia;
            const uint4* ra = Xm + (size_t)ia * quarter;
            const uint4* rb = Xm + (size_t)ib * quarter;
            float2 acc[2][RQ];
#pragma unroll
            for (int w = 0; w < 2; ++w)
#pragma unroll
                for (int q = 0; q < RQ; ++q) acc[w][q] = make_float2(0.f, 0.f);
            for (int c0 = lane; c0 < quarter; c0 += 32 * kApSegLoads) {
                uint4 xv[2][kApSegLoads];
#pragma unroll
                for (int u = 0; u < kApSegLoads; ++u) {
                    const bool in = c0 + 32 * u < quarter;
                    xv[0][u] = in ? ldg_l2hint(ra + c0 + 32 * u, pol) : make_uint4(zw, zw, zw, zw);
                    xv[1][u] = in ? ldg_l2hint(rb + c0 + 32 * u, pol) : make_uint4(zw, zw, zw, zw);
                }
#pragma unroll
                for (int u = 0; u < kApSegLoads; ++u) {
                    const int c4 = min(c0 + 32 * u, quarter - 1);
#pragma unroll
                    for (int q = 0; q < RQ; ++q) {
                        if constexpr (Q8) {
                            // 8 complex per load, two per 32-bit word (re, im, re, im)
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const float4 rr = reinterpret_cast<const float4*>(rsm[q])[4 * c4 + k];
#pragma unroll
                                for (int w = 0; w < 2; ++w) {
                                    const uint32_t wd = k == 0 ? xv[w][u].x : k == 1 ? xv[w][u].y
                                                      : k == 2 ? xv[w][u].z : xv[w][u].w;
                                    const float a0 = pc_q8(wd, 0), b0 = pc_q8(wd, 1);
                                    const float a1 = pc_q8(wd, 2), b1 = pc_q8(wd, 3);
                                    acc[w][q].x += a0 * rr.x - b0 * rr.y + a1 * rr.z - b1 * rr.w;
                                    acc[w][q].y += a0 * rr.y + b0 * rr.x + a1 * rr.w + b1 * rr.z;
                                }
                            }
                        } else {
                            const float4 r0 = reinterpret_cast<const float4*>(rsm[q])[2 * c4];
                            const float4 r1 = reinterpret_cast<const float4*>(rsm[q])[2 * c4 + 1];
#pragma unroll
                            for (int w = 0; w < 2; ++w) {
                                const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&xv[w][u].x));
                                const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&xv[w][u].y));
                                const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&xv[w][u].z));
                                const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&xv[w][u].w));
                                acc[w][q].x += f0.x * r0.x - f0.y * r0.y + f1.x * r0.z - f1.y * r0.w +
                                               f2.x * r1.x - f2.y * r1.y + f3.x * r1.z - f3.y * r1.w;
                                acc[w][q].y += f0.x * r0.y + f0.y * r0.x + f1.x * r0.w + f1.y * r0.z +
                                               f2.x * r1.y + f2.y * r1.x + f3.x * r1.w + f3.y * r1.z;
                            }
                        }
                    }
                }
            }
            // reduce-scatter: lane l ends with the warp sum of value l / kSpan
            float v[NV];
#pragma unroll
            for (int w = 0; w < 2; ++w)
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    v[(w * RQ + q) * 2] = acc[w][q].x;
                    v[(w * RQ + q) * 2 + 1] = acc[w][q].y;
                }
#pragma unroll
            for (int nn = NV, D = 16; nn > 1; nn >>= 1, D >>= 1) {
                const bool up = lane & D;
#pragma unroll
                for (int c = 0; c < nn / 2; ++c) {
                    const float send = up ? v[c] : v[c + nn / 2];
                    const float keep = up ? v[c + nn / 2] : v[c];
                    v[c] = keep + __shfl_xor_sync(0xffffffffu, send, D);
                }
            }
            float s1 = v[0];
#pragma unroll
            for (int D = 16 / NV; D >= 1; D >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, D);
            const float s2 = __shfl_down_sync(0xffffffffu, s1, kSpan);   // the next value (imaginary part)
            const int vi = lane / kSpan;
            if (lane % kSpan == 0 && (vi & 1) == 0) {
                const int w = vi / (2 * RQ), q = (vi >> 1) % RQ;
                if (w == 0 || p + 1 < cnt) {
                    const int i = w ? ib : ia;
                    const float sc = rscale[own_ptr[m] + i];
                    VT o;
                    o.x = s1 * sc;
                    o.y = s2 * sc;
                    y[(size_t)q * n_unique + ids[i]] = o;
                }
            }
        }
        g = e;
        ++m;
    }
}

template <int RQ, typename VT, bool Q8>
int launch_apply_seg(emsurf_handle* h, const VT* r, VT* y, cudaStream_t st) {
    static int occ[3][2][2] = {};
    int& o = occ[RQ][sizeof(VT) == sizeof(float2) ? 1 : 0][Q8 ? 1 : 0];
    if (!o) {
        int b = 0;
        EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pc_apply_seg_kernel<RQ, VT, Q8>, kApSegThreads, 0));
        o = std::max(b, 1);
    }
    const int blocks = std::max(1, std::min(h->num_sms * o, h->n_unique));
    pc_apply_seg_kernel<RQ, VT, Q8><<<blocks, kApSegThreads, 0, st>>>(
        h->pc_mat16, h->pc_rscale, h->pc_off, h->pc_ld, h->pc_own_ptr,
        h->pc_sub_ptr, h->pc_sub_ids, r, y, h->n_unique, h->M, h->n_unique);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}

template <int RQ, typename VO>
int launch_apply(emsurf_handle* h, VO* y, int r0, int nr, cudaStream_t st) {
    // resident blocks per SM (computed once; the library is compiled for one architecture)
    static int occ[9][2] = {};
    int& o = occ[RQ][sizeof(VO) == sizeof(float2) ? 1 : 0];
    if (!o) {
        int b = 0;
        EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pc_apply_kernel<RQ, VO>, kApThreads, 0));
        o = std::max(b, 1);
    }
    const int blocks = h->num_sms * o;
    pc_apply_kernel<RQ, VO><<<blocks, kApThreads, 0, st>>>(reinterpret_cast<const __half2*>(h->pc_mat16), h->pc_rscale,
                                                        h->pc_off, h->pc_ld, h->pc_own_ptr,
                                                        h->pc_sub_ptr, h->pc_sub_ids, h->pc_rs_off,
                                                        h->pc_rs + (size_t)r0 * h->pc_rs_stride,
                                                        h->pc_rs_stride, y, h->n_unique, h->M, h->n_unique, r0, nr);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}

}  // namespace

template <typename VT>
int pc_apply_t(emsurf_handle* h, const VT* r, VT* y, int R, cudaStream_t st) {
    if (R > h->max_rhs) {
        set_error("preconditioner: %d right-hand sides, handle holds %d", R, h->max_rhs);
        return EMSURF_EINVAL;
    }
    if (h->have_pc_tc && R >= kTcMinRhs) return pc_tc_apply<VT>(h, r, y, R, st);
    if (h->pc_int8)      // 8-bit rows: handles of one or two rhs, rows of up to kApSegMaxLd
        return R == 1 ? launch_apply_seg<1, VT, true>(h, r, y, st) : launch_apply_seg<2, VT, true>(h, r, y, st);
    if (R <= 2 && ((h->pc_nmax + 3) & ~3) <= kApSegMaxLd)
        return R == 1 ? launch_apply_seg<1, VT, false>(h, r, y, st) : launch_apply_seg<2, VT, false>(h, r, y, st);
    const int total = (int)h->pc_sub_total;
    pc_gather_kernel<VT><<<std::min((total + 255) / 256, h->num_sms * 8), 256, 0, st>>>(
        r, h->pc_sub_ids, h->pc_sub_cell, h->pc_sub_ptr, h->pc_rs_off, h->pc_rs, total, h->n_unique,
        h->pc_rs_stride, R);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    for (int r0 = 0; r0 < R; r0 += 8) {
        const int nr = std::min(8, R - r0);
        if (nr == 1) EMS_TRY((launch_apply<1, VT>(h, y, r0, nr, st)));
        else if (nr == 2) EMS_TRY((launch_apply<2, VT>(h, y, r0, nr, st)));
        else if (nr <= 4) EMS_TRY((launch_apply<4, VT>(h, y, r0, nr, st)));
        else EMS_TRY((launch_apply<8, VT>(h, y, r0, nr, st)));
    }
    return EMSURF_OK;
}

int pc_apply(emsurf_handle* h, const double2* r, double2* y, int R, cudaStream_t st) {
    return pc_apply_t<double2>(h, r, y, R, st);
}

int pc_apply_f32(emsurf_handle* h, const float2* r, float2* y, int R, cudaStream_t st) {
    return pc_apply_t<float2>(h, r, y, R, st);
}

// Subdomains, near tables, assembly and factorisation (create time).
// The near offset tables |dx|, |dy| <= 2 as [5][5][E][E] (zero outside the
// lattice), kept by the handle for the preconditioner's subdomain blocks.
int stage_near_tables(emsurf_handle* h, const emsurf_problem* p) {
    const int E = h->E, nx = h->nx, ny = h->ny;
    const size_t EE = (size_t)E * E;
    cudaStream_t st = h->setup_stream;
    double2 *nL = nullptr, *nK = nullptr;
    EMS_TRY(dev_alloc(h, (void**)&nL, 25 * EE * sizeof(double2)));
    EMS_TRY(dev_alloc(h, (void**)&nK, 25 * EE * sizeof(double2)));
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
    h->near_L = nL;
    h->near_K = nK;
    return EMSURF_OK;
}

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
    // LU factors n_m x n_m (temporary); owned inverse rows own_m x ld_m (kept)
    std::vector<int64_t> moff(M + 1, 0), xoff(M + 1, 0);
    std::vector<int32_t> ldv(M);
    int nmax_all = 0;
    for (int m = 0; m < M; ++m) nmax_all = std::max(nmax_all, nsz[m]);
    // 8-bit rows for the one- and two-rhs apply, when asked for and every row fits it
    const bool q8 = p->precond_int8 && h->max_rhs <= 2 && ((nmax_all + 7) & ~7) <= kApSegMaxLd;
    for (int m = 0; m < M; ++m) {
        moff[m + 1] = moff[m] + (int64_t)nsz[m] * nsz[m];
        // 16-byte loads: 4 complex of the FP16 rows, 8 of the 8-bit ones
        ldv[m] = q8 ? (nsz[m] + 7) & ~7 : (nsz[m] + 3) & ~3;
        xoff[m + 1] = xoff[m] + (int64_t)own[m] * ldv[m];
        h->pc_own_max = std::max(h->pc_own_max, own[m]);
    }
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
    std::vector<int32_t> own_ptr_host;
    EMS_TRY(up(&h->pc_off, xoff.data(), (size_t)M));
    EMS_TRY(up(&h->pc_ld, ldv.data(), (size_t)M));
    {
        // owned-row list, subdomain entry -> cell, FP32 gather buffer
        std::vector<int32_t> optr(M + 1, 0), scell(sids.size());
        std::vector<int64_t> rsoff(M + 1, 0);
        for (int m = 0; m < M; ++m) {
            optr[m + 1] = optr[m] + own[m];
            rsoff[m + 1] = rsoff[m] + ldv[m];
            for (int q = sptr[m]; q < sptr[m + 1]; ++q) scell[q] = m;
        }
        if (optr[M] != h->n_unique) {
            set_error("preconditioner: %d owned rows for %d unknowns", optr[M], h->n_unique);
            return EMSURF_EINVAL;
        }
        EMS_TRY(up(&h->pc_own_ptr, optr.data(), optr.size()));
        own_ptr_host = optr;
        EMS_TRY(up(&h->pc_sub_cell, scell.data(), scell.size()));
        EMS_TRY(up(&h->pc_rs_off, rsoff.data(), (size_t)M));
        h->pc_rs_stride = rsoff[M];
        EMS_TRY(dev_alloc(h, (void**)&h->pc_rs, (size_t)h->max_rhs * rsoff[M] * sizeof(float2)));
        EMS_CUDA(cudaMemsetAsync(h->pc_rs, 0, (size_t)h->max_rhs * rsoff[M] * sizeof(float2), st));
    }
    // FP32 inverse rows: a create-time temporary (the apply keeps FP16 rows)
    EMS_CUDA(cudaMalloc(&h->pc_mat, (size_t)xoff[M] * sizeof(float2)));
    EMS_CUDA(cudaMemsetAsync(h->pc_mat, 0, (size_t)xoff[M] * sizeof(float2), st));   // row padding
    int64_t* d_luoff = nullptr;
    int32_t* d_perm = nullptr;
    float2* d_lu = nullptr;
    EMS_CUDA(cudaMalloc(&d_luoff, sizeof(int64_t) * M));
    EMS_CUDA(cudaMemcpyAsync(d_luoff, moff.data(), sizeof(int64_t) * M, cudaMemcpyHostToDevice, st));
    EMS_CUDA(cudaMalloc(&d_perm, sids.size() * sizeof(int32_t)));
    EMS_CUDA(cudaMalloc(&d_lu, (size_t)moff[M] * sizeof(float2)));
    // near offset tables |dx|, |dy| <= 2 -> [5][5][E][E] (zero outside the lattice)
    const size_t EE = (size_t)E * E;
    // (kept by the handle: emsurf_create_like builds its preconditioner from them)
    const double2* nL = h->near_L;
    const double2* nK = h->near_K;
    (void)EE;
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
    pc_assemble_kernel<<<dim3(M, 64), 256, 0, st>>>(d_lu, d_luoff, h->pc_n, h->pc_sub_ptr, h->pc_sub_ids,
                                                    h->d_inv_ptr, h->d_inv_ent, h->d_inv_sgn, nL, nK, Zt,
                                                    h->d_type_map, nx, E, co[0], co[1], co[2], co[3]);
    EMS_CUDA(cudaGetLastError());
    int* dstat = nullptr;
    EMS_CUDA(cudaMalloc(&dstat, sizeof(int) * M));
    EMS_CUDA(cudaMemsetAsync(dstat, 0, sizeof(int) * M, st));
    const size_t lsm = (size_t)h->pc_nmax * kLuNB * sizeof(float2);
    EMS_TRY(set_smem_once(pc_lu_kernel, lsm));
    pc_lu_kernel<<<M, kLuThreads, lsm, st>>>(d_lu, d_luoff, h->pc_n, h->pc_sub_ptr, d_perm, dstat);
    EMS_CUDA(cudaGetLastError());
    const size_t ism = (size_t)kInvNR * h->pc_nmax * sizeof(float2);
    EMS_TRY(set_smem_once(pc_invrows_kernel, ism));
    pc_invrows_kernel<<<dim3((h->pc_own_max + kInvNR - 1) / kInvNR, M), kInvThreads, ism, st>>>(
        d_lu, d_luoff, h->pc_n, h->pc_own, h->pc_sub_ptr, d_perm, h->pc_mat, h->pc_off, h->pc_ld);
    EMS_CUDA(cudaGetLastError());
    std::vector<int> hs(M);
    EMS_CUDA(cudaMemcpyAsync(hs.data(), dstat, sizeof(int) * M, cudaMemcpyDeviceToHost, st));
    EMS_CUDA(cudaStreamSynchronize(st));
    cudaFree(dstat);
    cudaFree(d_lu);
    cudaFree(d_perm);
    cudaFree(d_luoff);

    if (own_zt) cudaFree(Zt);
    for (int m = 0; m < M; ++m)
        if (hs[m]) {
            cudaFree(h->pc_mat);
            h->pc_mat = nullptr;
            set_error("preconditioner block of cell %d is singular", m);
            return EMSURF_EINVAL;
        }
    h->pc_elems = xoff[M];
    h->pc_sub_total = (int64_t)sids.size();
    // FP16 (or 8-bit) rows with a per-row scale for the apply
    EMS_TRY(dev_alloc(h, &h->pc_mat16, (size_t)xoff[M] * (q8 ? 2 : 4)));
    EMS_TRY(dev_alloc(h, (void**)&h->pc_rscale, (size_t)h->n_unique * sizeof(float)));
    if (q8)
        pc_to_int8_kernel<<<h->num_sms * 16, 256, 0, st>>>(h->pc_mat, h->pc_off, h->pc_ld, h->pc_own_ptr, M,
                                                           h->n_unique, reinterpret_cast<uchar2*>(h->pc_mat16),
                                                           h->pc_rscale);
    else
        pc_to_half_kernel<<<h->num_sms * 16, 256, 0, st>>>(h->pc_mat, h->pc_off, h->pc_ld, h->pc_own_ptr, M,
                                                           h->n_unique, reinterpret_cast<__half2*>(h->pc_mat16),
                                                           h->pc_rscale);
    h->pc_int8 = q8;
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    h->have_pc = true;
    // many rhs: the apply as tensor-core GEMMs (with the handle's tensor-core option)
    int st_tc = EMSURF_OK;
    if (h->have_tc && h->max_rhs >= kTcMinRhs) st_tc = pc_tc_build(h, own_ptr_host);
    EMS_CUDA(cudaStreamSynchronize(st));
    cudaFree(h->pc_mat);
    h->pc_mat = nullptr;
    return st_tc;
}

}  // namespace emsurf
