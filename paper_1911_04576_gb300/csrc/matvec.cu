// The FFT-accelerated product y = U_o^T [Z_eq + Z_o] U_o x (Eq. MVP).
//
// Layouts in HBM (P = px*py bins, E RWGs, K = 2E, R right-hand sides):
//   Bhat [P][2][E][E]  Fourier-domain L^, K^ blocks, source-major (j, i):
//                      the bin multiply gives each thread one test row i and
//                      streams a column j across the warp (coalesced);
//   Zt   [T][K][K]     macromodels transposed (k' outer, k contiguous);
//   Xg,Yg [P][R][K]    padded grids, lanes (r, k) contiguous;
//   Ymm  [R][M][K]     macromodel products.
//
// Storing only L^ and K^ (not the full K x K block) is the paper's storage
// count 2^{d+1} N_eq^2 M complex numbers (Sec. IV-C): B(d) repeats L and K
// in its four quarters (Eq. blockZo with the coefficients of the scaled
// EFIE/MFIE form).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace emsurf {

namespace {

constexpr int kMmSplit = 8;   // k' chunks of the macromodel product

// ------------------------------------------------ placement of the tables
// Bhat[bin(d)][op][j][i] = table_op(d)[i][j] for one chunk of offsets;
// stage holds [nchunk][2][E][E] complex128 (row-major i, j).
template <typename T2>
__global__ void place_blocks_kernel(T2* __restrict__ Bhat, const double2* __restrict__ stage,
                                    const int* __restrict__ bins, int nchunk, int E) {
    __shared__ double2 tile[32][33];
    const int o = blockIdx.z / 2, op = blockIdx.z % 2;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const double2* src = stage + ((size_t)o * 2 + op) * E * E;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < E && j < E) ? src[(size_t)i * E + j] : make_double2(0, 0);
    }
    __syncthreads();
    T2* dst = Bhat + ((size_t)bins[o] * 2 + op) * E * E;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < E && j < E) {
            const double2 v = tile[threadIdx.x][r];
            dst[(size_t)j * E + i] = mk<T2>(v.x, v.y);
        }
    }
}

// Zt[t][k'][k] = Z[t][k][k']
template <typename T2>
__global__ void transpose_mm_kernel(T2* __restrict__ Zt, const double2* __restrict__ Z, int K) {
    __shared__ double2 tile[32][33];
    const int t = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const double2* src = Z + (size_t)t * K * K;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = r0 + r, j = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < K && j < K) ? src[(size_t)i * K + j] : make_double2(0, 0);
    }
    __syncthreads();
    T2* dst = Zt + (size_t)t * K * K;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = c0 + r, i = r0 + threadIdx.x;
        if (i < K && j < K) {
            const double2 v = tile[threadIdx.x][r];
            dst[(size_t)j * K + i] = mk<T2>(v.x, v.y);
        }
    }
}

__global__ void round_kernel(float2* __restrict__ dst, const double2* __restrict__ src, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = src[e];
        dst[e] = make_float2((float)v.x, (float)v.y);
    }
}

// Reciprocity of the spectrum: with L(-d) = L(d)^T and K(-d) = K(d)^T the
// blocks of bins k and -k are transposes, L^(-k) = L^(k)^T and
// K^(-k) = K^(k)^T.  out[0] = max over both operators of
// |O^(-k)[i][j] - O^(k)[j][i]|, out[1] = max |O^| (as ordered bit patterns
// of non-negative doubles).
__global__ void reciprocity_kernel(const double2* __restrict__ B, const int32_t* __restrict__ partner,
                                   int E, size_t nbins, unsigned long long* __restrict__ out) {
    const size_t EE = (size_t)E * E, total = nbins * 2 * EE;
    double dmax = 0.0, vmax = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t bin = e / (2 * EE), rem = e % (2 * EE);
        const int op = (int)(rem / EE), j = (int)((rem % EE) / E), i = (int)(rem % E);
        const double2 a = B[e];
        const double2 b = B[((size_t)partner[bin] * 2 + op) * EE + (size_t)i * E + j];
        dmax = fmax(dmax, fmax(fabs(a.x - b.x), fabs(a.y - b.y)));
        vmax = fmax(vmax, fmax(fabs(a.x), fabs(a.y)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(vmax));
    }
}

// Mirror relation of the spectrum for one mirror g of the box (det g = -1):
// with L(g d) = P L(d) P^T and K(g d) = -P K(d) P^T the blocks of bins k and
// g k obey O^(g k)[pi(i)][pi(j)] = s_op sign(i) sign(j) O^(k)[i][j], s_L = 1,
// s_K = -1.  perm[n] = pi(n) | (sign(n) < 0) << 31; image[bin] = g k.
// out[0] = max deviation, out[1] = max |O^| (ordered bit patterns).
__global__ void mirror_check_kernel(const double2* __restrict__ B, const uint32_t* __restrict__ perm,
                                    const int32_t* __restrict__ image, int E, size_t nbins,
                                    unsigned long long* __restrict__ out) {
    const size_t EE = (size_t)E * E, total = nbins * 2 * EE;
    double dmax = 0.0, vmax = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t bin = e / (2 * EE), rem = e % (2 * EE);
        const int op = (int)(rem / EE), j = (int)((rem % EE) / E), i = (int)(rem % E);
        const uint32_t pi = perm[i], pj = perm[j];
        const double f = ((pi ^ pj) >> 31 ? -1.0 : 1.0) * (op ? -1.0 : 1.0);
        const double2 a = B[e];
        const double2 b = B[((size_t)image[bin] * 2 + op) * EE + (size_t)(pj & 0x7fffffffu) * E + (pi & 0x7fffffffu)];
        dmax = fmax(dmax, fmax(fabs(b.x - f * a.x), fabs(b.y - f * a.y)));
        vmax = fmax(vmax, fmax(fabs(a.x), fabs(a.y)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(vmax));
    }
}

// half spectrum: dst[s] = (float) B^(st_bin[s]) for the stored bins
__global__ void half_round_kernel(float2* __restrict__ dst, const double2* __restrict__ src,
                                  const int32_t* __restrict__ st_bin, size_t per_bin, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t s = e / per_bin, r = e % per_bin;
        const double2 v = src[(size_t)st_bin[s] * per_bin + r];
        dst[e] = make_float2((float)v.x, (float)v.y);
    }
}

// ------------------------------------------------ K2: bin multiply
// Y^(k) = B^(k) X^(k) with B = [[a L, b K], [g K, d L]]:
//   y_J = a L^ x_J + b K^ x_M,   y_M = g K^ x_J + d L^ x_M.
// One CTA per bin (grid-stride), one thread per test row i.
template <typename T2, int RB>
__global__ void binmul_kernel(const T2* __restrict__ Bhat, const T2* __restrict__ Xh,
                              T2* __restrict__ Yh, int E, int nbins, int R, int r0,
                              T2 ca, T2 cb, T2 cg, T2 cd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* xs = reinterpret_cast<T2*>(smem_raw);   // [RB][2E]
    const int K = 2 * E;
    const T2 zero = mk<T2>(0.0, 0.0);
    for (int bin = blockIdx.x; bin < nbins; bin += gridDim.x) {
        __syncthreads();
        const T2* X = Xh + (size_t)bin * R * K;
        for (int e = threadIdx.x; e < RB * K; e += blockDim.x) {
            const int r = e / K, k = e - (e / K) * K;
            xs[e] = (r0 + r < R) ? X[(size_t)(r0 + r) * K + k] : zero;
        }
        __syncthreads();
        const T2* Lt = Bhat + (size_t)bin * 2 * E * E;
        const T2* Kt = Lt + (size_t)E * E;
        for (int i = threadIdx.x; i < E; i += blockDim.x) {
            T2 lj[RB], lm[RB], kj[RB], km[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) lj[r] = lm[r] = kj[r] = km[r] = zero;
#pragma unroll 8
            for (int j = 0; j < E; ++j) {
                const T2 l = __ldg(Lt + (size_t)j * E + i);
                const T2 kk = __ldg(Kt + (size_t)j * E + i);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const T2 xj = xs[r * K + j];
                    const T2 xm = xs[r * K + E + j];
                    cfma(lj[r], l, xj);
                    cfma(lm[r], l, xm);
                    cfma(kj[r], kk, xj);
                    cfma(km[r], kk, xm);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (r0 + r < R) {
                    T2* Y = Yh + ((size_t)bin * R + r0 + r) * K;
                    Y[i] = cadd(cmul(ca, lj[r]), cmul(cb, km[r]));
                    Y[E + i] = cadd(cmul(cg, kj[r]), cmul(cd, lm[r]));
                }
            }
        }
    }
}

// ------------------------------------------------ K2, FP32, one rhs: TMA-fed
// Persistent CTAs walk their bins as a sequence of stages; a stage is a block
// of JB source columns j of L^T and K^T (two contiguous JB x E slabs, since j
// is the outer index), brought into a ring of kBmStages shared-memory slots
// by 1-D bulk asynchronous copies (cp.async.bulk) signalled on mbarriers.
// The first stage of a bin also brings X^(bin).  Warp 0 lane 0 issues the
// copies; the other warps own one test row i each and release a slot with an
// mbarrier arrive.  Every wait is bounded: on expiry the kernel sets *err,
// the producer waits (bounded) for its copies in flight, and all return.
constexpr int kBmJB = 8;
constexpr int kBmStages = 4;
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kWaitLimit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Exercises the expiry path of mbar_wait: waits on an mbarrier that nothing
// arrives on, with a short limit, and reports like the production kernels.
__global__ void wait_selftest_kernel(long long limit, int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, limit)) atomicExch(err, 3);
}
// the same with an L2 policy (l2_evict_first for data read once per product)
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__global__ void binmul_tma_kernel(const float2* __restrict__ Bhat, const float2* __restrict__ Xh,
                                  float2* __restrict__ Yh, int E, int nbins, float2 ca, float2 cb,
                                  float2 cg, float2 cd, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stage_elems = 2 * kBmJB * E;
    float2* sbuf = reinterpret_cast<float2*>(smem_raw);
    float2* xbuf = sbuf + (size_t)kBmStages * stage_elems;      // [2][2E]
    uint64_t* full = reinterpret_cast<uint64_t*>(xbuf + 4 * E);
    uint64_t* empty = full + kBmStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (E + 31) / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nloc = (nbins - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int nj = (E + kBmJB - 1) / kBmJB;
    const long long total = (long long)nloc * nj;
    if (warp == 0) {
        if (lane != 0) return;
        const uint64_t pol = l2_evict_first();
        long long issued = 0;
        bool ok = true;
        for (long long q = 0; q < total; ++q) {
            const int s = (int)(q % kBmStages);
            if (q >= kBmStages && !mbar_wait(&empty[s], (uint32_t)((q / kBmStages - 1) & 1))) {
                ok = false;
                break;
            }
            const int t = (int)(q / nj), jb = (int)(q % nj);
            const int bin = (int)blockIdx.x + t * (int)gridDim.x;
            const int j0 = jb * kBmJB, jn = min(kBmJB, E - j0);
            const uint32_t bytes_op = (uint32_t)(jn * E * sizeof(float2));
            const uint32_t bytes_x = (uint32_t)(2 * E * sizeof(float2));
            mbar_expect_tx(&full[s], 2 * bytes_op + (jb == 0 ? bytes_x : 0u));
            const float2* src = Bhat + (size_t)bin * 2 * E * E + (size_t)j0 * E;
            float2* dst = sbuf + (size_t)s * stage_elems;
            bulk_g2s_hint(dst, src, bytes_op, &full[s], pol);
            bulk_g2s_hint(dst + kBmJB * E, src + (size_t)E * E, bytes_op, &full[s], pol);
            if (jb == 0) bulk_g2s(xbuf + (t & 1) * 2 * E, Xh + (size_t)bin * 2 * E, bytes_x, &full[s]);
            issued = q + 1;
        }
        if (!ok) {
            atomicExch(err, 1);
            // wait (bounded) for the copies still in flight before leaving
            for (long long q = (issued > kBmStages ? issued - kBmStages : 0); q < issued; ++q)
                mbar_wait(&full[q % kBmStages], (uint32_t)((q / kBmStages) & 1));
        }
        return;
    }
    const int i = (warp - 1) * 32 + lane;
    float2 lj = make_float2(0.f, 0.f), lm = lj, kj = lj, km = lj;
    for (long long q = 0; q < total; ++q) {
        const int s = (int)(q % kBmStages);
        const int t = (int)(q / nj), jb = (int)(q % nj);
        if (!mbar_wait(&full[s], (uint32_t)((q / kBmStages) & 1))) {
            atomicExch(err, 1);
            return;
        }
        if (jb == 0) lj = lm = kj = km = make_float2(0.f, 0.f);
        const float2* Ls = sbuf + (size_t)s * stage_elems;
        const float2* Ks = Ls + kBmJB * E;
        const float2* xs = xbuf + (t & 1) * 2 * E;
        const int j0 = jb * kBmJB, jn = min(kBmJB, E - j0);
        if (i < E) {
#pragma unroll
            for (int jj = 0; jj < kBmJB; ++jj) {
                if (jj < jn) {
                    const float2 l = Ls[jj * E + i];
                    const float2 k = Ks[jj * E + i];
                    const float2 xj = xs[j0 + jj];
                    const float2 xm = xs[E + j0 + jj];
                    cfma(lj, l, xj);
                    cfma(lm, l, xm);
                    cfma(kj, k, xj);
                    cfma(km, k, xm);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (jb == nj - 1 && i < E) {
            const int bin = (int)blockIdx.x + t * (int)gridDim.x;
            float2* Y = Yh + (size_t)bin * 2 * E;
            Y[i] = cadd(cmul(ca, lj), cmul(cb, km));
            Y[E + i] = cadd(cmul(cg, kj), cmul(cd, lm));
        }
    }
}

size_t binmul_tma_smem(int E) {
    return (size_t)kBmStages * 2 * kBmJB * E * sizeof(float2) + 4ull * E * sizeof(float2) +
           2ull * kBmStages * sizeof(uint64_t);
}

// ------------------------------------------------ K2, FP64 accuracy from FP32 arithmetic, one rhs
// The FP64 bin multiply is bound by this part's FP64 rate (~1/60 of FP32).
// Here every FP64 value v is held as a pair of floats, hi = rn(v) and
// lo = rn(v - hi) (|v - hi - lo| <= 2^-48 |v|), and each complex product is
// accumulated in double-single arithmetic: the rounding error of hi*hi is
// recovered exactly with an FMA, the cross terms hi*lo + lo*hi are added to
// it, and the partial sums are pairs (s, c) updated with Knuth's TwoSum, so
// each product term carries a relative error of a few 2^-48 (the lo*lo term,
// ~2^-48, is dropped).  The row sums are turned into FP64 at the end.  The
// spectrum planes hold the same bytes as the FP64 spectrum; one thread per
// test row as in binmul_tma_kernel, kDsJB-column slabs (hi and lo of L^ and
// K^) in a kDsStages-deep ring fed by bulk copies.
constexpr int kDsJB = 6;
constexpr int kDsStages = 3;

// (hi, lo) += (ah + al)(bh + bl); no operation is contracted or reassociated
__device__ __forceinline__ void ds_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);           // ah bh - p, exactly
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(hi, p);          // TwoSum(hi, p) = s + t exactly
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    lo = __fadd_rn(lo, __fadd_rn(t, e));
    hi = s;
}

struct DsC {   // complex double-single accumulator
    float rh, rl, ih, il;
};
__device__ __forceinline__ void ds_cmac(DsC& a, float2 xh, float2 xl, float2 bh, float2 bl) {
    ds_mac(a.rh, a.rl, xh.x, xl.x, bh.x, bl.x);
    ds_mac(a.rh, a.rl, -xh.y, -xl.y, bh.y, bl.y);
    ds_mac(a.ih, a.il, xh.x, xl.x, bh.y, bl.y);
    ds_mac(a.ih, a.il, xh.y, xl.y, bh.x, bl.x);
}
__device__ __forceinline__ double2 ds_value(const DsC& a) {
    return make_double2((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il);
}

// out[b][0][r] = rn(s v), out[b][1][r] = rn(s v - out[b][0][r]) for v = in[b][r],
// blocks b of `chunk` complex values; s = *scale (a power of two, exact), or 1
__global__ void split_hilo_kernel(float2* __restrict__ out, const double2* __restrict__ in, size_t chunk,
                                  size_t total, const double* __restrict__ scale) {
    const double sc = scale ? *scale : 1.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / chunk, r = e - b * chunk;
        const double2 v = make_double2(sc * in[e].x, sc * in[e].y);
        const float2 hi = make_float2((float)v.x, (float)v.y);
        const float2 lo = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
        out[b * 2 * chunk + r] = hi;
        out[b * 2 * chunk + chunk + r] = lo;
    }
}

// scale[r] = 2^-e with 2^(e-1) <= max over the r-th vector of |re|, |im| < 2^e
// (1 when the vector is zero or not finite): after it the vector's largest
// component lies in [0.5, 1), far from FP32 overflow, and FP32 subnormals only
// touch parts below 2^-100 of the largest.  Grid (blocks, R): every block
// folds its maximum into maxbits[r] (the bit patterns of non-negative doubles
// order like the values); the last block of rhs r to arrive (arrival counter)
// writes the scale and resets maxbits[r] and count[r] for the next product.
__global__ void __launch_bounds__(256) pow2_scale_kernel(const double2* __restrict__ v, size_t len,
                                                         unsigned long long* __restrict__ maxbits,
                                                         unsigned* __restrict__ count, double* __restrict__ scale) {
    __shared__ double s_m[256];
    __shared__ bool s_last;
    const int r = blockIdx.y;
    const double2* b = v + (size_t)r * len;
    double m = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fmax(fabs(b[e].x), fabs(b[e].y)));
    s_m[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s_m[threadIdx.x] = fmax(s_m[threadIdx.x], s_m[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(&maxbits[r], (unsigned long long)__double_as_longlong(s_m[0]));
        __threadfence();
        s_last = atomicAdd(&count[r], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double mx = __longlong_as_double((long long)atomicExch(&maxbits[r], 0ull));
        count[r] = 0u;
        scale[r] = (mx > 0.0 && mx <= 1.7e308) ? ldexp(1.0, -(ilogb(mx) + 1)) : 1.0;
    }
}

// grid-wide variant for one large array: per-CTA maxima in part[], then one CTA
__global__ void __launch_bounds__(256) absmax_part_kernel(const double2* __restrict__ v, size_t n,
                                                          double* __restrict__ part) {
    __shared__ double s_m[256];
    double m = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fmax(fabs(v[e].x), fabs(v[e].y)));
    s_m[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s_m[threadIdx.x] = fmax(s_m[threadIdx.x], s_m[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s_m[0];
}

// planes: [bin][hi, lo][op][j][i] float2; xs: [bin][hi, lo][2E]; Yh: [bin][2E] FP64
__global__ void binmul_ds_kernel(const float2* __restrict__ planes, const float2* __restrict__ xs,
                                 double2* __restrict__ Yh, int E, int nbins, double2 ca, double2 cb,
                                 double2 cg, double2 cd, int* __restrict__ err,
                                 const double* __restrict__ scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stage_elems = 4 * kDsJB * E;      // [hi, lo][L, K][kDsJB][E]
    float2* sbuf = reinterpret_cast<float2*>(smem_raw);
    float2* xbuf = sbuf + (size_t)kDsStages * stage_elems;      // [2 buffers][hi, lo][2E]
    uint64_t* full = reinterpret_cast<uint64_t*>(xbuf + 8 * E);
    uint64_t* empty = full + kDsStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (E + 31) / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kDsStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nloc = (nbins - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int nj = (E + kDsJB - 1) / kDsJB;
    const long long total = (long long)nloc * nj;
    const size_t EE = (size_t)E * E;
    if (warp == 0) {
        if (lane != 0) return;
        const uint64_t pol = l2_evict_first();
        const uint32_t bytes_x = (uint32_t)(4 * E * sizeof(float2));
        int s = 0, jb = 0, t = 0;
        uint32_t ph = 0;
        long long issued = 0;
        bool ok = true;
        for (long long q = 0; q < total; ++q) {
            if (q >= kDsStages && !mbar_wait(&empty[s], ph ^ 1u)) {
                ok = false;
                break;
            }
            const int bin = (int)blockIdx.x + t * (int)gridDim.x;
            const int j0 = jb * kDsJB, jn = min(kDsJB, E - j0);
            const uint32_t bytes_op = (uint32_t)(jn * E * sizeof(float2));
            mbar_expect_tx(&full[s], 4 * bytes_op + (jb == 0 ? bytes_x : 0u));
            float2* dst = sbuf + (size_t)s * stage_elems;
            for (int pl = 0; pl < 2; ++pl)
                for (int o = 0; o < 2; ++o)
                    bulk_g2s_hint(dst + (pl * 2 + o) * kDsJB * E,
                                  planes + (((size_t)bin * 2 + pl) * 2 + o) * EE + (size_t)j0 * E, bytes_op,
                                  &full[s], pol);
            if (jb == 0) bulk_g2s(xbuf + (t & 1) * 4 * E, xs + (size_t)bin * 4 * E, bytes_x, &full[s]);
            issued = q + 1;
            if (++s == kDsStages) { s = 0; ph ^= 1u; }
            if (++jb == nj) { jb = 0; ++t; }
        }
        if (!ok) {
            atomicExch(err, 1);
            for (long long u = (issued > kDsStages ? issued - kDsStages : 0); u < issued; ++u)
                mbar_wait(&full[u % kDsStages], (uint32_t)((u / kDsStages) & 1));
        }
        return;
    }
    const int i = (warp - 1) * 32 + lane;
    DsC lj{0.f, 0.f, 0.f, 0.f}, lm = lj, kj = lj, km = lj;
    int s = 0, jb = 0, t = 0;
    uint32_t ph = 0;
    for (long long q = 0; q < total; ++q) {
        if (!mbar_wait(&full[s], ph)) {
            atomicExch(err, 1);
            return;
        }
        const float2* S = sbuf + (size_t)s * stage_elems;
        const float2* X = xbuf + (t & 1) * 4 * E;       // [hi, lo][2E]
        const int j0 = jb * kDsJB, jn = min(kDsJB, E - j0);
        if (i < E) {
#pragma unroll
            for (int jj = 0; jj < kDsJB; ++jj) {
                if (jj < jn) {
                    const float2 lh = S[(0 * kDsJB + jj) * E + i], kh = S[(1 * kDsJB + jj) * E + i];
                    const float2 ll = S[(2 * kDsJB + jj) * E + i], kl = S[(3 * kDsJB + jj) * E + i];
                    const float2 xjh = X[j0 + jj], xmh = X[E + j0 + jj];
                    const float2 xjl = X[2 * E + j0 + jj], xml = X[3 * E + j0 + jj];
                    ds_cmac(lj, xjh, xjl, lh, ll);
                    ds_cmac(lm, xmh, xml, lh, ll);
                    ds_cmac(kj, xjh, xjl, kh, kl);
                    ds_cmac(km, xmh, xml, kh, kl);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (jb == nj - 1) {
            if (i < E) {
                const int bin = (int)blockIdx.x + t * (int)gridDim.x;
                double2* Y = Yh + (size_t)bin * 2 * E;
                const double u = 1.0 / (scale[0] * scale[2]);       // exact: powers of two
                const double2 yj = cadd(cmul(ca, ds_value(lj)), cmul(cb, ds_value(km)));
                const double2 ym = cadd(cmul(cg, ds_value(kj)), cmul(cd, ds_value(lm)));
                Y[i] = make_double2(u * yj.x, u * yj.y);
                Y[E + i] = make_double2(u * ym.x, u * ym.y);
            }
            lj = lm = kj = km = DsC{0.f, 0.f, 0.f, 0.f};
        }
        if (++s == kDsStages) { s = 0; ph ^= 1u; }
        if (++jb == nj) { jb = 0; ++t; }
    }
}

// Several rhs: RB of them per pass share each load of the hi/lo planes (the
// register-blocked form of binmul_kernel); X^ is split into hi/lo while it is
// staged in shared memory.  Compute-bound (about 60 FP32 operations per
// complex multiply-add), so the planes are streamed once per RB rhs.
template <int RB>
__global__ void binmul_ds_multi_kernel(const float2* __restrict__ planes, const double2* __restrict__ Xh,
                                       double2* __restrict__ Yh, int E, int nbins, int R, int r0,
                                       double2 ca, double2 cb, double2 cg, double2 cd,
                                       const double* __restrict__ scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* xh = reinterpret_cast<float2*>(smem_raw);   // [RB][2E] hi
    float2* xl = xh + (size_t)RB * 2 * E;               // [RB][2E] lo
    const int K = 2 * E;
    const size_t EE = (size_t)E * E;
    for (int bin = blockIdx.x; bin < nbins; bin += gridDim.x) {
        __syncthreads();
        const double2* X = Xh + (size_t)bin * R * K;
        for (int e = threadIdx.x; e < RB * K; e += blockDim.x) {
            const int r = e / K, k = e - r * K;
            double2 v = make_double2(0.0, 0.0);
            if (r0 + r < R) {
                const double sc = scale[2 + r0 + r];
                v = X[(size_t)(r0 + r) * K + k];
                v = make_double2(sc * v.x, sc * v.y);
            }
            const float2 hi = make_float2((float)v.x, (float)v.y);
            xh[e] = hi;
            xl[e] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
        }
        __syncthreads();
        const float2* Lh = planes + (size_t)bin * 4 * EE;
        const float2* Kh = Lh + EE;
        const float2* Ll = Lh + 2 * EE;
        const float2* Kl = Lh + 3 * EE;
        for (int i = threadIdx.x; i < E; i += blockDim.x) {
            DsC lj[RB], lm[RB], kj[RB], km[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) lj[r] = lm[r] = kj[r] = km[r] = DsC{0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
            for (int j = 0; j < E; ++j) {
                const size_t o = (size_t)j * E + i;
                const float2 lh = __ldg(Lh + o), kh = __ldg(Kh + o), ll = __ldg(Ll + o), kl = __ldg(Kl + o);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const float2 xjh = xh[r * K + j], xmh = xh[r * K + E + j];
                    const float2 xjl = xl[r * K + j], xml = xl[r * K + E + j];
                    ds_cmac(lj[r], xjh, xjl, lh, ll);
                    ds_cmac(lm[r], xmh, xml, lh, ll);
                    ds_cmac(kj[r], xjh, xjl, kh, kl);
                    ds_cmac(km[r], xmh, xml, kh, kl);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (r0 + r < R) {
                    double2* Y = Yh + ((size_t)bin * R + r0 + r) * K;
                    const double u = 1.0 / (scale[0] * scale[2 + r0 + r]);
                    const double2 yj = cadd(cmul(ca, ds_value(lj[r])), cmul(cb, ds_value(km[r])));
                    const double2 ym = cadd(cmul(cg, ds_value(kj[r])), cmul(cd, ds_value(lm[r])));
                    Y[i] = make_double2(u * yj.x, u * yj.y);
                    Y[E + i] = make_double2(u * ym.x, u * ym.y);
                }
            }
        }
    }
}

size_t binmul_ds_smem(int E) {
    return (size_t)kDsStages * 4 * kDsJB * E * sizeof(float2) + 8ull * E * sizeof(float2) +
           2ull * kDsStages * sizeof(uint64_t);
}

// ------------------------------------------------ K2, FP32, one rhs, half spectrum
// With reciprocal tables L^(-k) = L^(k)^T and K^(-k) = K^(k)^T, so only one
// bin k of each pair (k, -k) is stored and its blocks serve both:
// y(k) = B^(k) x(k) (one thread per test row, as in binmul_tma_kernel) and
// y_J(-k)[j] = a sum_i L[j][i] x_J(-k)[i] + b sum_i K[j][i] x_M(-k)[i]
// (y_M(-k) likewise with g, d), dot products along the contiguous test index
// of the slab's columns, computed by kPairColWarps further warps (two
// columns per warp, a warp reduction per slab).  Each stored slab is read
// from HBM once for both bins.  Self-paired bins (k = -k) take only the
// first product.
//
// Work split: the Q = nst * nj slabs (stored bins in order, nj slabs each)
// are cut into gridDim.x contiguous ranges whose lengths differ by at most
// one, so every CTA streams the same number of bytes and a bin may straddle
// CTAs.  A y(-k) output is complete within its slab.  The y(k) row sums of a
// bin that is not whole in one CTA are written per row warp as partials,
// part[cta][slot][2E] (slot 0: the range's first bin, 1: its last), and the
// warp whose arrival completes that (bin, warp) counter adds the partials
// of all contributing CTAs in CTA order (a deterministic sum), writes Y^ and
// resets the counter for the next launch.  No wait depends on another CTA.
constexpr int kPairStages = 3;     // ring depth
constexpr int kPairJB = 12;         // slab width (source columns per stage)
constexpr int kPairColWarps = 6;    // y(-k) warps
constexpr int kPairCpw = kPairJB / kPairColWarps;   // slab columns per y(-k) warp
constexpr int kPairNv = 8 * kPairCpw;               // floats reduced per lane and slab
constexpr int kPairUnroll = 5;      // row pairs per lane in flight in a y(-k) warp
constexpr int kPairMaxThreads = 576;
static_assert(kPairCpw * kPairColWarps == kPairJB && (kPairCpw == 1 || kPairCpw == 2),
              "one or two slab columns per y(-k) warp");

// the CTA whose slab range holds slab q (ranges [b Q / G, (b + 1) Q / G))
__device__ __forceinline__ int pair_cta_of(long long q, long long Q, int G) {
    return (int)(((q + 1) * G - 1) / Q);
}

__global__ void __launch_bounds__(kPairMaxThreads, 1) binmul_tma_pair_kernel(const float2* __restrict__ Bhat, const float2* __restrict__ Xh,
                                       float2* __restrict__ Yh, const int32_t* __restrict__ st_bin,
                                       const int32_t* __restrict__ st_part, int E, int nst, float2 ca,
                                       float2 cb, float2 cg, float2 cd, float2* __restrict__ part,
                                       int* __restrict__ cnt, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stage_elems = 2 * kPairJB * E;
    float2* sbuf = reinterpret_cast<float2*>(smem_raw);
    float2* xbuf = sbuf + (size_t)kPairStages * stage_elems;      // [2 buffers][x(k), x(-k)][2E]
    uint64_t* full = reinterpret_cast<uint64_t*>(xbuf + 8 * E);
    uint64_t* empty = full + kPairStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (E + 31) / 32;        // warps 1..ncw: y(k); the next kPairColWarps warps: y(-k)
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPairStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw + kPairColWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nj = (E + kPairJB - 1) / kPairJB;
    const int G = (int)gridDim.x;
    const long long Q = (long long)nst * nj;
    const long long q0 = (long long)blockIdx.x * Q / G, q1 = (long long)(blockIdx.x + 1) * Q / G;
    if (q0 >= q1) return;
    // position of the range's first slab; every role advances (s, ph, sb, jb,
    // t) by one slab per step (t counts the bins met, for the x double buffer)
    const int sb0 = (int)(q0 / nj), jb0 = (int)(q0 % nj);
    if (warp == 0) {
        if (lane != 0) return;
        const uint64_t pol = l2_evict_first();
        const uint32_t bytes_x = (uint32_t)(2 * E * sizeof(float2));
        int s = 0, sb = sb0, jb = jb0, t = 0;
        uint32_t ph = 0;
        long long issued = 0;
        bool ok = true;
        for (long long q = q0; q < q1; ++q) {
            if (q - q0 >= kPairStages && !mbar_wait(&empty[s], ph ^ 1u)) {
                ok = false;
                break;
            }
            const int j0 = jb * kPairJB, jn = min(kPairJB, E - j0);
            const uint32_t bytes_op = (uint32_t)(jn * E * sizeof(float2));
            const bool newbin = jb == 0 || q == q0;
            int bin = 0, prt = 0;
            if (newbin) {
                bin = st_bin[sb];
                prt = st_part[sb];
            }
            const uint32_t xb = newbin ? (prt != bin ? 2 * bytes_x : bytes_x) : 0u;
            mbar_expect_tx(&full[s], 2 * bytes_op + xb);
            const float2* src = Bhat + (size_t)sb * 2 * E * E + (size_t)j0 * E;
            float2* dst = sbuf + (size_t)s * stage_elems;
            bulk_g2s_hint(dst, src, bytes_op, &full[s], pol);
            bulk_g2s_hint(dst + kPairJB * E, src + (size_t)E * E, bytes_op, &full[s], pol);
            if (newbin) {
                float2* xd = xbuf + (t & 1) * 4 * E;
                bulk_g2s(xd, Xh + (size_t)bin * 2 * E, bytes_x, &full[s]);
                if (prt != bin) bulk_g2s(xd + 2 * E, Xh + (size_t)prt * 2 * E, bytes_x, &full[s]);
            }
            issued = q - q0 + 1;
            if (++s == kPairStages) { s = 0; ph ^= 1u; }
            if (++jb == nj) { jb = 0; ++sb; ++t; }
        }
        if (!ok) {
            atomicExch(err, 1);
            for (long long u = (issued > kPairStages ? issued - kPairStages : 0); u < issued; ++u)
                mbar_wait(&full[u % kPairStages], (uint32_t)((u / kPairStages) & 1));
        }
        return;
    }
    if (warp > ncw) {
        // ---- y(-k): columns cw + u kPairColWarps (u < kPairCpw) of every
        // slab, rows in pairs over the lanes
        const int cw = warp - ncw - 1;
        int s = 0, sb = sb0, jb = jb0, t = 0;
        uint32_t ph = 0;
        int bin = st_bin[sb], prt = st_part[sb];
        // after the reduce-scatter lane l holds value l >> (5 - log2 kPairNv);
        // lanes 0 .. 2 kPairCpw - 1 then gather the two complex sums of their
        // output (column u = l >> 1, J for even l, M for odd l)
        const int lo = lane & (2 * kPairCpw - 1), uo = lo >> 1;
        const int ip = 8 * uo + ((lo & 1) ? 4 : 0), iq = 8 * uo + ((lo & 1) ? 2 : 6);
        constexpr int kSpan = 32 / kPairNv;          // lanes per reduced value
        const float2 cP = (lo & 1) ? cg : ca, cQ = (lo & 1) ? cd : cb;
        const int cme = cw + uo * kPairColWarps;
        for (long long q = q0; q < q1; ++q) {
            if (!mbar_wait(&full[s], ph)) {
                atomicExch(err, 1);
                return;
            }
            if (prt != bin) {
                const int j0 = jb * kPairJB, jn = min(kPairJB, E - j0);
                const float2* Ls = sbuf + (size_t)s * stage_elems;
                const float2* xp = xbuf + (t & 1) * 4 * E + 2 * E;
                // a[u][pj, pm, qj, qm]: L x_J, L x_M, K x_J, K x_M of column u
                float2 a[kPairCpw][4];
#pragma unroll
                for (int u = 0; u < kPairCpw; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) a[u][v] = make_float2(0.f, 0.f);
                // rows in pairs (16-byte loads), kPairUnroll pairs per lane in
                // flight; columns past jn hold stale data that is read but never
                // written out
                for (int rb = 0; rb < E; rb += 64 * kPairUnroll) {
#pragma unroll
                    for (int it = 0; it < kPairUnroll; ++it) {
                        const int r = rb + 64 * it + 2 * lane;
                        if (r < E) {
                            const float4 xj = *reinterpret_cast<const float4*>(xp + r);
                            const float4 xm = *reinterpret_cast<const float4*>(xp + E + r);
                            const float2 xj0 = make_float2(xj.x, xj.y), xj1 = make_float2(xj.z, xj.w);
                            const float2 xm0 = make_float2(xm.x, xm.y), xm1 = make_float2(xm.z, xm.w);
#pragma unroll
                            for (int u = 0; u < kPairCpw; ++u) {
                                const float2* Lc = Ls + (cw + u * kPairColWarps) * E;
                                const float4 l = *reinterpret_cast<const float4*>(Lc + r);
                                const float4 k = *reinterpret_cast<const float4*>(Lc + kPairJB * E + r);
                                const float2 l0 = make_float2(l.x, l.y), l1 = make_float2(l.z, l.w);
                                const float2 k0 = make_float2(k.x, k.y), k1 = make_float2(k.z, k.w);
                                cfma(a[u][0], l0, xj0);
                                cfma(a[u][1], l0, xm0);
                                cfma(a[u][2], k0, xj0);
                                cfma(a[u][3], k0, xm0);
                                cfma(a[u][0], l1, xj1);
                                cfma(a[u][1], l1, xm1);
                                cfma(a[u][2], k1, xj1);
                                cfma(a[u][3], k1, xm1);
                            }
                        }
                    }
                }
                // kPairNv floats per lane -> reduce-scatter butterfly (half of
                // the values cross at each distance 16, 8, ...), then all-reduce
                // over the remaining distances
                float v[kPairNv];
#pragma unroll
                for (int u = 0; u < kPairCpw; ++u)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        v[8 * u + 2 * c] = a[u][c].x;
                        v[8 * u + 2 * c + 1] = a[u][c].y;
                    }
#pragma unroll
                for (int n = kPairNv, D = 16; n > 1; n >>= 1, D >>= 1) {
                    const bool up = lane & D;
#pragma unroll
                    for (int c = 0; c < n / 2; ++c) {
                        const float send = up ? v[c] : v[c + n / 2];
                        const float keep = up ? v[c + n / 2] : v[c];
                        v[c] = keep + __shfl_xor_sync(0xffffffffu, send, D);
                    }
                }
                float w1 = v[0];
#pragma unroll
                for (int D = 16 / kPairNv; D >= 1; D >>= 1) w1 += __shfl_xor_sync(0xffffffffu, w1, D);
                const float px = __shfl_sync(0xffffffffu, w1, kSpan * ip);
                const float py = __shfl_sync(0xffffffffu, w1, kSpan * (ip + 1));
                const float qx = __shfl_sync(0xffffffffu, w1, kSpan * iq);
                const float qy = __shfl_sync(0xffffffffu, w1, kSpan * (iq + 1));
                if (lane < 2 * kPairCpw && cme < jn) {
                    float2* Y = Yh + (size_t)prt * 2 * E + (lo & 1) * E;
                    Y[j0 + cme] = cadd(cmul(cP, make_float2(px, py)), cmul(cQ, make_float2(qx, qy)));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == kPairStages) { s = 0; ph ^= 1u; }
            if (++jb == nj) {
                jb = 0;
                ++sb;
                ++t;
                if (q + 1 < q1) {
                    bin = st_bin[sb];
                    prt = st_part[sb];
                }
            }
        }
        return;
    }
    // ---- y(k) = B^(k) x(k): one thread per test row
    const int w = warp - 1;
    const int i = w * 32 + lane;
    int s = 0, sb = sb0, jb = jb0, t = 0;
    uint32_t ph = 0;
    long long qb = (long long)sb0 * nj;     // first slab of bin sb
    float2 lj = make_float2(0.f, 0.f), lm = lj, kj = lj, km = lj;
    for (long long q = q0; q < q1; ++q) {
        if (!mbar_wait(&full[s], ph)) {
            atomicExch(err, 1);
            return;
        }
        const float2* Ls = sbuf + (size_t)s * stage_elems;
        const float2* Ks = Ls + kPairJB * E;
        const float2* xs = xbuf + (t & 1) * 4 * E;
        const int j0 = jb * kPairJB, jn = min(kPairJB, E - j0);
        if (i < E) {
            // x(k) of the slab's columns (broadcast reads, two complex per 16 bytes)
            float2 xjv[kPairJB], xmv[kPairJB];
            if (jn == kPairJB) {
                const float4* xj4 = reinterpret_cast<const float4*>(xs + j0);
                const float4* xm4 = reinterpret_cast<const float4*>(xs + E + j0);
#pragma unroll
                for (int p = 0; p < kPairJB / 2; ++p) {
                    const float4 a = xj4[p], b = xm4[p];
                    xjv[2 * p] = make_float2(a.x, a.y);
                    xjv[2 * p + 1] = make_float2(a.z, a.w);
                    xmv[2 * p] = make_float2(b.x, b.y);
                    xmv[2 * p + 1] = make_float2(b.z, b.w);
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < kPairJB; ++jj) {
                    xjv[jj] = jj < jn ? xs[j0 + jj] : make_float2(0.f, 0.f);
                    xmv[jj] = jj < jn ? xs[E + j0 + jj] : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int jj = 0; jj < kPairJB; ++jj) {
                if (jj < jn) {
                    const float2 l = Ls[jj * E + i];
                    const float2 k = Ks[jj * E + i];
                    cfma(lj, l, xjv[jj]);
                    cfma(lm, l, xmv[jj]);
                    cfma(kj, k, xjv[jj]);
                    cfma(km, k, xmv[jj]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (jb == nj - 1 || q == q1 - 1) {
            // this CTA's part of bin sb ends here
            const float2 y0 = cadd(cmul(ca, lj), cmul(cb, km));
            const float2 y1 = cadd(cmul(cg, kj), cmul(cd, lm));
            float2* Y = Yh + (size_t)st_bin[sb] * 2 * E;
            if (qb >= q0 && jb == nj - 1) {
                if (i < E) {
                    Y[i] = y0;
                    Y[E + i] = y1;
                }
            } else {
                float2* P = part + ((size_t)blockIdx.x * 2 + (t == 0 ? 0 : 1)) * 2 * E;
                if (i < E) {
                    P[i] = y0;
                    P[E + i] = y1;
                }
                __threadfence();
                __syncwarp();
                const int bf = pair_cta_of(qb, Q, G), bl = pair_cta_of(qb + nj - 1, Q, G);
                int* c = cnt + (size_t)sb * ncw + w;
                int old = 0;
                if (lane == 0) old = atomicAdd(c, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == bl - bf) {
                    // every contributor has written its partial
                    if (lane == 0) *c = 0;
                    __threadfence();
                    if (i < E) {
                        float2 a0 = make_float2(0.f, 0.f), a1 = a0;
                        for (int b = bf; b <= bl; ++b) {
                            const int sl = ((long long)b * Q / G) / nj == sb ? 0 : 1;
                            const float2* Pb = part + ((size_t)b * 2 + sl) * 2 * E;
                            a0 = cadd(a0, __ldcg(Pb + i));
                            a1 = cadd(a1, __ldcg(Pb + E + i));
                        }
                        Y[i] = a0;
                        Y[E + i] = a1;
                    }
                }
            }
            lj = lm = kj = km = make_float2(0.f, 0.f);
        }
        if (++s == kPairStages) { s = 0; ph ^= 1u; }
        if (++jb == nj) {
            jb = 0;
            ++sb;
            ++t;
            qb += nj;
        }
    }
}

size_t binmul_tma_pair_smem(int E) {
    return (size_t)kPairStages * 2 * kPairJB * E * sizeof(float2) + 8ull * E * sizeof(float2) +
           2ull * kPairStages * sizeof(uint64_t);
}

// ------------------------------------------------ K2, FP32, one rhs, mirror orbits
// With a mirror-symmetric box (union-jack mesh) the offset tables obey
// L(g d) = P_g L(d) P_g^T and K(g d) = det(g) P_g K(d) P_g^T for every g of
// the mirror group (x -> -x, y -> -y, and x <-> y on a square lattice), so
// the FFT-domain blocks of the bins g k of one orbit are
// B^(g k) = T_g B^(k) T_g^T, T_g = diag(P_g, det(g) P_g) on (J, M).  Only one
// bin k of each orbit is stored; with x~_j = T_g^T x(g k) gathered in shared
// memory, the bins of the orbit are G products with the same blocks:
// y(g k) = T_g B^(k) x~_j, one thread per test row i and G accumulator sets,
// so each stored slab is read from HBM once for all bins of its orbit.
// Work split, partial sums of straddling bins and their counters as in the
// pair kernel; the partials hold the unpermuted sums, the completing warp
// scatters y(g k) = T_g y~.
//
// Tables: orb_bin[s][j] the bin of slot j of stored bin s (-1: the orbit has
// fewer than G bins), orb_elem[s][j] its group element, orb_perm[e][n] the
// signed index of T_e: x~[n] = sign x[idx], y[idx] = sign y~[n], encoded as
// idx | (sign < 0) << 31.
constexpr int kOrbStages = 3;
// NT consumer threads per test row, each with G / NT accumulator sets (4):
// enough warps per SM to hide the shared-memory latency of the FMA stream
template <int NT>
constexpr int orb_max_threads() { return NT == 1 ? 384 : 640; }

template <int G, int JB, int NT>
__global__ void __launch_bounds__(orb_max_threads<NT>(), 1)
binmul_orbit_kernel(const float2* __restrict__ Bhat, const float2* __restrict__ Xh, float2* __restrict__ Yh,
                    const int32_t* __restrict__ orb_bin, const int32_t* __restrict__ orb_elem,
                    const uint32_t* __restrict__ orb_perm, int E, int nst, int n_elem, float2 ca, float2 cb,
                    float2 cg, float2 cd, float2* __restrict__ part, int* __restrict__ cnt,
                    int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stage_elems = 2 * JB * E;
    const int E2 = 2 * E;
    float2* sbuf = reinterpret_cast<float2*>(smem_raw);
    float2* xbuf = sbuf + (size_t)kOrbStages * stage_elems;         // [2][G][2E]
    uint32_t* ptab = reinterpret_cast<uint32_t*>(xbuf + 2 * G * E2); // [n_elem][2E]
    uint64_t* full = reinterpret_cast<uint64_t*>(ptab + (size_t)n_elem * E2 + ((n_elem * E2) & 1));
    uint64_t* empty = full + kOrbStages;
    uint64_t* pbar = empty + kOrbStages;     // consumer-only sync of the x~ gather
    constexpr int GS = G / NT;               // slots per consumer thread
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (E + 31) / 32;           // row warps of one slot group
    const int nthr = 32 * ncw * NT;          // consumer threads
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOrbStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw * NT);
        }
        mbar_init(pbar, ncw * NT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = threadIdx.x; e < n_elem * E2; e += blockDim.x) ptab[e] = orb_perm[e];
    __syncthreads();
    const int nj = (E + JB - 1) / JB;
    const int Gc = (int)gridDim.x;
    const long long Q = (long long)nst * nj;
    const long long q0 = (long long)blockIdx.x * Q / Gc, q1 = (long long)(blockIdx.x + 1) * Q / Gc;
    if (q0 >= q1) return;
    const int sb0 = (int)(q0 / nj), jb0 = (int)(q0 % nj);
    if (warp == 0) {
        if (lane != 0) return;
        const uint64_t pol = l2_evict_first();
        const uint32_t bytes_x = (uint32_t)(E2 * sizeof(float2));
        int s = 0, sb = sb0, jb = jb0, t = 0;
        uint32_t ph = 0;
        long long issued = 0;
        bool ok = true;
        for (long long q = q0; q < q1; ++q) {
            if (q - q0 >= kOrbStages && !mbar_wait(&empty[s], ph ^ 1u)) {
                ok = false;
                break;
            }
            const int j0 = jb * JB, jn = min(JB, E - j0);
            const uint32_t bytes_op = (uint32_t)(jn * E * sizeof(float2));
            const bool newbin = jb == 0 || q == q0;
            uint32_t xb = 0;
            int bins[G];
            if (newbin) {
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    bins[j] = orb_bin[(size_t)sb * G + j];
                    if (bins[j] >= 0) xb += bytes_x;
                }
            }
            mbar_expect_tx(&full[s], 2 * bytes_op + xb);
            const float2* src = Bhat + (size_t)sb * 2 * E * E + (size_t)j0 * E;
            float2* dst = sbuf + (size_t)s * stage_elems;
            bulk_g2s_hint(dst, src, bytes_op, &full[s], pol);
            bulk_g2s_hint(dst + JB * E, src + (size_t)E * E, bytes_op, &full[s], pol);
            if (newbin) {
                float2* xd = xbuf + (size_t)(t & 1) * G * E2;
#pragma unroll
                for (int j = 0; j < G; ++j)
                    if (bins[j] >= 0) bulk_g2s(xd + (size_t)j * E2, Xh + (size_t)bins[j] * E2, bytes_x, &full[s]);
            }
            issued = q - q0 + 1;
            if (++s == kOrbStages) { s = 0; ph ^= 1u; }
            if (++jb == nj) { jb = 0; ++sb; ++t; }
        }
        if (!ok) {
            atomicExch(err, 1);
            for (long long u = (issued > kOrbStages ? issued - kOrbStages : 0); u < issued; ++u)
                mbar_wait(&full[u % kOrbStages], (uint32_t)((u / kOrbStages) & 1));
        }
        return;
    }
    // ---- consumers: NT threads per test row i, slot group grp of GS slots
    const int tid = threadIdx.x - 32;
    const int w = warp - 1;                  // consumer warp (counter index)
    const int grp = w / ncw;
    const int i = (w - grp * ncw) * 32 + lane;
    const int j_lo = grp * GS;
    int s = 0, sb = sb0, jb = jb0, t = 0;
    uint32_t ph = 0, pph = 0;
    long long qb = (long long)sb0 * nj;
    // all consumer warps meet (bounded: on expiry the flag is set and the
    // warp leaves; the others' waits then expire too)
    auto consumers_meet = [&]() -> bool {
        __syncwarp();
        if (lane == 0) mbar_arrive(pbar);
        const bool ok = mbar_wait(pbar, pph);
        pph ^= 1u;
        return ok;
    };
    float2 lj[GS], lm[GS], kj[GS], km[GS];
#pragma unroll
    for (int j = 0; j < GS; ++j) lj[j] = lm[j] = kj[j] = km[j] = make_float2(0.f, 0.f);
    for (long long q = q0; q < q1; ++q) {
        if (!mbar_wait(&full[s], ph)) {
            atomicExch(err, 1);
            return;
        }
        float2* xs = xbuf + (size_t)(t & 1) * G * E2;
        if (jb == 0 || q == q0) {
            // x~_j = T_e^T x(bin_j) in place (zero for empty slots), in one
            // pass: every read before any write.  The G x 2E entries fit in
            // 2 GS registers per thread because there are at least NT E
            // consumer threads.
            float2 v[2 * GS];
#pragma unroll
            for (int c = 0; c < 2 * GS; ++c) {
                const int e = c * nthr + tid;
                v[c] = make_float2(0.f, 0.f);
                if (e < G * E2) {
                    const int j = e / E2, n = e - j * E2;
                    if (orb_bin[(size_t)sb * G + j] >= 0) {
                        const uint32_t pe = ptab[(size_t)orb_elem[(size_t)sb * G + j] * E2 + n];
                        const float2 a = xs[(size_t)j * E2 + (pe & 0x7fffffffu)];
                        v[c] = (pe >> 31) ? make_float2(-a.x, -a.y) : a;
                    }
                }
            }
            if (!consumers_meet()) {
                atomicExch(err, 1);
                return;
            }
#pragma unroll
            for (int c = 0; c < 2 * GS; ++c) {
                const int e = c * nthr + tid;
                if (e < G * E2) xs[e] = v[c];
            }
            if (!consumers_meet()) {
                atomicExch(err, 1);
                return;
            }
            // later bulk copies into this buffer are ordered after these writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        const float2* Ls = sbuf + (size_t)s * stage_elems;
        const float2* Ks = Ls + JB * E;
        const int j0 = jb * JB, jn = min(JB, E - j0);
        if (i < E) {
#pragma unroll
            for (int jj = 0; jj < JB; jj += 2) {
                if (jj < jn) {
                    // columns jj, jj + 1 (jn is even: E is even)
                    const float2 l0 = Ls[jj * E + i], l1 = Ls[(jj + 1) * E + i];
                    const float2 k0 = Ks[jj * E + i], k1 = Ks[(jj + 1) * E + i];
#pragma unroll
                    for (int j = 0; j < GS; ++j) {
                        const float2* xsj = xs + (size_t)(j_lo + j) * E2;
                        const float4 xj = *reinterpret_cast<const float4*>(xsj + j0 + jj);
                        const float4 xm = *reinterpret_cast<const float4*>(xsj + E + j0 + jj);
                        const float2 xj0 = make_float2(xj.x, xj.y), xj1 = make_float2(xj.z, xj.w);
                        const float2 xm0 = make_float2(xm.x, xm.y), xm1 = make_float2(xm.z, xm.w);
                        cfma(lj[j], l0, xj0);
                        cfma(lm[j], l0, xm0);
                        cfma(kj[j], k0, xj0);
                        cfma(km[j], k0, xm0);
                        cfma(lj[j], l1, xj1);
                        cfma(lm[j], l1, xm1);
                        cfma(kj[j], k1, xj1);
                        cfma(km[j], k1, xm1);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (jb == nj - 1 || q == q1 - 1) {
            // this CTA's part of stored bin sb ends here
            const bool whole = qb >= q0 && jb == nj - 1;
            float2* P = part + ((size_t)blockIdx.x * 2 + (t == 0 ? 0 : 1)) * G * E2;
#pragma unroll
            for (int jl = 0; jl < GS; ++jl) {
                const int j = j_lo + jl;
                const int bin = orb_bin[(size_t)sb * G + j];
                if (bin < 0 || i >= E) continue;
                const float2 y0 = cadd(cmul(ca, lj[jl]), cmul(cb, km[jl]));
                const float2 y1 = cadd(cmul(cg, kj[jl]), cmul(cd, lm[jl]));
                if (whole) {
                    const uint32_t* pt = ptab + (size_t)orb_elem[(size_t)sb * G + j] * E2;
                    const uint32_t p0 = pt[i], p1 = pt[E + i];
                    float2* Y = Yh + (size_t)bin * E2;
                    Y[p0 & 0x7fffffffu] = (p0 >> 31) ? make_float2(-y0.x, -y0.y) : y0;
                    Y[p1 & 0x7fffffffu] = (p1 >> 31) ? make_float2(-y1.x, -y1.y) : y1;
                } else {
                    P[(size_t)j * E2 + i] = y0;
                    P[(size_t)j * E2 + E + i] = y1;
                }
            }
            if (!whole) {
                __threadfence();
                __syncwarp();
                const int bf = pair_cta_of(qb, Q, Gc), bl = pair_cta_of(qb + nj - 1, Q, Gc);
                int* c = cnt + (size_t)sb * ncw * NT + w;
                int old = 0;
                if (lane == 0) old = atomicAdd(c, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == bl - bf) {
                    // every contributor has written its partial
                    if (lane == 0) *c = 0;
                    __threadfence();
                    if (i < E) {
                        for (int j = j_lo; j < j_lo + GS; ++j) {
                            const int bin = orb_bin[(size_t)sb * G + j];
                            if (bin < 0) continue;
                            float2 a0 = make_float2(0.f, 0.f), a1 = a0;
                            for (int b = bf; b <= bl; ++b) {
                                const int sl = ((long long)b * Q / Gc) / nj == sb ? 0 : 1;
                                const float2* Pb = part + ((size_t)b * 2 + sl) * G * E2 + (size_t)j * E2;
                                a0 = cadd(a0, __ldcg(Pb + i));
                                a1 = cadd(a1, __ldcg(Pb + E + i));
                            }
                            const uint32_t* pt = ptab + (size_t)orb_elem[(size_t)sb * G + j] * E2;
                            const uint32_t p0 = pt[i], p1 = pt[E + i];
                            float2* Y = Yh + (size_t)bin * E2;
                            Y[p0 & 0x7fffffffu] = (p0 >> 31) ? make_float2(-a0.x, -a0.y) : a0;
                            Y[p1 & 0x7fffffffu] = (p1 >> 31) ? make_float2(-a1.x, -a1.y) : a1;
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < GS; ++j) lj[j] = lm[j] = kj[j] = km[j] = make_float2(0.f, 0.f);
        }
        if (++s == kOrbStages) { s = 0; ph ^= 1u; }
        if (++jb == nj) {
            jb = 0;
            ++sb;
            ++t;
            qb += nj;
        }
    }
}

template <int G, int JB>
size_t binmul_orbit_smem(int E) {
    const size_t E2 = 2 * (size_t)E;
    const size_t n_elem = G;
    return (size_t)kOrbStages * 2 * JB * E * sizeof(float2) + 2 * G * E2 * sizeof(float2) +
           (n_elem * E2 + ((n_elem * E2) & 1)) * sizeof(uint32_t) + (2ull * kOrbStages + 1) * sizeof(uint64_t);
}

// ------------------------------------------------ K4: macromodel multiply
// Ymm[s][r][m][k] = sum_{k' in chunk s} Z~^{t(m)}[k][k'] x1[r][m][k'] for a
// group of up to G cells of one type (x1 = U_o x gathered on the fly).  The
// k' range is split over gridDim.y chunks so the product of a few dozen
// types fills the GPU; the crop/scatter kernel adds the chunk partials in a
// fixed order (deterministic).
struct MmBlock {
    int type, first, count;
};

// RB rhs per pass share every load of Z (register block G cells x RB rhs).
template <typename T2, int G, int RB>
__global__ void macromodel_kernel(const T2* __restrict__ Zt, const double2* __restrict__ x,
                                  const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn,
                                  const int32_t* __restrict__ type_cells,
                                  const MmBlock* __restrict__ blocks, T2* __restrict__ Ymm, int K,
                                  int M, int R, int n_unique, int chunk, const float2* __restrict__ xf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* xs = reinterpret_cast<T2*>(smem_raw);   // [RB][G][chunk]
    const MmBlock b = blocks[blockIdx.x];
    const int s = blockIdx.y;
    const int k0 = s * chunk, k1 = min(K, k0 + chunk), nk = k1 - k0;
    const T2 zero = mk<T2>(0.0, 0.0);
    const T2* Z = Zt + (size_t)b.type * K * K;
    for (int r0 = 0; r0 < R; r0 += RB) {
        __syncthreads();
        for (int e = threadIdx.x; e < RB * G * chunk; e += blockDim.x) {
            const int rr = e / (G * chunk), g = (e / chunk) % G, kk = e % chunk;
            T2 v = zero;
            if (r0 + rr < R && g < b.count && kk < nk) {
                const size_t loc = (size_t)type_cells[b.first + g] * K + k0 + kk;
                const size_t at = (size_t)(r0 + rr) * n_unique + idx[loc];
                if (xf) {
                    const float2 xv = xf[at];
                    const float sg = (float)sgn[loc];
                    if constexpr (sizeof(T2) == sizeof(float2)) v = make_float2(sg * xv.x, sg * xv.y);
                    else v = mk<T2>((double)(sg * xv.x), (double)(sg * xv.y));
                } else {
                    const double2 xv = x[at];
                    const double sg = (double)sgn[loc];
                    v = mk<T2>(sg * xv.x, sg * xv.y);
                }
            }
            xs[e] = v;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            T2 acc[RB][G];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int g = 0; g < G; ++g) acc[rr][g] = zero;
#pragma unroll 4
            for (int kk = 0; kk < nk; ++kk) {
                const T2 z = __ldg(Z + (size_t)(k0 + kk) * K + k);
#pragma unroll
                for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                    for (int g = 0; g < G; ++g) cfma(acc[rr][g], z, xs[(rr * G + g) * chunk + kk]);
            }
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (g < b.count && r0 + rr < R)
                        Ymm[(((size_t)s * R + r0 + rr) * M + type_cells[b.first + g]) * K + k] = acc[rr][g];
        }
    }
}

// Single-rhs FP32 variant: each thread owns two adjacent output rows and
// keeps eight 16-byte loads of Z in flight (the one-row kernel is bound by
// load latency at one rhs); the staged x1 is read two columns at a time.
constexpr int kMm2Unroll = 4;   // 16-byte loads per buffer (three blocks of 320 threads per SM)
template <int G>
__global__ void __launch_bounds__(320, 3)
macromodel2_kernel(const float2* __restrict__ Zt, const double2* __restrict__ x,
                   const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn,
                   const int32_t* __restrict__ type_cells, const MmBlock* __restrict__ blocks,
                   float2* __restrict__ Ymm, int K, int M, int n_unique, int chunk, const float2* __restrict__ xf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* xs = reinterpret_cast<float2*>(smem_raw);   // [G][chunk], chunk a multiple of kMm2Unroll
    const MmBlock b = blocks[blockIdx.x];
    const int s = blockIdx.y;
    const int k0 = s * chunk, k1 = min(K, k0 + chunk), nk = k1 - k0;
    // gather x1 (independent iterations: unrolled so their loads overlap)
#pragma unroll 4
    for (int e = threadIdx.x; e < G * chunk; e += blockDim.x) {
        const int g = e / chunk, kk = e % chunk;
        float2 v = make_float2(0.f, 0.f);
        if (g < b.count && kk < nk) {
            const size_t loc = (size_t)type_cells[b.first + g] * K + k0 + kk;
            const size_t at = idx[loc];
            const float sg = (float)sgn[loc];
            if (xf) {
                const float2 xv = xf[at];
                v = make_float2(sg * xv.x, sg * xv.y);
            } else {
                const double2 xv = x[at];
                v = make_float2((float)(sg * xv.x), (float)(sg * xv.y));
            }
        }
        xs[e] = v;
    }
    __syncthreads();
    const int K2 = K >> 1;
    const float4* Z4 = reinterpret_cast<const float4*>(Zt + (size_t)b.type * K * K + (size_t)k0 * K);
    const uint64_t pol = l2_evict_last();      // the macromodels are read by every product
    for (int k2 = threadIdx.x; k2 < K2; k2 += blockDim.x) {
        float2 a0[G], a1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) a0[g] = a1[g] = make_float2(0.f, 0.f);
        // register double buffer: the next block's loads are in flight while
        // the current one is multiplied
        float4 zb[2][kMm2Unroll];
        auto load = [&](float4 (&z)[kMm2Unroll], int kb) {
#pragma unroll
            for (int u = 0; u < kMm2Unroll; ++u)
                z[u] = kb + u < nk ? ldg_l2hint(Z4 + (size_t)(kb + u) * K2 + k2, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto mul = [&](const float4 (&z)[kMm2Unroll], int kb) {
#pragma unroll
            for (int u = 0; u < kMm2Unroll; u += 2) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    // x1 of columns kb+u, kb+u+1 (zero past nk, so no guard on the FMAs)
                    const float4 xv = *reinterpret_cast<const float4*>(xs + g * chunk + kb + u);
                    const float2 x0 = make_float2(xv.x, xv.y), x1 = make_float2(xv.z, xv.w);
                    cfma(a0[g], make_float2(z[u].x, z[u].y), x0);
                    cfma(a1[g], make_float2(z[u].z, z[u].w), x0);
                    cfma(a0[g], make_float2(z[u + 1].x, z[u + 1].y), x1);
                    cfma(a1[g], make_float2(z[u + 1].z, z[u + 1].w), x1);
                }
            }
        };
        load(zb[0], 0);
        for (int kb = 0; kb < nk; kb += 2 * kMm2Unroll) {
            if (kb + kMm2Unroll < nk) load(zb[1], kb + kMm2Unroll);
            mul(zb[0], kb);
            if (kb + kMm2Unroll >= nk) break;
            if (kb + 2 * kMm2Unroll < nk) load(zb[0], kb + 2 * kMm2Unroll);
            mul(zb[1], kb + kMm2Unroll);
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < b.count) {
                float2* y = Ymm + ((size_t)s * M + type_cells[b.first + g]) * K + 2 * k2;
                y[0] = a0[g];
                y[1] = a1[g];
            }
    }
}

// Single-rhs FP64-accuracy variant in double-single FP32 arithmetic (see
// binmul_ds_kernel): Z~ as FP32 hi/lo planes zp[t][hi, lo][k'][k], x1 split
// into hi/lo while it is gathered, each thread two output rows for up to G
// cells, products accumulated with ds_cmac, FP64 partial outputs.
constexpr int kMmDsUnroll = 2;
template <int G>
__global__ void __launch_bounds__(320, 2)
macromodel_ds_kernel(const float2* __restrict__ zp, const double2* __restrict__ x,
                     const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn,
                     const int32_t* __restrict__ type_cells, const MmBlock* __restrict__ blocks,
                     double2* __restrict__ Ymm, int K, int M, int chunk, const double* __restrict__ scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* xh = reinterpret_cast<float2*>(smem_raw);   // [G][chunk] hi
    float2* xl = xh + (size_t)G * chunk;                // [G][chunk] lo
    const MmBlock b = blocks[blockIdx.x];
    const double sx = scale[2], u = 1.0 / (scale[1] * scale[2]);
    const int s = blockIdx.y;
    const int k0 = s * chunk, k1 = min(K, k0 + chunk), nk = k1 - k0;
    for (int e = threadIdx.x; e < G * chunk; e += blockDim.x) {
        const int g = e / chunk, kk = e % chunk;
        double2 v = make_double2(0.0, 0.0);
        if (g < b.count && kk < nk) {
            const size_t loc = (size_t)type_cells[b.first + g] * K + k0 + kk;
            const double2 xv = x[idx[loc]];
            const double sg = (double)sgn[loc] * sx;
            v = make_double2(sg * xv.x, sg * xv.y);
        }
        const float2 hi = make_float2((float)v.x, (float)v.y);
        xh[e] = hi;
        xl[e] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
    }
    __syncthreads();
    const int K2 = K >> 1;
    const size_t KK = (size_t)K * K;
    const float4* Zh = reinterpret_cast<const float4*>(zp + (size_t)b.type * 2 * KK + (size_t)k0 * K);
    const float4* Zl = reinterpret_cast<const float4*>(zp + ((size_t)b.type * 2 + 1) * KK + (size_t)k0 * K);
    for (int k2 = threadIdx.x; k2 < K2; k2 += blockDim.x) {
        DsC a0[G], a1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) a0[g] = a1[g] = DsC{0.f, 0.f, 0.f, 0.f};
        for (int kb = 0; kb < nk; kb += kMmDsUnroll) {
            float4 zh[kMmDsUnroll], zl[kMmDsUnroll];
#pragma unroll
            for (int u = 0; u < kMmDsUnroll; ++u) {
                const bool in = kb + u < nk;
                zh[u] = in ? __ldg(Zh + (size_t)(kb + u) * K2 + k2) : make_float4(0.f, 0.f, 0.f, 0.f);
                zl[u] = in ? __ldg(Zl + (size_t)(kb + u) * K2 + k2) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kMmDsUnroll; ++u) {
                if (kb + u < nk) {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const float2 vh = xh[g * chunk + kb + u], vl = xl[g * chunk + kb + u];
                        ds_cmac(a0[g], vh, vl, make_float2(zh[u].x, zh[u].y), make_float2(zl[u].x, zl[u].y));
                        ds_cmac(a1[g], vh, vl, make_float2(zh[u].z, zh[u].w), make_float2(zl[u].z, zl[u].w));
                    }
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < b.count) {
                double2* y = Ymm + ((size_t)s * M + type_cells[b.first + g]) * K + 2 * k2;
                const double2 v0 = ds_value(a0[g]), v1 = ds_value(a1[g]);
                y[0] = make_double2(u * v0.x, u * v0.y);
                y[1] = make_double2(u * v1.x, u * v1.y);
            }
    }
}

// ------------------------------------------------ K3 tail: U_o^T
// y[r][u] = sum over local unknowns (m,k) of u: sign * y1[r][m][k]
// (sums in the grid's precision; V2 is the output vector type)
template <typename T2, typename V2>
__global__ void scatter_kernel(V2* __restrict__ y, const T2* __restrict__ y1,
                               const int32_t* __restrict__ ptr, const int32_t* __restrict__ ent,
                               const int8_t* __restrict__ esg, int MK, int R, int n_unique) {
    using S = decltype(y1[0].x);
    const size_t total = (size_t)R * n_unique;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(e % n_unique);
        const int r = (int)(e / n_unique);
        S ax = 0, ay = 0;
        for (int q = ptr[u]; q < ptr[u + 1]; ++q) {
            const T2 v = y1[(size_t)r * MK + ent[q]];
            const S s = (S)esg[q];
            ax += s * v.x;
            ay += s * v.y;
        }
        V2 o;
        o.x = ax;
        o.y = ay;
        y[e] = o;
    }
}

int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {
int orbit_spectrum(emsurf_handle* h, const emsurf_problem* pr, const double2* B64, bool* used);
}

// ---------------------------------------------------------------- build
// Places L(d), K(d) at grid point (dx mod px, dy mod py) -- the circulant's
// first column (Eq. LJV3 read by columns, d = test - source) -- and
// transforms the grid with the forward 2-D FFT: B^(k) = F[B](k).
template <typename T2>
int build_spectrum(emsurf_handle* h, Operator<T2>& op, const emsurf_problem* pr);

template <typename T2>
int build_operator(emsurf_handle* h, Operator<T2>& op, const emsurf_problem* pr, const Operator<T2>* share) {
    const int E = h->E, K = h->K;
    const size_t EE = (size_t)E * E;
    const int nox = 2 * h->nx - 1, noy = 2 * h->ny - 1;
    const size_t nbins = (size_t)h->nbins;
    cudaStream_t st = h->setup_stream;
    if (share) {
        // the spectrum of a handle of the same lattice (not owned here)
        op.Bhat = share->Bhat;
    } else {
        EMS_TRY(build_spectrum(h, op, pr));
    }
    // macromodels
    const size_t zbytes = (size_t)h->T * K * K * sizeof(double2);
    double2* zstage = nullptr;
    if (pr->tables_on_device) {
        zstage = const_cast<double2*>(reinterpret_cast<const double2*>(pr->macromodels));
    } else {
        EMS_CUDA(cudaMalloc(&zstage, zbytes));
        EMS_CUDA(cudaMemcpyAsync(zstage, pr->macromodels, zbytes, cudaMemcpyHostToDevice, st));
    }
    EMS_TRY(dev_alloc(h, (void**)&op.Zt, (size_t)h->T * K * K * sizeof(T2)));
    dim3 zg((K + 31) / 32, (K + 31) / 32, h->T);
    transpose_mm_kernel<T2><<<zg, dim3(32, 8), 0, st>>>(op.Zt, zstage, K);
    EMS_CUDA(cudaGetLastError());
    EMS_CUDA(cudaStreamSynchronize(st));
    if (!pr->tables_on_device) cudaFree(zstage);
    // work buffers
    const size_t grid_elems = nbins * (size_t)h->max_rhs * K;
    EMS_TRY(dev_alloc(h, (void**)&op.Xg, grid_elems * sizeof(T2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Yg, grid_elems * sizeof(T2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Ymm, (size_t)kMmSplit * h->max_rhs * h->M * K * sizeof(T2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Y1, (size_t)h->max_rhs * h->M * K * sizeof(T2)));
    for (int c = 0; c < 4; ++c) op.coef[c] = mk<T2>(pr->coef[c].re, pr->coef[c].im);
    (void)nox;
    (void)noy;
    (void)EE;
    return EMSURF_OK;
}

// The Fourier-domain blocks of Sec. IV-B from the offset tables.
template <typename T2>
int build_spectrum(emsurf_handle* h, Operator<T2>& op, const emsurf_problem* pr) {
    const int E = h->E;
    const size_t EE = (size_t)E * E;
    const int nox = 2 * h->nx - 1, noy = 2 * h->ny - 1;
    const size_t nbins = (size_t)h->nbins;
    // FP64 spectrum first (also the source of the FP32 copy)
    double2* B64 = nullptr;
    const size_t bbytes64 = nbins * 2 * EE * sizeof(double2);
    const bool direct64 = sizeof(T2) == sizeof(double2);
    if (direct64) {
        EMS_TRY(dev_alloc(h, (void**)&B64, bbytes64));
    } else {
        EMS_CUDA(cudaMalloc(&B64, bbytes64));
    }
    cudaStream_t st = h->setup_stream;
    EMS_CUDA(cudaMemsetAsync(B64, 0, bbytes64, st));
    // stage offsets in chunks of <= 256 MB
    const size_t per_off = 2 * EE * sizeof(double2);
    int chunk = (int)std::max<size_t>(1, (256ull << 20) / per_off);
    chunk = std::min(chunk, nox * noy);
    double2* stage = nullptr;
    int* dbins = nullptr;
    EMS_CUDA(cudaMalloc(&stage, per_off * chunk));
    EMS_CUDA(cudaMalloc(&dbins, sizeof(int) * chunk));
    std::vector<int> hb(chunk);
    const cudaMemcpyKind kind = pr->tables_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int o0 = 0; o0 < nox * noy; o0 += chunk) {
        const int nc = std::min(chunk, nox * noy - o0);
        for (int c = 0; c < nc; ++c) {
            const int o = o0 + c;
            const int dyi = o / nox, dxi = o % nox;
            const int dx = dxi - (h->nx - 1), dy = dyi - (h->ny - 1);
            const int bx = ((dx % h->px) + h->px) % h->px;
            const int by = ((dy % h->py) + h->py) % h->py;
            hb[c] = by * h->px + bx;
            EMS_CUDA(cudaMemcpyAsync(stage + (size_t)c * 2 * EE, pr->offset_L + (size_t)o * EE,
                                     EE * sizeof(double2), kind, st));
            EMS_CUDA(cudaMemcpyAsync(stage + (size_t)c * 2 * EE + EE, pr->offset_K + (size_t)o * EE,
                                     EE * sizeof(double2), kind, st));
        }
        EMS_CUDA(cudaMemcpyAsync(dbins, hb.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
        dim3 grid((E + 31) / 32, (E + 31) / 32, 2 * nc);
        place_blocks_kernel<double2><<<grid, dim3(32, 8), 0, st>>>(B64, stage, dbins, nc, E);
        EMS_CUDA(cudaGetLastError());
        EMS_CUDA(cudaStreamSynchronize(st));
    }
    cudaFree(stage);
    cudaFree(dbins);
    // 2-D forward FFT over bins: lanes = 2 E^2 block entries
    const long long lanes = 2LL * (long long)EE;
    EMS_TRY(fft_pass<double2>(B64, h->plan_x, lanes, h->py, (long long)h->px * lanes, -1, st));
    EMS_TRY(fft_pass<double2>(B64, h->plan_y, (long long)h->px * lanes, 1, 0, -1, st));
    if (direct64) {
        op.Bhat = reinterpret_cast<T2*>(B64);
    } else {
        // an FP32-only single-rhs handle of a mirror-symmetric box keeps one
        // bin per orbit (the same form a MIXED handle derives)
        bool orb = false;
        if (h->precision == EMSURF_FP32) {
            const int s = orbit_spectrum(h, pr, B64, &orb);
            if (s != EMSURF_OK) {
                cudaFree(B64);
                return s;
            }
        }
        if (orb) {
            cudaFree(B64);
            return EMSURF_OK;
        }
        EMS_TRY(dev_alloc(h, (void**)&op.Bhat, nbins * 2 * EE * sizeof(T2)));
        round_kernel<<<152 * 8, 256, 0, st>>>(reinterpret_cast<float2*>(op.Bhat), B64,
                                             nbins * 2 * EE);
        EMS_CUDA(cudaGetLastError());
        EMS_CUDA(cudaStreamSynchronize(st));
        cudaFree(B64);
    }
    return EMSURF_OK;
}

int derive_fp32_rest(emsurf_handle* h, const emsurf_problem* pr);

namespace {
constexpr int kOrbJB4 = 12;   // slab width of the 4-slot (x and y mirrors) orbit kernel
constexpr int kOrbJB8 = 8;    // and of the 8-slot one (with x <-> y)
constexpr int kOrbNT4 = 1;    // consumer threads per test row (4 accumulator sets each)
constexpr int kOrbNT8 = 2;

// The FP32 spectrum as one stored bin per mirror orbit, when the problem
// gives the box's mirrors and they hold on the FP64 blocks.  *used = false
// (and nothing allocated) otherwise.
int orbit_spectrum(emsurf_handle* h, const emsurf_problem* pr, const double2* B64, bool* used) {
    *used = false;
    const int E = h->E, px = h->px, py = h->py;
    const size_t EE = (size_t)E * E, nb = (size_t)h->nbins;
    cudaStream_t st = h->setup_stream;
    if (h->max_rhs != 1 || pr->tensor_cores || (E & 1) || !pr->sym_perm || !pr->sym_sign ||
        (pr->sym_mask & 3) != 3)
        return EMSURF_OK;
    for (int g = 0; g < 3; ++g) {
        if (!(pr->sym_mask & (1 << g))) continue;
        std::vector<char> hit(E, 0);
        for (int n = 0; n < E; ++n) {
            const int m = pr->sym_perm[(size_t)g * E + n], sg = pr->sym_sign[(size_t)g * E + n];
            if (m < 0 || m >= E || (sg != 1 && sg != -1) || hit[m]) {
                set_error("sym_perm/sym_sign of mirror %d is not a signed permutation of %d entries", g, E);
                return EMSURF_EINVAL;
            }
            hit[m] = 1;
        }
    }
    const bool diag = (pr->sym_mask & 4) && px == py && h->nx == h->ny;
    const int G = diag ? 8 : 4, JB = diag ? kOrbJB8 : kOrbJB4, NT = diag ? kOrbNT8 : kOrbNT4;
    const size_t smem = diag ? binmul_orbit_smem<8, kOrbJB8>(E) : binmul_orbit_smem<4, kOrbJB4>(E);
    const int ncw = (E + 31) / 32;
    const int maxt = diag ? orb_max_threads<kOrbNT8>() : orb_max_threads<kOrbNT4>();
    if (smem > 227 * 1024 || 32 * (1 + NT * ncw) > maxt || (E + JB - 1) / JB < kOrbStages) return EMSURF_OK;
    // the generators' relations on the FP64 blocks
    {
        std::vector<uint32_t> pt(E);
        std::vector<int32_t> img(nb);
        uint32_t* dpt = nullptr;
        int32_t* dimg = nullptr;
        unsigned long long* dout = nullptr;
        EMS_CUDA(cudaMalloc(&dpt, E * sizeof(uint32_t)));
        EMS_CUDA(cudaMalloc(&dimg, nb * sizeof(int32_t)));
        EMS_CUDA(cudaMalloc(&dout, 2 * sizeof(unsigned long long)));
        bool holds = true;
        for (int g = 0; g < (diag ? 3 : 2) && holds; ++g) {
            for (int n = 0; n < E; ++n)
                pt[n] = (uint32_t)pr->sym_perm[(size_t)g * E + n] |
                        (pr->sym_sign[(size_t)g * E + n] < 0 ? 0x80000000u : 0u);
            for (int ky = 0; ky < py; ++ky)
                for (int kx = 0; kx < px; ++kx) img[(size_t)ky * px + kx] = orbit_image(1 << g, kx, ky, px, py);
            EMS_CUDA(cudaMemcpyAsync(dpt, pt.data(), E * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
            EMS_CUDA(cudaMemcpyAsync(dimg, img.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            EMS_CUDA(cudaMemsetAsync(dout, 0, 2 * sizeof(unsigned long long), st));
            mirror_check_kernel<<<152 * 8, 256, 0, st>>>(B64, dpt, dimg, E, nb, dout);
            EMS_CUDA(cudaGetLastError());
            unsigned long long hout[2] = {0, 0};
            EMS_CUDA(cudaMemcpyAsync(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost, st));
            EMS_CUDA(cudaStreamSynchronize(st));
            double dmax, vmax;
            std::memcpy(&dmax, &hout[0], sizeof(double));
            std::memcpy(&vmax, &hout[1], sizeof(double));
            holds = vmax > 0.0 && dmax <= 1e-12 * vmax;
        }
        cudaFree(dpt);
        cudaFree(dimg);
        cudaFree(dout);
        if (!holds) return EMSURF_OK;
    }
    // the signed permutations T_e of the group elements and the orbits
    // (host logic in the setup library)
    const int E2 = 2 * E;
    std::vector<uint32_t> tperm;
    mirror_group_perms(E, G, pr->sym_perm, pr->sym_sign, tperm);
    std::vector<int32_t> rep, obin, oelem;
    mirror_orbits(px, py, G, rep, obin, oelem);
    const int nst = (int)rep.size();
    int32_t *drep = nullptr, *dob = nullptr, *doe = nullptr;
    uint32_t* dtp = nullptr;
    EMS_TRY(dev_alloc(h, (void**)&drep, rep.size() * sizeof(int32_t)));
    EMS_TRY(dev_alloc(h, (void**)&dob, obin.size() * sizeof(int32_t)));
    EMS_TRY(dev_alloc(h, (void**)&doe, oelem.size() * sizeof(int32_t)));
    EMS_TRY(dev_alloc(h, (void**)&dtp, tperm.size() * sizeof(uint32_t)));
    EMS_CUDA(cudaMemcpyAsync(drep, rep.data(), rep.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    EMS_CUDA(cudaMemcpyAsync(dob, obin.data(), obin.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    EMS_CUDA(cudaMemcpyAsync(doe, oelem.data(), oelem.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    EMS_CUDA(cudaMemcpyAsync(dtp, tperm.data(), tperm.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    h->nst = nst;
    h->d_st_bin = drep;
    h->d_orb_bin = dob;
    h->d_orb_elem = doe;
    h->d_orb_perm = dtp;
    h->orb_G = G;
    const long long nslab = (long long)nst * ((E + JB - 1) / JB);
    h->pair_grid = (int)std::min<long long>(std::max(1, h->num_sms), nslab);
    EMS_TRY(dev_alloc(h, (void**)&h->d_pair_part, (size_t)h->pair_grid * 2 * G * E2 * sizeof(float2)));
    h->pair_cnt_bytes = (size_t)nst * ncw * NT * sizeof(int);
    EMS_TRY(dev_alloc(h, (void**)&h->d_pair_cnt, h->pair_cnt_bytes));
    EMS_CUDA(cudaMemsetAsync(h->d_pair_cnt, 0, h->pair_cnt_bytes, st));
    EMS_TRY(dev_alloc(h, (void**)&h->op32.Bhat, (size_t)nst * 2 * EE * sizeof(float2)));
    half_round_kernel<<<152 * 8, 256, 0, st>>>(h->op32.Bhat, B64, drep, 2 * EE, (size_t)nst * 2 * EE);
    EMS_CUDA(cudaGetLastError());
    EMS_CUDA(cudaStreamSynchronize(st));   // the host vectors above go out of scope
    h->orb32 = true;
    *used = true;
    return EMSURF_OK;
}
}  // namespace

// The stored-bin lists of a shared handle's partial FP32 spectrum (pairs or
// mirror orbits); the kernels' partial sums and counters are per-handle work
// space.
int adopt_fp32_form(emsurf_handle* h, const emsurf_handle* share) {
    h->half32 = share->half32;
    h->nst = share->nst;
    h->d_st_bin = share->d_st_bin;
    h->d_st_part = share->d_st_part;
    h->orb32 = share->orb32;
    h->orb_G = share->orb_G;
    h->d_orb_bin = share->d_orb_bin;
    h->d_orb_elem = share->d_orb_elem;
    h->d_orb_perm = share->d_orb_perm;
    if (h->half32 || h->orb32) {
        const int ncw = (h->E + 31) / 32;
        const int slots = h->orb32 ? h->orb_G : 2;
        h->pair_grid = share->pair_grid;
        EMS_TRY(dev_alloc(h, (void**)&h->d_pair_part, (size_t)h->pair_grid * 2 * slots * 2 * h->E * sizeof(float2)));
        h->pair_cnt_bytes = share->pair_cnt_bytes;
        EMS_TRY(dev_alloc(h, (void**)&h->d_pair_cnt, h->pair_cnt_bytes));
        EMS_CUDA(cudaMemsetAsync(h->d_pair_cnt, 0, h->pair_cnt_bytes, h->setup_stream));
    }
    return EMSURF_OK;
}

// FP32 operator of a MIXED handle: round the resident FP64 spectrum and
// macromodels instead of transforming the tables a second time.
int derive_fp32_operator(emsurf_handle* h, const emsurf_problem* pr, const emsurf_handle* share) {
    const int K = h->K;
    const size_t EE = (size_t)h->E * h->E;
    const size_t nb = (size_t)h->nbins;
    cudaStream_t st = h->setup_stream;
    Operator<float2>& op = h->op32;
    if (share) {
        op.Bhat = share->op32.Bhat;
        EMS_TRY(adopt_fp32_form(h, share));
        return derive_fp32_rest(h, pr);
    }
    {
        bool orb = false;
        EMS_TRY(orbit_spectrum(h, pr, h->op64.Bhat, &orb));
        if (orb) return derive_fp32_rest(h, pr);
    }
    // With reciprocal tables L^(-k) = L^(k)^T and K^(-k) = K^(k)^T: single-rhs
    // handles without the tensor-core planes keep one bin of each pair
    // (k, -k) (checked here on the FP64 spectrum, to 1e-12 of its largest
    // entry).
    bool half = false;
    std::vector<int32_t> partner(nb), sbin, spart;
    for (int ky = 0; ky < h->py; ++ky)
        for (int kx = 0; kx < h->px; ++kx)
            partner[(size_t)ky * h->px + kx] = ((h->py - ky) % h->py) * h->px + (h->px - kx) % h->px;
    const int ncw = (h->E + 31) / 32;
    if (h->max_rhs == 1 && !pr->tensor_cores && (h->E & 1) == 0 && binmul_tma_pair_smem(h->E) <= 227 * 1024 &&
        32 * (1 + ncw + kPairColWarps) <= kPairMaxThreads && (h->E + kPairJB - 1) / kPairJB >= kPairStages) {
        int32_t* dpart = nullptr;
        unsigned long long* dout = nullptr;
        EMS_CUDA(cudaMalloc(&dpart, nb * sizeof(int32_t)));
        EMS_CUDA(cudaMalloc(&dout, 2 * sizeof(unsigned long long)));
        EMS_CUDA(cudaMemcpyAsync(dpart, partner.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        EMS_CUDA(cudaMemsetAsync(dout, 0, 2 * sizeof(unsigned long long), st));
        reciprocity_kernel<<<152 * 8, 256, 0, st>>>(h->op64.Bhat, dpart, h->E, nb, dout);
        EMS_CUDA(cudaGetLastError());
        unsigned long long hout[2] = {0, 0};
        EMS_CUDA(cudaMemcpyAsync(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost, st));
        EMS_CUDA(cudaStreamSynchronize(st));
        cudaFree(dpart);
        cudaFree(dout);
        double dmax, vmax;
        std::memcpy(&dmax, &hout[0], sizeof(double));
        std::memcpy(&vmax, &hout[1], sizeof(double));
        half = vmax > 0.0 && dmax <= 1e-12 * vmax;
    }
    if (half) {
        for (size_t b = 0; b < nb; ++b)
            if ((int32_t)b <= partner[b]) {
                sbin.push_back((int32_t)b);
                spart.push_back(partner[b]);
            }
        h->nst = (int)sbin.size();
        int32_t *dsb = nullptr, *dsp = nullptr;
        EMS_TRY(dev_alloc(h, (void**)&dsb, sbin.size() * sizeof(int32_t)));
        EMS_TRY(dev_alloc(h, (void**)&dsp, spart.size() * sizeof(int32_t)));
        EMS_CUDA(cudaMemcpyAsync(dsb, sbin.data(), sbin.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        EMS_CUDA(cudaMemcpyAsync(dsp, spart.data(), spart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        h->d_st_bin = dsb;
        h->d_st_part = dsp;
        // slab ranges of the pair kernel: one per SM, none empty; partial row
        // sums of straddling bins and their arrival counters (kept at zero
        // between launches)
        const long long nslab = (long long)h->nst * ((h->E + kPairJB - 1) / kPairJB);
        h->pair_grid = (int)std::min<long long>(std::max(1, h->num_sms), nslab);
        EMS_TRY(dev_alloc(h, (void**)&h->d_pair_part, (size_t)h->pair_grid * 2 * 2 * h->E * sizeof(float2)));
        h->pair_cnt_bytes = (size_t)h->nst * ncw * sizeof(int);
        EMS_TRY(dev_alloc(h, (void**)&h->d_pair_cnt, h->pair_cnt_bytes));
        EMS_CUDA(cudaMemsetAsync(h->d_pair_cnt, 0, h->pair_cnt_bytes, st));
        EMS_TRY(dev_alloc(h, (void**)&op.Bhat, (size_t)h->nst * 2 * EE * sizeof(float2)));
        half_round_kernel<<<152 * 8, 256, 0, st>>>(op.Bhat, h->op64.Bhat, dsb, 2 * EE, (size_t)h->nst * 2 * EE);
        EMS_CUDA(cudaGetLastError());
        EMS_CUDA(cudaStreamSynchronize(st));   // the host vectors above go out of scope
        h->half32 = true;
    } else {
        EMS_TRY(dev_alloc(h, (void**)&op.Bhat, nb * 2 * EE * sizeof(float2)));
        round_kernel<<<152 * 8, 256, 0, st>>>(op.Bhat, h->op64.Bhat, nb * 2 * EE);
        EMS_CUDA(cudaGetLastError());
    }
    return derive_fp32_rest(h, pr);
}

// the FP32 macromodels and work buffers of a MIXED handle
int derive_fp32_rest(emsurf_handle* h, const emsurf_problem* pr) {
    const int K = h->K;
    const size_t nb = (size_t)h->nbins;
    cudaStream_t st = h->setup_stream;
    Operator<float2>& op = h->op32;
    EMS_TRY(dev_alloc(h, (void**)&op.Zt, (size_t)h->T * K * K * sizeof(float2)));
    round_kernel<<<152 * 8, 256, 0, st>>>(op.Zt, h->op64.Zt, (size_t)h->T * K * K);
    EMS_CUDA(cudaGetLastError());
    const size_t grid_elems = nb * (size_t)h->max_rhs * K;
    EMS_TRY(dev_alloc(h, (void**)&op.Xg, grid_elems * sizeof(float2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Yg, grid_elems * sizeof(float2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Ymm, (size_t)kMmSplit * h->max_rhs * h->M * K * sizeof(float2)));
    EMS_TRY(dev_alloc(h, (void**)&op.Y1, (size_t)h->max_rhs * h->M * K * sizeof(float2)));
    for (int c = 0; c < 4; ++c) op.coef[c] = mk<float2>(pr->coef[c].re, pr->coef[c].im);
    return EMSURF_OK;
}

// FP32 hi/lo planes of the FP64 spectrum and macromodels for the
// double-single kernels (left out, and the FP64 kernels used, when the
// single-rhs kernel's shape does not fit or the device-memory budget has no
// room for them).
int build_ds_planes(emsurf_handle* h, const emsurf_handle* share) {
    const int E = h->E;
    const int ncw = (E + 31) / 32;
    if (binmul_ds_smem(E) > 227 * 1024 || 32 * (1 + ncw) > 1024 || (E + kDsJB - 1) / kDsJB < kDsStages)
        return EMSURF_OK;
    const size_t nb = (size_t)h->nbins, EE = (size_t)E * E;
    const size_t pbytes = nb * 2 * 2 * EE * sizeof(float2), xbytes = nb * 2 * 2 * E * sizeof(float2);
    if (share && !share->ds_planes) return EMSURF_OK;          // products use the shared FP64 spectrum
    if (!share && h->budget > 0 && h->device_bytes + (int64_t)(pbytes + xbytes) > h->budget) return EMSURF_OK;
    if (share) h->ds_planes = share->ds_planes;
    else EMS_TRY(dev_alloc(h, (void**)&h->ds_planes, pbytes));
    EMS_TRY(dev_alloc(h, (void**)&h->ds_x, xbytes));
    EMS_TRY(dev_alloc(h, (void**)&h->d_ds_scale, sizeof(double) * (2 + std::max(1, h->max_rhs))));
    EMS_TRY(dev_alloc(h, (void**)&h->d_ds_max, sizeof(unsigned long long) * std::max(1, h->max_rhs)));
    EMS_TRY(dev_alloc(h, (void**)&h->d_ds_cnt, sizeof(unsigned) * std::max(1, h->max_rhs)));
    EMS_CUDA(cudaMemsetAsync(h->d_ds_max, 0, sizeof(unsigned long long) * std::max(1, h->max_rhs), h->setup_stream));
    EMS_CUDA(cudaMemsetAsync(h->d_ds_cnt, 0, sizeof(unsigned) * std::max(1, h->max_rhs), h->setup_stream));
    // operator scales: the largest component of the spectrum (of the
    // macromodels) maps into [0.5, 1), exactly (powers of two)
    const size_t KK = (size_t)h->K * h->K;
    double* part = nullptr;
    EMS_CUDA(cudaMalloc(&part, sizeof(double) * 2 * 1024));
    double hs[2] = {1.0, 1.0};
    {
        std::vector<double> hp(2 * 1024);
        if (!share) absmax_part_kernel<<<1024, 256, 0, h->setup_stream>>>(h->op64.Bhat, nb * 2 * EE, part);
        absmax_part_kernel<<<1024, 256, 0, h->setup_stream>>>(h->op64.Zt, (size_t)h->T * KK, part + 1024);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * 2 * 1024, cudaMemcpyDeviceToHost, h->setup_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->setup_stream);
        cudaFree(part);
        if (e != cudaSuccess) {
            set_error("operator scale: %s", cudaGetErrorString(e));
            return EMSURF_ECUDA;
        }
        for (int w = share ? 1 : 0; w < 2; ++w) {
            double mx = 0.0;
            for (int i = 0; i < 1024; ++i) mx = std::max(mx, hp[w * 1024 + i]);
            if (mx > 0.0 && std::isfinite(mx)) hs[w] = std::ldexp(1.0, -(std::ilogb(mx) + 1));
        }
        if (share) hs[0] = share->h_ds_scale0;
        h->h_ds_scale0 = hs[0];
        EMS_CUDA(cudaMemcpyAsync(h->d_ds_scale, hs, sizeof(hs), cudaMemcpyHostToDevice, h->setup_stream));
        EMS_CUDA(cudaStreamSynchronize(h->setup_stream));
    }
    if (!share) {
        split_hilo_kernel<<<152 * 16, 256, 0, h->setup_stream>>>(h->ds_planes, h->op64.Bhat, 2 * EE, nb * 2 * EE,
                                                                 h->d_ds_scale);
        EMS_CUDA(cudaGetLastError());
    }
    // the macromodels likewise (the transposed Z~ of each type)
    const size_t zbytes = (size_t)h->T * 2 * KK * sizeof(float2);
    if ((h->K & 1) == 0 && (h->budget <= 0 || h->device_bytes + (int64_t)zbytes <= h->budget)) {
        EMS_TRY(dev_alloc(h, (void**)&h->ds_zt, zbytes));
        split_hilo_kernel<<<152 * 16, 256, 0, h->setup_stream>>>(h->ds_zt, h->op64.Zt, KK, (size_t)h->T * KK,
                                                                 h->d_ds_scale + 1);
        EMS_CUDA(cudaGetLastError());
    }
    return EMSURF_OK;
}

// ---------------------------------------------------------------- apply
template <typename T2>
int apply_operator_io(emsurf_handle* h, Operator<T2>& op, const double2* x, const float2* xf,
                      double2* y, float2* yf, int R, cudaStream_t st) {
    const int E = h->E, K = h->K, px = h->px, py = h->py;
    const long long lanes = (long long)R * K;
    const bool f64 = sizeof(T2) == sizeof(double2);
    const int ph_fft = f64 ? EMS_PH_FFT64 : EMS_PH_FFT32;
    const int ph_bin = f64 ? EMS_PH_BINMUL64 : EMS_PH_BINMUL32;
    const int ph_mm = f64 ? EMS_PH_MM64 : EMS_PH_MM32;
    // K4 runs on the handle's side stream (it reads only x and writes only
    // the partials Ymm that the inverse transform adds).  FP32 products fork
    // before the forward transform, so the macromodel product starts while
    // the transform runs; FP64-accuracy products fork after the per-rhs
    // scales it reads.  The tensor-core variant (>= 8 rhs) stays on the
    // caller's stream.
    const bool side = h->side_stream && !(h->have_tc && R >= kTcMinRhs);
    const bool early_fork = side && std::is_same<T2, float2>::value;
    if (early_fork) {
        EMS_CUDA(cudaEventRecord(h->ev_fork, st));
        EMS_CUDA(cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0));
    }
    prof_mark(h, ph_fft, true, st);
    // K1: x-pass over the cell rows iy < ny reading x1 = U_o x directly
    // (points ix >= nx are the zero padding), then the y-pass with rows
    // iy >= ny taken as zero
    const bool fused = fft2d_fused_ok(px, py);
    if (fused) {
        // one launch: gather, both 1-D transforms, X^ stored
        EMS_TRY(fft2d_forward<T2>(op.Xg, px, lanes, h->nx, h->ny, K, h->n_unique, h->plan_x.tw, x, xf,
                                  h->d_uo_index, h->d_uo_sign, st));
    } else {
        EMS_TRY(fft_pass_gather<T2>(op.Xg, h->plan_x, lanes, h->ny, (long long)px * lanes, h->nx, x,
                                    h->d_uo_index, h->d_uo_sign, h->nx, K, h->n_unique, st, xf));
        EMS_TRY(fft_pass<T2>(op.Xg, h->plan_y, (long long)px * lanes, 1, 0, -1, st, h->ny, py));
    }
    prof_mark(h, ph_fft, false, st);
    if constexpr (std::is_same<T2, double2>::value) {
        if (h->ds_planes && x) {
            // per-rhs powers of two for the double-single operands of this product
            const int nbl = (int)std::min<size_t>(((size_t)h->n_unique + 1023) / 1024, (size_t)h->num_sms);
            pow2_scale_kernel<<<dim3(nbl, R), 256, 0, st>>>(x, (size_t)h->n_unique, h->d_ds_max, h->d_ds_cnt,
                                                            h->d_ds_scale + 2);
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
        }
    }
    cudaStream_t mst = st;
    if (side) {
        if (!early_fork) {
            EMS_CUDA(cudaEventRecord(h->ev_fork, st));
            EMS_CUDA(cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0));
        }
        mst = h->side_stream;
    }
    prof_mark(h, ph_mm, true, mst);
    // K splits of the macromodel product: as many as fill one wave of
    // resident CTAs (a partial second wave would double its time), at most
    // kMmSplit and at least 32 columns each
    bool mm_done = false;
    if constexpr (std::is_same<T2, float2>::value) {
        if (h->have_tc && R >= kTcMinRhs) {
            EMS_TRY(tc_macromodel(h, x, xf, op.Ymm, R, mst));
            mm_done = true;
        }
    }
    const bool blk4 = R >= 4;      // 4 rhs share each load of Z
    const int variant = (std::is_same<T2, float2>::value ? 0 : 1) + (blk4 ? 2 : 0);
    int& mthreads = h->mm_threads[variant];
    if (!mthreads) {
        // one thread per output row, capped by what the kernel's registers allow
        cudaFuncAttributes fa;
        if (blk4) EMS_CUDA(cudaFuncGetAttributes(&fa, macromodel_kernel<T2, kMmGroup, 4>));
        else EMS_CUDA(cudaFuncGetAttributes(&fa, macromodel_kernel<T2, kMmGroup, 1>));
        mthreads = std::max(32, (std::min(fa.maxThreadsPerBlock, ((K + 31) / 32) * 32) / 32) * 32);
    }
    int nsplit = std::max(1, std::min(kMmSplit, K / 32));
    {
        int& occ = h->mm_occ[variant];
        if (!occ) {
            int b = 0;
            const size_t sm = (size_t)(blk4 ? 4 : 1) * kMmGroup * ((K + 1) / 2) * sizeof(T2);
            if (blk4)
                EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, macromodel_kernel<T2, kMmGroup, 4>,
                                                                       mthreads, sm));
            else
                EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, macromodel_kernel<T2, kMmGroup, 1>,
                                                                       mthreads, sm));
            occ = std::max(b, 1);
        }
        const int slots = h->num_sms * occ;
        nsplit = std::max(1, std::min(nsplit, slots / std::max(1, h->n_mm_blocks)));
    }
    {
        // the staged x1 block (rhs block x kMmGroup cells x chunk) must fit in shared memory
        const size_t per_col = (size_t)(blk4 ? 4 : 1) * kMmGroup * sizeof(T2);
        const int max_chunk = (int)((200u * 1024u) / per_col);
        nsplit = std::max(nsplit, (K + max_chunk - 1) / max_chunk);
        nsplit = std::min(nsplit, kMmSplit);
    }
    if (mm_done) nsplit = 1;   // the tensor-core product wrote Ymm[0] whole
    if constexpr (std::is_same<T2, float2>::value) {
        if (!mm_done && R == 1 && (K & 1) == 0) {
            // one rhs: the two-rows-per-thread kernel (K split to fill one wave)
            int& occ2 = h->mm2_occ;
            const int threads2 = std::min(320, ((K / 2 + 31) / 32) * 32);
            const int nblk = h->n_mm_blocks;
            if (!occ2) {
                int b2 = 0;
                EMS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, macromodel2_kernel<kMmGroup>, threads2,
                                                                       (size_t)kMmGroup * ((K + 1) / 2) * sizeof(float2)));
                occ2 = std::max(b2, 1);
            }
            int ns2 = std::max(1, std::min(kMmSplit, K / 64));
            ns2 = std::max(1, std::min(ns2, h->num_sms * occ2 / std::max(1, nblk)));
            int chunk2 = (K + ns2 - 1) / ns2;
            // a multiple of the unroll: the paired x1 reads of a row stay inside it
            chunk2 = (chunk2 + kMm2Unroll - 1) / kMm2Unroll * kMm2Unroll;
            ns2 = (K + chunk2 - 1) / chunk2;
            const size_t sm = (size_t)kMmGroup * chunk2 * sizeof(float2);
            EMS_TRY(set_smem_once(macromodel2_kernel<kMmGroup>, sm));
            macromodel2_kernel<kMmGroup><<<dim3(nblk, ns2), threads2, sm, mst>>>(
                op.Zt, x, h->d_uo_index, h->d_uo_sign, h->d_type_cells,
                reinterpret_cast<const MmBlock*>(h->d_mm_blocks), op.Ymm, K, h->M, h->n_unique, chunk2, xf);
            EMS_CUDA(cudaGetLastError());
            nsplit = ns2;
            mm_done = true;
        }
    }
    if constexpr (std::is_same<T2, double2>::value) {
        if (!mm_done && R == 1 && h->ds_zt) {
            // one rhs, FP64 accuracy from double-single FP32 arithmetic
            const int threads2 = std::min(320, ((K / 2 + 31) / 32) * 32);
            const int nblk = h->n_mm_blocks;
            int ns2 = std::max(1, std::min(kMmSplit, K / 64));
            ns2 = std::max(1, std::min(ns2, h->num_sms * 2 / std::max(1, nblk)));
            int chunk2 = (K + ns2 - 1) / ns2;
            chunk2 = (chunk2 + kMmDsUnroll - 1) / kMmDsUnroll * kMmDsUnroll;
            ns2 = (K + chunk2 - 1) / chunk2;
            const size_t sm = (size_t)2 * kMmGroup * chunk2 * sizeof(float2);
            EMS_TRY(set_smem_once(macromodel_ds_kernel<kMmGroup>, sm));
            macromodel_ds_kernel<kMmGroup><<<dim3(nblk, ns2), threads2, sm, mst>>>(
                h->ds_zt, x, h->d_uo_index, h->d_uo_sign, h->d_type_cells,
                reinterpret_cast<const MmBlock*>(h->d_mm_blocks), op.Ymm, K, h->M, chunk2, h->d_ds_scale);
            EMS_CUDA(cudaGetLastError());
            nsplit = ns2;
            mm_done = true;
        }
    }
    if (!mm_done) {
        const int nblk = h->n_mm_blocks;
        const int chunk = (K + nsplit - 1) / nsplit;
        const MmBlock* blocks = reinterpret_cast<const MmBlock*>(h->d_mm_blocks);
        if (blk4) {
            const size_t sm = (size_t)4 * kMmGroup * chunk * sizeof(T2);
            EMS_TRY(set_smem_once(macromodel_kernel<T2, kMmGroup, 4>, sm));
            macromodel_kernel<T2, kMmGroup, 4><<<dim3(nblk, nsplit), mthreads, sm, mst>>>(
                op.Zt, x, h->d_uo_index, h->d_uo_sign, h->d_type_cells, blocks, op.Ymm, K, h->M, R,
                h->n_unique, chunk, xf);
        } else {
            macromodel_kernel<T2, kMmGroup, 1><<<dim3(nblk, nsplit), mthreads,
                                                 (size_t)kMmGroup * chunk * sizeof(T2), mst>>>(
                op.Zt, x, h->d_uo_index, h->d_uo_sign, h->d_type_cells, blocks, op.Ymm, K, h->M, R,
                h->n_unique, chunk, xf);
        }
        EMS_CUDA(cudaGetLastError());
    }
    prof_mark(h, ph_mm, false, mst);
    if (side) EMS_CUDA(cudaEventRecord(h->ev_join, mst));
    prof_mark(h, ph_bin, true, st);
    // K2
    const int threads = std::min(1024, ((E + 31) / 32) * 32);
    const int nb = h->nbins;
    bool bin_done = false;
    if constexpr (std::is_same<T2, float2>::value) {
        if (h->have_tc && R >= kTcMinRhs) {
            EMS_TRY(tc_binmul(h, op.Xg, op.Yg, R, op.coef, st));
            bin_done = true;
        }
    }
    if constexpr (std::is_same<T2, float2>::value) {
        if (!bin_done && h->orb32) {
            // one stored bin per mirror orbit: one read serves every bin of the orbit
            if (h->orb_G == 8) {
                const int thr = 32 * (1 + kOrbNT8 * ((E + 31) / 32));
                const size_t smem = binmul_orbit_smem<8, kOrbJB8>(E);
                EMS_TRY(set_smem_once(binmul_orbit_kernel<8, kOrbJB8, kOrbNT8>, smem));
                binmul_orbit_kernel<8, kOrbJB8, kOrbNT8><<<h->pair_grid, thr, smem, st>>>(
                    op.Bhat, op.Xg, op.Yg, h->d_orb_bin, h->d_orb_elem, h->d_orb_perm, E, h->nst, 8, op.coef[0],
                    op.coef[1], op.coef[2], op.coef[3], h->d_pair_part, h->d_pair_cnt, h->d_err);
            } else {
                const int thr = 32 * (1 + kOrbNT4 * ((E + 31) / 32));
                const size_t smem = binmul_orbit_smem<4, kOrbJB4>(E);
                EMS_TRY(set_smem_once(binmul_orbit_kernel<4, kOrbJB4, kOrbNT4>, smem));
                binmul_orbit_kernel<4, kOrbJB4, kOrbNT4><<<h->pair_grid, thr, smem, st>>>(
                    op.Bhat, op.Xg, op.Yg, h->d_orb_bin, h->d_orb_elem, h->d_orb_perm, E, h->nst, 4, op.coef[0],
                    op.coef[1], op.coef[2], op.coef[3], h->d_pair_part, h->d_pair_cnt, h->d_err);
            }
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
            bin_done = true;
        }
        if (!bin_done && h->half32) {
            // half spectrum (single rhs): one read of each stored bin serves k and -k
            const size_t smem = binmul_tma_pair_smem(E);
            EMS_TRY(set_smem_once(binmul_tma_pair_kernel, smem));
            binmul_tma_pair_kernel<<<h->pair_grid, 32 * (1 + (E + 31) / 32 + kPairColWarps), smem, st>>>(
                op.Bhat, op.Xg, op.Yg, h->d_st_bin, h->d_st_part, E, h->nst, op.coef[0], op.coef[1], op.coef[2],
                op.coef[3], h->d_pair_part, h->d_pair_cnt, h->d_err);
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
            bin_done = true;
        }
        const size_t smem = binmul_tma_smem(E);
        // the x double buffer needs at least kBmStages stages per bin
        if (!bin_done && R == 1 && smem <= 227 * 1024 && E + 32 <= 1024 && (E + kBmJB - 1) / kBmJB >= kBmStages) {
            EMS_TRY(set_smem_once(binmul_tma_kernel, smem));
            const int grid = std::min(nb, std::max(1, h->num_sms));
            binmul_tma_kernel<<<grid, 32 * (1 + (E + 31) / 32), smem, st>>>(
                op.Bhat, op.Xg, op.Yg, E, nb, op.coef[0], op.coef[1], op.coef[2], op.coef[3], h->d_err);
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
            bin_done = true;
        }
    }
    if constexpr (std::is_same<T2, double2>::value) {
        if (!bin_done && R == 1 && h->ds_planes) {
            // FP64 accuracy from FP32 hi/lo arithmetic (the FP64 rate is ~1/60 of FP32)
            const size_t lanes2 = (size_t)2 * E;
            split_hilo_kernel<<<grid_for((size_t)nb * lanes2, 256), 256, 0, st>>>(h->ds_x, op.Xg, lanes2,
                                                                                (size_t)nb * lanes2,
                                                                                h->d_ds_scale + 2);
            EMS_CUDA(cudaGetLastError());
            const size_t smem = binmul_ds_smem(E);
            EMS_TRY(set_smem_once(binmul_ds_kernel, smem));
            const int grid = std::min(nb, std::max(1, h->num_sms));
            binmul_ds_kernel<<<grid, 32 * (1 + (E + 31) / 32), smem, st>>>(
                h->ds_planes, h->ds_x, op.Yg, E, nb, op.coef[0], op.coef[1], op.coef[2], op.coef[3], h->d_err,
                h->d_ds_scale);
            EMS_CUDA(cudaGetLastError());
            h->launches += 2;
            bin_done = true;
        }
        if (!bin_done && R > 1 && h->ds_planes) {
            // several rhs: FP64 accuracy from double-single FP32 arithmetic,
            // four rhs per pass over the planes
            constexpr int RBd = 4;
            const size_t smem = (size_t)2 * RBd * 2 * E * sizeof(float2);
            EMS_TRY(set_smem_once(binmul_ds_multi_kernel<RBd>, smem));
            const int grid = std::min(nb, 152 * 8);
            for (int r0 = 0; r0 < R; r0 += RBd) {
                binmul_ds_multi_kernel<RBd><<<grid, threads, smem, st>>>(h->ds_planes, op.Xg, op.Yg, E, nb, R, r0,
                                                                      op.coef[0], op.coef[1], op.coef[2],
                                                                      op.coef[3], h->d_ds_scale);
                EMS_CUDA(cudaGetLastError());
                h->launches += 1;
            }
            bin_done = true;
        }
    }
    if (!bin_done) {
        int rb = 1;
        if (R >= 4) rb = 4;
        else if (R >= 2) rb = 2;
        for (int r0 = 0; r0 < R; r0 += rb) {
            const size_t smem = (size_t)rb * K * sizeof(T2);
            const int grid = std::min(nb, 152 * 8);
            if (rb == 4) {
                binmul_kernel<T2, 4><<<grid, threads, smem, st>>>(op.Bhat, op.Xg, op.Yg, E, nb, R, r0,
                                                                  op.coef[0], op.coef[1], op.coef[2], op.coef[3]);
            } else if (rb == 2) {
                binmul_kernel<T2, 2><<<grid, threads, smem, st>>>(op.Bhat, op.Xg, op.Yg, E, nb, R, r0,
                                                                  op.coef[0], op.coef[1], op.coef[2], op.coef[3]);
            } else {
                binmul_kernel<T2, 1><<<grid, threads, smem, st>>>(op.Bhat, op.Xg, op.Yg, E, nb, R, r0,
                                                                  op.coef[0], op.coef[1], op.coef[2], op.coef[3]);
            }
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
        }
    }
    prof_mark(h, ph_bin, false, st);
    if (side) EMS_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));      // the partials are in Ymm
    prof_mark(h, ph_fft, true, st);
    // K3: inverse y-pass on all columns, inverse x-pass on the rows kept
    if (fused) {
        EMS_TRY(fft2d_inverse<T2>(op.Yg, px, lanes, h->nx, h->ny, K, h->M, R, nsplit, 1.0 / (double)h->nbins,
                                  h->plan_x.tw, op.Ymm, op.Y1, st));
    } else {
        EMS_TRY(fft_pass<T2>(op.Yg, h->plan_y, (long long)px * lanes, 1, 0, +1, st, py, h->ny));
        EMS_TRY(fft_pass_crop<T2>(op.Yg, h->plan_x, lanes, h->ny, (long long)px * lanes, h->nx, op.Ymm,
                                  nsplit, R, h->M, K, 1.0 / (double)h->nbins, op.Y1, st));
    }
    prof_mark(h, ph_fft, false, st);
    prof_mark(h, EMS_PH_SCATTER, true, st);
    if (yf)
        scatter_kernel<T2, float2><<<grid_for((size_t)R * h->n_unique, 256), 256, 0, st>>>(
            yf, op.Y1, h->d_inv_ptr, h->d_inv_ent, h->d_inv_sgn, h->M * K, R, h->n_unique);
    else
        scatter_kernel<T2, double2><<<grid_for((size_t)R * h->n_unique, 256), 256, 0, st>>>(
            y, op.Y1, h->d_inv_ptr, h->d_inv_ent, h->d_inv_sgn, h->M * K, R, h->n_unique);
    EMS_CUDA(cudaGetLastError());
    prof_mark(h, EMS_PH_SCATTER, false, st);
    h->launches += fused ? 4 : 6;   // FFTs (2 fused or 4 passes), macromodel, scatter
    return EMSURF_OK;
}

template int build_operator<double2>(emsurf_handle*, Operator<double2>&, const emsurf_problem*,
                                     const Operator<double2>*);
template int build_operator<float2>(emsurf_handle*, Operator<float2>&, const emsurf_problem*,
                                    const Operator<float2>*);
template <typename T2>
int apply_operator(emsurf_handle* h, Operator<T2>& op, const double2* x, double2* y, int R,
                   cudaStream_t st) {
    return apply_operator_io<T2>(h, op, x, nullptr, y, nullptr, R, st);
}

int apply_operator_f32(emsurf_handle* h, const float2* x, float2* y, int R, cudaStream_t st) {
    return apply_operator_io<float2>(h, h->op32, nullptr, x, nullptr, y, R, st);
}

template int apply_operator<double2>(emsurf_handle*, Operator<double2>&, const double2*, double2*,
                                     int, cudaStream_t);
template int apply_operator<float2>(emsurf_handle*, Operator<float2>&, const double2*, double2*,
                                    int, cudaStream_t);

}  // namespace emsurf

namespace emsurf {
int wait_selftest(emsurf_handle* h, long long limit, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit, h->d_err);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}
}  // namespace emsurf
