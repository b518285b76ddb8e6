// Lane-vectorised mixed-radix FFT passes for the lattice grids.
//
// Sec. IV-B evaluates each Toeplitz block product with the FFT of its
// circulant embedding (Eqs. LJV3-LJV5) and generalises to 2-D lattices with
// 2-D FFTs.  Here every 2-D transform is two 1-D passes.  A pass transforms
// data[outer][P][inner] along P; the `inner` dimension holds independent
// sequences (local unknowns k, right-hand sides, or block entries (op,j,i))
// that sit next to each other in memory, so one CTA loads a P x W tile whose
// rows are W contiguous lanes (coalesced), transforms all W lanes in shared
// memory with a Stockham autosort mixed-radix algorithm (radices 2,3,4,5,7;
// Govindaraju et al., SC 2008), and writes the tile back.
//
// Pruning: only the first p_in points along P are read (the rest are the
// zero padding of the circulant embedding) and only the first p_out are
// written (the crop of the inverse transform).  The forward pass over the
// cell rows can read its input straight from the unique-unknown vector
// through U_o (x1 = U_o x, Eq. MVP), so no padded grid is ever written.
//
// Grid sizes used by the lattices here have compile-time kernels (radices,
// strides and twiddle indices are constants, twiddles sit in shared memory);
// any other 2,3,5,7-smooth size runs a generic kernel.
#include <cmath>

#include "common.cuh"

namespace emsurf {

namespace {

constexpr int kFftThreads = 256;
constexpr int kMaxRadix = 7;

// ---------------------------------------------------------------- radices
constexpr int rad_count(int P) {
    int n = 0;
    const int qs[5] = {4, 2, 3, 5, 7};
    for (int i = 0; i < 5; ++i)
        while (P % qs[i] == 0 && P > 1) {
            P /= qs[i];
            ++n;
        }
    return n;
}
constexpr int rad_at(int P, int s) {
    int n = 0;
    const int qs[5] = {4, 2, 3, 5, 7};
    for (int i = 0; i < 5; ++i)
        while (P % qs[i] == 0 && P > 1) {
            if (n == s) return qs[i];
            P /= qs[i];
            ++n;
        }
    return 1;
}

template <typename T2>
__device__ __forceinline__ T2 mul_i(T2 a, int s) {   // a * (s i), s = +-1
    T2 r;
    r.x = -s * a.y;
    r.y = s * a.x;
    return r;
}
template <typename T2>
__device__ __forceinline__ T2 csub2(T2 a, T2 b) {
    T2 r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}

// One Stockham stage of radix R (compile time) over all W lanes.
template <typename T2, int W, int P, int R, int NS, int SIGN>
__device__ __forceinline__ void stage(const T2* __restrict__ in, T2* __restrict__ out,
                                      const T2* __restrict__ tw) {
    constexpr int NR = P / R;
    constexpr int tstep = P / (NS * R);
    constexpr int qstep = P / R;
    for (int e = threadIdx.x; e < NR * W; e += blockDim.x) {
        const int j = e / W, l = e % W;
        const int jm = j % NS;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T2 a = in[(j + r * NR) * W + l];
            v[r] = (r == 0 || NS == 1) ? a : cmul(a, tw[jm * r * tstep]);
        }
        const int idxD = (j / NS) * NS * R + jm;
        if constexpr (R == 2) {
            out[idxD * W + l] = cadd(v[0], v[1]);
            out[(idxD + NS) * W + l] = csub2(v[0], v[1]);
        } else if constexpr (R == 4) {
            // w_4 = e^{SIGN 2 pi i / 4} = SIGN i
            const T2 s02 = cadd(v[0], v[2]), d02 = csub2(v[0], v[2]);
            const T2 s13 = cadd(v[1], v[3]), d13 = csub2(v[1], v[3]);
            out[idxD * W + l] = cadd(s02, s13);
            out[(idxD + NS) * W + l] = cadd(d02, mul_i(d13, SIGN));
            out[(idxD + 2 * NS) * W + l] = csub2(s02, s13);
            out[(idxD + 3 * NS) * W + l] = csub2(d02, mul_i(d13, SIGN));
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                T2 acc = v[0];
#pragma unroll
                for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((q * r) % R) * qstep]));
                out[(idxD + q * NS) * W + l] = acc;
            }
        }
    }
}

template <typename T2, int W, int P, int S, int NS, int SIGN>
struct Stages {
    // returns the buffer holding the result
    static __device__ __forceinline__ T2* run(T2* in, T2* out, const T2* tw) {
        if constexpr (S < rad_count(P)) {
            constexpr int R = rad_at(P, S);
            stage<T2, W, P, R, NS, SIGN>(in, out, tw);
            __syncthreads();
            return Stages<T2, W, P, S + 1, NS * R, SIGN>::run(out, in, tw);
        } else {
            return in;
        }
    }
};

// Gather source of the forward pass over cell rows: element (row iy, point
// ix, lane L = r*K + k) = sign * x[r][uo_index[(iy*nx + ix)*K + k]].
struct GatherSrc {
    const double2* x;
    const int32_t* idx;
    const int8_t* sgn;
    int nx, K, n_unique;
    const float2* xf;   // FP32 source instead of x when not null
};

// sign * x[r][u] of the gather, from the FP64 or the FP32 source; an FP32
// source into an FP32 grid needs no FP64 arithmetic
template <typename T2>
__device__ __forceinline__ T2 gather_value(const GatherSrc& gs, int r, size_t loc) {
    const size_t at = (size_t)r * gs.n_unique + gs.idx[loc];
    if (gs.xf) {
        const float2 xv = gs.xf[at];
        const float s = (float)gs.sgn[loc];
        if constexpr (sizeof(T2) == sizeof(float2)) return make_float2(s * xv.x, s * xv.y);
        else return mk<T2>((double)(s * xv.x), (double)(s * xv.y));
    }
    const double2 xv = gs.x[at];
    const double s = (double)gs.sgn[loc];
    return mk<T2>(s * xv.x, s * xv.y);
}

// Store epilogue of the inverse pass over the kept rows: point ix < nx of row
// iy, lane L = r*K + k, goes to y1[r][iy*nx + ix][k] = scale * value +
// sum_s mm[s][r][m][k] (the macromodel partials).
template <typename T2>
struct CropEpi {
    const T2* mm;
    T2* y1;
    int nsplit, R, M, nx, K;
    double scale;
};

template <typename T2>
__device__ __forceinline__ void crop_store(const CropEpi<T2>& ep, int iy, int p, long long L, T2 v) {
    const int r = (int)(L / ep.K), k = (int)(L % ep.K);
    const size_t m = (size_t)iy * ep.nx + p;
    // in the precision of the grid (no FP64 arithmetic on the FP32 path)
    using S = decltype(v.x);
    const S sc = (S)ep.scale;
    S ax = v.x * sc, ay = v.y * sc;
    for (int s = 0; s < ep.nsplit; ++s) {
        const T2 z = ep.mm[(((size_t)s * ep.R + r) * ep.M + m) * ep.K + k];
        ax += z.x;
        ay += z.y;
    }
    T2 o;
    o.x = ax;
    o.y = ay;
    ep.y1[((size_t)r * ep.M + m) * ep.K + k] = o;
}

template <typename T2, int W, int P, int SIGN, bool GATHER, bool EPI>
__global__ void __launch_bounds__(kFftThreads)
fft_fixed_kernel(T2* __restrict__ data, long long inner, long long outer_stride, int p_in, int p_out,
                 const double2* __restrict__ twg, GatherSrc gs, CropEpi<T2> ep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* buf0 = reinterpret_cast<T2*>(smem_raw);
    T2* buf1 = buf0 + P * W;
    T2* tw = buf1 + P * W;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const double2 w = twg[e];
        tw[e] = mk<T2>(w.x, SIGN < 0 ? w.y : -w.y);
    }
    const long long lane0 = (long long)blockIdx.x * W;
    const int wl = (int)min((long long)W, inner - lane0);
    T2* base = data + (long long)blockIdx.y * outer_stride + lane0;
    const T2 zero = mk<T2>(0.0, 0.0);
    for (int e = threadIdx.x; e < P * W; e += blockDim.x) {
        const int p = e / W, l = e % W;
        T2 v = zero;
        if (l < wl && p < p_in) {
            if constexpr (GATHER) {
                const long long L = lane0 + l;
                const int r = (int)(L / gs.K), k = (int)(L % gs.K);
                const size_t loc = ((size_t)blockIdx.y * gs.nx + p) * gs.K + k;
                v = gather_value<T2>(gs, r, loc);
            } else {
                v = base[(long long)p * inner + l];
            }
        }
        buf0[e] = v;
    }
    __syncthreads();
    const T2* res = Stages<T2, W, P, 0, 1, SIGN>::run(buf0, buf1, tw);
    for (int e = threadIdx.x; e < p_out * W; e += blockDim.x) {
        const int p = e / W, l = e % W;
        if (l < wl) {
            if constexpr (EPI) crop_store(ep, blockIdx.y, p, lane0 + l, res[e]);
            else base[(long long)p * inner + l] = res[e];
        }
    }
}

// ---------------------------------------------------------------- generic
struct RadList {
    int n;
    int r[16];
};

template <typename T2>
__device__ __forceinline__ T2 tw_at(const double2* __restrict__ tw, int k, int sign) {
    double2 w = tw[k];
    return mk<T2>(w.x, sign < 0 ? w.y : -w.y);
}

template <typename T2, int W>
__global__ void __launch_bounds__(kFftThreads)
fft_pass_kernel(T2* __restrict__ data, int P, long long inner, long long outer_stride, int p_in,
                int p_out, const double2* __restrict__ tw, RadList rad, int sign, GatherSrc gs,
                int gather, CropEpi<T2> ep, int epi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* buf0 = reinterpret_cast<T2*>(smem_raw);
    T2* buf1 = buf0 + (size_t)P * W;
    const long long lane0 = (long long)blockIdx.x * W;
    const int wl = (int)min((long long)W, inner - lane0);
    T2* base = data + (long long)blockIdx.y * outer_stride + lane0;
    const T2 zero = mk<T2>(0.0, 0.0);

    for (int e = threadIdx.x; e < P * W; e += blockDim.x) {
        const int p = e / W, l = e - (e / W) * W;
        T2 v = zero;
        if (l < wl && p < p_in) {
            if (gather) {
                const long long L = lane0 + l;
                const int r = (int)(L / gs.K), k = (int)(L % gs.K);
                const size_t loc = ((size_t)blockIdx.y * gs.nx + p) * gs.K + k;
                v = gather_value<T2>(gs, r, loc);
            } else {
                v = base[(long long)p * inner + l];
            }
        }
        buf0[e] = v;
    }
    __syncthreads();

    T2* in = buf0;
    T2* out = buf1;
    int Ns = 1;
    for (int s = 0; s < rad.n; ++s) {
        const int R = rad.r[s];
        const int NR = P / R;
        const int tstep = P / (Ns * R);   // twiddle stride of w_{Ns R}
        const int qstep = P / R;          // stride of w_R
        for (int e = threadIdx.x; e < NR * W; e += blockDim.x) {
            const int j = e / W, l = e - (e / W) * W;
            const int jm = j % Ns;
            T2 v[kMaxRadix];
#pragma unroll
            for (int r = 0; r < kMaxRadix; ++r) {
                if (r < R) {
                    T2 a = in[(j + r * NR) * W + l];
                    v[r] = (r == 0 || jm == 0) ? a : cmul(a, tw_at<T2>(tw, jm * r * tstep, sign));
                }
            }
            const int idxD = (j / Ns) * Ns * R + jm;
#pragma unroll
            for (int q = 0; q < kMaxRadix; ++q) {
                if (q < R) {
                    T2 acc = v[0];
#pragma unroll
                    for (int r = 1; r < kMaxRadix; ++r) {
                        if (r < R) acc = cadd(acc, cmul(v[r], tw_at<T2>(tw, ((q * r) % R) * qstep, sign)));
                    }
                    out[(idxD + q * Ns) * W + l] = acc;
                }
            }
        }
        Ns *= R;
        T2* t = in;
        in = out;
        out = t;
        __syncthreads();
    }

    for (int e = threadIdx.x; e < p_out * W; e += blockDim.x) {
        const int p = e / W, l = e - (e / W) * W;
        if (l < wl) {
            if (epi) crop_store(ep, blockIdx.y, p, lane0 + l, in[e]);
            else base[(long long)p * inner + l] = in[e];
        }
    }
}

// lanes per CTA: the largest of 32, 16, 8 whose two buffers fit in 96 KB
template <typename T2>
constexpr int lanes_for(int P) {
    return (2 * P * 32 * (int)sizeof(T2) <= 96 * 1024) ? 32
         : (2 * P * 16 * (int)sizeof(T2) <= 96 * 1024) ? 16 : 8;
}

template <typename T2, int P, int SIGN, bool GATHER, bool EPI>
int launch_fixed(T2* data, const FftPlan& plan, long long inner, long long outer,
                 long long outer_stride, int p_in, int p_out, const GatherSrc& gs,
                 const CropEpi<T2>& ep, cudaStream_t st) {
    constexpr int W = lanes_for<T2>(P);
    const size_t smem = (2ull * P * W + P) * sizeof(T2);
    auto kern = fft_fixed_kernel<T2, W, P, SIGN, GATHER, EPI>;
    EMS_TRY(set_smem_once(kern, smem));
    const long long gx = (inner + W - 1) / W;
    dim3 grid((unsigned)gx, (unsigned)outer);
    kern<<<grid, kFftThreads, smem, st>>>(data, inner, outer_stride, p_in, p_out, plan.tw, gs, ep);
    EMS_CUDA(cudaGetLastError());
    return EMSURF_OK;
}

template <typename T2, int W>
int launch_generic(T2* data, const FftPlan& plan, long long inner, long long outer,
                   long long outer_stride, int p_in, int p_out, int sign, const GatherSrc& gs,
                   bool gather, const CropEpi<T2>& ep, bool epi, cudaStream_t st) {
    RadList rl;
    rl.n = plan.nrad;
    for (int i = 0; i < 16; ++i) rl.r[i] = plan.rad[i];
    const size_t smem = 2ull * plan.P * W * sizeof(T2);
    EMS_TRY(set_smem_once(fft_pass_kernel<T2, W>, smem));
    const long long gx = (inner + W - 1) / W;
    dim3 grid((unsigned)gx, (unsigned)outer);
    fft_pass_kernel<T2, W><<<grid, kFftThreads, smem, st>>>(data, plan.P, inner, outer_stride, p_in,
                                                            p_out, plan.tw, rl, sign, gs, gather ? 1 : 0,
                                                            ep, epi ? 1 : 0);
    EMS_CUDA(cudaGetLastError());
    return EMSURF_OK;
}

template <typename T2, int SIGN, bool GATHER, bool EPI>
int dispatch_fixed(int P, T2* data, const FftPlan& plan, long long inner, long long outer,
                   long long os, int p_in, int p_out, const GatherSrc& gs, const CropEpi<T2>& ep,
                   cudaStream_t st, bool* done) {
    *done = true;
#define EMS_FFT_CASE(N) \
    case N: return launch_fixed<T2, N, SIGN, GATHER, EPI>(data, plan, inner, outer, os, p_in, p_out, gs, ep, st);
    switch (P) {
        EMS_FFT_CASE(5)
        EMS_FFT_CASE(8)
        EMS_FFT_CASE(15)
        EMS_FFT_CASE(16)
        EMS_FFT_CASE(24)
        EMS_FFT_CASE(32)
        EMS_FFT_CASE(48)
        EMS_FFT_CASE(64)
        EMS_FFT_CASE(96)
        EMS_FFT_CASE(128)
        EMS_FFT_CASE(200)
        default: *done = false; return EMSURF_OK;
    }
#undef EMS_FFT_CASE
}

template <typename T2>
int pass_impl(T2* data, const FftPlan& plan, long long inner, long long outer, long long outer_stride,
              int sign, int p_in, int p_out, const GatherSrc& gs, bool gather, const CropEpi<T2>& ep,
              bool epi, cudaStream_t st) {
    if (outer <= 0 || inner <= 0) return EMSURF_OK;
    if (outer > 65535 || (inner + 7) / 8 > 2147483647LL) {
        set_error("fft_pass: grid too large (outer %lld, lanes %lld)", outer, inner);
        return EMSURF_EINVAL;
    }
    p_in = p_in < 0 ? plan.P : std::min(p_in, plan.P);
    p_out = p_out < 0 ? plan.P : std::min(p_out, plan.P);
    bool done = false;
    int s = EMSURF_OK;
    if (sign < 0 && gather)
        s = dispatch_fixed<T2, -1, true, false>(plan.P, data, plan, inner, outer, outer_stride, p_in, p_out, gs, ep, st, &done);
    else if (sign < 0)
        s = dispatch_fixed<T2, -1, false, false>(plan.P, data, plan, inner, outer, outer_stride, p_in, p_out, gs, ep, st, &done);
    else if (epi)
        s = dispatch_fixed<T2, +1, false, true>(plan.P, data, plan, inner, outer, outer_stride, p_in, p_out, gs, ep, st, &done);
    else
        s = dispatch_fixed<T2, +1, false, false>(plan.P, data, plan, inner, outer, outer_stride, p_in, p_out, gs, ep, st, &done);
    if (s != EMSURF_OK || done) return s;
    const size_t per_lane = 2ull * plan.P * sizeof(T2);
    if (per_lane * 32 <= 200 * 1024)
        return launch_generic<T2, 32>(data, plan, inner, outer, outer_stride, p_in, p_out, sign, gs, gather, ep, epi, st);
    if (per_lane * 16 <= 200 * 1024)
        return launch_generic<T2, 16>(data, plan, inner, outer, outer_stride, p_in, p_out, sign, gs, gather, ep, epi, st);
    if (per_lane * 8 <= 200 * 1024)
        return launch_generic<T2, 8>(data, plan, inner, outer, outer_stride, p_in, p_out, sign, gs, gather, ep, epi, st);
    set_error("FFT length %d too large for one shared-memory pass", plan.P);
    return EMSURF_EINVAL;
}

}  // namespace

int smallest_smooth_at_least(int n) {
    for (int m = (n < 1 ? 1 : n);; ++m) {
        int t = m;
        for (int p : {2, 3, 5})
            while (t % p == 0) t /= p;
        if (t == 1) return m;
    }
}

int fft_plan_create(FftPlan& plan, int P) {
    int t = P, n = 0;
    int rad[16];
    while (t % 4 == 0 && n < 16) { rad[n++] = 4; t /= 4; }
    while (t % 2 == 0 && n < 16) { rad[n++] = 2; t /= 2; }
    while (t % 3 == 0 && n < 16) { rad[n++] = 3; t /= 3; }
    while (t % 5 == 0 && n < 16) { rad[n++] = 5; t /= 5; }
    while (t % 7 == 0 && n < 16) { rad[n++] = 7; t /= 7; }
    if (t != 1 || P < 1) {
        set_error("FFT length %d has a prime factor other than 2, 3, 5, 7", P);
        return EMSURF_EINVAL;
    }
    plan.P = P;
    plan.nrad = n;
    for (int i = 0; i < 16; ++i) plan.rad[i] = i < n ? rad[i] : 0;
    std::vector<double2> h(P);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < P; ++k) {
        // exact values on the axes; host libm elsewhere
        const double ang = two_pi * (double)k / (double)P;
        double c = std::cos(ang), s = std::sin(ang);
        if (4 * k == P) { c = 0.0; s = 1.0; }
        if (2 * k == P) { c = -1.0; s = 0.0; }
        if (4 * k == 3 * P) { c = 0.0; s = -1.0; }
        h[k] = make_double2(c, -s);
    }
    EMS_CUDA(cudaMalloc(&plan.tw, sizeof(double2) * P));
    EMS_CUDA(cudaMemcpy(plan.tw, h.data(), sizeof(double2) * P, cudaMemcpyHostToDevice));
    return EMSURF_OK;
}

void fft_plan_destroy(FftPlan& plan) {
    if (plan.tw) cudaFree(plan.tw);
    plan.tw = nullptr;
}

template <typename T2>
int fft_pass(T2* data, const FftPlan& plan, long long inner, long long outer,
             long long outer_stride, int sign, cudaStream_t st, int p_in, int p_out) {
    GatherSrc gs{nullptr, nullptr, nullptr, 0, 1, 0, nullptr};
    CropEpi<T2> ep{nullptr, nullptr, 0, 1, 1, 1, 1, 1.0};
    return pass_impl<T2>(data, plan, inner, outer, outer_stride, sign, p_in, p_out, gs, false, ep,
                         false, st);
}

template <typename T2>
int fft_pass_gather(T2* data, const FftPlan& plan, long long inner, long long outer,
                    long long outer_stride, int p_in, const double2* x, const int32_t* idx,
                    const int8_t* sgn, int nx, int K, int n_unique, cudaStream_t st, const float2* xf) {
    GatherSrc gs{x, idx, sgn, nx, K, n_unique, xf};
    CropEpi<T2> ep{nullptr, nullptr, 0, 1, 1, 1, 1, 1.0};
    return pass_impl<T2>(data, plan, inner, outer, outer_stride, -1, p_in, plan.P, gs, true, ep, false,
                         st);
}

template <typename T2>
int fft_pass_crop(T2* data, const FftPlan& plan, long long inner, long long outer,
                  long long outer_stride, int nx, const T2* mm, int nsplit, int R, int M, int K,
                  double scale, T2* y1, cudaStream_t st) {
    GatherSrc gs{nullptr, nullptr, nullptr, 0, 1, 0, nullptr};
    CropEpi<T2> ep{mm, y1, nsplit, R, M, nx, K, scale};
    return pass_impl<T2>(data, plan, inner, outer, outer_stride, +1, plan.P, nx, gs, false, ep, true,
                         st);
}

template int fft_pass<double2>(double2*, const FftPlan&, long long, long long, long long, int,
                               cudaStream_t, int, int);
template int fft_pass<float2>(float2*, const FftPlan&, long long, long long, long long, int,
                              cudaStream_t, int, int);
template int fft_pass_gather<double2>(double2*, const FftPlan&, long long, long long, long long, int,
                                      const double2*, const int32_t*, const int8_t*, int, int, int,
                                      cudaStream_t, const float2*);
template int fft_pass_gather<float2>(float2*, const FftPlan&, long long, long long, long long, int,
                                     const double2*, const int32_t*, const int8_t*, int, int, int,
                                     cudaStream_t, const float2*);
template int fft_pass_crop<double2>(double2*, const FftPlan&, long long, long long, long long, int,
                                    const double2*, int, int, int, int, double, double2*, cudaStream_t);
template int fft_pass_crop<float2>(float2*, const FftPlan&, long long, long long, long long, int,
                                   const float2*, int, int, int, int, double, float2*, cudaStream_t);

}  // namespace emsurf
