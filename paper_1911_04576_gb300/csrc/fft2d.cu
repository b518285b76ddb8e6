// Fused 2-D transforms of one product's grids (Sec. IV-B: the circulant
// embedding of the block-Toeplitz lattice operator, applied with 2-D FFTs).
//
// The pass-based transforms (fft.cu) run each 2-D FFT as two launches with
// the grid written to global memory in between.  For square grids of up to
// 64 x 64 points a CTA here holds a whole P x P grid for W lanes (local
// unknowns k of one or more rhs) in shared memory and does the gather of
// x1 = U_o x, both 1-D transforms and the store of X^ in one launch; the
// inverse does both inverse transforms, the crop to the lattice, the 1/P
// scale and the addition of the macromodel partials in one launch.
//
// Layouts in shared memory (W lanes contiguous):
//   rows:    A[ix][iy * W + w]  (the x-transform's lanes are (iy, w))
//   columns: B[iy][kx * W + w]  (the y-transform's lanes are (kx, w))
// The 1-D transforms are Stockham autosort stages (radices 4, 2, 3, 5, 7;
// Govindaraju et al., SC 2008) over a runtime number of lanes.
#include "common.cuh"

namespace emsurf {
namespace {


constexpr int f2_rad_count(int P) {
    int n = 0;
    const int qs[5] = {4, 2, 3, 5, 7};
    for (int i = 0; i < 5; ++i)
        while (P % qs[i] == 0 && P > 1) {
            P /= qs[i];
            ++n;
        }
    return n;
}
constexpr int f2_rad_at(int P, int s) {
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
__device__ __forceinline__ T2 f2_sub(T2 a, T2 b) {
    T2 r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}
template <typename T2>
__device__ __forceinline__ T2 f2_muli(T2 a, int s) {   // a * (s i)
    T2 r;
    r.x = -s * a.y;
    r.y = s * a.x;
    return r;
}

// one radix-R Stockham stage over nl lanes: element (p, l) at p * nl + l
template <typename T2, int P, int R, int NS, int SIGN>
__device__ __forceinline__ void f2_stage(const T2* __restrict__ in, T2* __restrict__ out,
                                         const T2* __restrict__ tw, int nl) {
    constexpr int NR = P / R;
    constexpr int tstep = P / (NS * R);
    constexpr int qstep = P / R;
    for (int e = threadIdx.x; e < NR * nl; e += blockDim.x) {
        const int j = e / nl, l = e - j * nl;
        const int jm = j % NS;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T2 a = in[(j + r * NR) * nl + l];
            v[r] = (r == 0 || NS == 1) ? a : cmul(a, tw[jm * r * tstep]);
        }
        const int d = (j / NS) * NS * R + jm;
        if constexpr (R == 2) {
            out[d * nl + l] = cadd(v[0], v[1]);
            out[(d + NS) * nl + l] = f2_sub(v[0], v[1]);
        } else if constexpr (R == 4) {
            const T2 s02 = cadd(v[0], v[2]), d02 = f2_sub(v[0], v[2]);
            const T2 s13 = cadd(v[1], v[3]), d13 = f2_sub(v[1], v[3]);
            out[d * nl + l] = cadd(s02, s13);
            out[(d + NS) * nl + l] = cadd(d02, f2_muli(d13, SIGN));
            out[(d + 2 * NS) * nl + l] = f2_sub(s02, s13);
            out[(d + 3 * NS) * nl + l] = f2_sub(d02, f2_muli(d13, SIGN));
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                T2 acc = v[0];
#pragma unroll
                for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((q * r) % R) * qstep]));
                out[(d + q * NS) * nl + l] = acc;
            }
        }
    }
}

template <typename T2, int P, int S, int NS, int SIGN>
struct F2Stages {
    // transforms in place between the two buffers; returns the one holding the result
    static __device__ __forceinline__ T2* run(T2* in, T2* out, const T2* tw, int nl) {
        if constexpr (S < f2_rad_count(P)) {
            constexpr int R = f2_rad_at(P, S);
            f2_stage<T2, P, R, NS, SIGN>(in, out, tw, nl);
            __syncthreads();
            return F2Stages<T2, P, S + 1, NS * R, SIGN>::run(out, in, tw, nl);
        } else {
            return in;
        }
    }
};

// lanes per CTA: at most what keeps the grid of W lanes twice (ping-pong)
// within ~96 KB (one lane when the grid alone is larger).  The launch takes
// the widest W while that still gives at least one CTA per SM (measured at
// 16x16, K = 576, one rhs: W = 4 with 512 threads 10.1 + 12.2 us per
// forward + inverse pair, W = 1 with 256 threads 12.3 + 13.7 us).
template <typename T2, int P>
constexpr int f2_max_lanes() {
    constexpr int per = 2 * P * P * (int)sizeof(T2);
    return per * 8 <= 96 * 1024 ? 8 : per * 4 <= 96 * 1024 ? 4 : per * 2 <= 96 * 1024 ? 2 : 1;
}

template <typename T2, int P, int W>
constexpr size_t f2_smem() {
    return (size_t)(2 * P * P * W + P) * sizeof(T2);
}

template <int W>
constexpr int f2_threads() { return W >= 4 ? 512 : 256; }

int f2_pick_lanes(int max_w, long long lanes) {
    static int sm_count[64] = {};      // per device, filled on first use
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        if (!sm_count[dev]) cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
        if (sm_count[dev] > 0) sms = sm_count[dev];
    }
    for (int w = max_w; w > 1; w >>= 1)
        if ((lanes + w - 1) / w >= (long long)sms * 9 / 10) return w;
    return 1;
}

template <typename T2, int SIGN>
__device__ __forceinline__ void f2_twiddles(T2* tw, const double2* __restrict__ twg, int P) {
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const double2 w = twg[e];
        tw[e] = mk<T2>(w.x, SIGN < 0 ? w.y : -w.y);
    }
}

// X^[ky * P + kx][lane] of x1 = U_o x (sign * x[r][uo_index[(iy nx + ix) K + k]],
// lane = r K + k), zero outside the lattice
template <typename T2, int P, int W>
__global__ void __launch_bounds__(f2_threads<W>())
fft2d_fwd_kernel(T2* __restrict__ Xg, long long lanes, int nx, int ny, int K, int n_unique,
                 const double2* __restrict__ twg, const double2* __restrict__ x, const float2* __restrict__ xf,
                 const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    T2* b1 = b0 + P * P * W;
    T2* tw = b1 + P * P * W;
    f2_twiddles<T2, -1>(tw, twg, P);
    const long long lane0 = (long long)blockIdx.x * W;
    const int wl = (int)min((long long)W, lanes - lane0);
    const int nlx = ny * W;
    // gather the cell rows into A[ix][iy * W + w]
    for (int e = threadIdx.x; e < P * nlx; e += blockDim.x) {
        const int ix = e / nlx, rem = e - ix * nlx, iy = rem / W, w = rem - iy * W;
        T2 v = mk<T2>(0.0, 0.0);
        if (ix < nx && w < wl) {
            const long long L = lane0 + w;
            const int r = (int)(L / K), k = (int)(L - (long long)r * K);
            const size_t loc = ((size_t)iy * nx + ix) * K + k;
            const size_t at = (size_t)r * n_unique + idx[loc];
            if (xf) {
                const float s = (float)sgn[loc];
                const float2 xv = xf[at];
                v = mk<T2>((double)(s * xv.x), (double)(s * xv.y));
                if constexpr (sizeof(T2) == sizeof(float2)) v = make_float2(s * xv.x, s * xv.y);
            } else {
                const double s = (double)sgn[loc];
                const double2 xv = x[at];
                v = mk<T2>(s * xv.x, s * xv.y);
            }
        }
        b0[e] = v;
    }
    __syncthreads();
    T2* r1 = F2Stages<T2, P, 0, 1, -1>::run(b0, b1, tw, nlx);
    T2* o1 = r1 == b0 ? b1 : b0;
    // columns: B[iy][kx * W + w], rows iy >= ny are the zero padding
    const int nly = P * W;
    for (int e = threadIdx.x; e < P * nly; e += blockDim.x) {
        const int iy = e / nly, rem = e - iy * nly, kx = rem / W, w = rem - kx * W;
        o1[e] = iy < ny ? r1[kx * nlx + iy * W + w] : mk<T2>(0.0, 0.0);
    }
    __syncthreads();
    T2* r2 = F2Stages<T2, P, 0, 1, -1>::run(o1, r1, tw, nly);
    for (int e = threadIdx.x; e < P * P * W; e += blockDim.x) {
        const int bin = e / W, w = e - bin * W;
        if (w < wl) Xg[(size_t)bin * lanes + lane0 + w] = r2[e];
    }
}

// y1[r][iy nx + ix][k] = scale * IFFT2(Y^)[iy][ix] + sum_s mm[s][r][m][k] for
// the lattice points (the crop of the circulant embedding)
template <typename T2, int P, int W>
__global__ void __launch_bounds__(f2_threads<W>())
fft2d_inv_kernel(const T2* __restrict__ Yg, long long lanes, int nx, int ny, int K, int M, int R,
                 int nsplit, double scale, const double2* __restrict__ twg, const T2* __restrict__ mm,
                 T2* __restrict__ y1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    T2* b1 = b0 + P * P * W;
    T2* tw = b1 + P * P * W;
    f2_twiddles<T2, +1>(tw, twg, P);
    const long long lane0 = (long long)blockIdx.x * W;
    const int wl = (int)min((long long)W, lanes - lane0);
    const int nly = P * W;
    for (int e = threadIdx.x; e < P * P * W; e += blockDim.x) {
        const int bin = e / W, w = e - bin * W;
        b0[e] = w < wl ? Yg[(size_t)bin * lanes + lane0 + w] : mk<T2>(0.0, 0.0);
    }
    __syncthreads();
    T2* r1 = F2Stages<T2, P, 0, 1, +1>::run(b0, b1, tw, nly);
    T2* o1 = r1 == b0 ? b1 : b0;
    // rows kept (iy < ny) into A[kx][iy * W + w]
    const int nlx = ny * W;
    for (int e = threadIdx.x; e < P * nlx; e += blockDim.x) {
        const int kx = e / nlx, rem = e - kx * nlx, iy = rem / W, w = rem - iy * W;
        o1[e] = r1[iy * nly + kx * W + w];
    }
    __syncthreads();
    T2* r2 = F2Stages<T2, P, 0, 1, +1>::run(o1, r1, tw, nlx);
    using S = decltype(r2[0].x);
    const S sc = (S)scale;
    for (int e = threadIdx.x; e < nx * nlx; e += blockDim.x) {
        const int ix = e / nlx, rem = e - ix * nlx, iy = rem / W, w = rem - iy * W;
        if (w >= wl) continue;
        const long long L = lane0 + w;
        const int r = (int)(L / K), k = (int)(L - (long long)r * K);
        const size_t m = (size_t)iy * nx + ix;
        const T2 v = r2[e];
        S ax = v.x * sc, ay = v.y * sc;
        for (int s = 0; s < nsplit; ++s) {
            const T2 z = mm[(((size_t)s * R + r) * M + m) * K + k];
            ax += z.x;
            ay += z.y;
        }
        T2 o;
        o.x = ax;
        o.y = ay;
        y1[((size_t)r * M + m) * K + k] = o;
    }
}

template <typename T2, int P, int W>
int f2_fwd_w(T2* Xg, long long lanes, int nx, int ny, int K, int n_unique, const double2* tw, const double2* x,
             const float2* xf, const int32_t* idx, const int8_t* sgn, cudaStream_t st) {
    constexpr size_t smem = f2_smem<T2, P, W>();
    EMS_TRY(set_smem_once(fft2d_fwd_kernel<T2, P, W>, smem));
    fft2d_fwd_kernel<T2, P, W><<<(unsigned)((lanes + W - 1) / W), f2_threads<W>(), smem, st>>>(
        Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn);
    EMS_CUDA(cudaGetLastError());
    return EMSURF_OK;
}

template <typename T2, int P, int W>
int f2_inv_w(const T2* Yg, long long lanes, int nx, int ny, int K, int M, int R, int nsplit, double scale,
             const double2* tw, const T2* mm, T2* y1, cudaStream_t st) {
    constexpr size_t smem = f2_smem<T2, P, W>();
    EMS_TRY(set_smem_once(fft2d_inv_kernel<T2, P, W>, smem));
    fft2d_inv_kernel<T2, P, W><<<(unsigned)((lanes + W - 1) / W), f2_threads<W>(), smem, st>>>(
        Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1);
    EMS_CUDA(cudaGetLastError());
    return EMSURF_OK;
}

template <typename T2, int P>
int f2_fwd(T2* Xg, long long lanes, int nx, int ny, int K, int n_unique, const double2* tw, const double2* x,
           const float2* xf, const int32_t* idx, const int8_t* sgn, cudaStream_t st) {
    constexpr int MW = f2_max_lanes<T2, P>();
    const int w = f2_pick_lanes(MW, lanes);
    if constexpr (MW >= 8) if (w == 8) return f2_fwd_w<T2, P, 8>(Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn, st);
    if constexpr (MW >= 4) if (w == 4) return f2_fwd_w<T2, P, 4>(Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn, st);
    if constexpr (MW >= 2) if (w == 2) return f2_fwd_w<T2, P, 2>(Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn, st);
    return f2_fwd_w<T2, P, 1>(Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn, st);
}

template <typename T2, int P>
int f2_inv(const T2* Yg, long long lanes, int nx, int ny, int K, int M, int R, int nsplit, double scale,
           const double2* tw, const T2* mm, T2* y1, cudaStream_t st) {
    constexpr int MW = f2_max_lanes<T2, P>();
    const int w = f2_pick_lanes(MW, lanes);
    if constexpr (MW >= 8) if (w == 8) return f2_inv_w<T2, P, 8>(Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1, st);
    if constexpr (MW >= 4) if (w == 4) return f2_inv_w<T2, P, 4>(Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1, st);
    if constexpr (MW >= 2) if (w == 2) return f2_inv_w<T2, P, 2>(Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1, st);
    return f2_inv_w<T2, P, 1>(Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1, st);
}

}  // namespace

bool fft2d_fused_ok(int px, int py) {
    if (px != py) return false;
    switch (px) {
        case 5: case 8: case 15: case 16: case 24: case 32: case 48: case 64: return true;
        default: return false;
    }
}

#define EMS_F2_SIZES(X) X(5) X(8) X(15) X(16) X(24) X(32) X(48) X(64)

template <typename T2>
int fft2d_forward(T2* Xg, int P, long long lanes, int nx, int ny, int K, int n_unique, const double2* tw,
                  const double2* x, const float2* xf, const int32_t* idx, const int8_t* sgn, cudaStream_t st) {
    switch (P) {
#define EMS_F2_CASE(N) \
    case N: return f2_fwd<T2, N>(Xg, lanes, nx, ny, K, n_unique, tw, x, xf, idx, sgn, st);
        EMS_F2_SIZES(EMS_F2_CASE)
#undef EMS_F2_CASE
        default: set_error("fused 2-D FFT: no kernel for %d x %d", P, P); return EMSURF_EINVAL;
    }
}

template <typename T2>
int fft2d_inverse(const T2* Yg, int P, long long lanes, int nx, int ny, int K, int M, int R, int nsplit,
                  double scale, const double2* tw, const T2* mm, T2* y1, cudaStream_t st) {
    switch (P) {
#define EMS_F2_CASE(N) \
    case N: return f2_inv<T2, N>(Yg, lanes, nx, ny, K, M, R, nsplit, scale, tw, mm, y1, st);
        EMS_F2_SIZES(EMS_F2_CASE)
#undef EMS_F2_CASE
        default: set_error("fused 2-D FFT: no kernel for %d x %d", P, P); return EMSURF_EINVAL;
    }
}

template int fft2d_forward<float2>(float2*, int, long long, int, int, int, int, const double2*, const double2*,
                                   const float2*, const int32_t*, const int8_t*, cudaStream_t);
template int fft2d_forward<double2>(double2*, int, long long, int, int, int, int, const double2*,
                                    const double2*, const float2*, const int32_t*, const int8_t*, cudaStream_t);
template int fft2d_inverse<float2>(const float2*, int, long long, int, int, int, int, int, int, double,
                                   const double2*, const float2*, float2*, cudaStream_t);
template int fft2d_inverse<double2>(const double2*, int, long long, int, int, int, int, int, int, double,
                                    const double2*, const double2*, double2*, cudaStream_t);

}  // namespace emsurf
