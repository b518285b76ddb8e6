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
// Govindaraju et al., SC 2008), and writes the tile back in place.
#include <cmath>

#include "common.cuh"

namespace emsurf {

namespace {

struct RadList {
    int n;
    int r[16];
};

constexpr int kFftThreads = 256;
constexpr int kMaxRadix = 7;

template <typename T2>
__device__ __forceinline__ T2 tw_at(const double2* __restrict__ tw, int k, int sign) {
    double2 w = tw[k];
    return mk<T2>(w.x, sign < 0 ? w.y : -w.y);
}

template <typename T2, int W>
__global__ void __launch_bounds__(kFftThreads)
fft_pass_kernel(T2* __restrict__ data, int P, long long inner, long long outer_stride,
                const double2* __restrict__ tw, RadList rad, int sign) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* buf0 = reinterpret_cast<T2*>(smem_raw);
    T2* buf1 = buf0 + (size_t)P * W;
    const long long lane0 = (long long)blockIdx.x * W;
    const int wl = (int)min((long long)W, inner - lane0);
    T2* base = data + (long long)blockIdx.y * outer_stride + lane0;
    const T2 zero = mk<T2>(0.0, 0.0);

    for (int e = threadIdx.x; e < P * W; e += blockDim.x) {
        const int p = e / W, l = e - (e / W) * W;
        buf0[e] = (l < wl) ? base[(long long)p * inner + l] : zero;
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
                    v[r] = (r == 0 || jm == 0) ? a : cmul(a, tw_at<T2>(tw, (jm * r * tstep) % P, sign));
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

    for (int e = threadIdx.x; e < P * W; e += blockDim.x) {
        const int p = e / W, l = e - (e / W) * W;
        if (l < wl) base[(long long)p * inner + l] = in[e];
    }
}

template <typename T2, int W>
int launch_pass(T2* data, const FftPlan& plan, long long inner, long long outer,
                long long outer_stride, int sign, cudaStream_t st) {
    RadList rl;
    rl.n = plan.nrad;
    for (int i = 0; i < 16; ++i) rl.r[i] = plan.rad[i];
    const size_t smem = 2ull * plan.P * W * sizeof(T2);
    EMS_CUDA(cudaFuncSetAttribute(fft_pass_kernel<T2, W>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long gx = (inner + W - 1) / W;
    if (outer > 65535 || gx > 2147483647LL) {
        set_error("fft_pass: grid too large (outer %lld, lanes %lld)", outer, inner);
        return EMSURF_EINVAL;
    }
    dim3 grid((unsigned)gx, (unsigned)outer);
    fft_pass_kernel<T2, W><<<grid, kFftThreads, smem, st>>>(data, plan.P, inner, outer_stride,
                                                            plan.tw, rl, sign);
    EMS_CUDA(cudaGetLastError());
    return EMSURF_OK;
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
             long long outer_stride, int sign, cudaStream_t st) {
    if (outer <= 0 || inner <= 0) return EMSURF_OK;
    const size_t per_lane = 2ull * plan.P * sizeof(T2);
    if (per_lane * 32 <= 200 * 1024)
        return launch_pass<T2, 32>(data, plan, inner, outer, outer_stride, sign, st);
    if (per_lane * 16 <= 200 * 1024)
        return launch_pass<T2, 16>(data, plan, inner, outer, outer_stride, sign, st);
    if (per_lane * 8 <= 200 * 1024)
        return launch_pass<T2, 8>(data, plan, inner, outer, outer_stride, sign, st);
    set_error("FFT length %d too large for one shared-memory pass", plan.P);
    return EMSURF_EINVAL;
}

template int fft_pass<double2>(double2*, const FftPlan&, long long, long long, long long, int,
                               cudaStream_t);
template int fft_pass<float2>(float2*, const FftPlan&, long long, long long, long long, int,
                              cudaStream_t);

}  // namespace emsurf
