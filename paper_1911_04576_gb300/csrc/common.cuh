// Shared device helpers and the handle layout of the emsurf library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "emsurf.h"

namespace emsurf {

constexpr int kMmGroup = 4;   // cells of one type per macromodel CTA

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define EMS_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) {                                               \
            ::emsurf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,     \
                                cudaGetErrorString(_e));                       \
            return EMSURF_ECUDA;                                               \
        }                                                                      \
    } while (0)

#define EMS_TRY(expr)                                                          \
    do {                                                                       \
        int _s = (expr);                                                       \
        if (_s != EMSURF_OK) return _s;                                        \
    } while (0)

// Set a kernel's dynamic shared-memory limit once per (kernel, device): the
// call is costly on the host and the attribute persists for the process.
int set_smem_attr(const void* kernel, size_t bytes);
template <typename F>
int set_smem_once(F* kernel, size_t bytes) {
    return set_smem_attr(reinterpret_cast<const void*>(kernel), bytes);
}

// ---------------------------------------------------------------- complex
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}

// ---------------------------------------------------------------- L2 priority
// Data streamed once per product (the Fourier-domain blocks, the
// preconditioner rows) is loaded with an evict-first L2 policy and data
// reused by every product (the macromodels) with evict-last, so the 129 MB L2
// keeps the reused arrays between products.  Both are hints (createpolicy,
// L2::cache_hint); results do not depend on them.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ldg_l2hint(const uint4* a, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ldg_l2hint(const float4* a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}

template <typename T2> struct Real;
template <> struct Real<double2> { using type = double; };
template <> struct Real<float2> { using type = float; };

template <typename T2> __host__ __device__ __forceinline__ T2 mk(double re, double im);
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) {
    return make_double2(re, im);
}
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
    return make_float2((float)re, (float)im);
}

// ---------------------------------------------------------------- FFT plan
// One 1-D transform length P = product of radices (each 2, 3, 4, 5 or 7) with
// a device table tw[k] = exp(-2 pi i k / P), k in [0, P), from host libm.
struct FftPlan {
    int P = 0;
    int nrad = 0;
    int rad[16] = {0};
    double2* tw = nullptr;   // device
};

int fft_plan_create(FftPlan& plan, int P);
// fused 2-D transforms of square grids up to 64 x 64 (fft2d.cu)
bool fft2d_fused_ok(int px, int py);
template <typename T2>
int fft2d_forward(T2* Xg, int P, long long lanes, int nx, int ny, int K, int n_unique, const double2* tw,
                  const double2* x, const float2* xf, const int32_t* idx, const int8_t* sgn, cudaStream_t st);
template <typename T2>
int fft2d_inverse(const T2* Yg, int P, long long lanes, int nx, int ny, int K, int M, int R, int nsplit,
                  double scale, const double2* tw, const T2* mm, T2* y1, cudaStream_t st);
void fft_plan_destroy(FftPlan& plan);

// In-place 1-D transform along p of data[outer][P][inner] (inner contiguous
// lanes, outer stride outer_stride elements).  sign = -1 forward, +1 inverse
// (unscaled).  Only points p < p_in are read (the rest are zero) and only
// p < p_out are written; -1 means P.
template <typename T2>
int fft_pass(T2* data, const FftPlan& plan, long long inner, long long outer,
             long long outer_stride, int sign, cudaStream_t st, int p_in = -1, int p_out = -1);

// Forward pass over the cell rows whose input is read through U_o from the
// unique-unknown vector x ([R][n_unique]); lane L = r*K + k, row iy = outer
// index, point ix < p_in = nx.
template <typename T2>
int fft_pass_gather(T2* data, const FftPlan& plan, long long inner, long long outer,
                    long long outer_stride, int p_in, const double2* x, const int32_t* idx,
                    const int8_t* sgn, int nx, int K, int n_unique, cudaStream_t st,
                    const float2* xf = nullptr);

// Inverse pass over the kept rows (outer = ny) whose store writes only points
// ix < nx, as y1[r][iy*nx+ix][k] = scale * value + sum_s mm[s][r][m][k].
template <typename T2>
int fft_pass_crop(T2* data, const FftPlan& plan, long long inner, long long outer,
                  long long outer_stride, int nx, const T2* mm, int nsplit, int R, int M, int K,
                  double scale, T2* y1, cudaStream_t st);

int smallest_smooth_at_least(int n);   // smallest 2^a 3^b 5^c >= n

// ---------------------------------------------------------------- operator
// Fourier-domain blocks of one precision: B^[bin][op][j][i] (op 0 = L, 1 = K,
// stored transposed: source index j outer, test index i contiguous) and the
// macromodels transposed Zt[type][k'][k].
template <typename T2>
struct Operator {
    T2* Bhat = nullptr;
    T2* Zt = nullptr;
    T2* Xg = nullptr;      // work grid [bins][R][2E] (forward)
    T2* Yg = nullptr;      // work grid [bins][R][2E] (inverse)
    T2* Ymm = nullptr;     // macromodel partial outputs [split][R][M][2E]
    T2* Y1 = nullptr;      // local-space product [R][M][2E]
    T2 coef[4];
};

}  // namespace emsurf

// Per-phase CUDA-event timers (recorded on the launching stream).
struct PhaseTimer {
    std::vector<cudaEvent_t> ev;   // pairs (start, stop)
    size_t used = 0;               // events in use
};
enum { EMS_PH_BINMUL32 = 0, EMS_PH_BINMUL64, EMS_PH_MM32, EMS_PH_MM64, EMS_PH_FFT32, EMS_PH_FFT64,
       EMS_PH_ARNOLDI, EMS_PH_SCATTER, EMS_PH_PRECOND, EMS_NPHASE };

struct emsurf_handle {
    int device = 0;
    int nx = 0, ny = 0, E = 0, K = 0, M = 0, T = 0, n_unique = 0, max_rhs = 1;
    int px = 0, py = 0, nbins = 0;
    int precision = EMSURF_FP64;
    int64_t device_bytes = 0;
    int64_t budget = 0;
    emsurf::FftPlan plan_x, plan_y;
    // U_o: forward map and its inverse (CSR over unique unknowns)
    int32_t* d_uo_index = nullptr;
    int8_t* d_uo_sign = nullptr;
    int32_t* d_inv_ptr = nullptr;     // [n_unique + 1]
    int32_t* d_inv_ent = nullptr;     // [M*K] local unknown (m*K + k), signed via d_inv_sgn
    int8_t* d_inv_sgn = nullptr;
    int32_t* d_type_map = nullptr;    // [M]
    int32_t* d_type_cells = nullptr;  // cells grouped by type [M]
    int32_t* d_type_ptr = nullptr;    // [T + 1]
    std::vector<int32_t> h_type_ptr;
    void* d_mm_blocks = nullptr;      // macromodel work list (type, first, count)
    int n_mm_blocks = 0;
    emsurf::Operator<double2> op64;
    emsurf::Operator<float2> op32;
    bool have64 = false, have32 = false;
    int num_sms = 0;
    // half FP32 spectrum (reciprocal tables, single rhs): stored bins and partners
    bool half32 = false;
    int nst = 0;
    int32_t* d_st_bin = nullptr;
    int32_t* d_st_part = nullptr;
    // FP32 blocks of one bin per orbit of the box's mirror group (single
    // rhs): nst stored bins (d_st_bin their representatives), orb_G slots each
    bool orb32 = false;
    int orb_G = 0;
    int32_t* d_orb_bin = nullptr;     // [nst][orb_G] bin of each slot (-1: none)
    int32_t* d_orb_elem = nullptr;    // [nst][orb_G] its group element
    uint32_t* d_orb_perm = nullptr;   // [orb_G][2E] signed index of T_e
    // FP64-accuracy single-rhs bin multiply from FP32 hi/lo pairs: spectrum
    // planes [bin][hi, lo][op][j][i] and the split X^ [bin][hi, lo][2E]
    float2* ds_planes = nullptr;
    float2* ds_x = nullptr;
    float2* ds_zt = nullptr;          // the macromodels as hi/lo planes [t][hi, lo][k'][k]
    // powers of two that keep the double-single operands inside FP32's
    // exponent range: [0] spectrum planes, [1] macromodel planes (both were
    // split from the FP64 values times these), [2 + r] rhs r of the current
    // product (from max |x_r|); the kernels divide their FP64 outputs back
    double* d_ds_scale = nullptr;
    double h_ds_scale0 = 1.0;         // the spectrum planes' scale (host copy)
    unsigned long long* d_ds_max = nullptr;   // per-rhs running maxima of the scale kernel (kept at 0)
    unsigned* d_ds_cnt = nullptr;             // its per-rhs block arrival counters (kept at 0)
    int pair_grid = 0;                // CTAs of the pair kernel (equal slab ranges)
    float2* d_pair_part = nullptr;    // partial row sums of straddling bins [cta][2][2E]
    int* d_pair_cnt = nullptr;        // arrival counters [stored bin][row warp]
    size_t pair_cnt_bytes = 0;
    // BF16x3 split planes of the FP32 operator for the tensor-core bin multiply
    bool have_tc = false;
    void* tc_Bh = nullptr;          // spectrum hi/lo [bin][op][2i+c][ej] bf16
    void* tc_Bl = nullptr;
    void* tc_Xh = nullptr;          // X^ planes hi/lo [bin][rows][ej] bf16
    void* tc_Xl = nullptr;
    int tc_ej = 0, tc_rows = 0, tc_kp = 0;
    void* tc_Zh = nullptr;          // macromodel planes hi/lo [t][2k+c][kp] bf16
    void* tc_Zl = nullptr;
    void* tc_Mh = nullptr;          // x1 tiles of the macromodel product hi/lo [tile][128][kp]
    void* tc_Ml = nullptr;
    std::vector<void*> tc_mm_tiles;   // per rhs count: device (type, first column) tile list
    std::vector<int> tc_mm_ntiles;
    // tensor maps: X hi, X lo, B hi, B lo (bin multiply); x1 hi, x1 lo, Z hi, Z lo (macromodels)
    alignas(64) unsigned char tc_maps[12][128];
    int tc_variant = 0;                    // bin multiply ring shape picked by the autotuner
    float tc_tune_ms[2] = {0.f, 0.f};      // the two shapes' times at create
    int mm_occ[4] = {0, 0, 0, 0};          // resident macromodel CTAs per SM (FP32, FP64; x 1 / 4 rhs)
    int mm_threads[4] = {0, 0, 0, 0};      // macromodel block size per variant
    int mm2_occ = 0;                       // resident single-rhs FP32 macromodel CTAs per SM
    cudaStream_t setup_stream = nullptr;   // stream of the create-time work
    cudaStream_t side_stream = nullptr;    // the macromodel product beside the bin multiply
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // near-field preconditioner (restricted additive Schwarz, FP32 LU blocks)
    bool have_pc = false;
    int pc_nmax = 0;
    int64_t pc_elems = 0;           // sum over cells of own_m * ld_m (stored entries)
    int64_t pc_sub_total = 0;       // sum over cells of n_m
    int pc_own_max = 0;
    float2* pc_mat = nullptr;       // owned rows of A_m^{-1} in FP32 (create time only): own_m x ld_m per cell
    void* pc_mat16 = nullptr;       // the same rows as FP16 (re, im) pairs (or 8-bit, pc_int8), scaled per row
    bool pc_int8 = false;           // rows stored as offset-binary 8-bit pairs (1-2 rhs handles that ask)
    float* pc_rscale = nullptr;     // [n_unique] scale of each owned row
    int64_t* pc_off = nullptr;      // [M] element offset of each cell's rows
    int32_t* pc_ld = nullptr;       // [M] row length (n_m rounded up to even)
    int32_t* pc_own_ptr = nullptr;  // [M+1] first owned row of each cell in the row list
    int32_t* pc_sub_cell = nullptr; // cell of each subdomain entry
    int64_t* pc_rs_off = nullptr;   // [M] start of each cell's segment in pc_rs
    float2* pc_rs = nullptr;        // [max_rhs][pc_rs_stride] gathered r (FP32)
    int64_t pc_rs_stride = 0;
    // tensor-core apply (>= kTcMinRhs rhs): bf16 planes of the owned rows and of r per cell
    bool have_pc_tc = false;
    void* pc_tc_Xh = nullptr;       // [2 n_unique][np]
    void* pc_tc_Xl = nullptr;
    void* pc_tc_Rh = nullptr;       // [M][128][np]
    void* pc_tc_Rl = nullptr;
    void* pc_tc_items = nullptr;    // (cell, first owned row) per item
    int pc_tc_nitems = 0, pc_tc_np = 0;
    alignas(64) unsigned char pc_tc_maps[4][128];
    const double2* near_L = nullptr;  // near offset tables [5][5][E][E] (|dx|, |dy| <= 2)
    const double2* near_K = nullptr;
    int32_t* pc_n = nullptr;        // [M] subdomain sizes
    int32_t* pc_own = nullptr;      // [M] owned unknowns (first in each subdomain)
    int32_t* pc_sub_ptr = nullptr;  // [M+1]
    int32_t* pc_sub_ids = nullptr;  // unique ids of each subdomain
    int* d_err = nullptr;             // device error flag of bounded waits (0 = ok)
    unsigned* d_grid_bar = nullptr;   // [2] count and generation of the cooperative Arnoldi step's grid barrier
    bool coop_ok = true;              // the cooperative Arnoldi step may be used (no overlapping solves)
    // GMRES workspace (FP64), allocated lazily by emsurf_solve
    void* gm = nullptr;
    // tracing: kernel launches issued by this handle, optional phase timers
    int64_t launches = 0;
    bool prof_on = false;
    uint32_t prof_mask = 0xffffffffu;      // phases recorded while prof_on
    PhaseTimer prof[EMS_NPHASE];
    std::vector<void*> allocations;
};

namespace emsurf {
int dev_alloc(emsurf_handle* h, void** p, size_t bytes);
// free one of the handle's allocations before destroy (bytes as allocated)
void dev_free(emsurf_handle* h, void* p, size_t bytes);
// record the start (begin = true) or end of a phase on stream st if profiling
void prof_mark(emsurf_handle* h, int phase, bool begin, cudaStream_t st);

// a triangle mesh with RWG slots, host arrays (see emsurf_setup_box_mesh)
struct MeshView {
    const double* verts;
    const int32_t* tris;
    const int32_t* slot_rwg;
    const int8_t* slot_sgn;
    int T, E;
};
// the configurations' cell (slab + patch): the two region surfaces (air,
// slab) and U of Eq. incidence1 as, per region, the region-local unknown
// (J of RWG r: r, M: E_v + r) and sign of every X~ column (-1: absent);
// X~ = [interior unknowns (n_int) | J_eq (E) | M_eq (E)]
struct SlabRegionMesh {
    std::vector<double> verts;
    std::vector<int32_t> tris, slot_rwg;
    std::vector<int8_t> slot_sgn;
    int T = 0, E = 0;
};
struct SlabPlan {
    SlabRegionMesh region[2];
    int n_int = 0, N = 0, E = 0;
    std::vector<int32_t> copy[2];
    std::vector<int8_t> sgn[2];
};
int slab_cell_plan(double a, double b, double h, int n, const double* zlevels, double side,
                   int patch_n, int ring_layers, SlabPlan& out);
int slab_top(double a, double b, double z, int n, double side, int patch_n, int ring_layers,
             std::vector<double>& verts, std::vector<int32_t>& tris, std::vector<int32_t>& edges,
             std::vector<int32_t>& tplus, std::vector<int32_t>& tminus,
             std::vector<int32_t>& slot_rwg, std::vector<int8_t>& slot_sgn,
             std::vector<int8_t>& on_patch);
// complex wavenumber k = kr + j ki (Im k < 0 in a lossy region, e^{jwt})
int tabulate_blocks_cx(const MeshView& test, const MeshView& src, const double* shifts,
                       const int8_t* singular, int nb, double kr, double ki, double2* L,
                       double2* K, cudaStream_t st);
// Galerkin L, K [nb][test E][src E] on the device for nb test-mesh shifts
int tabulate_blocks(const MeshView& test, const MeshView& src, const double* shifts,
                    const int8_t* singular, int nb, double k, double2* L, double2* K,
                    cudaStream_t st);
template <typename T2>
int build_operator(emsurf_handle* h, Operator<T2>& op, const emsurf_problem* pr,
                   const Operator<T2>* share = nullptr);
// share: a handle of the same lattice whose Fourier-domain blocks are reused
int derive_fp32_operator(emsurf_handle* h, const emsurf_problem* pr, const emsurf_handle* share = nullptr);
// mirror orbits of the spectrum's bins (setup.cpp): the bin of group element
// e (bit 0: x mirror, bit 1: y mirror, bit 2: x <-> y, applied first) acting
// on bin (kx, ky); the signed permutations T_e [G][2E] (index | sign << 31)
// composed from the box's mirror permutations; the orbits, one
// representative (the smallest bin) each, G slots (bin, element) per
// representative, bin -1 past the orbit's size
int orbit_image(int e, int kx, int ky, int px, int py);
void mirror_group_perms(int E, int G, const int32_t* perm, const int8_t* sign, std::vector<uint32_t>& tperm);
void mirror_orbits(int px, int py, int G, std::vector<int32_t>& rep, std::vector<int32_t>& obin,
                   std::vector<int32_t>& oelem);
int adopt_fp32_form(emsurf_handle* h, const emsurf_handle* share);
int clear_wait_error(emsurf_handle* h);
int build_ds_planes(emsurf_handle* h, const emsurf_handle* share = nullptr);
int grid_barrier_selftest(emsurf_handle* h, long long limit, cudaStream_t st);
template <typename T2>
int apply_operator(emsurf_handle* h, Operator<T2>& op, const double2* x, double2* y, int nrhs,
                   cudaStream_t st);
// FP32 operator on FP32 vectors [R][n_unique] (the inner solve of MIXED)
int apply_operator_f32(emsurf_handle* h, const float2* x, float2* y, int R, cudaStream_t st);
int pc_build(emsurf_handle* h, const emsurf_problem* p);
int stage_near_tables(emsurf_handle* h, const emsurf_problem* p);
int wait_selftest(emsurf_handle* h, long long limit, cudaStream_t st);
// tensor-core bin multiply (BF16x3) for nrhs >= kTcMinRhs
constexpr int kTcMinRhs = 8;
int tc_build(emsurf_handle* h, const emsurf_handle* share = nullptr);
int tc_binmul(emsurf_handle* h, const float2* X, float2* Y, int R, const float2* coef, cudaStream_t st);
int tc_macromodel(emsurf_handle* h, const double2* x, const float2* xf, float2* Ymm, int R, cudaStream_t st);
int pc_tc_build(emsurf_handle* h, const std::vector<int32_t>& own_ptr);
template <typename VT>
int pc_tc_apply(emsurf_handle* h, const VT* r, VT* y, int R, cudaStream_t st);
int pc_apply(emsurf_handle* h, const double2* r, double2* y, int R, cudaStream_t st);
int pc_apply_f32(emsurf_handle* h, const float2* r, float2* y, int R, cudaStream_t st);
int gmres_solve(emsurf_handle* h, const double2* b, double2* x, int nrhs,
                const emsurf_solve_opts* o, emsurf_solve_info* info, cudaStream_t st);
}  // namespace emsurf
