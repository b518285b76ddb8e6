// Bin multiply on the tensor cores for many right-hand sides (Sec. IV-B,
// Eqs. LJV3-LJV5 per bin): with R rhs the product B^(k) X^(k) of every bin
// is a complex GEMM (E x E by E x R, twice: L^ and K^), which at R >= 8 is
// compute-bound on the FP32 pipes.  Here it runs as BF16x3 split precision
// on tcgen05 with FP32 accumulation in TMEM:
//   v = hi + lo (both bf16, hi = rn(v), lo = rn(v - hi)),
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// which keeps ~16 significant bits per factor (relative error per product
// term <= 3 * 2^-18).  The split planes take the same bytes as the FP32
// complex spectrum, so the kernel stays bound by streaming the spectrum.
//
// Complex arithmetic as real GEMMs.  For one bin, operator op in {L, K},
// test row i, source j:  the "B" operand holds the spectrum as real rows
// m = 2 i + c (c = 0 real part, 1 imaginary part) over j; the "A" operand
// holds the X^ planes as real rows rho = 4 r + q (q = 0 Re x_J, 1 Im x_J,
// 2 Re x_M, 3 Im x_M) over j, 32 rhs per pass (M = 128).  D_op[rho][m] =
// sum_j A[rho][j] B_op[m][j]; then, e.g., (L x_J)_i = (D_L[4r][2i] -
// D_L[4r+1][2i+1]) + i (D_L[4r+1][2i] + D_L[4r][2i+1]), combined into
// y_J = a L x_J + b K x_M and y_M = g K x_J + d L x_M in the epilogue.
//
// Kernel: persistent, one CTA per SM, items = (rhs group, bin, chunk of 48
// test rows).  Warp 0 issues TMA tensor loads (64B swizzle) of 32-source
// stages into a 5-deep ring; warp 1 issues the MMAs (M = 128, N = 96,
// K = 16) into one of two TMEM accumulator sets; warps 2-5 drain the other
// set (tcgen05.ld), combine and store Y^.  Every wait is bounded: on expiry
// the kernel sets the error flag, waits (bounded) for its copies and MMAs in
// flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

constexpr int kTcM = 128;          // A rows: 32 rhs x 4 planes
constexpr int kTcRhs = 32;
constexpr int kTcN = 96;           // B rows per item: 48 test rows x (re, im)
constexpr int kTcKc = 64;          // sources per stage (128 bytes of bf16)
constexpr int kTcStages = 2;
constexpr int kTcThreads = 192;    // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kTcABytes = kTcM * 128;      // 16 KB
constexpr int kTcBBytes = kTcN * 128;      // 12 KB
constexpr int kTcStageBytes = 2 * kTcABytes + 4 * kTcBBytes;   // A hi/lo, B hi/lo x (L, K)
constexpr int kTcSmem = 1024 + kTcStages * kTcStageBytes;
constexpr uint32_t kTcTmemCols = 512;     // two accumulator sets of 2 x 96 columns
constexpr long long kTcWait = 1LL << 22;
// The bin multiply's ring, two shapes chosen per handle by timing them at
// create (the spectrum stream is latency-bound per SM, throughput = bytes in
// flight / DRAM latency, so the deeper ring usually wins):
//   KC = 32 sources per stage (64-byte rows, 64B swizzle), 5 stages of 40 KB;
//   KC = 64 sources per stage (128-byte rows, 128B swizzle), 2 stages of 80 KB.
template <int KC>
struct BmShape {
    static constexpr int ABytes = kTcM * KC * 2;
    static constexpr int BBytes = kTcN * KC * 2;
    static constexpr int StageBytes = 2 * ABytes + 4 * BBytes;
};
template <int KC, int STAGES>
constexpr int bm_smem() {
    return 1024 + STAGES * BmShape<KC>::StageBytes;
}
static_assert(bm_smem<32, 5>() <= 227 * 1024 && bm_smem<64, 2>() <= 227 * 1024, "bin multiply ring exceeds shared memory");
// instruction descriptor: kind::f16, bf16 x bf16 -> f32, K-major A and B, N = 96, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < kTcWait; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// the same for 64B swizzle (64-byte rows, 8-row groups 512 B apart)
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | (32ull << 32) | (1ull << 46) | (4ull << 61);
}
template <int KC>
__device__ __forceinline__ uint64_t bm_desc(uint32_t addr) {
    if constexpr (KC == 64) return sdesc(addr);
    else return sdesc64(addr);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

struct TcArgs {
    float2* Y;            // [bins][R][2E]
    int E, nbins, R, groups, chunks, nk, items;
    float2 ca, cb, cg, cd;
    int* err;
};

template <int KC, int STAGES>
__global__ void __launch_bounds__(kTcThreads, 1)
binmul_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                 const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, TcArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf[2], acce[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&accf[a], 1);
            bar_init(&acce[a], 4);
        }
        bar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const int E = g.E, K2 = 2 * g.E;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES] = {};
            for (int item = blockIdx.x; item < g.items && !*(volatile int*)&abort_flag; item += gridDim.x) {
                const int grp = item / (g.nbins * g.chunks), rem = item % (g.nbins * g.chunks);
                const int bin = rem / g.chunks, ch = rem % g.chunks;
                for (int ks = 0; ks < g.nk; ++ks) {
                    if (!bar_wait(&empty[stage], phase ^ 1)) {
                        atomicExch(g.err, 4);
                        *(volatile int*)&abort_flag = 1;
                        break;
                    }
                    unsigned char* st = smem + stage * BmShape<KC>::StageBytes;
                    bar_expect(&full[stage], BmShape<KC>::StageBytes);
                    const int j0 = ks * KC;
                    tma3d(st, &mAh, j0, kTcM * grp, bin, &full[stage]);
                    tma3d(st + BmShape<KC>::ABytes, &mAl, j0, kTcM * grp, bin, &full[stage]);
                    for (int op = 0; op < 2; ++op) {
                        unsigned char* b = st + 2 * BmShape<KC>::ABytes + op * 2 * BmShape<KC>::BBytes;
                        tma3d(b, &mBh, j0, kTcN * ch, 2 * bin + op, &full[stage]);
                        tma3d(b + BmShape<KC>::BBytes, &mBl, j0, kTcN * ch, 2 * bin + op, &full[stage]);
                    }
                    ++issued[stage];
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            // every copy this thread issued has landed before the CTA can exit
            for (int s = 0; s < STAGES; ++s)
                if (issued[s] && !bar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1))) atomicExch(g.err, 4);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool any = false;
            for (int item = blockIdx.x; item < g.items && !*(volatile int*)&abort_flag; item += gridDim.x) {
                if (!bar_wait(&acce[acc], aphase ^ 1)) {
                    atomicExch(g.err, 5);
                    *(volatile int*)&abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dL = tmem + (uint32_t)(acc * 256), dK = dL + kTcN;
                bool ok = true;
                for (int ks = 0; ks < g.nk; ++ks) {
                    if (!bar_wait(&full[stage], phase)) {
                        atomicExch(g.err, 6);
                        *(volatile int*)&abort_flag = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = saddr(smem + stage * BmShape<KC>::StageBytes);
                    const uint32_t ah = st, al = st + BmShape<KC>::ABytes;
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint32_t off = 32u * kk;
                        const uint64_t dah = bm_desc<KC>(ah + off), dal = bm_desc<KC>(al + off);
                        for (int op = 0; op < 2; ++op) {
                            const uint32_t b = st + 2 * BmShape<KC>::ABytes + op * 2 * BmShape<KC>::BBytes;
                            const uint64_t dbh = bm_desc<KC>(b + off), dbl = bm_desc<KC>(b + BmShape<KC>::BBytes + off);
                            const uint32_t d = op ? dK : dL;
                            mma_bf16(d, dah, dbh, (ks > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(d, dah, dbl, 1u);
                            mma_bf16(d, dal, dbh, 1u);
                        }
                    }
                    mma_commit(&empty[stage]);   // the stage is free once these MMAs have read it
                    any = true;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&accf[acc]);
                if (++acc == 2) {
                    acc = 0;
                    aphase ^= 1;
                }
            }
            // all issued MMAs complete before teardown
            if (any) {
                mma_commit(&mma_done);
                if (!bar_wait(&mma_done, 0)) atomicExch(g.err, 7);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int qd = warp & 3;                 // TMEM lane quadrant of this warp
        const int rho = 32 * qd + lane, rl = rho >> 2, q = rho & 3;
        const int base = lane & ~3;
        int acc = 0;
        uint32_t aphase = 0;
        for (int item = blockIdx.x; item < g.items && !*(volatile int*)&abort_flag; item += gridDim.x) {
            const int grp = item / (g.nbins * g.chunks), rem = item % (g.nbins * g.chunks);
            const int bin = rem / g.chunks, ch = rem % g.chunks;
            if (!bar_wait(&accf[acc], aphase)) {
                if (lane == 0) atomicExch(g.err, 8);
                *(volatile int*)&abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int r = kTcRhs * grp + rl;
            const uint32_t t0 = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(acc * 256);
            float2* Yb = g.Y + ((size_t)bin * g.R + (r < g.R ? r : 0)) * K2;
            for (int c0 = 0; c0 < kTcN; c0 += 32) {
                uint32_t a[32], b[32];
                tmem_ld32(t0 + c0, a);
                tmem_ld32(t0 + kTcN + c0, b);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                for (int t = 0; t < 16; ++t) {
                    float LR[4], LI[4], KR[4], KI[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        LR[s] = __shfl_sync(0xffffffffu, __uint_as_float(a[2 * t]), base + s);
                        LI[s] = __shfl_sync(0xffffffffu, __uint_as_float(a[2 * t + 1]), base + s);
                        KR[s] = __shfl_sync(0xffffffffu, __uint_as_float(b[2 * t]), base + s);
                        KI[s] = __shfl_sync(0xffffffffu, __uint_as_float(b[2 * t + 1]), base + s);
                    }
                    const int i = ch * (kTcN / 2) + c0 / 2 + t;
                    if (r < g.R && i < E && q < 2) {
                        float2 y;
                        if (q == 0) {
                            // y_J = a L x_J + b K x_M
                            const float uR = LR[0] - LI[1], uI = LR[1] + LI[0];
                            const float wR = KR[2] - KI[3], wI = KR[3] + KI[2];
                            y.x = g.ca.x * uR - g.ca.y * uI + g.cb.x * wR - g.cb.y * wI;
                            y.y = g.ca.x * uI + g.ca.y * uR + g.cb.x * wI + g.cb.y * wR;
                            Yb[i] = y;
                        } else {
                            // y_M = g K x_J + d L x_M
                            const float wR = KR[0] - KI[1], wI = KR[1] + KI[0];
                            const float uR = LR[2] - LI[3], uI = LR[3] + LI[2];
                            y.x = g.cg.x * wR - g.cg.y * wI + g.cd.x * uR - g.cd.y * uI;
                            y.y = g.cg.x * wI + g.cg.y * wR + g.cd.x * uI + g.cd.y * uR;
                            Yb[E + i] = y;
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(&acce[acc]);
            if (++acc == 2) {
                acc = 0;
                aphase ^= 1;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

// Split planes of the spectrum, test-major: out[bin][op][2i+c][j] = hi/lo of
// (c ? Im : Re) Bhat[bin][op][j][i] (source-major FP32), rows padded to ej.
__global__ void tc_split_spectrum_kernel(const float2* __restrict__ Bhat, __nv_bfloat16* __restrict__ hi,
                                         __nv_bfloat16* __restrict__ lo, int E, int ej, int z0) {
    __shared__ float2 tile[32][33];
    const int bo = z0 + (int)blockIdx.z;        // bin * 2 + op (launches cover <= 65535 at a time)
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const float2* src = Bhat + (size_t)bo * E * E;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (j < E && i < E) ? src[(size_t)j * E + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // write rows m = 2i + c, columns j (j < ej; padding columns are zero)
    for (int r = threadIdx.y; r < 64; r += blockDim.y) {
        const int il = r >> 1, c = r & 1, i = i0 + il, j = j0 + threadIdx.x;
        if (i >= E || j >= ej) continue;
        const float v = c ? tile[threadIdx.x][il].y : tile[threadIdx.x][il].x;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        const size_t at = ((size_t)bo * 2 * E + (size_t)(2 * i + c)) * ej + j;
        hi[at] = h;
        lo[at] = l;
    }
}

// Split planes of X^: out[bin][4r+q][j], q = (Re x_J, Im x_J, Re x_M, Im x_M),
// zero for r >= R and j >= E.
__global__ void tc_split_x_kernel(const float2* __restrict__ X, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, int E, int ej, int R, int rows, size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % ej);
        const size_t br = e / ej;
        const int rho = (int)(br % rows);
        const size_t bin = br / rows;
        const int r = rho >> 2, q = rho & 3;
        float v = 0.f;
        if (r < R && j < E) {
            const float2 x = X[(bin * R + r) * (size_t)(2 * E) + (q >> 1) * E + j];
            v = (q & 1) ? x.y : x.x;
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// ---------------------------------------------------------------- macromodels
// The per-type macromodel product (Eq. Zmacromodel_Array) with many rhs is a
// complex GEMM per type t: Y1[r][m] = Z~^t x1[r][m] for the cells m of type
// t, i.e. K x K times K x (cells_t R).  Same BF16x3 scheme: "A" = the x1
// planes of a tile of 64 complex columns (cell, rhs) of one type, rows
// rho = 2c + q (q = Re, Im of column c); "B" = the Z~^t planes, rows
// m = 2k + c over k'.  Re y_k = D[2c][2k] - D[2c+1][2k+1],
// Im y_k = D[2c+1][2k] + D[2c][2k+1].  Items = (tile, chunk of 48 rows k),
// 3 stages of 56 KB, one TMEM accumulator set of 96 columns per item
// (two sets alternate).
constexpr int kMmStageBytes = 2 * kTcABytes + 2 * kTcBBytes;   // 56 KB
constexpr int kMmStages = 3;
constexpr int kMmSmem = 1024 + kMmStages * kMmStageBytes;
constexpr uint32_t kMmTmemCols = 256;

struct MmArgs {
    float2* Y;                    // Ymm[0] = [R][M][K]
    const int2* tiles;            // (type, first column)
    const int32_t* type_ptr;      // [T+1] cells of each type in type_cells
    const int32_t* type_cells;
    int K, M, R, ntiles, chunks, nk, items;
    int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1)
mm_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
             const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, MmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kMmStages], empty[kMmStages], accf[2], acce[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kMmTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMmStages; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&accf[a], 1);
            bar_init(&acce[a], 4);
        }
        bar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[kMmStages] = {0, 0, 0};
            for (int item = blockIdx.x; item < g.items && !*abort_v; item += gridDim.x) {
                const int tile = item / g.chunks, ch = item % g.chunks;
                const int type = g.tiles[tile].x;
                for (int ks = 0; ks < g.nk; ++ks) {
                    if (!bar_wait(&empty[stage], phase ^ 1)) {
                        atomicExch(g.err, 9);
                        *abort_v = 1;
                        break;
                    }
                    unsigned char* st = smem + stage * kMmStageBytes;
                    bar_expect(&full[stage], kMmStageBytes);
                    const int j0 = ks * kTcKc;
                    tma3d(st, &mAh, j0, 0, tile, &full[stage]);
                    tma3d(st + kTcABytes, &mAl, j0, 0, tile, &full[stage]);
                    tma3d(st + 2 * kTcABytes, &mBh, j0, kTcN * ch, type, &full[stage]);
                    tma3d(st + 2 * kTcABytes + kTcBBytes, &mBl, j0, kTcN * ch, type, &full[stage]);
                    ++issued[stage];
                    if (++stage == kMmStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            for (int s = 0; s < kMmStages; ++s) {
                // the n-th use of a stage completes phase n-1 of its full barrier
                if (issued[s] && !bar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1))) atomicExch(g.err, 9);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool any = false;
            for (int item = blockIdx.x; item < g.items && !*abort_v; item += gridDim.x) {
                if (!bar_wait(&acce[acc], aphase ^ 1)) {
                    atomicExch(g.err, 10);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d = tmem + (uint32_t)(acc * 128);
                bool ok = true;
                for (int ks = 0; ks < g.nk; ++ks) {
                    if (!bar_wait(&full[stage], phase)) {
                        atomicExch(g.err, 11);
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = saddr(smem + stage * kMmStageBytes);
                    const uint32_t ah = st, al = st + kTcABytes, bh = st + 2 * kTcABytes, bl = bh + kTcBBytes;
                    for (int kk = 0; kk < kTcKc / 16; ++kk) {
                        const uint32_t off = 32u * kk;
                        mma_bf16(d, sdesc(ah + off), sdesc(bh + off), (ks > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(d, sdesc(ah + off), sdesc(bl + off), 1u);
                        mma_bf16(d, sdesc(al + off), sdesc(bh + off), 1u);
                    }
                    mma_commit(&empty[stage]);
                    any = true;
                    if (++stage == kMmStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&accf[acc]);
                if (++acc == 2) {
                    acc = 0;
                    aphase ^= 1;
                }
            }
            if (any) {
                mma_commit(&mma_done);
                if (!bar_wait(&mma_done, 0)) atomicExch(g.err, 12);
            }
        }
    } else {
        const int qd = warp & 3;
        const int rho = 32 * qd + lane, c = rho >> 1, q = rho & 1;
        int acc = 0;
        uint32_t aphase = 0;
        for (int item = blockIdx.x; item < g.items && !*abort_v; item += gridDim.x) {
            const int tile = item / g.chunks, ch = item % g.chunks;
            const int2 tl = g.tiles[tile];
            if (!bar_wait(&accf[acc], aphase)) {
                if (lane == 0) atomicExch(g.err, 13);
                *abort_v = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int col = tl.y + c;
            const int n_t = g.type_ptr[tl.x + 1] - g.type_ptr[tl.x];
            const bool valid = col < n_t * g.R;
            float2* Yc = g.Y;
            if (valid) {
                const int slot = col / g.R, r = col % g.R;
                const int cell = g.type_cells[g.type_ptr[tl.x] + slot];
                Yc = g.Y + ((size_t)r * g.M + cell) * g.K;
            }
            const uint32_t t0 = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(acc * 128);
            for (int c0 = 0; c0 < kTcN; c0 += 32) {
                uint32_t a[32];
                tmem_ld32(t0 + c0, a);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                for (int t = 0; t < 16; ++t) {
                    const float pR = __shfl_xor_sync(0xffffffffu, __uint_as_float(a[2 * t]), 1);
                    const float pI = __shfl_xor_sync(0xffffffffu, __uint_as_float(a[2 * t + 1]), 1);
                    const int k = ch * (kTcN / 2) + c0 / 2 + t;
                    if (valid && q == 0 && k < g.K) {
                        // own row = Re x (2c), partner = Im x (2c+1)
                        float2 y;
                        y.x = __uint_as_float(a[2 * t]) - pI;
                        y.y = pR + __uint_as_float(a[2 * t + 1]);
                        Yc[k] = y;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(&acce[acc]);
            if (++acc == 2) {
                acc = 0;
                aphase ^= 1;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmTmemCols));
}

// x1 planes of the macromodel tiles: out[tile][2c+q][k'] = hi/lo of
// (q ? Im : Re)(sign * x[r][U_o index]) for column c = (cell slot, rhs) of
// the tile's type; zero past the type's columns and for k' >= K.
__global__ void tc_mm_gather_kernel(const double2* __restrict__ x, const float2* __restrict__ xf,
                                    const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn,
                                    const int2* __restrict__ tiles, const int32_t* __restrict__ type_ptr,
                                    const int32_t* __restrict__ type_cells, __nv_bfloat16* __restrict__ hi,
                                    __nv_bfloat16* __restrict__ lo, int K, int kp, int R, int n_unique,
                                    size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(e % kp);
        const size_t tr = e / kp;
        const int rho = (int)(tr % kTcM);
        const int tile = (int)(tr / kTcM);
        const int2 tl = tiles[tile];
        const int col = tl.y + (rho >> 1), q = rho & 1;
        const int n_t = type_ptr[tl.x + 1] - type_ptr[tl.x];
        float v = 0.f;
        if (col < n_t * R && kk < K) {
            const int slot = col / R, r = col % R;
            const int cell = type_cells[type_ptr[tl.x] + slot];
            const size_t loc = (size_t)cell * K + kk;
            const size_t at = (size_t)r * n_unique + idx[loc];
            const float s = (float)sgn[loc];
            if (xf) v = s * (q ? xf[at].y : xf[at].x);
            else v = s * (float)(q ? x[at].y : x[at].x);
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// ---------------------------------------------------------------- preconditioner
// The restricted additive Schwarz apply with many rhs is a complex GEMM per
// cell: y[own rows] = X_m (own_m x n_m) r[S_m] (n_m x R).  Same BF16x3
// scheme as the macromodels: "A" = the gathered r planes of cell m (rows
// 2c + q for rhs c < 64, over the subdomain index j), "B" = the planes of
// the owned inverse rows (one flat list over all cells, rows 2g + c for
// owned row g).  Items = (cell, 48 owned rows); the K loop covers n_m.
struct PcArgs {
    void* y;                       // [R][n_unique], float2 or double2
    int y_f32;
    const int2* items;             // (cell, first owned row)
    const int32_t* own_ptr;        // [M+1]
    const int32_t* nsz;            // [M]
    const int32_t* sub_ptr;
    const int32_t* sub_ids;
    int R, n_unique, nitems;
    int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1)
pc_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
             const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, PcArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kMmStages], empty[kMmStages], accf[2], acce[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kMmTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMmStages; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&accf[a], 1);
            bar_init(&acce[a], 4);
        }
        bar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[kMmStages] = {0, 0, 0};
            for (int item = blockIdx.x; item < g.nitems && !*abort_v; item += gridDim.x) {
                const int2 it = g.items[item];
                const int nk = (g.nsz[it.x] + kTcKc - 1) / kTcKc;
                const int brow = 2 * (g.own_ptr[it.x] + it.y);
                for (int ks = 0; ks < nk; ++ks) {
                    if (!bar_wait(&empty[stage], phase ^ 1)) {
                        atomicExch(g.err, 14);
                        *abort_v = 1;
                        break;
                    }
                    unsigned char* st = smem + stage * kMmStageBytes;
                    bar_expect(&full[stage], kMmStageBytes);
                    const int j0 = ks * kTcKc;
                    tma3d(st, &mAh, j0, 0, it.x, &full[stage]);
                    tma3d(st + kTcABytes, &mAl, j0, 0, it.x, &full[stage]);
                    tma3d(st + 2 * kTcABytes, &mBh, j0, brow, 0, &full[stage]);
                    tma3d(st + 2 * kTcABytes + kTcBBytes, &mBl, j0, brow, 0, &full[stage]);
                    ++issued[stage];
                    if (++stage == kMmStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            for (int s = 0; s < kMmStages; ++s)
                if (issued[s] && !bar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1))) atomicExch(g.err, 14);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t phase = 0, aphase = 0;
            bool any = false;
            for (int item = blockIdx.x; item < g.nitems && !*abort_v; item += gridDim.x) {
                const int nk = (g.nsz[g.items[item].x] + kTcKc - 1) / kTcKc;
                if (!bar_wait(&acce[acc], aphase ^ 1)) {
                    atomicExch(g.err, 15);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d = tmem + (uint32_t)(acc * 128);
                bool ok = true;
                for (int ks = 0; ks < nk; ++ks) {
                    if (!bar_wait(&full[stage], phase)) {
                        atomicExch(g.err, 16);
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = saddr(smem + stage * kMmStageBytes);
                    const uint32_t ah = st, al = st + kTcABytes, bh = st + 2 * kTcABytes, bl = bh + kTcBBytes;
                    for (int kk = 0; kk < kTcKc / 16; ++kk) {
                        const uint32_t off = 32u * kk;
                        mma_bf16(d, sdesc(ah + off), sdesc(bh + off), (ks > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(d, sdesc(ah + off), sdesc(bl + off), 1u);
                        mma_bf16(d, sdesc(al + off), sdesc(bh + off), 1u);
                    }
                    mma_commit(&empty[stage]);
                    any = true;
                    if (++stage == kMmStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&accf[acc]);
                if (++acc == 2) {
                    acc = 0;
                    aphase ^= 1;
                }
            }
            if (any) {
                mma_commit(&mma_done);
                if (!bar_wait(&mma_done, 0)) atomicExch(g.err, 17);
            }
        }
    } else {
        const int qd = warp & 3;
        const int rho = 32 * qd + lane, c = rho >> 1, q = rho & 1;
        int acc = 0;
        uint32_t aphase = 0;
        for (int item = blockIdx.x; item < g.nitems && !*abort_v; item += gridDim.x) {
            const int2 it = g.items[item];
            if (!bar_wait(&accf[acc], aphase)) {
                if (lane == 0) atomicExch(g.err, 18);
                *abort_v = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int own = g.own_ptr[it.x + 1] - g.own_ptr[it.x];
            const int32_t* sub = g.sub_ids + g.sub_ptr[it.x];
            const uint32_t t0 = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(acc * 128);
            for (int c0 = 0; c0 < kTcN; c0 += 32) {
                uint32_t a[32];
                tmem_ld32(t0 + c0, a);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                for (int t = 0; t < 16; ++t) {
                    const float pR = __shfl_xor_sync(0xffffffffu, __uint_as_float(a[2 * t]), 1);
                    const float pI = __shfl_xor_sync(0xffffffffu, __uint_as_float(a[2 * t + 1]), 1);
                    const int i = it.y + c0 / 2 + t;
                    if (q == 0 && c < g.R && i < own) {
                        const float yr = __uint_as_float(a[2 * t]) - pI;
                        const float yi = pR + __uint_as_float(a[2 * t + 1]);
                        const size_t at = (size_t)c * g.n_unique + sub[i];
                        if (g.y_f32) static_cast<float2*>(g.y)[at] = make_float2(yr, yi);
                        else static_cast<double2*>(g.y)[at] = make_double2((double)yr, (double)yi);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(&acce[acc]);
            if (++acc == 2) {
                acc = 0;
                aphase ^= 1;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmTmemCols));
}

// planes of the owned inverse rows: out[2g + c][j] = hi/lo of (c ? Im : Re)
// X_m[i][j] for owned row g = own_ptr[m] + i, zero for j >= n_m
__global__ void pc_tc_split_rows_kernel(const float2* __restrict__ X, const int64_t* __restrict__ xoff,
                                        const int32_t* __restrict__ ldx, const int32_t* __restrict__ nsz,
                                        const int32_t* __restrict__ own_ptr, int M, int np,
                                        __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                        size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % np);
        const size_t rc = e / np;
        const int c = (int)(rc & 1);
        const int gr = (int)(rc >> 1);
        int lo_ = 0, hi_ = M;
        while (hi_ - lo_ > 1) {
            const int mid = (lo_ + hi_) >> 1;
            if (own_ptr[mid] <= gr) lo_ = mid; else hi_ = mid;
        }
        const int m = lo_, i = gr - own_ptr[m];
        float v = 0.f;
        if (j < nsz[m]) {
            const float2 x = X[xoff[m] + (size_t)i * ldx[m] + j];
            v = c ? x.y : x.x;
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// gathered r planes per cell: out[m][2c+q][j] = hi/lo of (q ? Im : Re)
// r[c][sub_m[j]] for rhs c < R and j < n_m, zero otherwise
template <typename VT>
__global__ void pc_tc_gather_kernel(const VT* __restrict__ r, const int32_t* __restrict__ sub_ptr,
                                    const int32_t* __restrict__ sub_ids, const int32_t* __restrict__ nsz,
                                    int R, int n_unique, int np, __nv_bfloat16* __restrict__ hi,
                                    __nv_bfloat16* __restrict__ lo, size_t total) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % np);
        const size_t mr = e / np;
        const int rho = (int)(mr % kTcM);
        const int m = (int)(mr / kTcM);
        const int cc = rho >> 1, q = rho & 1;
        float v = 0.f;
        if (cc < R && j < nsz[m]) {
            const VT x = r[(size_t)cc * n_unique + sub_ids[sub_ptr[m] + j]];
            v = (float)(q ? x.y : x.x);
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode3d(CUtensorMap* map, void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
             CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            !p) {
            set_error("tensor-core path: cuTensorMapEncodeTiled is not available");
            return EMSURF_ECUDA;
        }
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * 2, d0 * 2 * d1};
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tensor-core path: tensor map encoding failed (%d)", (int)r);
        return EMSURF_ECUDA;
    }
    return EMSURF_OK;
}

}  // namespace

int tc_tune(emsurf_handle* h);

// Create-time: split planes of the FP32 spectrum and the tensor maps.
int tc_build(emsurf_handle* h, const emsurf_handle* share) {
    const int E = h->E;
    const int ej = (E + 7) & ~7;     // rows of 16-byte multiples
    const int rows = 4 * kTcRhs * ((h->max_rhs + kTcRhs - 1) / kTcRhs);
    const size_t nb = (size_t)h->nbins;
    const size_t spec = nb * 2 * 2 * E * ej;
    if (share) {
        // the spectrum planes of a handle of the same lattice (not owned)
        h->tc_Bh = share->tc_Bh;
        h->tc_Bl = share->tc_Bl;
    } else {
        EMS_TRY(dev_alloc(h, (void**)&h->tc_Bh, spec * sizeof(__nv_bfloat16)));
        EMS_TRY(dev_alloc(h, (void**)&h->tc_Bl, spec * sizeof(__nv_bfloat16)));
        EMS_CUDA(cudaMemsetAsync(h->tc_Bh, 0, spec * sizeof(__nv_bfloat16), h->setup_stream));
        EMS_CUDA(cudaMemsetAsync(h->tc_Bl, 0, spec * sizeof(__nv_bfloat16), h->setup_stream));
    }
    const size_t xs = nb * rows * ej;
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Xh, xs * sizeof(__nv_bfloat16)));
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Xl, xs * sizeof(__nv_bfloat16)));
    if (!share) {
        for (size_t z0 = 0; z0 < nb * 2; z0 += 65535) {
            const dim3 grid((E + 31) / 32, (E + 31) / 32, (unsigned)std::min<size_t>(65535, nb * 2 - z0));
            tc_split_spectrum_kernel<<<grid, dim3(32, 8), 0, h->setup_stream>>>(
                h->op32.Bhat, reinterpret_cast<__nv_bfloat16*>(h->tc_Bh), reinterpret_cast<__nv_bfloat16*>(h->tc_Bl),
                E, ej, (int)z0);
            EMS_CUDA(cudaGetLastError());
            h->launches += 1;
        }
    }
    static_assert(sizeof(CUtensorMap) <= sizeof(h->tc_maps[0]), "tensor map storage");
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(h->tc_maps);
    // maps of both ring shapes: [0..3] 32-source boxes (64B swizzle), [8..11] 64-source boxes (128B)
    EMS_TRY(encode3d(&m[0], h->tc_Xh, ej, rows, nb, 32, kTcM, CU_TENSOR_MAP_SWIZZLE_64B));
    EMS_TRY(encode3d(&m[1], h->tc_Xl, ej, rows, nb, 32, kTcM, CU_TENSOR_MAP_SWIZZLE_64B));
    EMS_TRY(encode3d(&m[2], h->tc_Bh, ej, 2 * E, 2 * nb, 32, kTcN, CU_TENSOR_MAP_SWIZZLE_64B));
    EMS_TRY(encode3d(&m[3], h->tc_Bl, ej, 2 * E, 2 * nb, 32, kTcN, CU_TENSOR_MAP_SWIZZLE_64B));
    EMS_TRY(encode3d(&m[8], h->tc_Xh, ej, rows, nb, 64, kTcM));
    EMS_TRY(encode3d(&m[9], h->tc_Xl, ej, rows, nb, 64, kTcM));
    EMS_TRY(encode3d(&m[10], h->tc_Bh, ej, 2 * E, 2 * nb, 64, kTcN));
    EMS_TRY(encode3d(&m[11], h->tc_Bl, ej, 2 * E, 2 * nb, 64, kTcN));
    h->tc_ej = ej;
    h->tc_rows = rows;
    // macromodel planes: Z~ [t][2k+c][kp] and x1 tiles [tile][128][kp]
    const int K = h->K, kp = (K + 7) & ~7;
    const size_t zs = (size_t)h->T * 2 * K * kp;
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Zh, zs * sizeof(__nv_bfloat16)));
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Zl, zs * sizeof(__nv_bfloat16)));
    EMS_CUDA(cudaMemsetAsync(h->tc_Zh, 0, zs * sizeof(__nv_bfloat16), h->setup_stream));
    EMS_CUDA(cudaMemsetAsync(h->tc_Zl, 0, zs * sizeof(__nv_bfloat16), h->setup_stream));
    const dim3 zgrid((K + 31) / 32, (K + 31) / 32, (unsigned)h->T);
    tc_split_spectrum_kernel<<<zgrid, dim3(32, 8), 0, h->setup_stream>>>(
        h->op32.Zt, reinterpret_cast<__nv_bfloat16*>(h->tc_Zh), reinterpret_cast<__nv_bfloat16*>(h->tc_Zl), K, kp, 0);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    int maxtiles = 0;
    for (int t = 0; t < h->T; ++t)
        maxtiles += ((h->h_type_ptr[t + 1] - h->h_type_ptr[t]) * h->max_rhs + 63) / 64;
    maxtiles = std::max(maxtiles, 1);
    const size_t ms = (size_t)maxtiles * kTcM * kp;
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Mh, ms * sizeof(__nv_bfloat16)));
    EMS_TRY(dev_alloc(h, (void**)&h->tc_Ml, ms * sizeof(__nv_bfloat16)));
    EMS_TRY(encode3d(&m[4], h->tc_Mh, kp, kTcM, maxtiles, kTcKc, kTcM));
    EMS_TRY(encode3d(&m[5], h->tc_Ml, kp, kTcM, maxtiles, kTcKc, kTcM));
    EMS_TRY(encode3d(&m[6], h->tc_Zh, kp, 2 * K, h->T, kTcKc, kTcN));
    EMS_TRY(encode3d(&m[7], h->tc_Zl, kp, 2 * K, h->T, kTcKc, kTcN));
    h->tc_kp = kp;
    h->tc_mm_tiles.assign(h->max_rhs + 1, nullptr);
    h->tc_mm_ntiles.assign(h->max_rhs + 1, 0);
    h->have_tc = true;
    if (share) {
        h->tc_variant = share->tc_variant;
        h->tc_tune_ms[0] = share->tc_tune_ms[0];
        h->tc_tune_ms[1] = share->tc_tune_ms[1];
    } else {
        EMS_TRY(tc_tune(h));
    }
    return EMSURF_OK;
}

// Macromodel products of R rhs on the tensor cores into Ymm[0] ([R][M][K]).
int tc_macromodel(emsurf_handle* h, const double2* x, const float2* xf, float2* Ymm, int R, cudaStream_t st) {
    const int K = h->K, kp = h->tc_kp;
    if (!h->tc_mm_tiles[R]) {
        // tiles of 64 columns (cell slot, rhs) per type, for this rhs count
        std::vector<int2> tl;
        for (int t = 0; t < h->T; ++t) {
            const int ncol = (h->h_type_ptr[t + 1] - h->h_type_ptr[t]) * R;
            for (int c0 = 0; c0 < ncol; c0 += 64) tl.push_back(make_int2(t, c0));
        }
        if (tl.empty()) tl.push_back(make_int2(0, 1 << 30));
        int2* d = nullptr;
        EMS_TRY(dev_alloc(h, (void**)&d, tl.size() * sizeof(int2)));
        EMS_CUDA(cudaMemcpy(d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice));
        h->tc_mm_tiles[R] = d;
        h->tc_mm_ntiles[R] = (int)tl.size();
    }
    const int ntiles = h->tc_mm_ntiles[R];
    const int2* tiles = static_cast<const int2*>(h->tc_mm_tiles[R]);
    const size_t total = (size_t)ntiles * kTcM * kp;
    tc_mm_gather_kernel<<<(int)std::min<size_t>((total + 255) / 256, (size_t)h->num_sms * 16), 256, 0, st>>>(
        x, xf, h->d_uo_index, h->d_uo_sign, tiles, h->d_type_ptr, h->d_type_cells,
        reinterpret_cast<__nv_bfloat16*>(h->tc_Mh), reinterpret_cast<__nv_bfloat16*>(h->tc_Ml), K, kp, R,
        h->n_unique, total);
    EMS_CUDA(cudaGetLastError());
    MmArgs a;
    a.Y = Ymm;
    a.tiles = tiles;
    a.type_ptr = h->d_type_ptr;
    a.type_cells = h->d_type_cells;
    a.K = K;
    a.M = h->M;
    a.R = R;
    a.ntiles = ntiles;
    a.chunks = (2 * K + kTcN - 1) / kTcN;
    a.nk = (kp + kTcKc - 1) / kTcKc;
    a.items = ntiles * a.chunks;
    a.err = h->d_err;
    EMS_TRY(set_smem_once(mm_tc_kernel, (size_t)kMmSmem));
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(h->tc_maps);
    mm_tc_kernel<<<std::min(a.items, h->num_sms), kTcThreads, kMmSmem, st>>>(m[4], m[5], m[6], m[7], a);
    EMS_CUDA(cudaGetLastError());
    h->launches += 2;
    return EMSURF_OK;
}

// launch of the bin multiply's kernel in ring shape `variant` (0: 32 x 5, 1: 64 x 2)
int tc_binmul_launch(emsurf_handle* h, float2* Y, int R, const float2* coef, int variant, cudaStream_t st) {
    const int E = h->E, ej = h->tc_ej;
    const size_t nb = (size_t)h->nbins;
    TcArgs a;
    a.Y = Y;
    a.E = E;
    a.nbins = (int)nb;
    a.R = R;
    a.groups = (R + kTcRhs - 1) / kTcRhs;
    a.chunks = (2 * E + kTcN - 1) / kTcN;
    const int kc = variant == 0 ? 32 : 64;
    a.nk = (ej + kc - 1) / kc;
    a.items = a.groups * a.nbins * a.chunks;
    a.ca = coef[0];
    a.cb = coef[1];
    a.cg = coef[2];
    a.cd = coef[3];
    a.err = h->d_err;
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(h->tc_maps);
    const int grid = std::min(a.items, h->num_sms);
    if (variant == 0) {
        constexpr int sm = bm_smem<32, 5>();
        EMS_TRY(set_smem_once(binmul_tc_kernel<32, 5>, (size_t)sm));
        binmul_tc_kernel<32, 5><<<grid, kTcThreads, sm, st>>>(m[0], m[1], m[2], m[3], a);
    } else {
        constexpr int sm = bm_smem<64, 2>();
        EMS_TRY(set_smem_once(binmul_tc_kernel<64, 2>, (size_t)sm));
        binmul_tc_kernel<64, 2><<<grid, kTcThreads, sm, st>>>(m[8], m[9], m[10], m[11], a);
    }
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return EMSURF_OK;
}

// Y^ = B^ X^ for every bin on the tensor cores (R rhs, FP32 grids [bins][R][2E]).
int tc_binmul(emsurf_handle* h, const float2* X, float2* Y, int R, const float2* coef, cudaStream_t st) {
    const int E = h->E, ej = h->tc_ej, rows = h->tc_rows;
    const size_t nb = (size_t)h->nbins;
    const size_t xs = nb * rows * ej;
    tc_split_x_kernel<<<(int)std::min<size_t>((xs + 255) / 256, (size_t)h->num_sms * 16), 256, 0, st>>>(
        X, reinterpret_cast<__nv_bfloat16*>(h->tc_Xh), reinterpret_cast<__nv_bfloat16*>(h->tc_Xl), E, ej, R, rows, xs);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    return tc_binmul_launch(h, Y, R, coef, h->tc_variant, st);
}

// The project's autotuner for the bin multiply's ring shape: both shapes
// run twice on this handle's spectrum (max_rhs rhs; the values in the X^
// planes do not change the time), CUDA events on the setup stream, the
// faster one kept.  Shared handles take their share's choice.
int tc_tune(emsurf_handle* h) {
    cudaStream_t st = h->setup_stream;
    const float2 coef[4] = {make_float2(1.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(1.f, 0.f)};
    float best = 1e30f;
    cudaEvent_t e0, e1;
    EMS_CUDA(cudaEventCreate(&e0));
    EMS_CUDA(cudaEventCreate(&e1));
    int status = EMSURF_OK;
    for (int v = 0; v < 2 && !status; ++v) {
        status = tc_binmul_launch(h, h->op32.Yg, h->max_rhs, coef, v, st);          // warm-up
        if (status) break;
        cudaEventRecord(e0, st);
        status = tc_binmul_launch(h, h->op32.Yg, h->max_rhs, coef, v, st);
        cudaEventRecord(e1, st);
        if (status) break;
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            set_error("tensor-core autotune: event timing failed");
            status = EMSURF_ECUDA;
            break;
        }
        h->tc_tune_ms[v] = ms;
        if (ms < best) {
            best = ms;
            h->tc_variant = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

}  // namespace emsurf

namespace emsurf {

// Create-time: planes of the owned inverse rows, gather buffer, items, maps.
int pc_tc_build(emsurf_handle* h, const std::vector<int32_t>& optr) {
    const int np = (h->pc_nmax + 7) & ~7;
    const size_t rows = (size_t)2 * h->n_unique;
    EMS_TRY(dev_alloc(h, (void**)&h->pc_tc_Xh, rows * np * sizeof(__nv_bfloat16)));
    EMS_TRY(dev_alloc(h, (void**)&h->pc_tc_Xl, rows * np * sizeof(__nv_bfloat16)));
    const size_t total = rows * np;
    pc_tc_split_rows_kernel<<<(int)std::min<size_t>((total + 255) / 256, (size_t)h->num_sms * 16), 256, 0,
                              h->setup_stream>>>(h->pc_mat, h->pc_off, h->pc_ld, h->pc_n, h->pc_own_ptr, h->M, np,
                                                 reinterpret_cast<__nv_bfloat16*>(h->pc_tc_Xh),
                                                 reinterpret_cast<__nv_bfloat16*>(h->pc_tc_Xl), total);
    EMS_CUDA(cudaGetLastError());
    h->launches += 1;
    const size_t gs = (size_t)h->M * kTcM * np;
    EMS_TRY(dev_alloc(h, (void**)&h->pc_tc_Rh, gs * sizeof(__nv_bfloat16)));
    EMS_TRY(dev_alloc(h, (void**)&h->pc_tc_Rl, gs * sizeof(__nv_bfloat16)));
    std::vector<int2> items;
    for (int m = 0; m < h->M; ++m)
        for (int i0 = 0; i0 < optr[m + 1] - optr[m]; i0 += kTcN / 2) items.push_back(make_int2(m, i0));
    if (items.empty()) items.push_back(make_int2(0, 1 << 30));
    int2* d = nullptr;
    EMS_TRY(dev_alloc(h, (void**)&d, items.size() * sizeof(int2)));
    EMS_CUDA(cudaMemcpy(d, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    h->pc_tc_items = d;
    h->pc_tc_nitems = (int)items.size();
    h->pc_tc_np = np;
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(h->pc_tc_maps);
    EMS_TRY(encode3d(&m[0], h->pc_tc_Rh, np, kTcM, h->M, kTcKc, kTcM));
    EMS_TRY(encode3d(&m[1], h->pc_tc_Rl, np, kTcM, h->M, kTcKc, kTcM));
    EMS_TRY(encode3d(&m[2], h->pc_tc_Xh, np, rows, 1, kTcKc, kTcN));
    EMS_TRY(encode3d(&m[3], h->pc_tc_Xl, np, rows, 1, kTcKc, kTcN));
    h->have_pc_tc = true;
    return EMSURF_OK;
}

template <typename VT>
int pc_tc_apply(emsurf_handle* h, const VT* r, VT* y, int R, cudaStream_t st) {
    const int np = h->pc_tc_np;
    const size_t gs = (size_t)h->M * kTcM * np;
    pc_tc_gather_kernel<VT><<<(int)std::min<size_t>((gs + 255) / 256, (size_t)h->num_sms * 16), 256, 0, st>>>(
        r, h->pc_sub_ptr, h->pc_sub_ids, h->pc_n, R, h->n_unique, np,
        reinterpret_cast<__nv_bfloat16*>(h->pc_tc_Rh), reinterpret_cast<__nv_bfloat16*>(h->pc_tc_Rl), gs);
    EMS_CUDA(cudaGetLastError());
    PcArgs a;
    a.y = y;
    a.y_f32 = std::is_same<VT, float2>::value ? 1 : 0;
    a.items = static_cast<const int2*>(h->pc_tc_items);
    a.own_ptr = h->pc_own_ptr;
    a.nsz = h->pc_n;
    a.sub_ptr = h->pc_sub_ptr;
    a.sub_ids = h->pc_sub_ids;
    a.R = R;
    a.n_unique = h->n_unique;
    a.nitems = h->pc_tc_nitems;
    a.err = h->d_err;
    EMS_TRY(set_smem_once(pc_tc_kernel, (size_t)kMmSmem));
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(h->pc_tc_maps);
    pc_tc_kernel<<<std::min(a.nitems, h->num_sms), kTcThreads, kMmSmem, st>>>(m[0], m[1], m[2], m[3], a);
    EMS_CUDA(cudaGetLastError());
    h->launches += 2;
    return EMSURF_OK;
}

template int pc_tc_apply<double2>(emsurf_handle*, const double2*, double2*, int, cudaStream_t);
template int pc_tc_apply<float2>(emsurf_handle*, const float2*, float2*, int, cudaStream_t);

}  // namespace emsurf

extern "C" {

EMSURF_API int emsurf_tc_tuning(const emsurf_handle* h, int32_t* sources_per_stage, int32_t* stages,
                                double* ms_shapes) {
    if (!h) { emsurf::set_error("emsurf_tc_tuning: NULL handle"); return EMSURF_EINVAL; }
    if (!h->have_tc) {
        if (sources_per_stage) *sources_per_stage = 0;
        if (stages) *stages = 0;
        if (ms_shapes) ms_shapes[0] = ms_shapes[1] = 0.0;
        return EMSURF_OK;
    }
    if (sources_per_stage) *sources_per_stage = h->tc_variant == 0 ? 32 : 64;
    if (stages) *stages = h->tc_variant == 0 ? 5 : 2;
    if (ms_shapes) {
        ms_shapes[0] = h->tc_tune_ms[0];
        ms_shapes[1] = h->tc_tune_ms[1];
    }
    return EMSURF_OK;
}

}  // extern "C"
