// C ABI entry points: create / matvec / solve / query / destroy.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "common.cuh"

namespace emsurf {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int set_smem_attr(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> have;
    int dev = 0;
    EMS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(dev, kernel);
    auto it = have.find(key);
    if (it != have.end() && it->second >= bytes) return EMSURF_OK;
    EMS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have[key] = bytes;
    return EMSURF_OK;
}

int dev_alloc(emsurf_handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (h->budget > 0 && h->device_bytes + (int64_t)bytes > h->budget) {
        set_error("device memory budget exceeded: %lld + %zu > %lld bytes",
                  (long long)h->device_bytes, bytes, (long long)h->budget);
        return EMSURF_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return EMSURF_ENOMEM;
    }
    h->allocations.push_back(*p);
    h->device_bytes += (int64_t)bytes;
    return EMSURF_OK;
}

void dev_free(emsurf_handle* h, void* p, size_t bytes) {
    if (!p) return;
    for (size_t i = 0; i < h->allocations.size(); ++i)
        if (h->allocations[i] == p) {
            cudaFree(p);
            h->allocations.erase(h->allocations.begin() + (long)i);
            h->device_bytes -= (int64_t)std::max<size_t>(bytes, 16);
            return;
        }
}

namespace {

class DeviceGuard {
public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        ok_ = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() { cudaSetDevice(prev_); }
    bool ok() const { return ok_; }

private:
    int prev_ = 0;
    bool ok_ = false;
};

int validate(const emsurf_problem* p) {
    if (!p) { set_error("problem is NULL"); return EMSURF_EINVAL; }
    if (p->nx < 1 || p->ny < 1 || p->n_edges < 1 || p->n_types < 1 || p->n_unique < 1) {
        set_error("nx, ny, n_edges, n_types, n_unique must be >= 1");
        return EMSURF_EINVAL;
    }
    if (p->max_rhs < 1 || p->max_rhs > 64) {
        set_error("max_rhs must be in [1, 64]");
        return EMSURF_EINVAL;
    }
    if (p->precision < EMSURF_FP64 || p->precision > EMSURF_MIXED) {
        set_error("unknown precision %d", p->precision);
        return EMSURF_EINVAL;
    }
    if (!p->type_map || !p->macromodels || !p->offset_L || !p->offset_K || !p->uo_index ||
        !p->uo_sign) {
        set_error("a required input pointer is NULL");
        return EMSURF_EINVAL;
    }
    if ((p->grid_px && p->grid_px < 2 * p->nx - 1) || (p->grid_py && p->grid_py < 2 * p->ny - 1)) {
        set_error("grid must be at least (2nx-1) x (2ny-1)");
        return EMSURF_EINVAL;
    }
    const int64_t M = (int64_t)p->nx * p->ny, K = 2LL * p->n_edges;
    if (M * K > INT32_MAX) { set_error("too many local unknowns"); return EMSURF_EINVAL; }
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(p->coef[c].re) || !std::isfinite(p->coef[c].im)) {
            set_error("coef[%d] is not finite", c);
            return EMSURF_EINVAL;
        }
    if (!p->tables_on_device) {
        // host inputs: a NaN or an infinity would spread through every product
        const size_t nz = (size_t)p->n_types * (size_t)K * (size_t)K;
        const size_t nt = (size_t)(2 * p->nx - 1) * (size_t)(2 * p->ny - 1) * (size_t)p->n_edges * p->n_edges;
        const struct { const emsurf_c128* a; size_t n; const char* name; } arrays[3] = {
            {p->macromodels, nz, "macromodels"}, {p->offset_L, nt, "offset_L"}, {p->offset_K, nt, "offset_K"}};
        for (const auto& t : arrays)
            for (size_t i = 0; i < t.n; ++i)
                if (!std::isfinite(t.a[i].re) || !std::isfinite(t.a[i].im)) {
                    set_error("%s[%zu] is not finite", t.name, i);
                    return EMSURF_EINVAL;
                }
    }
    for (int64_t m = 0; m < M; ++m)
        if (p->type_map[m] < 0 || p->type_map[m] >= p->n_types) {
            set_error("type_map[%lld] = %d out of range", (long long)m, p->type_map[m]);
            return EMSURF_EINVAL;
        }
    for (int64_t e = 0; e < M * K; ++e) {
        if (p->uo_index[e] < 0 || p->uo_index[e] >= p->n_unique) {
            set_error("uo_index[%lld] = %d out of range", (long long)e, p->uo_index[e]);
            return EMSURF_EINVAL;
        }
        if (p->uo_sign[e] != 1 && p->uo_sign[e] != -1) {
            set_error("uo_sign[%lld] = %d is not +-1", (long long)e, (int)p->uo_sign[e]);
            return EMSURF_EINVAL;
        }
    }
    return EMSURF_OK;
}

template <typename T>
int upload(emsurf_handle* h, T** d, const T* src, size_t n) {
    EMS_TRY(dev_alloc(h, (void**)d, n * sizeof(T)));
    EMS_CUDA(cudaMemcpyAsync(*d, src, n * sizeof(T), cudaMemcpyHostToDevice, h->setup_stream));
    return EMSURF_OK;
}

int create_impl(const emsurf_problem* p, emsurf_handle* h, const emsurf_handle* share) {
    h->device = p->device;
    h->setup_stream = reinterpret_cast<cudaStream_t>(p->stream);
    h->nx = p->nx;
    h->ny = p->ny;
    h->E = p->n_edges;
    h->K = 2 * p->n_edges;
    h->M = p->nx * p->ny;
    h->T = p->n_types;
    h->n_unique = p->n_unique;
    h->max_rhs = p->max_rhs;
    h->precision = p->precision;
    h->budget = p->device_mem_budget;
    h->px = share ? share->px : p->grid_px ? p->grid_px : smallest_smooth_at_least(2 * p->nx - 1);
    h->py = share ? share->py : p->grid_py ? p->grid_py : smallest_smooth_at_least(2 * p->ny - 1);
    h->nbins = h->px * h->py;
    EMS_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    EMS_CUDA(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    EMS_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    EMS_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    EMS_TRY(dev_alloc(h, (void**)&h->d_err, sizeof(int)));
    EMS_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->setup_stream));
    EMS_TRY(dev_alloc(h, (void**)&h->d_grid_bar, 2 * sizeof(unsigned)));
    EMS_CUDA(cudaMemsetAsync(h->d_grid_bar, 0, 2 * sizeof(unsigned), h->setup_stream));
    EMS_TRY(fft_plan_create(h->plan_x, h->px));
    EMS_TRY(fft_plan_create(h->plan_y, h->py));
    const int M = h->M, K = h->K;
    const size_t MK = (size_t)M * K;
    // U_o and its inverse (CSR by unique unknown, local entries in scan order)
    EMS_TRY(upload(h, &h->d_uo_index, p->uo_index, MK));
    EMS_TRY(upload(h, &h->d_uo_sign, p->uo_sign, MK));
    std::vector<int32_t> ptr(h->n_unique + 1, 0), ent(MK);
    std::vector<int8_t> esg(MK);
    for (size_t e = 0; e < MK; ++e) ptr[p->uo_index[e] + 1]++;
    for (int u = 0; u < h->n_unique; ++u) ptr[u + 1] += ptr[u];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t e = 0; e < MK; ++e) {
        const int u = p->uo_index[e];
        ent[fill[u]] = (int32_t)e;
        esg[fill[u]] = p->uo_sign[e];
        fill[u]++;
    }
    for (int u = 0; u < h->n_unique; ++u)
        if (ptr[u + 1] == ptr[u]) {
            set_error("unique unknown %d is referenced by no local unknown", u);
            return EMSURF_EINVAL;
        }
    EMS_TRY(upload(h, &h->d_inv_ptr, ptr.data(), ptr.size()));
    EMS_TRY(upload(h, &h->d_inv_ent, ent.data(), MK));
    EMS_TRY(upload(h, &h->d_inv_sgn, esg.data(), MK));
    // cells grouped by type; macromodel work list in groups of 8 cells
    std::vector<int32_t> tptr(h->T + 1, 0), cells(M);
    for (int m = 0; m < M; ++m) tptr[p->type_map[m] + 1]++;
    for (int t = 0; t < h->T; ++t) tptr[t + 1] += tptr[t];
    {
        std::vector<int32_t> f(tptr.begin(), tptr.end() - 1);
        for (int m = 0; m < M; ++m) cells[f[p->type_map[m]]++] = m;
    }
    std::vector<int32_t> blocks;
    for (int t = 0; t < h->T; ++t)
        for (int s = tptr[t]; s < tptr[t + 1]; s += kMmGroup) {
            blocks.push_back(t);
            blocks.push_back(s);
            blocks.push_back(std::min(kMmGroup, tptr[t + 1] - s));
        }
    h->h_type_ptr = tptr;
    h->n_mm_blocks = (int)(blocks.size() / 3);
    EMS_TRY(upload(h, &h->d_type_map, p->type_map, (size_t)M));
    EMS_TRY(upload(h, &h->d_type_cells, cells.data(), (size_t)M));
    EMS_TRY(upload(h, &h->d_type_ptr, tptr.data(), tptr.size()));
    int32_t* dblk = nullptr;
    EMS_TRY(upload(h, &dblk, blocks.data(), blocks.size()));
    h->d_mm_blocks = dblk;
    // operators
    if (h->precision == EMSURF_FP64 || h->precision == EMSURF_MIXED) {
        EMS_TRY(build_operator<double2>(h, h->op64, p, share ? &share->op64 : nullptr));
        h->have64 = true;
    }
    if (h->precision == EMSURF_FP32) {
        EMS_TRY(build_operator<float2>(h, h->op32, p, share ? &share->op32 : nullptr));
        if (share) EMS_TRY(adopt_fp32_form(h, share));
        h->have32 = true;
    } else if (h->precision == EMSURF_MIXED) {
        EMS_TRY(derive_fp32_operator(h, p, share));
        h->have32 = true;
    }
    if (h->have64) EMS_TRY(build_ds_planes(h, share));
    if (p->tensor_cores && h->have32 && h->E >= 64) EMS_TRY(tc_build(h, share));
    if (share) {
        h->near_L = share->near_L;
        h->near_K = share->near_K;
    } else {
        EMS_TRY(stage_near_tables(h, p));
    }
    if (p->precond_overlap > 0.0 && p->unknown_xy) {
        if (!(p->cell_a > 0.0) || !(p->cell_b > 0.0)) {
            set_error("the preconditioner needs cell_a, cell_b > 0");
            return EMSURF_EINVAL;
        }
        EMS_TRY(pc_build(h, p));
    }
    EMS_CUDA(cudaStreamSynchronize(h->setup_stream));
    // with the double-single planes every FP64-accuracy bin multiply reads
    // them (one rhs and several), so the complex128 spectrum is not needed
    // after create: its bytes (those of the planes) are given back
    if (h->have64 && h->ds_planes && h->op64.Bhat) {
        dev_free(h, h->op64.Bhat, (size_t)h->nbins * 2 * (size_t)h->E * h->E * sizeof(double2));
        h->op64.Bhat = nullptr;
    }
    return EMSURF_OK;
}

void free_handle(emsurf_handle* h) {
    for (auto& pt : h->prof)
        for (cudaEvent_t e : pt.ev) cudaEventDestroy(e);
    if (h->side_stream) {
        cudaStreamSynchronize(h->side_stream);
        cudaStreamDestroy(h->side_stream);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (void* p : h->allocations) cudaFree(p);
    h->allocations.clear();
    fft_plan_destroy(h->plan_x);
    fft_plan_destroy(h->plan_y);
    delete h;
}

}  // namespace

void prof_mark(emsurf_handle* h, int phase, bool begin, cudaStream_t st) {
    if (!h->prof_on || !((h->prof_mask >> phase) & 1u)) return;
    PhaseTimer& pt = h->prof[phase];
    // a begin takes a fresh pair; an end closes the pair opened last
    if (begin) {
        if (pt.used + 2 > pt.ev.size())
            for (int i = 0; i < 2; ++i) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) { h->prof_on = false; return; }
                pt.ev.push_back(e);
            }
        cudaEventRecord(pt.ev[pt.used], st);
        pt.used += 2;
    } else if (pt.used >= 2) {
        cudaEventRecord(pt.ev[pt.used - 1], st);
    }
}

void gmres_release(emsurf_handle* h);

// Clears the bounded-wait error flag and the state an aborted launch may
// have left behind (the pair kernel's arrival counters, the grid barrier of
// the cooperative Arnoldi step).
int clear_wait_error(emsurf_handle* h) {
    EMS_CUDA(cudaDeviceSynchronize());
    EMS_CUDA(cudaMemset(h->d_err, 0, sizeof(int)));
    if (h->d_pair_cnt) EMS_CUDA(cudaMemset(h->d_pair_cnt, 0, h->pair_cnt_bytes));
    if (h->d_ds_max) EMS_CUDA(cudaMemset(h->d_ds_max, 0, sizeof(unsigned long long) * std::max(1, h->max_rhs)));
    if (h->d_ds_cnt) EMS_CUDA(cudaMemset(h->d_ds_cnt, 0, sizeof(unsigned) * std::max(1, h->max_rhs)));
    if (h->d_grid_bar) EMS_CUDA(cudaMemset(h->d_grid_bar, 0, 2 * sizeof(unsigned)));
    return EMSURF_OK;
}

}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API const char* emsurf_last_error(void) { return g_err; }

EMSURF_API int emsurf_create(const emsurf_problem* problem, emsurf_handle** out) {
    if (!out) { set_error("out is NULL"); return EMSURF_EINVAL; }
    *out = nullptr;
    EMS_TRY(validate(problem));
    DeviceGuard dg(problem->device);
    if (!dg.ok()) { set_error("cannot select device %d", problem->device); return EMSURF_EINVAL; }
    emsurf_handle* h = new (std::nothrow) emsurf_handle();
    if (!h) { set_error("host allocation failed"); return EMSURF_ENOMEM; }
    const int s = create_impl(problem, h, nullptr);
    if (s != EMSURF_OK) {
        cudaStreamSynchronize(h->setup_stream);
        gmres_release(h);
        free_handle(h);
        return s;
    }
    *out = h;
    return EMSURF_OK;
}

EMSURF_API int emsurf_create_like(const emsurf_problem* problem, const emsurf_handle* share,
                                  emsurf_handle** out) {
    if (!out || !share || !problem) { set_error("emsurf_create_like: NULL argument"); return EMSURF_EINVAL; }
    *out = nullptr;
    // the tables are not read: stand-ins pass the pointer checks
    emsurf_problem p = *problem;
    if (!p.offset_L) p.offset_L = p.macromodels;
    if (!p.offset_K) p.offset_K = p.macromodels;
    const int save_dev = p.tables_on_device;
    p.tables_on_device = 1;                 // skip the host scan of tables that are not read
    EMS_TRY(validate(&p));
    p.tables_on_device = save_dev;
    if (p.nx != share->nx || p.ny != share->ny || p.n_edges != share->E || p.precision != share->precision ||
        p.device != share->device || (p.grid_px && p.grid_px != share->px) || (p.grid_py && p.grid_py != share->py)) {
        set_error("emsurf_create_like: lattice, RWG count, grid, precision or device differ from the shared handle");
        return EMSURF_EINVAL;
    }
    const bool tc_wanted = p.tensor_cores && p.precision != EMSURF_FP64 && p.n_edges >= 64;
    if ((share->half32 || share->orb32) && (p.max_rhs != 1 || tc_wanted)) {
        set_error("emsurf_create_like: the shared handle keeps part of the FP32 spectrum (one rhs, no tensor "
                  "cores); this problem needs the full spectrum");
        return EMSURF_EINVAL;
    }
    if (tc_wanted && !share->have_tc) {
        set_error("emsurf_create_like: tensor cores asked for, the shared handle has no tensor-core planes");
        return EMSURF_EINVAL;
    }
    if (!p.tables_on_device) {
        const size_t nz = (size_t)p.n_types * (size_t)(2 * p.n_edges) * (size_t)(2 * p.n_edges);
        for (size_t i = 0; i < nz; ++i)
            if (!std::isfinite(p.macromodels[i].re) || !std::isfinite(p.macromodels[i].im)) {
                set_error("macromodels[%zu] is not finite", i);
                return EMSURF_EINVAL;
            }
    }
    DeviceGuard dg(p.device);
    if (!dg.ok()) { set_error("cannot select device %d", p.device); return EMSURF_EINVAL; }
    emsurf_handle* h = new (std::nothrow) emsurf_handle();
    if (!h) { set_error("host allocation failed"); return EMSURF_ENOMEM; }
    const int s = create_impl(&p, h, share);
    if (s != EMSURF_OK) {
        cudaStreamSynchronize(h->setup_stream);
        gmres_release(h);
        free_handle(h);
        return s;
    }
    *out = h;
    return EMSURF_OK;
}

EMSURF_API int emsurf_matvec(emsurf_handle* h, const emsurf_c128* x, emsurf_c128* y, int32_t nrhs,
                             int32_t precision, void* stream) {
    if (!h || !x || !y) { set_error("NULL handle or vector"); return EMSURF_EINVAL; }
    if (nrhs < 1 || nrhs > h->max_rhs) {
        set_error("nrhs %d outside [1, %d]", nrhs, h->max_rhs);
        return EMSURF_EINVAL;
    }
    const size_t n = (size_t)nrhs * h->n_unique;
    const char* xa = reinterpret_cast<const char*>(x);
    const char* ya = reinterpret_cast<const char*>(y);
    if (xa < ya + n * sizeof(emsurf_c128) && ya < xa + n * sizeof(emsurf_c128)) {
        set_error("x and y overlap");
        return EMSURF_EINVAL;
    }
    DeviceGuard dg(h->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (precision == EMSURF_FP64) {
        if (!h->have64) { set_error("FP64 operator not resident"); return EMSURF_EINVAL; }
        return apply_operator<double2>(h, h->op64, reinterpret_cast<const double2*>(x),
                                       reinterpret_cast<double2*>(y), nrhs, st);
    }
    if (precision == EMSURF_FP32) {
        if (!h->have32) { set_error("FP32 operator not resident"); return EMSURF_EINVAL; }
        return apply_operator<float2>(h, h->op32, reinterpret_cast<const double2*>(x),
                                      reinterpret_cast<double2*>(y), nrhs, st);
    }
    set_error("matvec precision must be EMSURF_FP64 or EMSURF_FP32");
    return EMSURF_EINVAL;
}

EMSURF_API int emsurf_operator_info(const emsurf_handle* h, int32_t* stored_bins, int32_t* tensor_cores) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    if (stored_bins) *stored_bins = (h->half32 || h->orb32) ? h->nst : h->nbins;
    if (tensor_cores) *tensor_cores = h->have_tc ? 1 : 0;
    return EMSURF_OK;
}

EMSURF_API int emsurf_operator_layout(const emsurf_handle* h, int32_t* form, int32_t* bins_per_stored) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    const int f = h->orb32 ? 2 : h->half32 ? 1 : 0;
    if (form) *form = f;
    if (bins_per_stored) *bins_per_stored = f == 2 ? h->orb_G : f == 1 ? 2 : 1;
    return EMSURF_OK;
}

EMSURF_API int emsurf_precond_info(const emsurf_handle* h, int64_t* factor_entries,
                                   int64_t* subdomain_total, int32_t* max_subdomain) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    if (factor_entries) *factor_entries = h->have_pc ? h->pc_elems : 0;
    if (subdomain_total) *subdomain_total = h->have_pc ? h->pc_sub_total : 0;
    if (max_subdomain) *max_subdomain = h->have_pc ? h->pc_nmax : 0;
    return EMSURF_OK;
}

EMSURF_API int emsurf_precond_apply(emsurf_handle* h, const emsurf_c128* r, emsurf_c128* y,
                                    int32_t nrhs, void* stream) {
    if (!h || !r || !y) { set_error("NULL handle or vector"); return EMSURF_EINVAL; }
    if (!h->have_pc) { set_error("no preconditioner was built for this handle"); return EMSURF_EINVAL; }
    if (nrhs < 1 || nrhs > h->max_rhs) {
        set_error("nrhs %d outside [1, %d]", nrhs, h->max_rhs);
        return EMSURF_EINVAL;
    }
    const size_t n = (size_t)nrhs * h->n_unique * sizeof(emsurf_c128);
    const char* ra = reinterpret_cast<const char*>(r);
    const char* ya = reinterpret_cast<const char*>(y);
    if (ra < ya + n && ya < ra + n) { set_error("r and y overlap"); return EMSURF_EINVAL; }
    DeviceGuard dg(h->device);
    return pc_apply(h, reinterpret_cast<const double2*>(r), reinterpret_cast<double2*>(y), nrhs,
                    reinterpret_cast<cudaStream_t>(stream));
}

EMSURF_API int emsurf_solve(emsurf_handle* h, const emsurf_c128* b, emsurf_c128* x, int32_t nrhs,
                            const emsurf_solve_opts* opts, emsurf_solve_info* info, void* stream) {
    if (!h || !b || !x || !opts) { set_error("NULL argument"); return EMSURF_EINVAL; }
    if (nrhs < 1 || nrhs > h->max_rhs) {
        set_error("nrhs %d outside [1, %d]", nrhs, h->max_rhs);
        return EMSURF_EINVAL;
    }
    if (!(opts->rtol > 0.0) || opts->restart < 1 || opts->restart > 64 || opts->max_iters < 1 ||
        !(opts->max_ms >= 0.0)) {
        set_error("need rtol > 0, restart in [1, 64], max_iters >= 1");
        return EMSURF_EINVAL;
    }
    if (opts->solver < 0 || opts->solver > 3) {
        set_error("solver must be 0..3");
        return EMSURF_EINVAL;
    }
    const int mode = opts->solver ? opts->solver
                                  : (h->precision == EMSURF_MIXED ? 3 : (h->precision == EMSURF_FP32 ? 2 : 1));
    if ((mode == 1 || mode == 3) && !h->have64) {
        set_error("solver needs the FP64 operator, which is not resident");
        return EMSURF_EINVAL;
    }
    if ((mode == 2 || mode == 3) && !h->have32) {
        set_error("solver needs the FP32 operator, which is not resident");
        return EMSURF_EINVAL;
    }
    if (mode == 3 && opts->max_refine < 1) {
        set_error("mixed solve needs max_refine >= 1");
        return EMSURF_EINVAL;
    }
    DeviceGuard dg(h->device);
    return gmres_solve(h, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x), nrhs,
                       opts, info, reinterpret_cast<cudaStream_t>(stream));
}

EMSURF_API int emsurf_query(const emsurf_handle* h, int32_t* grid_px, int32_t* grid_py,
                            int64_t* device_bytes) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    if (grid_px) *grid_px = h->px;
    if (grid_py) *grid_py = h->py;
    if (device_bytes) *device_bytes = h->device_bytes;
    return EMSURF_OK;
}

EMSURF_API int emsurf_profile(emsurf_handle* h, int32_t enable) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    if (enable) for (auto& pt : h->prof) pt.used = 0;
    h->prof_on = enable != 0;
    h->prof_mask = 0xffffffffu;
    return EMSURF_OK;
}

EMSURF_API int emsurf_profile_phases(emsurf_handle* h, uint32_t phase_mask) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    for (auto& pt : h->prof) pt.used = 0;
    h->prof_on = phase_mask != 0;
    h->prof_mask = phase_mask;
    return EMSURF_OK;
}

EMSURF_API int emsurf_profile_read(emsurf_handle* h, int32_t phase, double* total_ms,
                                   int64_t* count) {
    if (!h || phase < 0 || phase >= EMS_NPHASE) { set_error("bad handle or phase"); return EMSURF_EINVAL; }
    DeviceGuard dg(h->device);
    PhaseTimer& pt = h->prof[phase];
    double ms = 0.0;
    for (size_t i = 0; i < pt.used; i += 2) {
        float t = 0.0f;
        EMS_CUDA(cudaEventSynchronize(pt.ev[i + 1]));
        EMS_CUDA(cudaEventElapsedTime(&t, pt.ev[i], pt.ev[i + 1]));
        ms += t;
    }
    if (total_ms) *total_ms = ms;
    if (count) *count = (int64_t)(pt.used / 2);
    return EMSURF_OK;
}

EMSURF_API int emsurf_check(emsurf_handle* h) {
    if (!h) { set_error("NULL handle"); return EMSURF_EINVAL; }
    DeviceGuard dg(h->device);
    EMS_CUDA(cudaDeviceSynchronize());
    int flag = 0;
    EMS_CUDA(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        EMS_TRY(clear_wait_error(h));
        set_error("a bounded device wait expired (flag %d); results of the affected calls are invalid", flag);
        return EMSURF_ETIMEDOUT;
    }
    return EMSURF_OK;
}

EMSURF_API int emsurf_selftest_wait(emsurf_handle* h, int64_t limit, void* stream) {
    if (!h || limit < 1 || limit > (1LL << 22)) {
        set_error("emsurf_selftest_wait: NULL handle or limit outside [1, 2^22]");
        return EMSURF_EINVAL;
    }
    DeviceGuard dg(h->device);
    EMS_TRY(wait_selftest(h, (long long)limit, reinterpret_cast<cudaStream_t>(stream)));
    return grid_barrier_selftest(h, (long long)limit, reinterpret_cast<cudaStream_t>(stream));
}

EMSURF_API int emsurf_launch_count(const emsurf_handle* h, int64_t* launches) {
    if (!h || !launches) { set_error("NULL argument"); return EMSURF_EINVAL; }
    *launches = h->launches;
    return EMSURF_OK;
}

EMSURF_API void emsurf_destroy(emsurf_handle* h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    gmres_release(h);
    free_handle(h);
}

}  // extern "C"
