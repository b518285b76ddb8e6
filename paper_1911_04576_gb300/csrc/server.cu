// Solve server: continuous batching of whole lattice solves on one GPU.
//
// Not part of the paper (which solves one array at a time on a CPU); it
// serves many independent instances of Eq. final.  A request describes one
// lattice (box geometry, cell types, type map, plane waves); a worker builds
// everything on the device -- U_o (host setup), offset tables and
// macromodels (GPU), the FFT-domain operator, the excitation -- solves with
// GMRES and copies the currents back.  Up to max_active requests run at once,
// each on its own non-blocking CUDA stream and host thread, so their kernels
// overlap on the GPU.  Admission is first-fit by an upper estimate of a
// request's device memory against the server's budget: requests that arrive
// while others run are admitted as soon as a slot and enough memory are
// free; a request whose estimate exceeds the whole budget is refused at
// submit (EMSURF_EBUSY).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace emsurf {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    uint64_t ticket = 0;
    emsurf_request req{};
    std::vector<double> sides, khat, ehat;
    std::vector<int32_t> tmap;
    int64_t est = 0;
    int status = EMSURF_EAGAIN;
    int32_t n_unique = 0;
    std::vector<emsurf_solve_info> info;
    Clock::time_point t_submit, t_start, t_setup, t_end;
    bool done = false;
    int64_t peak_bytes = 0;
};

int64_t request_bytes(const emsurf_request& q) {
    const int64_t E = 18LL * q.n * q.n, K = 2 * E;
    const int64_t px = smallest_smooth_at_least(2 * q.nx - 1);
    const int64_t py = smallest_smooth_at_least(2 * q.ny - 1);
    const int64_t P = px * py, M = (int64_t)q.nx * q.ny, R = std::max(1, q.nrhs);
    const int64_t tables = 2LL * (2 * q.nx - 1) * (2 * q.ny - 1) * E * E * 16;
    const int64_t mm = (int64_t)q.n_types * K * K * 16;
    const int64_t b64 = 2LL * E * E * P * 16, b32 = 2LL * E * E * P * 8;
    int64_t op = 0;
    if (q.precision == EMSURF_FP64) op = b64 + mm;
    else if (q.precision == EMSURF_FP32) op = b32 + b64 + mm;          // FP64 spectrum is a temporary
    else op = b64 + b32 + mm + mm / 2;
    // FP32 hi/lo planes of the FP64 spectrum and macromodels (= their FP64 bytes)
    if (q.precision != EMSURF_FP32) op += b64 + P * 4LL * E * 8 + mm;
    // BF16x3 planes of the tensor-core path: spectrum (= b32) + X^ planes
    if (q.precision != EMSURF_FP64 && q.nrhs >= kTcMinRhs && E >= 64)
        op += b32 + P * 4LL * 32 * ((R + 31) / 32) * E * 4;
    const int64_t work = 2LL * P * R * K * 16 + 10LL * R * M * K * 16;
    int64_t krylov = (int64_t)(std::max(q.opts.restart, 1) + 8) * R * M * K * 16;
    int64_t pc = 0;
    if (q.precond_overlap > 0.0) {
        const int64_t nm = std::min<int64_t>(1100, 3 * K / 2);          // largest subdomain
        pc = M * nm * nm * 8 + 2 * M * nm * 4 + 50LL * E * E * 16;
        krylov += (int64_t)std::max(q.opts.restart, 1) * R * M * K * 16;   // Z_j of flexible GMRES
    }
    int64_t cell = 0;                  // slab macromodels: elimination buffers (interior <= ~450)
    if (q.slab_t > 0.0) cell = 2LL * q.n_types * (K + 450) * (K + 450) * 16 + q.n_types * 8LL * 400 * 400 * 16;
    return tables + mm + op + work + krylov + pc + cell + (768LL << 20);   // + tabulation scratch, slack
}

}  // namespace
}  // namespace emsurf

struct emsurf_server {
    int device = 0;
    int64_t budget = 0;
    int max_active = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<emsurf::Job>> queue;
    std::map<uint64_t, std::shared_ptr<emsurf::Job>> jobs;
    int64_t in_use = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
};

namespace emsurf {
namespace {

int run_job(emsurf_server* sv, Job& jb, cudaStream_t st) {
    const emsurf_request& q = jb.req;
    EMS_CUDA(cudaSetDevice(sv->device));
    const int E = 18 * q.n * q.n, K = 2 * E, M = q.nx * q.ny;
    std::vector<int32_t> idx((size_t)M * K);
    std::vector<int8_t> sgn((size_t)M * K);
    int32_t nu = 0;
    EMS_TRY(emsurf_setup_overlap(q.n, q.nx, q.ny, idx.data(), sgn.data(), &nu));
    jb.n_unique = nu;
    const size_t tab = (size_t)(2 * q.nx - 1) * (2 * q.ny - 1) * E * E;
    void *L = nullptr, *Kt = nullptr, *Z = nullptr, *V = nullptr, *X = nullptr;
    emsurf_handle* hd = nullptr;
    int s = EMSURF_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (s) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("server: device allocation of %zu bytes failed", bytes);
            s = EMSURF_ENOMEM;
        }
    };
    alloc(&L, tab * sizeof(double2));
    alloc(&Kt, tab * sizeof(double2));
    alloc(&Z, (size_t)q.n_types * K * K * sizeof(double2));
    // slab cells: box rows end at the slab top (junction with S_eq)
    std::vector<double> zl;
    if (!s && q.slab_t > 0.0) {
        zl.resize(q.n + 1);
        s = emsurf_setup_slab_zlevels(q.h, q.n, q.slab_t, zl.data());
    }
    const double* zp = zl.empty() ? nullptr : zl.data();
    if (!s) s = emsurf_tabulate_offsets(q.a, q.b, q.h, q.n, zp, q.nx, q.ny, q.k0,
                                        static_cast<emsurf_c128*>(L), static_cast<emsurf_c128*>(Kt), st);
    if (!s && zp)
        s = emsurf_macromodel_slab_patch(q.a, q.b, q.h, q.n, zp, q.n_types, jb.sides.data(), q.patch_n,
                                         q.ring_layers > 0 ? q.ring_layers : 3, q.slab_eps, q.k0,
                                         static_cast<emsurf_c128*>(Z), st);
    else if (!s)
        s = emsurf_macromodel_pec_patch(q.a, q.b, q.h, q.n, q.n_types, jb.sides.data(), q.patch_z,
                                        q.patch_n, q.k0, static_cast<emsurf_c128*>(Z), st);
    if (!s) {
        emsurf_problem p{};
        p.nx = q.nx;
        p.ny = q.ny;
        p.n_edges = E;
        p.n_types = q.n_types;
        p.n_unique = nu;
        p.max_rhs = q.nrhs;
        p.type_map = jb.tmap.data();
        p.macromodels = static_cast<const emsurf_c128*>(Z);
        p.offset_L = static_cast<const emsurf_c128*>(L);
        p.offset_K = static_cast<const emsurf_c128*>(Kt);
        p.coef[0] = {0.0, q.k0};
        p.coef[1] = {1.0, 0.0};
        p.coef[2] = {-1.0, 0.0};
        p.coef[3] = {0.0, q.k0};
        p.uo_index = idx.data();
        p.uo_sign = sgn.data();
        p.precision = q.precision;
        p.tables_on_device = 1;
        p.device = sv->device;
        p.stream = st;
        // many right-hand sides: FP32 products as tensor-core GEMMs
        p.tensor_cores = (q.precision != EMSURF_FP64 && q.nrhs >= kTcMinRhs) ? 1 : 0;
        std::vector<double> xy;
        if (q.precond_overlap > 0.0) {
            xy.resize((size_t)2 * nu);
            s = emsurf_setup_unknown_xy(q.a, q.b, q.h, q.n, q.nx, q.ny, idx.data(), nu, xy.data());
            p.unknown_xy = xy.data();
            p.cell_a = q.a;
            p.cell_b = q.b;
            p.precond_overlap = q.precond_overlap;
        }
        if (!s) s = emsurf_create(&p, &hd);
        // solves of several requests overlap on the device, so their Arnoldi
        // steps must not rely on every block of a launch being resident
        if (!s) hd->coop_ok = false;
    }
    cudaFree(L);
    cudaFree(Kt);
    cudaFree(Z);
    alloc(&V, (size_t)q.nrhs * nu * sizeof(double2));
    alloc(&X, (size_t)q.nrhs * nu * sizeof(double2));
    if (!s) s = emsurf_excitation(hd, q.a, q.b, q.h, q.n, zp, q.k0, q.nrhs, jb.khat.data(), jb.ehat.data(),
                                  static_cast<emsurf_c128*>(V), st);
    jb.t_setup = Clock::now();
    if (!s) {
        jb.info.assign(q.nrhs, emsurf_solve_info{});
        s = emsurf_solve(hd, static_cast<emsurf_c128*>(V), static_cast<emsurf_c128*>(X), q.nrhs, &q.opts,
                         jb.info.data(), st);
        if ((s == EMSURF_OK || s == EMSURF_ENOTCONV) && q.x_out) {
            if (cudaMemcpyAsync(q.x_out, X, (size_t)q.nrhs * nu * sizeof(double2), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                set_error("server: copy of the solution failed");
                s = EMSURF_ECUDA;
            }
        }
    }
    if (hd) {
        int64_t b = 0;
        emsurf_query(hd, nullptr, nullptr, &b);
        jb.peak_bytes = b;
        emsurf_destroy(hd);
    }
    cudaFree(V);
    cudaFree(X);
    return s;
}

void worker_main(emsurf_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Job> jb;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stopping && sv->queue.empty()) break;
                // first fit: the oldest queued request whose estimate fits now
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
                    if ((*it)->est <= sv->budget - sv->in_use) {
                        jb = *it;
                        sv->queue.erase(it);
                        break;
                    }
                if (jb) break;
                sv->cv_work.wait(lk);
            }
            if (!jb) break;
            sv->in_use += jb->est;
        }
        jb->t_start = Clock::now();
        const int s = run_job(sv, *jb, st);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            jb->t_end = Clock::now();
            jb->status = s;
            jb->done = true;
            sv->in_use -= jb->est;
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

void fill_result(const Job& jb, emsurf_result* out) {
    if (!out) return;
    *out = emsurf_result{};
    out->status = jb.status;
    out->n_unique = jb.n_unique;
    out->nrhs = jb.req.nrhs;
    if (!jb.info.empty()) {
        out->info = jb.info[0];
        for (const auto& i : jb.info) {
            out->info.rel_residual = std::max(out->info.rel_residual, i.rel_residual);
            out->info.converged = out->info.converged && i.converged;
        }
    }
    out->queue_ms = ms_between(jb.t_submit, jb.t_start);
    out->setup_ms = ms_between(jb.t_start, jb.t_setup);
    out->solve_ms = ms_between(jb.t_setup, jb.t_end);
    out->latency_ms = ms_between(jb.t_submit, jb.t_end);
    out->est_bytes = jb.est;
    out->handle_bytes = jb.peak_bytes;
}

}  // namespace
}  // namespace emsurf

using namespace emsurf;

extern "C" {

EMSURF_API int emsurf_request_bytes(const emsurf_request* req, int64_t* bytes) {
    if (!req || !bytes || req->n < 1 || req->nx < 1 || req->ny < 1 || req->nrhs < 1) {
        set_error("emsurf_request_bytes: bad request");
        return EMSURF_EINVAL;
    }
    *bytes = request_bytes(*req);
    return EMSURF_OK;
}

EMSURF_API int emsurf_server_create(const emsurf_server_opts* opts, emsurf_server** out) {
    if (!opts || !out || opts->max_active < 1 || opts->max_active > 64) {
        set_error("emsurf_server_create: need options with 1 <= max_active <= 64");
        return EMSURF_EINVAL;
    }
    *out = nullptr;
    EMS_CUDA(cudaSetDevice(opts->device));
    size_t free_b = 0, total_b = 0;
    EMS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    emsurf_server* sv = new emsurf_server();
    sv->device = opts->device;
    sv->budget = opts->device_mem_budget > 0 ? opts->device_mem_budget : (int64_t)free_b;
    sv->max_active = opts->max_active;
    for (int i = 0; i < sv->max_active; ++i) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return EMSURF_OK;
}

EMSURF_API int emsurf_submit(emsurf_server* sv, const emsurf_request* req, uint64_t* ticket) {
    if (!sv || !req || !ticket) { set_error("emsurf_submit: NULL argument"); return EMSURF_EINVAL; }
    const emsurf_request& q = *req;
    if (q.n < 1 || q.nx < 1 || q.ny < 1 || q.n_types < 1 || q.nrhs < 1 || q.nrhs > 64 || !q.patch_sides ||
        !q.type_map || !q.khat || !q.ehat || !(q.k0 > 0.0) ||
        (q.precision != EMSURF_FP64 && q.precision != EMSURF_FP32 && q.precision != EMSURF_MIXED) ||
        !(q.opts.rtol > 0.0) || q.opts.restart < 1 || q.opts.restart > 64 || q.opts.max_iters < 1) {
        set_error("emsurf_submit: invalid request");
        return EMSURF_EINVAL;
    }
    for (int m = 0; m < q.nx * q.ny; ++m)
        if (q.type_map[m] < 0 || q.type_map[m] >= q.n_types) {
            set_error("emsurf_submit: type_map[%d] out of range", m);
            return EMSURF_EINVAL;
        }
    auto jb = std::make_shared<Job>();
    jb->req = q;
    jb->est = request_bytes(q);
    if (jb->est > sv->budget) {
        set_error("emsurf_submit: request needs ~%lld bytes, the budget is %lld", (long long)jb->est,
                  (long long)sv->budget);
        return EMSURF_EBUSY;
    }
    jb->sides.assign(q.patch_sides, q.patch_sides + q.n_types);
    jb->tmap.assign(q.type_map, q.type_map + q.nx * q.ny);
    jb->khat.assign(q.khat, q.khat + 3 * q.nrhs);
    jb->ehat.assign(q.ehat, q.ehat + 3 * q.nrhs);
    jb->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) { set_error("emsurf_submit: server is stopping"); return EMSURF_EBUSY; }
        jb->ticket = sv->next_ticket++;
        sv->jobs[jb->ticket] = jb;
        sv->queue.push_back(jb);
        *ticket = jb->ticket;
    }
    sv->cv_work.notify_all();
    return EMSURF_OK;
}

EMSURF_API int emsurf_poll(emsurf_server* sv, uint64_t ticket, emsurf_result* out) {
    if (!sv) { set_error("emsurf_poll: NULL server"); return EMSURF_EINVAL; }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) { set_error("emsurf_poll: unknown ticket %llu", (unsigned long long)ticket); return EMSURF_EINVAL; }
    if (!it->second->done) return EMSURF_EAGAIN;
    fill_result(*it->second, out);
    sv->jobs.erase(it);
    return EMSURF_OK;
}

EMSURF_API int emsurf_wait(emsurf_server* sv, uint64_t ticket, int64_t timeout_ms, emsurf_result* out) {
    if (!sv) { set_error("emsurf_wait: NULL server"); return EMSURF_EINVAL; }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) { set_error("emsurf_wait: unknown ticket %llu", (unsigned long long)ticket); return EMSURF_EINVAL; }
    auto jb = it->second;
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(std::max<int64_t>(0, timeout_ms)),
                              [&] { return jb->done; })) {
        set_error("emsurf_wait: ticket %llu not done after %lld ms", (unsigned long long)ticket,
                  (long long)timeout_ms);
        return EMSURF_ETIMEDOUT;
    }
    fill_result(*jb, out);
    sv->jobs.erase(ticket);
    return EMSURF_OK;
}

EMSURF_API void emsurf_server_destroy(emsurf_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
}

}  // extern "C"
