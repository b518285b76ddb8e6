// Solve server: continuous batching of whole lattice solves on one GPU.
//
// Not part of the paper (which solves one array at a time on a CPU); it
// serves many independent instances of Eq. final.  A request describes one
// lattice (box geometry, cell types, type map, plane waves); a worker builds
// what it needs on the device -- U_o (host setup), offset tables and
// macromodels (GPU), the FFT-domain operator, the excitation -- solves with
// GMRES and copies the currents back.  Up to max_active requests run at once,
// each on its own non-blocking CUDA stream and host thread, so their kernels
// overlap on the GPU.
//
// Resident operators.  The Fourier-domain blocks depend only on the box
// geometry, the lattice size, the wavenumber and the precision (not on the
// type map), and the macromodels only on the cell library: both are cached.
// The first request of a lattice builds a full handle and leaves it in the
// cache; later requests of that lattice build a light handle that reads its
// blocks (emsurf_create_like: macromodel copies, work space and
// preconditioner only).  Macromodel libraries are cached across lattice
// sizes.  Cached entries count against the budget and are evicted, least
// recently used first, when an admitted request needs the room.
//
// Admission is first-fit by an upper estimate of a request's device memory
// (the whole build on a cache miss, the request's own part on a hit) against
// what the budget has left; a request that cannot fit even in an empty
// server is refused at submit (EMSURF_EBUSY).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <cstdio>
#include <list>
#include <map>
#include <memory>
#include <string>
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
    std::string op_key, mm_key;
    bool hit = false;              // the operator was cached when admitted
    bool op_build = false;         // this job builds the operator's cache entry
    bool mm_build = false;         // ... and the library's
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
    int64_t new_bytes = 0;         // cache entries this job created
    std::atomic<int> phase{0};     // EMSURF_PHASE_* (emsurf_request_phase)
};

// the cache keys: the operator's (geometry, lattice, wavenumber, precision,
// spectrum form) and the macromodel library's (geometry, cell library)
int spectrum_form(const emsurf_request& q) {
    const int E = 18 * q.n * q.n;
    if (q.precision == EMSURF_FP64) return 0;
    if (q.nrhs >= kTcMinRhs && E >= 64) return 3;      // tensor-core planes
    return q.nrhs == 1 ? 1 : 2;                          // part (pairs or mirror orbits) / full FP32 spectrum
}

std::string cell_key(const emsurf_request& q) {
    char b[256];
    std::snprintf(b, sizeof(b), "%.17g|%.17g|%.17g|%d|%.17g|%.17g|%.17g|%.17g|%d|%d|%.17g", q.a, q.b, q.h, q.n,
                  q.slab_t, q.slab_eps.re, q.slab_eps.im, q.slab_t > 0.0 ? 0.0 : q.patch_z, q.patch_n,
                  q.ring_layers, q.k0);
    return b;
}

std::string operator_key(const emsurf_request& q) {
    char b[96];
    std::snprintf(b, sizeof(b), "|%d|%d|%d|%d", q.nx, q.ny, q.precision, spectrum_form(q));
    std::string k = cell_key(q) + b;
    // the slab's permittivity and the patches do not enter the blocks, the rows do
    return k;
}

std::string library_key(const emsurf_request& q) {
    std::string k = cell_key(q);
    char b[32];
    for (int t = 0; t < q.n_types; ++t) {
        std::snprintf(b, sizeof(b), "|%.17g", q.patch_sides[t]);
        k += b;
    }
    return k;
}

// device bytes of the blocks a full handle keeps (what the cache holds)
int64_t operator_bytes(const emsurf_request& q) {
    const int64_t E = 18LL * q.n * q.n;
    const int64_t P = (int64_t)smallest_smooth_at_least(2 * q.nx - 1) * smallest_smooth_at_least(2 * q.ny - 1);
    const int64_t b64 = 2LL * E * E * P * 16, b32 = 2LL * E * E * P * 8;
    int64_t op = b64;                                   // FP64 spectrum or its hi/lo planes
    if (q.precision != EMSURF_FP64) op += spectrum_form(q) == 1 ? b32 / 2 : b32;
    if (spectrum_form(q) == 3) op += b32;               // tensor-core planes
    return op + 50LL * E * E * 16;                      // + near tables
}

// Upper estimate of a request's device memory, by part: offset tables (a
// build-time temporary), the blocks a full handle keeps (operator_bytes), the
// handle's own macromodel copies, work grids, Krylov basis, preconditioner,
// the macromodel library (input array and, for slab cells, its build
// scratch) and slack.
struct Estimate {
    int64_t tables = 0, blocks = 0, own = 0, library = 0, slack = 0;
    int64_t full() const { return tables + blocks + own + library + slack; }
    int64_t shared(bool library_cached) const { return own + (library_cached ? 0 : library) + slack; }
};

Estimate estimate(const emsurf_request& q) {
    Estimate e;
    const int64_t E = 18LL * q.n * q.n, K = 2 * E;
    const int64_t px = smallest_smooth_at_least(2 * q.nx - 1);
    const int64_t py = smallest_smooth_at_least(2 * q.ny - 1);
    const int64_t P = px * py, M = (int64_t)q.nx * q.ny, R = std::max(1, q.nrhs);
    e.tables = 2LL * (2 * q.nx - 1) * (2 * q.ny - 1) * E * E * 16;
    const int64_t mm = (int64_t)q.n_types * K * K * 16;
    const int64_t b64 = 2LL * E * E * P * 16;
    // during create the FP64 spectrum and its hi/lo planes coexist before the
    // spectrum is given back
    e.blocks = operator_bytes(q) + b64;
    // macromodel copies: FP64 (+ its hi/lo planes), FP32 (MIXED / FP32), bf16 planes
    e.own = mm * (q.precision == EMSURF_FP32 ? 1 : 2) + (q.precision == EMSURF_MIXED ? mm / 2 : 0);
    if (spectrum_form(q) == 3) e.own += mm / 2 + P * 4LL * 32 * ((R + 31) / 32) * E * 4;
    const int64_t work = 2LL * P * R * K * 16 + 10LL * R * M * K * 16;
    int64_t krylov = (int64_t)(std::max(q.opts.restart, 1) + 8) * R * M * K * 16;
    int64_t pc = 0;
    if (q.precond_overlap > 0.0) {
        const int64_t nm = std::min<int64_t>(1100, 3 * K / 2);          // largest subdomain
        pc = M * nm * nm * 8 + 2 * M * nm * 4;
        krylov += (int64_t)std::max(q.opts.restart, 1) * R * M * K * 16;   // Z_j of flexible GMRES
    }
    e.own += work + krylov + pc;
    e.library = mm;
    if (q.slab_t > 0.0) e.library += 2LL * q.n_types * (K + 450) * (K + 450) * 16 + q.n_types * 8LL * 400 * 400 * 16;
    e.slack = 768LL << 20;                              // tabulation scratch, allocator slack
    return e;
}

int64_t request_bytes(const emsurf_request& q) { return estimate(q).full(); }

}  // namespace
}  // namespace emsurf

namespace emsurf {
namespace {
struct OpEntry {                   // a full handle whose blocks later requests read
    emsurf_handle* h = nullptr;
    int64_t bytes = 0;
    int refs = 0;                  // jobs using it now
    bool ready = false;            // built (else being built by a job)
    uint64_t last_use = 0;
};
struct MmEntry {                   // device macromodels [T][K][K] of a cell library
    void* Z = nullptr;
    int64_t bytes = 0;
    int refs = 0;
    bool ready = false;
    uint64_t last_use = 0;
};
}  // namespace
}  // namespace emsurf

struct emsurf_server {
    int device = 0;
    int64_t budget = 0;
    int max_active = 1;
    bool cache_on = true;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_cache;
    std::map<std::string, emsurf::OpEntry> ops;
    std::map<std::string, emsurf::MmEntry> mms;
    uint64_t use_clock = 0;
    int64_t cached_bytes = 0;      // part of in_use held by idle and busy cache entries
    int64_t evictions = 0;
    std::deque<std::shared_ptr<emsurf::Job>> queue;
    std::map<uint64_t, std::shared_ptr<emsurf::Job>> jobs;
    int64_t in_use = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
};

namespace emsurf {
namespace {

// Builds the macromodels of the request's cell library into a new device
// array (a cache entry or the job's own).
int build_library(const emsurf_request& q, const Job& jb, const double* zp, void** Zout, cudaStream_t st) {
    const int K = 36 * q.n * q.n;
    const size_t bytes = (size_t)q.n_types * K * K * sizeof(double2);
    void* Z = nullptr;
    if (cudaMalloc(&Z, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("server: device allocation of %zu bytes failed", bytes);
        return EMSURF_ENOMEM;
    }
    int s;
    if (zp)
        s = emsurf_macromodel_slab_patch(q.a, q.b, q.h, q.n, zp, q.n_types, jb.sides.data(), q.patch_n,
                                         q.ring_layers > 0 ? q.ring_layers : 3, q.slab_eps, q.k0,
                                         static_cast<emsurf_c128*>(Z), st);
    else
        s = emsurf_macromodel_pec_patch(q.a, q.b, q.h, q.n, q.n_types, jb.sides.data(), q.patch_z, q.patch_n,
                                        q.k0, static_cast<emsurf_c128*>(Z), st);
    if (s) {
        cudaFree(Z);
        return s;
    }
    *Zout = Z;
    return EMSURF_OK;
}

// The cache entry `key` of map m once its builder has published it, or
// nullptr if the build failed (the entry was dropped).  The caller holds a
// reference taken at admission.  Called with the lock held.
template <typename Entry>
Entry* wait_entry(emsurf_server* sv, std::map<std::string, Entry>& m, const std::string& key,
                  std::unique_lock<std::mutex>& lk) {
    for (;;) {
        auto it = m.find(key);
        if (it == m.end()) return nullptr;
        if (it->second.ready) {
            it->second.last_use = ++sv->use_clock;
            return &it->second;
        }
        sv->cv_cache.wait(lk);       // another job is building it
    }
}

int run_job(emsurf_server* sv, Job& jb, cudaStream_t st) {
    const emsurf_request& q = jb.req;
    // no early return below: the cache entries this job was admitted to
    // build must be published or dropped, or the jobs waiting on them would
    // wait for ever
    int s = EMSURF_OK;
    if (cudaSetDevice(sv->device) != cudaSuccess) {
        cudaGetLastError();
        set_error("server: cudaSetDevice failed");
        s = EMSURF_ECUDA;
    }
    const int E = 18 * q.n * q.n, K = 2 * E, M = q.nx * q.ny;
    std::vector<int32_t> idx((size_t)M * K);
    std::vector<int8_t> sgn((size_t)M * K);
    int32_t nu = 0;
    if (!s) s = emsurf_setup_overlap(q.n, q.nx, q.ny, idx.data(), sgn.data(), &nu);
    jb.n_unique = nu;
    // slab cells: box rows end at the slab top (junction with S_eq)
    std::vector<double> zl;
    if (!s && q.slab_t > 0.0) {
        zl.resize(q.n + 1);
        s = emsurf_setup_slab_zlevels(q.h, q.n, q.slab_t, zl.data());
    }
    const double* zp = zl.empty() ? nullptr : zl.data();
    // ---- macromodel library (cached across lattices)
    void* Z = nullptr;
    MmEntry* me = nullptr;
    if (sv->cache_on) {
        if (jb.mm_build) {
            jb.phase = EMSURF_PHASE_LIBRARY;
            if (!s) s = build_library(q, jb, zp, &Z, st);
            std::lock_guard<std::mutex> lk(sv->mu);
            me = &sv->mms[jb.mm_key];
            if (s) {
                sv->mms.erase(jb.mm_key);
                me = nullptr;
            } else {
                me->Z = Z;
                me->bytes = (int64_t)q.n_types * K * K * 16;
                me->ready = true;
                me->last_use = ++sv->use_clock;
                jb.new_bytes += me->bytes;
            }
            sv->cv_cache.notify_all();
        } else {
            jb.phase = EMSURF_PHASE_WAIT_LIBRARY;
            std::unique_lock<std::mutex> lk(sv->mu);
            me = wait_entry(sv, sv->mms, jb.mm_key, lk);
            if (me) Z = me->Z;
            else if (!s) {
                set_error("server: the cell library's macromodels could not be built");
                s = EMSURF_ECUDA;
            }
        }
    } else if (!s) {
        jb.phase = EMSURF_PHASE_LIBRARY;
        s = build_library(q, jb, zp, &Z, st);
    }
    // ---- the operator: a cached full handle, or a new one
    emsurf_handle* base = nullptr;     // cached handle whose blocks are read
    emsurf_handle* hd = nullptr;       // the handle this job solves with
    OpEntry* oe = nullptr;
    const bool build_op = !sv->cache_on || jb.op_build;
    if (sv->cache_on) {
        std::unique_lock<std::mutex> lk(sv->mu);
        if (jb.op_build) {
            oe = &sv->ops[jb.op_key];
        } else {
            jb.phase = EMSURF_PHASE_WAIT_OPERATOR;
            oe = wait_entry(sv, sv->ops, jb.op_key, lk);
            if (oe) base = oe->h;
            else if (!s) {
                set_error("server: the lattice's operator could not be built");
                s = EMSURF_ECUDA;
            }
        }
    }
    emsurf_problem p{};
    std::vector<double> xy;
    std::vector<int32_t> mperm((size_t)3 * E);
    std::vector<int8_t> msign((size_t)3 * E);
    if (!s) {
        p.nx = q.nx;
        p.ny = q.ny;
        p.n_edges = E;
        p.n_types = q.n_types;
        p.n_unique = nu;
        p.max_rhs = q.nrhs;
        p.type_map = jb.tmap.data();
        p.macromodels = static_cast<const emsurf_c128*>(Z);
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
        p.tensor_cores = spectrum_form(q) == 3 ? 1 : 0;
        // the box's mirrors (one stored bin per orbit for single-rhs FP32 products)
        int32_t mask = 0;
        s = emsurf_setup_box_mirrors(q.a, q.b, q.n, mperm.data(), msign.data(), &mask);
        p.sym_mask = mask;
        p.sym_perm = mperm.data();
        p.sym_sign = msign.data();
        if (q.precond_overlap > 0.0) {
            xy.resize((size_t)2 * nu);
            s = emsurf_setup_unknown_xy(q.a, q.b, q.h, q.n, q.nx, q.ny, idx.data(), nu, xy.data());
            p.unknown_xy = xy.data();
            p.cell_a = q.a;
            p.cell_b = q.b;
            p.precond_overlap = q.precond_overlap;
        }
    }
    jb.phase = EMSURF_PHASE_OPERATOR;
    if (!s && base) {
        s = emsurf_create_like(&p, base, &hd);
    } else if (!s) {
        const size_t tab = (size_t)(2 * q.nx - 1) * (2 * q.ny - 1) * E * E;
        void *L = nullptr, *Kt = nullptr;
        if (cudaMalloc(&L, tab * sizeof(double2)) != cudaSuccess || cudaMalloc(&Kt, tab * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            set_error("server: device allocation of the offset tables failed");
            s = EMSURF_ENOMEM;
        }
        if (!s) s = emsurf_tabulate_offsets(q.a, q.b, q.h, q.n, zp, q.nx, q.ny, q.k0,
                                            static_cast<emsurf_c128*>(L), static_cast<emsurf_c128*>(Kt), st);
        p.offset_L = static_cast<const emsurf_c128*>(L);
        p.offset_K = static_cast<const emsurf_c128*>(Kt);
        if (!s) s = emsurf_create(&p, &hd);
        cudaFree(L);
        cudaFree(Kt);
    }
    // solves of several requests overlap on the device, so their Arnoldi
    // steps must not rely on every block of a launch being resident
    if (!s) hd->coop_ok = false;
    if (oe && build_op) {
        // publish the new full handle (or drop the entry if it failed)
        std::lock_guard<std::mutex> lk(sv->mu);
        if (s || !hd) {
            sv->ops.erase(jb.op_key);
            oe = nullptr;
        } else {
            int64_t b = 0;
            emsurf_query(hd, nullptr, nullptr, &b);
            oe->h = hd;
            oe->bytes = b;
            oe->ready = true;
            oe->last_use = ++sv->use_clock;
            jb.new_bytes += b;
        }
        sv->cv_cache.notify_all();
    }
    void *V = nullptr, *X = nullptr;
    if (!s && (cudaMalloc(&V, (size_t)q.nrhs * nu * sizeof(double2)) != cudaSuccess ||
               cudaMalloc(&X, (size_t)q.nrhs * nu * sizeof(double2)) != cudaSuccess)) {
        cudaGetLastError();
        set_error("server: device allocation of the rhs failed");
        s = EMSURF_ENOMEM;
    }
    if (!s) s = emsurf_excitation(hd, q.a, q.b, q.h, q.n, zp, q.k0, q.nrhs, jb.khat.data(), jb.ehat.data(),
                                  static_cast<emsurf_c128*>(V), st);
    jb.t_setup = Clock::now();
    jb.phase = EMSURF_PHASE_SOLVE;
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
    }
    cudaFree(V);
    cudaFree(X);
    // a cached full handle stays (with the solve's work space: its bytes are
    // counted again); a light handle or an uncached one goes
    const bool keep_hd = oe && build_op && hd && hd == oe->h;
    if (keep_hd) {
        std::lock_guard<std::mutex> lk(sv->mu);
        jb.new_bytes += jb.peak_bytes - oe->bytes;
        oe->bytes = jb.peak_bytes;
    }
    if (hd && !keep_hd) emsurf_destroy(hd);
    if (!sv->cache_on && Z) cudaFree(Z);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (oe) oe->refs -= 1;
        if (me) me->refs -= 1;
    }
    sv->cv_work.notify_all();        // idle entries may make room for queued requests
    return s;
}

// Evicts idle cache entries, least recently used first, until `need` bytes
// fit in the budget; returns whether they do.  Called with the lock held.
bool make_room(emsurf_server* sv, int64_t need) {
    while (sv->in_use + need > sv->budget) {
        uint64_t best = UINT64_MAX;
        int kind = -1;
        std::string key;
        for (auto& kv : sv->ops)
            if (kv.second.ready && kv.second.refs == 0 && kv.second.last_use < best) {
                best = kv.second.last_use;
                kind = 0;
                key = kv.first;
            }
        for (auto& kv : sv->mms)
            if (kv.second.ready && kv.second.refs == 0 && kv.second.last_use < best) {
                best = kv.second.last_use;
                kind = 1;
                key = kv.first;
            }
        if (kind < 0) return false;
        if (kind == 0) {
            OpEntry& e = sv->ops[key];
            emsurf_destroy(e.h);
            sv->in_use -= e.bytes;
            sv->cached_bytes -= e.bytes;
            sv->ops.erase(key);
        } else {
            MmEntry& e = sv->mms[key];
            cudaFree(e.Z);
            sv->in_use -= e.bytes;
            sv->cached_bytes -= e.bytes;
            sv->mms.erase(key);
        }
        sv->evictions += 1;
    }
    return true;
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
                // (after evicting idle cache entries if needed)
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                    Job& j = **it;
                    const Estimate e = estimate(j.req);
                    const bool op_c = sv->cache_on && sv->ops.count(j.op_key);
                    const bool mm_c = sv->cache_on && sv->mms.count(j.mm_key);
                    const int64_t need = op_c ? e.shared(mm_c) : e.full() - (mm_c ? e.library : 0);
                    // the entries this job would reuse stay pinned while room
                    // is made: evicting one of them here would leave the job
                    // waiting for an entry that nobody builds
                    OpEntry* pin_op = op_c ? &sv->ops[j.op_key] : nullptr;
                    MmEntry* pin_mm = mm_c ? &sv->mms[j.mm_key] : nullptr;
                    if (pin_op) pin_op->refs += 1;
                    if (pin_mm) pin_mm->refs += 1;
                    const bool room = make_room(sv, need);
                    if (pin_op) pin_op->refs -= 1;
                    if (pin_mm) pin_mm->refs -= 1;
                    if (room) {
                        j.est = need;
                        j.hit = op_c;
                        if (sv->cache_on) {
                            // references (or the build) are taken now, so no
                            // eviction can remove what this job counts on
                            OpEntry& oe = sv->ops[j.op_key];
                            oe.refs += 1;
                            j.op_build = !op_c;
                            MmEntry& me = sv->mms[j.mm_key];
                            me.refs += 1;
                            j.mm_build = !mm_c;
                        }
                        jb = *it;
                        jb->phase = EMSURF_PHASE_ADMITTED;
                        sv->queue.erase(it);
                        break;
                    }
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
            // the reservation goes; entries this job added to the cache stay
            sv->in_use += jb->new_bytes - jb->est;
            sv->cached_bytes += jb->new_bytes;
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
    out->cache_hit = jb.hit ? 1 : 0;
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
    sv->cache_on = opts->no_cache == 0;
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
        !(q.opts.rtol > 0.0) || q.opts.restart < 1 || q.opts.restart > 64 || q.opts.max_iters < 1 ||
        !(q.opts.max_ms >= 0.0)) {
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
    jb->op_key = operator_key(q);
    jb->mm_key = library_key(q);
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

EMSURF_API int emsurf_request_phase(emsurf_server* sv, uint64_t ticket, int32_t* phase) {
    if (!sv || !phase) { set_error("emsurf_request_phase: NULL argument"); return EMSURF_EINVAL; }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) {
        set_error("emsurf_request_phase: unknown ticket %llu", (unsigned long long)ticket);
        return EMSURF_EINVAL;
    }
    *phase = it->second->done ? EMSURF_PHASE_DONE : it->second->phase.load();
    return EMSURF_OK;
}

EMSURF_API int emsurf_cancel(emsurf_server* sv, uint64_t ticket) {
    if (!sv) { set_error("emsurf_cancel: NULL server"); return EMSURF_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(ticket);
        if (it == sv->jobs.end()) {
            set_error("emsurf_cancel: unknown ticket %llu", (unsigned long long)ticket);
            return EMSURF_EINVAL;
        }
        auto q = std::find(sv->queue.begin(), sv->queue.end(), it->second);
        if (q == sv->queue.end()) {
            set_error("emsurf_cancel: ticket %llu is no longer queued", (unsigned long long)ticket);
            return EMSURF_EBUSY;
        }
        Job& jb = *it->second;
        sv->queue.erase(q);
        jb.t_start = jb.t_setup = jb.t_end = Clock::now();
        jb.status = EMSURF_ECANCELED;
        jb.done = true;
    }
    sv->cv_done.notify_all();
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
    cudaSetDevice(sv->device);
    for (auto& kv : sv->ops)
        if (kv.second.h) emsurf_destroy(kv.second.h);
    for (auto& kv : sv->mms)
        if (kv.second.Z) cudaFree(kv.second.Z);
    delete sv;
}

EMSURF_API int emsurf_server_stats(emsurf_server* sv, int64_t* cached_bytes, int32_t* operators,
                                   int32_t* libraries, int64_t* evictions) {
    if (!sv) { set_error("emsurf_server_stats: NULL server"); return EMSURF_EINVAL; }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (cached_bytes) *cached_bytes = sv->cached_bytes;
    if (operators) *operators = (int32_t)sv->ops.size();
    if (libraries) *libraries = (int32_t)sv->mms.size();
    if (evictions) *evictions = sv->evictions;
    return EMSURF_OK;
}

}  // extern "C"
