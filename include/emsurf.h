/*
 * emsurf -- C ABI of the FFT-accelerated macromodel solver for inhomogeneous
 * electromagnetic surfaces (Patel, Triverio, Hum).
 *
 * The library solves Eq. final,  U_o^T [Z_eq + Z_o] U_o Y~ = U_o^T V,
 * for the equivalent currents on the box surfaces S_eq^(m) of an Nx x Ny
 * lattice of unit cells (Sec. III), with matrix-vector products done by the
 * circulant-embedded FFT of Sec. IV-B generalised to 2-D lattices.
 *
 * Conventions shared by every entry point
 *   - complex numbers are interleaved (re, im) doubles (emsurf_c128);
 *   - E = n_edges RWG functions per box; K = 2E local unknowns per box,
 *     ordered (J_1..J_E, M_1..M_E) with x_J = eta0*J and x_M = M;
 *   - cells are numbered m = iy*nx + ix;
 *   - lattice offsets d = (dx, dy) = test cell - source cell;
 *   - vectors of unique unknowns are [nrhs][n_unique] complex128 DEVICE
 *     arrays on the handle's device, owned by the caller;
 *   - calls are ordered on the given CUDA stream (NULL = legacy default);
 *     emsurf_solve synchronises that stream before it returns;
 *   - every call returns an emsurf_status; on EMSURF_EINVAL no output is
 *     written; emsurf_last_error() gives a thread-local message.
 */
#ifndef EMSURF_H
#define EMSURF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMSURF_API __attribute__((visibility("default")))

typedef struct { double re, im; } emsurf_c128;

typedef enum {
    EMSURF_OK = 0,
    EMSURF_EINVAL = 1,      /* bad argument; nothing written                  */
    EMSURF_ENOMEM = 2,      /* device or host allocation failed / over budget */
    EMSURF_ECUDA = 3,       /* a CUDA call failed                             */
    EMSURF_ENOTCONV = 4,    /* solver hit max_iters; best iterate written     */
    EMSURF_EAGAIN = 5,      /* request still pending                          */
    EMSURF_ETIMEDOUT = 6,   /* a bounded wait ran out                         */
    EMSURF_EBUSY = 7        /* request can never be admitted                  */
} emsurf_status;

/* Storage/arithmetic of the Fourier-domain blocks and macromodels.
 * FP64: complex128 storage and FP64 arithmetic.
 * FP32: complex64 storage, FP32 arithmetic (FFTs, bin multiply, macromodel).
 * MIXED: both operators resident; emsurf_solve runs FP32 inner GMRES with
 *        FP64 residual refinement.                                         */
typedef enum { EMSURF_FP64 = 0, EMSURF_FP32 = 1, EMSURF_MIXED = 2 } emsurf_precision;

typedef struct emsurf_handle emsurf_handle;

/* Problem statement of Eq. final (Sec. III-D).
 *  type_map     [ny*nx] cell -> macromodel type in [0, n_types)       (host)
 *  macromodels  [n_types][K][K] Z~_eq,eq of Eq. Zmacromodel, row-major
 *  offset_L/K   [2ny-1][2nx-1][E][E] Galerkin L(d), K(d) between a test box
 *               at offset d and the source box (Eqs. out, blockZo), index
 *               [dy+ny-1][dx+nx-1][test RWG][source RWG]
 *  coef         (a, b, g, d): B(d) = [[a L(d), b K(d)], [g K(d), d L(d)]]
 *  uo_index     [nx*ny*K] unique unknown of local unknown (m, k), in
 *               [0, n_unique)  (U_o of Eq. connections_IUI)           (host)
 *  uo_sign      [nx*ny*K] +1 / -1                                      (host)
 *  grid_px/py   FFT grid; 0 = smallest 2,3,5-smooth >= 2N-1; else >= 2N-1
 *  max_rhs      largest nrhs later passed to matvec/solve (>= 1)
 *  tables_on_device  0: offset_L/K and macromodels are host pointers;
 *                    1: they are device pointers on `device`
 * The handle copies everything it needs; the caller may free the inputs
 * after emsurf_create returns.                                            */
typedef struct {
    int32_t nx, ny;
    int32_t n_edges;
    int32_t n_types;
    int32_t n_unique;
    int32_t max_rhs;
    const int32_t* type_map;
    const emsurf_c128* macromodels;
    const emsurf_c128* offset_L;
    const emsurf_c128* offset_K;
    emsurf_c128 coef[4];
    const int32_t* uo_index;
    const int8_t* uo_sign;
    int32_t grid_px, grid_py;
    int32_t precision;
    int32_t tables_on_device;
    int64_t device_mem_budget;   /* bytes; 0 = no limit; ENOMEM if exceeded */
    int32_t device;
} emsurf_problem;

typedef struct {
    double rtol;          /* stop on ||b - A x|| / ||b|| <= rtol               */
    int32_t restart;      /* GMRES restart length m (1..64)                    */
    int32_t max_iters;    /* total inner iterations across restarts/refines    */
    int32_t max_refine;   /* MIXED only: outer FP64 refinement steps           */
    double inner_rtol;    /* MIXED only: inner FP32 solve tolerance (0 = 1e-4) */
} emsurf_solve_opts;

typedef struct {
    int32_t iters;        /* inner GMRES iterations (Arnoldi steps)            */
    int32_t refinements;  /* FP64 residual refinements (MIXED)                 */
    int32_t n_matvec;     /* operator applications                             */
    int32_t converged;    /* 1 if rel_residual <= rtol                          */
    double rel_residual;  /* true ||b - A x|| / ||b|| in FP64 at return         */
    double ms_total;      /* wall time of the call                             */
} emsurf_solve_info;

/* Build the FFT-domain operator (Sec. IV-B, Eqs. LJV3-LJV5 with the
 * circulant's first column as generator, generalised to 2-D, Sec. IV-B last
 * paragraph) and all device state.  Allocates device memory owned by the
 * handle.  Errors: EINVAL (shape/index/sign out of range), ENOMEM, ECUDA.  */
EMSURF_API int emsurf_create(const emsurf_problem* problem, emsurf_handle** out);

/* y = U_o^T [Z_eq + Z_o] U_o x  (Eq. MVP) for nrhs right-hand sides.
 * x, y: device [nrhs][n_unique] complex128; must not overlap.
 * precision: EMSURF_FP64 or EMSURF_FP32 (the operator must be resident).
 * Errors: EINVAL (nrhs outside 1..max_rhs, null pointers, operator absent). */
EMSURF_API int emsurf_matvec(emsurf_handle* h, const emsurf_c128* x, emsurf_c128* y,
                             int32_t nrhs, int32_t precision, void* stream);

/* Solve Eq. final for nrhs right-hand sides b with restarted GMRES on the
 * device (Sec. IV-A; zero initial guess, classical Gram-Schmidt applied
 * twice, Givens rotations, FP64 Krylov vectors).  x: device output.
 * info: host array [nrhs] or NULL.  Returns ENOTCONV (x = best iterate) if
 * any right-hand side did not reach rtol within max_iters.              */
EMSURF_API int emsurf_solve(emsurf_handle* h, const emsurf_c128* b, emsurf_c128* x,
                            int32_t nrhs, const emsurf_solve_opts* opts,
                            emsurf_solve_info* info, void* stream);

/* Grid chosen by emsurf_create, unknown count and bytes of device memory
 * held by the handle.                                                     */
EMSURF_API int emsurf_query(const emsurf_handle* h, int32_t* grid_px, int32_t* grid_py,
                            int64_t* device_bytes);

EMSURF_API void emsurf_destroy(emsurf_handle* h);

/* Thread-local message of the last failing call on this thread.          */
EMSURF_API const char* emsurf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EMSURF_H */
