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
 *     written; emsurf_last_error() gives a thread-local message;
 *   - a handle keeps per-handle device workspaces (FFT grids, split
 *     operands, Krylov basis, preconditioner buffers), so it serves one call
 *     at a time: calls on one handle from different host threads or streams
 *     must be serialised by the caller (different handles are independent).
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
    EMSURF_EBUSY = 7,       /* request can never be admitted                  */
    EMSURF_ECANCELED = 8    /* request withdrawn before it ran                */
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
 *               with no prime factor above 7 (EINVAL otherwise)
 *  max_rhs      largest nrhs later passed to matvec/solve (>= 1).  Handles
 *               holding the FP64 operator also keep its spectrum and the
 *               macromodels as FP32 hi/lo planes (same bytes) for the
 *               double-single FP64-accuracy kernels, when device_mem_budget
 *               leaves room.  Their operands are scaled by powers of two
 *               (the spectrum and the macromodels at create, each rhs of a
 *               product by its largest component) and the FP64 results
 *               scaled back, so FP32's exponent range limits only parts
 *               more than ~2^100 below the largest of their array (relative
 *               error per term a few 2^-48 of that largest).  The FP32
 *               operator (EMSURF_FP32, MIXED) stores complex64 values and
 *               needs table and macromodel entries inside FP32's range.
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
    void* stream;                /* CUDA stream for the setup work of
                                    emsurf_create (NULL = legacy default);
                                    create synchronises it before returning */
    /* Near-field preconditioner (Eq. final_precond), built when
     * precond_overlap > 0 and unknown_xy != NULL: restricted additive
     * Schwarz over cell subdomains, subdomain m = unknowns whose RWG edge
     * midpoint lies in cell m's footprint (cell_a x cell_b, centred at
     * (ix*cell_a, iy*cell_b)) grown by precond_overlap metres.  unknown_xy:
     * host [n_unique][2] edge-midpoint x, y of each unique unknown
     * (emsurf_setup_unknown_xy).  At most 1100 unknowns per subdomain.      */
    const double* unknown_xy;
    double cell_a, cell_b;
    double precond_overlap;
    /* 1: also keep BF16x3 split planes of the FP32 operator (same bytes as
     * its complex64 spectrum) and run FP32 products with nrhs >= 8 as
     * tensor-core GEMMs per bin (tcgen05, FP32 accumulation; relative error
     * per product term <= 3 * 2^-18 instead of 2^-24).  Needs an FP32
     * operator (EMSURF_FP32 or EMSURF_MIXED) and E >= 64; ignored otherwise. */
    int32_t tensor_cores;
    /* Mirror symmetries of the box (emsurf_setup_box_mirrors), optional:
     * sym_mask bits 0 (x -> -x), 1 (y -> -y), 2 (x <-> y); sym_perm [3][E],
     * sym_sign [3][E] host (NULL with sym_mask 0).  With bits 0 and 1, a
     * MIXED handle with max_rhs 1 and no tensor cores keeps the FP32 blocks
     * of one bin per orbit {(+-kx, +-ky)} (with bit 2 on a square lattice and
     * grid also (+-ky, +-kx)), about a quarter (an eighth) of the bins, and
     * reads each once per product for every bin of its orbit.  The mirror
     * relations are checked on the FP64 blocks at create (to 1e-12 of their
     * largest entry); where they do not hold the handle keeps half of the
     * bins (reciprocity) as without mirrors.  No counterpart in the paper.  */
    int32_t sym_mask;
    const int32_t* sym_perm;
    const int8_t* sym_sign;
    /* 1: store the preconditioner's owned inverse rows as 8-bit integers
     * with one FP32 scale per row (absolute error <= 1/254 of the row's
     * largest component per entry, half the bytes of the FP16 rows) for
     * handles with max_rhs <= 2 and subdomains of up to 1024 unknowns;
     * 0 (or otherwise): FP16 rows.  No counterpart in the paper.           */
    int32_t precond_int8;
} emsurf_problem;

typedef struct {
    double rtol;          /* stop on ||b - A x|| / ||b|| <= rtol               */
    int32_t restart;      /* GMRES restart length m (1..64)                    */
    int32_t max_iters;    /* total inner iterations across restarts/refines    */
    int32_t max_refine;   /* MIXED only: outer FP64 refinement steps           */
    double inner_rtol;    /* MIXED only: floor of the inner FP32 solve tolerance,
                             which is max(floor, 0.5 rtol / current residual)
                             (0 = 1e-6; 3e-5 on the tensor-core operator)     */
    int32_t solver;       /* 0: by handle precision; 1: FP64-operator GMRES;
                             2: FP32-operator GMRES; 3: mixed refinement.
                             The operators it needs must be resident.         */
    int32_t precond;      /* 0: right-precondition with the handle's near-field
                             preconditioner if it was built; -1: do not      */
    double max_ms;        /* wall-time limit (ms, 0 = none), checked at every
                             GMRES restart and refinement: past it the solve
                             stops as if max_iters were spent (ENOTCONV,
                             x = best iterate)                                */
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

/* emsurf_create for a lattice whose Fourier-domain blocks another handle
 * already holds (no counterpart in the paper; used by the serving cache):
 * the new handle reads `share`'s spectra (FP64 or its double-single planes,
 * FP32, tensor-core planes) instead of building its own, and builds only
 * what depends on the problem's macromodels and type map (macromodel
 * copies, work space, preconditioner).  offset_L/offset_K are not read
 * (may be NULL); nx, ny, n_edges, precision, device and the grid must match
 * `share`; a share that keeps part of the FP32 spectrum (single rhs, no
 * tensor cores) serves only such problems, and tensor cores need a share
 * that has their planes.  `share` must outlive the new handle and must not
 * be destroyed first; the two may run calls at the same time (the shared
 * blocks are only read).  Errors: as emsurf_create, EINVAL on a mismatch. */
EMSURF_API int emsurf_create_like(const emsurf_problem* problem, const emsurf_handle* share,
                                  emsurf_handle** out);

/* y = U_o^T [Z_eq + Z_o] U_o x  (Eq. MVP) for nrhs right-hand sides.
 * x, y: device [nrhs][n_unique] complex128; must not overlap.
 * precision: EMSURF_FP64 or EMSURF_FP32 (the operator must be resident).
 * Errors: EINVAL (nrhs outside 1..max_rhs, null pointers, operator absent). */
EMSURF_API int emsurf_matvec(emsurf_handle* h, const emsurf_c128* x, emsurf_c128* y,
                             int32_t nrhs, int32_t precision, void* stream);

/* Solve Eq. final for nrhs right-hand sides b with restarted GMRES on the
 * device (Sec. IV-A; zero initial guess, classical Gram-Schmidt with a
 * second pass when ||w'|| < ||w|| / sqrt 10, Givens rotations; FP64 Krylov
 * vectors, FP32 ones inside the MIXED refinement).  x: device output.
 * info: host array [nrhs] or NULL.  Returns ENOTCONV (x = best iterate) if
 * any right-hand side did not reach rtol within max_iters.  With one rhs
 * each Arnoldi step is one cooperative launch whose blocks wait for each
 * other (bounded): solves of other handles running at the same time on the
 * device can make those waits expire, which returns ETIMEDOUT instead of
 * hanging; the server (emsurf_submit) runs its solves without it.        */
EMSURF_API int emsurf_solve(emsurf_handle* h, const emsurf_c128* b, emsurf_c128* x,
                            int32_t nrhs, const emsurf_solve_opts* opts,
                            emsurf_solve_info* info, void* stream);

/* y = M^{-1} r with the handle's near-field preconditioner (restricted
 * additive Schwarz over cells, the grouping of Eq. final_precond's near
 * field used here): y = sum_m Rt_m^T A_m^{-1} R_m r, A_m the exact block of
 * Eq. final on subdomain m, factored in complex FP32; its owned rows of
 * A_m^{-1} are applied from FP16 copies scaled per row (relative error per
 * entry <= 2^-11), or as BF16x3 tensor-core GEMMs for >= 8 rhs.  r, y: device
 * [nrhs][n_unique] complex128, must not overlap; nrhs <= max_rhs.
 * Errors: EINVAL (no preconditioner built, bad nrhs or pointers).        */
EMSURF_API int emsurf_precond_apply(emsurf_handle* h, const emsurf_c128* r, emsurf_c128* y,
                                    int32_t nrhs, void* stream);

/* Sizes of the near-field preconditioner: stored entries of the owned rows
 * of the subdomain inverses (complex FP16 pairs, 4 bytes each, plus one FP32
 * scale per row), sum of n_m, and the largest n_m; all 0 if none.        */
EMSURF_API int emsurf_precond_info(const emsurf_handle* h, int64_t* factor_entries,
                                   int64_t* subdomain_total, int32_t* max_subdomain);

/* FP32 operator layout: spectrum bins it stores (grid_px * grid_py; for a
 * single-rhs handle one bin per mirror orbit, about a quarter or an eighth
 * of that, when sym_mask gave the box's mirrors, else about half when the
 * tables are reciprocal: one bin of each pair (k, -k), Sec. IV-B with
 * L(-d) = L(d)^T) and whether the tensor-core planes were built (1) or not
 * (0).                                                                    */
EMSURF_API int emsurf_operator_info(const emsurf_handle* h, int32_t* stored_bins, int32_t* tensor_cores);

/* Form of the FP32 spectrum: 0 every bin, 1 one bin per pair (k, -k)
 * (reciprocity), 2 one bin per mirror orbit; bins_per_stored: the most bins
 * one stored bin serves (1, 2, or the mirror group's order 4 or 8).       */
EMSURF_API int emsurf_operator_layout(const emsurf_handle* h, int32_t* form, int32_t* bins_per_stored);

/* Ring shape of the tensor-core bin multiply chosen at create by timing
 * both shapes on the handle's spectrum (the library's own autotuner; no
 * counterpart in the paper): sources per pipeline stage (32 or 64), stages
 * (5 or 2), and the two shapes' times in ms ([0]: 32 x 5, [1]: 64 x 2);
 * all zero for a handle without tensor-core planes.                       */
EMSURF_API int emsurf_tc_tuning(const emsurf_handle* h, int32_t* sources_per_stage, int32_t* stages,
                                double* ms_shapes);

/* Grid chosen by emsurf_create, unknown count and bytes of device memory
 * held by the handle.                                                     */
EMSURF_API int emsurf_query(const emsurf_handle* h, int32_t* grid_px, int32_t* grid_py,
                            int64_t* device_bytes);

EMSURF_API void emsurf_destroy(emsurf_handle* h);

/* Tracing (no counterpart in the paper, which reports wall-clock phases
 * only): CUDA-event timers around each phase of emsurf_matvec, recorded on
 * the caller's stream while enabled.  enable != 0 clears and starts
 * recording; 0 stops.  Phases: 0 bin multiply FP32, 1 bin multiply FP64,
 * 2 macromodel multiply FP32, 3 macromodel FP64, 4 FFT passes + gather FP32,
 * 5 the same FP64, 6 Arnoldi orthogonalisation/norm/Givens kernels of
 * emsurf_solve, 7 crop + U_o^T scatter of emsurf_matvec, 8 near-field
 * preconditioner applications of emsurf_solve.  emsurf_profile_read synchronises on the recorded events
 * and returns the summed milliseconds and the number of intervals.       */
EMSURF_API int emsurf_profile(emsurf_handle* h, int32_t enable);
/* As emsurf_profile(h, 1) but recording only the phases whose bit is set in
 * phase_mask (bit i = phase i; 0 stops): fewer events on the stream when
 * one kernel is timed inside a longer run.                                */
EMSURF_API int emsurf_profile_phases(emsurf_handle* h, uint32_t phase_mask);
EMSURF_API int emsurf_profile_read(emsurf_handle* h, int32_t phase, double* total_ms,
                                   int64_t* count);

/* Synchronise the handle's device and report whether any bounded device
 * wait of this handle's kernels expired since the last check
 * (EMSURF_ETIMEDOUT, flag cleared) -- the kernels give up instead of
 * hanging, so the context stays usable.  emsurf_solve does the same check
 * before it returns.                                                      */
EMSURF_API int emsurf_check(emsurf_handle* h);

/* Self-test of the bounded-wait paths (no counterpart in the paper): one
 * kernel waits on an mbarrier that nothing arrives on, another at a grid
 * barrier for a block that is never launched, each at most `limit` polls
 * (1..2^22); on expiry they set the handle's error flag exactly as the bin
 * multiply's and the cooperative Arnoldi step's waits do.  The next
 * emsurf_check returns ETIMEDOUT and clears the flag and the barrier
 * state.  Nothing faults or hangs.                                        */
EMSURF_API int emsurf_selftest_wait(emsurf_handle* h, int64_t limit, void* stream);

/* Number of CUDA kernels this handle has launched since creation.        */
EMSURF_API int emsurf_launch_count(const emsurf_handle* h, int64_t* launches);

/* ------------------------------------------------------------------------
 * Setup helpers (host).  Canonical meshes and the overlap map, by integer
 * index arithmetic.  Output arrays are caller-allocated host arrays sized by
 * the *_counts calls; nothing is written on EINVAL.
 *
 * Box S_eq of cell (0,0) (Sec. II-A): x in [-a/2,a/2], y in [-b/2,b/2],
 * z in [0,h], n x n quads per face, opposite faces identical (translates).
 * Vertices: surface grid points (i,j,k) in lexicographic order; faces
 * x-,x+,y-,y+,z-,z+ with in-plane axes (j,k),(i,k),(i,j); quad (u,v) is
 * cut, for even n, along the diagonal pointing at the face centre:
 * triangles (c00,c10,c11),(c00,c11,c01) when (2u+1 < n) == (2v+1 < n),
 * else (c00,c10,c01),(c10,c11,c01); for odd n always the first way;
 * index face*2n^2 + 2(v*n+u) + {0,1}.
 * RWG edges (Eqs. Hdiscretebox/Ediscretebox): distinct vertex pairs sorted
 * lexicographically; T+ = lower triangle; slot i of a triangle = edge
 * opposite vertex i; slot_rwg = RWG index (-1 if none), slot_sgn = +1 on T+.
 * zlevels: optional [n+1] z of the grid rows (NULL = uniform).
 *   verts [V][3], tris [T][3], edges [E][2], tplus/tminus [E],
 *   slot_rwg [T][3], slot_sgn [T][3].                                      */
EMSURF_API int emsurf_setup_box_counts(int32_t n, int32_t* n_verts, int32_t* n_tris,
                                       int32_t* n_edges);
EMSURF_API int emsurf_setup_box_mesh(double a, double b, double h, int32_t n,
                                     const double* zlevels, double* verts, int32_t* tris,
                                     int32_t* edges, int32_t* tplus, int32_t* tminus,
                                     int32_t* slot_rwg, int8_t* slot_sgn);

/* Mirror symmetries of the box mesh (no counterpart in the paper: they let
 * the FFT-domain blocks of mirrored bins share storage).  Mirror g (0:
 * x -> -x, 1: y -> -y, 2: x <-> y, the last only when a == b) maps RWG
 * function e of the box onto sign[g][e] * RWG perm[g][e]; bit g of *mask is
 * set when g maps the mesh onto itself (for n even all three; for n odd
 * only x <-> y).  perm [3][E], sign [3][E]
 * host, E = 18 n^2; entries of mirrors not in the mask are unspecified.
 * The offset tables then satisfy L(g d) = P_g L(d) P_g^T and
 * K(g d) = -P_g K(d) P_g^T (P_g e_e = sign[g][e] e_perm[g][e]); see
 * sym_mask in emsurf_problem.  Errors: EINVAL (n < 1, bad sides, NULL).   */
EMSURF_API int emsurf_setup_box_mirrors(double a, double b, int32_t n, int32_t* perm, int8_t* sign,
                                        int32_t* mask);

/* The host logic of the mirror-orbit spectrum (exposed for tests and
 * tools).  Group element e = bits (x mirror, y mirror, x <-> y applied
 * first) acts on bin (kx, ky) of a px x py grid as k -> (+-kx, +-ky) mod
 * the grid; n_elem is 4 (x and y mirrors) or 8 (with x <-> y; px == py).
 * emsurf_setup_mirror_orbits: the orbits, each represented by its smallest
 * bin index: *n_stored representatives rep[s] and n_elem slots each,
 * slot_bin[s][j] (-1 past the orbit's size) and slot_elem[s][j] with
 * slot_bin = e(rep); arrays of px*py (rep) and px*py*n_elem entries, or
 * NULL to get *n_stored only.
 * emsurf_setup_mirror_group: tperm[e][2E] = index | (sign < 0) << 31 of
 * T_e = diag(P_e, det(e) P_e), P_e = Px^a Py^b Pd^c composed from the
 * mirrors of emsurf_setup_box_mirrors (perm/sign [3][E]), det(e) =
 * (-1)^(a+b+c); the FFT-domain blocks obey B^(e k) = T_e B^(k) T_e^T.    */
EMSURF_API int emsurf_setup_mirror_orbits(int32_t px, int32_t py, int32_t n_elem, int32_t* n_stored,
                                          int32_t* rep, int32_t* slot_bin, int32_t* slot_elem);
EMSURF_API int emsurf_setup_mirror_group(int32_t n_edges, int32_t n_elem, const int32_t* perm, const int8_t* sign,
                                         uint32_t* tperm);

/* Flat square PEC patch (Sec. II-A: J only on PEC) of side `side` centred
 * on the cell axis at height z, n x n quads each cut along (c00,c11);
 * vertices (i,j) at index i*(n+1)+j; RWGs on interior edges only.         */
EMSURF_API int emsurf_setup_patch_counts(int32_t n, int32_t* n_verts, int32_t* n_tris,
                                         int32_t* n_edges);
EMSURF_API int emsurf_setup_patch_mesh(double side, double z, int32_t n, double* verts,
                                       int32_t* tris, int32_t* edges, int32_t* tplus,
                                       int32_t* tminus, int32_t* slot_rwg, int8_t* slot_sgn);

/* Row heights of a box whose bottom slab_t is a dielectric slab (the
 * configurations' cell; Sec. II-A asks the interface to meet S_eq on mesh
 * edges, the junction of Fig. composite): zlevels [n+1] = 0, slab_t, then
 * uniform up to h.  n >= 2, 0 < slab_t < h.                               */
EMSURF_API int emsurf_setup_slab_zlevels(double h, int32_t n, double slab_t, double* zlevels);

/* The slab-top interface of that cell at height z (Sec. II-A: all surfaces
 * inside S_eq meshed; the interface conforms to the box rows and the patch):
 * vertices = the patch grid (patch_n+1)^2 at index i*(patch_n+1)+j, then
 * ring_layers - 1 rings of 4 patch_n points on the rectangles of half-width
 * side/2 + (a/2 - side/2) (k/ring_layers)^2 (likewise in y), then the 4n
 * footprint boundary points (the box vertices of grid row 1), every ring
 * walked counter-clockwise from its (-,-) corner.  Triangles: the patch
 * quads (as emsurf_setup_patch_mesh), the ring bands, and a last band zipped
 * from each corner onto the footprint boundary.  side <= 0: no patch, the
 * n x n footprint grid (inner points i-major, then the boundary).  RWGs on
 * interior edges; on_patch [T] = 1 for patch triangles.                    */
EMSURF_API int emsurf_setup_slab_top_counts(double a, double b, int32_t n, double side,
                                            int32_t patch_n, int32_t ring_layers,
                                            int32_t* n_verts, int32_t* n_tris, int32_t* n_edges);
EMSURF_API int emsurf_setup_slab_top_mesh(double a, double b, double z, int32_t n, double side,
                                          int32_t patch_n, int32_t ring_layers, double* verts,
                                          int32_t* tris, int32_t* edges, int32_t* tplus,
                                          int32_t* tminus, int32_t* slot_rwg, int8_t* slot_sgn,
                                          int8_t* on_patch);

/* Sizes of that cell's interior system: unknowns eliminated by the Schur
 * complement (n_interior) and RWGs of the air and slab region surfaces
 * (region_edges[2]).                                                      */
EMSURF_API int emsurf_setup_slab_cell_counts(double a, double b, double h, int32_t n,
                                             const double* zlevels, double side, int32_t patch_n,
                                             int32_t ring_layers, int32_t* n_interior,
                                             int32_t* region_edges);

/* Edge-midpoint (x, y) of every unique unknown of an nx x ny lattice
 * (box of cell (ix,iy) centred at (ix*a, iy*b)), from the canonical box
 * mesh and the overlap map: xy host [n_unique][2].                        */
EMSURF_API int emsurf_setup_unknown_xy(double a, double b, double h, int32_t n, int32_t nx,
                                       int32_t ny, const int32_t* uo_index, int32_t n_unique,
                                       double* xy);

/* U_o of Eq. connections_IUI (Sec. III-D, rule 1 with Delta -> 0 of
 * Fig. connections) for an nx x ny lattice of boxes meshed n x n per face:
 * RWGs of different boxes whose edges coincide and that share a coincident
 * triangle are one unique unknown, signed so the coincident halves cancel
 * (J^(m) = -J^(m') on a shared face).  Unique unknowns are numbered by first
 * appearance over (cell m = iy*nx+ix, local k).  uo_index/uo_sign:
 * [nx*ny*36n^2] host outputs; n_unique: out.                              */
EMSURF_API int emsurf_setup_overlap(int32_t n, int32_t nx, int32_t ny, int32_t* uo_index,
                                    int8_t* uo_sign, int32_t* n_unique);

/* ------------------------------------------------------------------------
 * Operator tabulation on the device (setup of Eq. out / Eq. blockZo).
 *   L[b][m][n] = int int [Lam_m.Lam_n - div Lam_m div' Lam_n / k^2] G
 *   K[b][m][n] = int int Lam_m(r) . [grad_r G(r,r') x Lam_n(r')]   (p.v.)
 * with G = e^{-jkR}/(4 pi R) (Eqs. SIE_LOperator1, SIE_KOperator1), test
 * mesh translated by shifts[b] relative to the source mesh.  7-point
 * degree-5 rule on both triangles; for singular[b] != 0 the 1/R and
 * grad(1/R) parts are integrated over the source triangle in closed form.
 * Meshes are host arrays as produced by the setup helpers; L, K are device
 * [n_blocks][test_E][src_E] complex128.  Synchronises `stream`.           */
EMSURF_API int emsurf_tabulate(const double* test_verts, const int32_t* test_tris,
                               const int32_t* test_slot_rwg, const int8_t* test_slot_sgn,
                               int32_t test_T, int32_t test_E, const double* src_verts,
                               const int32_t* src_tris, const int32_t* src_slot_rwg,
                               const int8_t* src_slot_sgn, int32_t src_T, int32_t src_E,
                               const double* shifts, const int8_t* singular, int32_t n_blocks,
                               double k, emsurf_c128* L, emsurf_c128* K, void* stream);

/* emsurf_tabulate for callers that must not allocate device memory.  The
 * paper has no counterpart; this exists for hosts that cannot call
 * cudaMalloc at this point -- for example a plugin inside another
 * application's memory pool, a process under a fixed device-memory quota,
 * or code running while its host holds an allocator lock.  Same arguments,
 * same results as emsurf_tabulate; the caller still provides L and K.  It
 * makes no cudaMalloc/cudaFree or other allocating call: its scratch is one
 * static 64 MiB device array per GPU, which every GPU that loads the library
 * keeps until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture.  Meshes whose per-block
 * triangle-pair scratch (test_T * src_T * 288 bytes) plus geometry exceeds
 * the array are rejected with EMSURF_EINVAL and a message giving the bytes
 * needed.  All calls share the array and it keeps the previous call's
 * contents (every value is written before it is read, so nothing is
 * cleared); calls that overlap on the GPU -- from two host threads or two
 * streams -- race on it and must be serialised by the caller.  Synchronises
 * `stream`.                                                               */
EMSURF_API int emsurf_tabulate_noalloc(const double* test_verts, const int32_t* test_tris,
                                       const int32_t* test_slot_rwg, const int8_t* test_slot_sgn,
                                       int32_t test_T, int32_t test_E, const double* src_verts,
                                       const int32_t* src_tris, const int32_t* src_slot_rwg,
                                       const int8_t* src_slot_sgn, int32_t src_T, int32_t src_E,
                                       const double* shifts, const int8_t* singular,
                                       int32_t n_blocks, double k, emsurf_c128* L, emsurf_c128* K,
                                       void* stream);

/* Offset tables of an nx x ny lattice of boxes (period a, b; height h; n x n
 * per face, rows at zlevels or uniform if NULL): L, K device [2ny-1][2nx-1][E][E] indexed [dy+ny-1][dx+nx-1],
 * d = test cell - source cell; closed-form singular parts for touching
 * boxes (|dx|, |dy| <= 1).  The tables are the reciprocal part of the
 * one-sided blocks of emsurf_tabulate, T(d) = (T1(d) + T1(-d)^T) / 2, so
 * L(-d) = L(d)^T and K(-d) = K(d)^T hold exactly (the one-sided closed-form
 * integration breaks them at touching offsets).  The layout emsurf_create
 * takes; with reciprocal tables it stores half of the FP32 spectrum.      */
EMSURF_API int emsurf_tabulate_offsets(double a, double b, double h, int32_t n,
                                       const double* zlevels, int32_t nx, int32_t ny, double k,
                                       emsurf_c128* L, emsurf_c128* K, void* stream);

/* Macromodels Z~ of Eq. Zmacromodel of the patch-on-slab cell (Secs. II-A..D
 * with two interior regions): a dielectric slab of relative permittivity
 * eps_slab (lossy: Im < 0 under e^{jwt}) fills the bottom of the box up to
 * the first row boundary zlevels[1] of the side faces, a flat PEC square
 * patch of side sides[t] (patch_n x patch_n quads; sides[t] <= 0: slab
 * only) lies centred on the slab top, air above.  Box rows at zlevels
 * ([n+1], zlevels[0] = 0, zlevels[n] = h; see emsurf_setup_slab_zlevels).
 * The slab top is meshed by emsurf_setup_slab_top_mesh (ring_layers graded
 * rings around the patch).  Per region v the tested block
 * [[jk0 L_v, K_v], [-K_v, jk0 eps_v L_v]] with k_v = k0 sqrt(eps_v)
 * (Eq. ch5_macromodel_composite_SIE_Block); U (Eq. incidence1) joins them by
 * the rules of Sec. II-C: interface (J, M shared, rule 1), PEC at the
 * interface (one J per side, rule 2), PEC-dielectric junction (J shared,
 * rule 3), and the junction of the interface with S_eq (label 2 of
 * Fig. composite); Z~ is the Schur complement of U^T Z U (Eq. mmm_mult)
 * on the interior unknowns.  Z: device [n_types][K][K] complex128.  EINVAL
 * for n < 2, a patch that does not fit inside the footprint, Re eps <= 0 or
 * Im eps > 0, or a singular interior block.  Synchronises `stream`.       */
EMSURF_API int emsurf_macromodel_slab_patch(double a, double b, double h, int32_t n,
                                            const double* zlevels, int32_t n_types,
                                            const double* sides, int32_t patch_n,
                                            int32_t ring_layers, emsurf_c128 eps_slab, double k0,
                                            emsurf_c128* Z, void* stream);

/* Macromodels Z~ of Eq. Zmacromodel for cells holding one flat PEC square
 * patch of side sides[t] (centred, height patch_z, patch_n x patch_n quads)
 * in a free-space box: Schur complement of the patch unknowns of the
 * interior system [[jk L_ee, K_ee, jk L_ep], [-K_ee, jk L_ee, -K_ep],
 * [jk L_pe, K_pe, jk L_pp]] (Secs. II-B..D).  sides[t] <= 0: empty box.
 * Z: device [n_types][K][K] complex128.  EINVAL if a patch does not fit
 * strictly inside the box or has more than 100 RWGs.                      */
EMSURF_API int emsurf_macromodel_pec_patch(double a, double b, double h, int32_t n,
                                           int32_t n_types, const double* sides, double patch_z,
                                           int32_t patch_n, double k, emsurf_c128* Z,
                                           void* stream);

/* Excitation V~ = U_o^T V of Eq. final for nrhs plane waves
 * E_inc = ehat e^{-jk khat.r} (|E_inc| = 1 V/m): rows J test E_inc, rows M
 * test eta0 H_inc = (khat x ehat) e^{..} (Eq. out).  khat, ehat: host
 * [nrhs][3] unit vectors; V: device [nrhs][n_unique].  The box geometry
 * (a, b, h, n, zlevels: row heights or NULL for uniform) must be the one
 * the handle's tables were built for.                                     */
EMSURF_API int emsurf_excitation(emsurf_handle* h, double a, double b, double hgt, int32_t n,
                                 const double* zlevels, double k, int32_t nrhs, const double* khat,
                                 const double* ehat, emsurf_c128* V, void* stream);

/* Far field radiated by solved currents Y~ (device [nrhs][n_unique]) in
 * ndir directions rhat (host [ndir][3] unit vectors): F (device
 * [nrhs][ndir][3]) with E ~ F e^{-jkr}/r, and optionally the bistatic RCS
 * sigma = 4 pi |F|^2 (device [nrhs][ndir], m^2; NULL to skip).  Box
 * geometry as for emsurf_excitation.  The sum over cells of the lattice
 * phases runs in FP64 for FP64 handles and in FP32 for FP32 / MIXED handles
 * (relative error ~1e-6 of the largest term: negligible in dB wherever
 * sigma lies within ~60 dB of its maximum); the per-box radiation integrals
 * are FP64.                                                               */
EMSURF_API int emsurf_far_field(emsurf_handle* h, double a, double b, double hgt, int32_t n,
                                const double* zlevels, double k, const emsurf_c128* Y,
                                int32_t nrhs, int32_t ndir, const double* rhat, emsurf_c128* F,
                                double* rcs, void* stream);

/* ------------------------------------------------------------------------
 * Serving (no counterpart in the paper, which solves one array at a time):
 * continuous batching of whole lattice solves.  A request describes one
 * lattice; a server worker builds it on the device (U_o, offset tables,
 * macromodels, FFT-domain operator, excitation) -- or takes the resident
 * blocks of an earlier request of the same lattice and cell library --
 * solves Eq. final and copies the currents to x_out.  Requests with nrhs >= 8 and an FP32 operator use
 * the tensor-core bin multiply (see tensor_cores in emsurf_problem).  Up to
 * max_active requests run at once, each on its
 * own non-blocking stream; a queued request is admitted (first fit) when a
 * slot is free and its device-memory estimate (emsurf_request_bytes) fits
 * in what the budget has left.                                            */
typedef struct emsurf_server emsurf_server;

typedef struct {
    int32_t device;
    int64_t device_mem_budget;   /* bytes admitted at once; 0 = free memory   */
    int32_t max_active;          /* concurrent solves, 1..64                  */
    int32_t no_cache;            /* 1: build every request from scratch; 0:
                                    keep each lattice's Fourier-domain blocks
                                    and each cell library's macromodels
                                    resident (within the budget, least
                                    recently used evicted first) and build
                                    later requests of the same lattice with
                                    emsurf_create_like                        */
} emsurf_server_opts;

typedef struct {
    double a, b, h;              /* cell period x, y and box height (m)       */
    int32_t n;                   /* box faces meshed n x n (K = 36 n^2)       */
    int32_t nx, ny;              /* lattice                                   */
    double k0;                   /* free-space wavenumber (1/m)               */
    int32_t n_types;
    const double* patch_sides;   /* [n_types] PEC patch side (m), <= 0 empty  */
    double patch_z;              /* patch height (m)                          */
    int32_t patch_n;             /* patch mesh patch_n x patch_n              */
    const int32_t* type_map;     /* [ny*nx] cell -> type                      */
    int32_t nrhs;                /* plane waves, 1..64                        */
    const double* khat;          /* [nrhs][3] propagation directions          */
    const double* ehat;          /* [nrhs][3] polarisations                   */
    int32_t precision;           /* EMSURF_FP64 / FP32 / MIXED                */
    emsurf_solve_opts opts;
    emsurf_c128* x_out;          /* host [nrhs][n_unique] or NULL; must stay
                                    valid until the result is collected       */
    double precond_overlap;      /* near-field preconditioner margin (m),
                                    <= 0: none                                */
    double slab_t;               /* > 0: patch-on-slab cells (slab thickness,
                                    m; the patch lies on the slab top and
                                    patch_z is ignored); 0: free-space cells  */
    emsurf_c128 slab_eps;        /* slab relative permittivity (Im <= 0)      */
    int32_t ring_layers;         /* slab-top rings around the patch (0 = 3)   */
} emsurf_request;

typedef struct {
    int32_t status;              /* status of the solve (OK, ENOTCONV, ...)   */
    int32_t n_unique, nrhs;
    emsurf_solve_info info;      /* worst residual / all-converged over rhs   */
    double queue_ms;             /* submit -> admitted                        */
    double setup_ms;             /* tables, macromodels, operator, excitation */
    double solve_ms;             /* GMRES and the copy of x                   */
    double latency_ms;           /* submit -> done                            */
    int64_t est_bytes;           /* admission estimate                        */
    int64_t handle_bytes;        /* device bytes the solve handle held        */
    int32_t cache_hit;           /* 1: the lattice's blocks were resident     */
} emsurf_result;

EMSURF_API int emsurf_server_create(const emsurf_server_opts* opts, emsurf_server** out);
/* Admission estimate of a request in bytes of device memory.              */
EMSURF_API int emsurf_request_bytes(const emsurf_request* req, int64_t* bytes);
/* Queue a request (its small arrays are copied; x_out is not).  EBUSY if
 * its estimate exceeds the whole budget or the server is stopping.        */
EMSURF_API int emsurf_submit(emsurf_server* s, const emsurf_request* req, uint64_t* ticket);
/* EAGAIN while queued or running; OK with the result once done (the ticket
 * is then forgotten); EINVAL for an unknown ticket.                       */
EMSURF_API int emsurf_poll(emsurf_server* s, uint64_t ticket, emsurf_result* out);
/* As poll, but blocks up to timeout_ms; ETIMEDOUT if not done by then.    */
EMSURF_API int emsurf_wait(emsurf_server* s, uint64_t ticket, int64_t timeout_ms,
                           emsurf_result* out);
/* Where a request is: queued, admitted, building (or waiting for another
 * request to build) the cell library or the lattice's operator, solving,
 * done.  EINVAL for an unknown (or already collected) ticket.            */
enum {
    EMSURF_PHASE_QUEUED = 0,
    EMSURF_PHASE_ADMITTED = 1,
    EMSURF_PHASE_LIBRARY = 2,
    EMSURF_PHASE_WAIT_LIBRARY = 3,
    EMSURF_PHASE_WAIT_OPERATOR = 4,
    EMSURF_PHASE_OPERATOR = 5,
    EMSURF_PHASE_SOLVE = 6,
    EMSURF_PHASE_DONE = 7
};
EMSURF_API int emsurf_request_phase(emsurf_server* s, uint64_t ticket, int32_t* phase);
/* Withdraws a request that is still queued (not yet admitted): OK, and its
 * result (collected by poll/wait) has status ECANCELED; EBUSY once it runs
 * (its opts.max_ms bounds it); EINVAL for an unknown ticket.             */
EMSURF_API int emsurf_cancel(emsurf_server* s, uint64_t ticket);
/* Stops accepting requests, finishes the queued and running ones, frees
 * them and the resident blocks.                                           */
EMSURF_API void emsurf_server_destroy(emsurf_server* s);
/* Resident cache: device bytes held, cached lattices (operators), cached
 * cell libraries, entries evicted so far.                                 */
EMSURF_API int emsurf_server_stats(emsurf_server* s, int64_t* cached_bytes, int32_t* operators,
                                   int32_t* libraries, int64_t* evictions);

/* Thread-local message of the last failing call on this thread.          */
EMSURF_API const char* emsurf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EMSURF_H */
