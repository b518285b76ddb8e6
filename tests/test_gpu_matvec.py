"""GPU parity of the FFT matvec (Eq. MVP via Sec. IV-B) against the oracle's
direct offset sum, through the C ABI.

Tolerances: FP64 path rel-L2 <= 1e-10 per product (the accuracy target of
the FP64 plain path).  FP32 path: complex64 storage and FP32 arithmetic give
per-product errors ~ sqrt(number of terms) * 2^-24 * (condition of the
sums), about 1e-6 here for E up to 288 and random phases; 3e-5 rel-L2 bounds
it with margin on these inputs.
"""
import numpy as np
import pytest

from oracle import lattice
from oracle.mesh import box_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.PERIOD
H = W.BOX_H
COEF = (1j * W.K0, 1.0, -1.0, 1j * W.K0)
TOL64 = 1e-10
TOL32 = 3e-5


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def random_case(n, nx, ny, T, seed):
    box = box_mesh(A, A, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, seed)
    Z = W.random_macromodels(T, 2 * E, seed + 1)
    tmap = np.random.default_rng(seed + 2).integers(0, T, nx * ny).astype(np.int32)
    return E, idx, sgn, nu, Lt, Kt, Z, tmap


def run_matvec(B, h, x, prec):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, prec)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("n,nx,ny,R", [(1, 1, 1, 1), (2, 2, 2, 1), (2, 3, 5, 2), (2, 4, 4, 3),
                                       (3, 3, 3, 1), (2, 5, 1, 4), (1, 7, 6, 5)])
def test_matvec_parity_random_tables(emsurf_lib, n, nx, ny, R):
    from paper_1911_04576_gb300 import binding as B
    seed = 100 * n + 10 * nx + ny
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 3, seed)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED,
                        max_rhs=max(R, 2))
    x = W.random_vectors(R, nu, seed + 3)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    y64 = run_matvec(B, h, x, B.FP64)
    y32 = run_matvec(B, h, x, B.FP32)
    for r in range(R):
        assert relerr(y64[r], yref[r]) <= TOL64
        assert relerr(y32[r], yref[r]) <= TOL32
    B.emsurf_check(h)
    h.close()


def test_grid_size_does_not_change_result(emsurf_lib):
    """Any grid >= 2N-1 embeds the Toeplitz blocks exactly: 2N-1 (the paper's
    5x5 circulant for N = 3), the 2,3,5-smooth default and 2N agree."""
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 3, 4
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 2, 77)
    x = W.random_vectors(1, nu, 78)
    ys = []
    for grid in [(0, 0), (2 * nx - 1, 2 * ny - 1), (2 * nx, 2 * ny), (10, 9)]:
        h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, grid=grid)
        assert B.emsurf_query(h)[:2] == ((5, 8) if grid == (0, 0) else grid)
        ys.append(run_matvec(B, h, x, B.FP64))
        h.close()
    for y in ys[1:]:
        assert relerr(y, ys[0]) <= 1e-13


def test_matvec_full_size_sampled(emsurf_lib):
    """16x16 lattice, K = 576, 32 types, one rhs: the bench's launch
    configuration; 32 sampled outputs recomputed one by one by the oracle."""
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = W.random_tables(w.nx, w.ny, w.E, 1600)
    Z = W.random_macromodels(w.n_types, w.K, 1601)
    tmap = W.type_map(w)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED)
    x = W.random_vectors(1, nu, 1602)
    rows = np.sort(np.random.default_rng(1603).choice(nu, 32, replace=False))
    rows[0], rows[-1] = 0, nu - 1
    yref = lattice.matvec_direct_rows(x[0], rows, Lt, Kt, COEF, Z, tmap, idx, sgn, w.nx, w.ny)
    y64 = run_matvec(B, h, x, B.FP64)[0]
    y32 = run_matvec(B, h, x, B.FP32)[0]
    assert relerr(y64[rows], yref) <= TOL64
    assert relerr(y32[rows], yref) <= TOL32
    # repeated calls are bit-identical (no atomics, fixed reduction order)
    assert np.array_equal(run_matvec(B, h, x, B.FP64)[0], y64)
    assert np.array_equal(run_matvec(B, h, x, B.FP32)[0], y32)
    B.emsurf_check(h)          # no bounded device wait expired
    h.close()
    # the same workload with reciprocal tables: half of the FP32 spectrum
    # (514 of 1024 bins), bins straddling the pair kernel's CTA ranges
    Lt, Kt = reciprocal(Lt), reciprocal(Kt)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED)
    assert B.emsurf_operator_info(h) == (514, False)
    yref = lattice.matvec_direct_rows(x[0], rows, Lt, Kt, COEF, Z, tmap, idx, sgn, w.nx, w.ny)
    y32 = run_matvec(B, h, x, B.FP32)[0]
    assert relerr(y32[rows], yref) <= TOL32
    assert relerr(run_matvec(B, h, x, B.FP64)[0][rows], yref) <= TOL64
    # deterministic: the partial row sums are added in a fixed order
    assert np.array_equal(run_matvec(B, h, x, B.FP32)[0], y32)
    B.emsurf_check(h)
    h.close()


def test_invalid_calls_rejected(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(1, 2, 2, 1, 5)
    h = B.emsurf_create(2, 2, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.FP64, max_rhs=2)
    x = torch.zeros(3, nu, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_matvec(h, x, y, B.FP64)           # nrhs 3 > max_rhs 2
    assert e.value.status == B.EMSURF_EINVAL
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_matvec(h, x[:1], y[:1], B.FP32)   # FP32 operator not resident
    assert e.value.status == B.EMSURF_EINVAL
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_matvec(h, x[:1], x[:1], B.FP64)   # in place
    assert e.value.status == B.EMSURF_EINVAL
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_create(2, 2, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, device_mem_budget=1024)
    assert e.value.status == B.EMSURF_ENOMEM
    h.close()


def test_bounded_wait_expiry_is_reported(emsurf_lib):
    """Device waits that nothing satisfies (an mbarrier wait and a grid
    barrier) give up after their limit, the host reads ETIMEDOUT once, and
    the context stays usable (the product afterwards is still exact, a solve
    afterwards runs)."""
    from paper_1911_04576_gb300 import binding as B
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(2, 3, 2, 2, 77)
    h = B.emsurf_create(3, 2, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED)
    B.emsurf_check(h)
    B.emsurf_selftest_wait(h, 2000)
    with pytest.raises(B.EmsurfError) as ei:
        B.emsurf_check(h)
    assert ei.value.status == B.EMSURF_ETIMEDOUT
    B.emsurf_check(h)                       # the flag was cleared
    x = W.random_vectors(1, nu, 78)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, 3, 2)
    assert relerr(run_matvec(B, h, x, B.FP32)[0], yref[0]) <= TOL32
    B.emsurf_check(h)
    with pytest.raises(B.EmsurfError):
        B.emsurf_selftest_wait(h, 0)        # limit outside [1, 2^22]
    # the grid barrier of the cooperative Arnoldi step was reset with the
    # flag: a solve afterwards runs its steps to the end without expiry
    import torch
    b = torch.from_numpy(W.random_vectors(1, nu, 79)).cuda()
    st, info = B.emsurf_solve(h, b, torch.zeros_like(b), rtol=1e-10, restart=8, max_iters=16, max_refine=2)
    assert st in (B.EMSURF_OK, B.EMSURF_ENOTCONV) and info[0]["iters"] > 0
    B.emsurf_check(h)
    h.close()


def reciprocal(T):
    """Reciprocal part of a table: T(d) <- (T(d) + T(-d)^T) / 2."""
    return 0.5 * (T + np.swapaxes(T[::-1, ::-1], 2, 3))


@pytest.mark.parametrize("n,nx,ny,grid", [(2, 3, 2, (0, 0)), (2, 4, 4, (8, 8)), (3, 2, 3, (0, 0)),
                                          (2, 5, 3, (10, 6))])
def test_half_spectrum_parity(emsurf_lib, n, nx, ny, grid):
    """Reciprocal tables (L(-d) = L(d)^T, K(-d) = K(d)^T) on a single-rhs MIXED
    handle: the FP32 operator stores one bin of each pair (k, -k) and the
    paired kernel applies B^(k) to x(k) and B^(k)^T to x(-k).  Same FP32 bar
    against the oracle; odd and even grids (1, 2 or 4 self-paired bins)."""
    from paper_1911_04576_gb300 import binding as B
    seed = 700 + 10 * nx + ny
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 3, seed)
    Lt, Kt = reciprocal(Lt), reciprocal(Kt)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, grid=grid)
    x = W.random_vectors(1, nu, seed + 3)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    assert relerr(run_matvec(B, h, x, B.FP32)[0], yref[0]) <= TOL32
    assert relerr(run_matvec(B, h, x, B.FP64)[0], yref[0]) <= TOL64
    # the FP32 spectrum is (about) half of a non-reciprocal handle's
    Lr, Kr = W.random_tables(nx, ny, E, seed)
    h2 = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lr, Kr, COEF, idx, sgn, precision=B.MIXED, grid=grid)
    px, py, bytes_half = B.emsurf_query(h)
    bytes_full = B.emsurf_query(h2)[2]
    P = px * py
    stored = (P + sum(1 for kx in range(px) for ky in range(py)
                      if (2 * kx) % px == 0 and (2 * ky) % py == 0)) // 2
    assert B.emsurf_operator_info(h) == (stored, False)
    assert B.emsurf_operator_info(h2) == (P, False)
    # (minus the stored-bin index arrays and the pair kernel's partial row
    # sums [CTA][2][2E] and arrival counters [stored bin][row warp])
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scratch_max = sms * 2 * 2 * E * 8 + stored * -(-E // 32) * 4
    saved = (P - stored) * 2 * E * E * 8 - (bytes_full - bytes_half)
    assert -4096 <= saved <= scratch_max + 8 * stored + 4096, (saved, scratch_max)
    B.emsurf_check(h)
    h.close()
    h2.close()


@pytest.mark.parametrize("n,nx,ny", [(2, 3, 2), (3, 2, 3)])
def test_fp64_single_rhs_double_single(emsurf_lib, n, nx, ny):
    """Single-rhs handles take the FP64 bin multiply in double-single FP32
    arithmetic (hi/lo planes, exact product errors, TwoSum sums): each product
    term carries a few 2^-48 of relative error, so the FP64 product meets a
    bar 100x below the FP64 path's 1e-10 (1e-12 rel-L2 against the oracle),
    for one rhs and on a two-rhs handle (the register-blocked variant)."""
    from paper_1911_04576_gb300 import binding as B
    seed = 900 + 10 * nx + ny
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 2, seed)
    x = W.random_vectors(1, nu, seed + 3)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    for R in (1, 2):
        h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, max_rhs=R)
        assert relerr(run_matvec(B, h, x, B.FP64)[0], yref[0]) <= 1e-12
        B.emsurf_check(h)
        h.close()


@pytest.mark.parametrize("sx,sop", [(2.0 ** 100, 1.0), (2.0 ** -100, 1.0), (1.0, 2.0 ** 90), (2.0 ** -60, 2.0 ** -80)])
def test_double_single_outside_fp32_range(emsurf_lib, sx, sop):
    """The double-single FP64-accuracy product keeps its 1e-12 bar when x or
    the operator (tables and macromodels) lies far outside FP32's exponent
    range: operands are scaled by powers of two before the hi/lo split and
    the FP64 results scaled back.  One rhs (TMA-fed kernel, double-single
    macromodel product) and two rhs (register-blocked kernel), FP64 handles
    (no complex64 operator, whose storage would overflow)."""
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 3, 2
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 2, 950)
    Lt, Kt, Z = Lt * sop, Kt * sop, Z * sop
    x = W.random_vectors(2, nu, 951) * sx
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    for R in (1, 2):
        h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.FP64, max_rhs=R)
        y = run_matvec(B, h, x[:R], B.FP64)
        for r in range(R):
            assert np.all(np.isfinite(y[r])) and relerr(y[r], yref[r]) <= 1e-12, (R, r)
        B.emsurf_check(h)
        h.close()


@pytest.mark.parametrize("n,nx,ny,P,R", [(2, 4, 4, 8, 1), (2, 3, 3, 5, 3), (2, 8, 7, 16, 2), (1, 12, 12, 24, 2),
                                         (2, 16, 16, 32, 1), (1, 20, 24, 48, 1), (2, 16, 16, 32, 5),
                                         (2, 6, 6, 16, 9)])
def test_fused_2d_fft_matches_passes(emsurf_lib, n, nx, ny, P, R):
    """Square grids up to 64 x 64 take the fused 2-D transforms (gather, both
    passes and the crop/epilogue in one launch each); a taller grid takes the
    pass-based ones.  Both embeddings are exact (any grid >= 2N - 1),
    so FP64 products agree to rounding and both match the oracle.  The lane
    counts (rhs x 2E) cover one, two and four lanes per CTA."""
    from paper_1911_04576_gb300 import binding as B
    seed = 1300 + P + nx
    E, idx, sgn, nu, Lt, Kt, Z, tmap = random_case(n, nx, ny, 2, seed)
    x = W.random_vectors(R, nu, seed + 5)
    Q = P + 1                      # a taller grid with no prime factor above 7
    while any(Q % f == 0 for f in (11, 13, 17, 19, 23, 29, 31)):
        Q += 1
    ys = {}
    for grid in ((P, P), (P, Q)):
        h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, max_rhs=R,
                            grid=grid)
        ys[grid] = (run_matvec(B, h, x, B.FP64), run_matvec(B, h, x, B.FP32))
        B.emsurf_check(h)
        h.close()
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    for r in range(R):
        assert relerr(ys[(P, P)][0][r], ys[(P, Q)][0][r]) <= 1e-13
        assert relerr(ys[(P, P)][0][r], yref[r]) <= TOL64
        assert relerr(ys[(P, P)][1][r], yref[r]) <= TOL32
