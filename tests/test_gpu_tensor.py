"""GPU parity of the tensor-core bin multiply (BF16x3 split precision on
tcgen05, FP32 accumulation) used for FP32 products with nrhs >= 8.

Tolerance.  Each factor is split v = hi + lo with hi = rn_bf16(v),
lo = rn_bf16(v - hi), so |v - hi - lo| <= 2^-18 |v|; dropping lo*lo leaves a
relative error per product term of at most 3 * 2^-18 (FP32 accumulation
adds 2^-24 per addition).  An output sums 2E such terms; its relative error
is bounded by 3 * 2^-18 * (sum_j |b_j||x_j|) / |sum_j b_j x_j|, and for the
random-phase tables and vectors used here that ratio is about sqrt(2E).
The FFTs add FP32 rounding only.  The bar is TOL = 3 * 2^-18 * sqrt(2E)
(1.1e-3 at E = 288, 4.3e-4 at E = 72) in rel-L2 against the oracle's
FFT-free direct product.  Solves keep their FP64-refined bars.
"""
import numpy as np
import pytest

from oracle import lattice, macromodel, operators, precond, solve
from oracle.mesh import box_mesh, patch_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.PERIOD
H = W.BOX_H
COEF = (1j * W.K0, 1.0, -1.0, 1j * W.K0)


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def tol(E):
    return 3 * 2.0 ** -18 * np.sqrt(2 * E)


@pytest.mark.parametrize("n,nx,ny,R", [(2, 3, 2, 8), (3, 2, 3, 13), (4, 2, 2, 32), (2, 4, 3, 40)])
def test_tc_matvec_parity(emsurf_lib, n, nx, ny, R):
    import torch
    from paper_1911_04576_gb300 import binding as B
    seed = 1000 + 100 * n + 10 * nx + ny
    box = box_mesh(A, A, H, n)
    E = box.n_rwg
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    Lt, Kt = W.random_tables(nx, ny, E, seed)
    Z = W.random_macromodels(3, 2 * E, seed + 1)
    tmap = np.random.default_rng(seed + 2).integers(0, 3, nx * ny).astype(np.int32)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, max_rhs=R,
                        tensor_cores=True)
    x = W.random_vectors(R, nu, seed + 3)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, B.FP32)
    y = yd.cpu().numpy()
    errs = [relerr(y[r], yref[r]) for r in range(R)]
    assert max(errs) <= tol(E), (max(errs), tol(E))
    # the split planes exist: the handle holds the bf16 hi/lo spectrum on top
    h0 = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, max_rhs=R)
    px, py, _ = B.emsurf_query(h)
    assert B.emsurf_query(h)[2] - B.emsurf_query(h0)[2] >= px * py * 2 * 2 * E * E * 2 * 2
    h0.close()
    # fewer rhs than the threshold take the FP32 kernels on the same handle
    B.emsurf_matvec(h, xd[:2].contiguous(), yd[:2], B.FP32)
    y2 = yd[:2].cpu().numpy()
    assert max(relerr(y2[r], yref[r]) for r in range(2)) <= 3e-5
    B.emsurf_check(h)
    h.close()


def test_tc_mixed_solve_multi_rhs(emsurf_lib):
    """Preconditioned MIXED solve of 8 right-hand sides with the tensor-core
    FP32 operator: FP64 refinement brings every solution to the dense-LU
    answer within the plain MIXED bar."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice3x3_k324"]
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = lattice.offset_tables(box, w.nx, w.ny, A, A, W.K0)
    Z = np.stack([macromodel.pec_patch(box, patch_mesh(s, W.PATCH_Z, w.patch_n), W.K0)
                  for s in W.patch_sides(w)])
    tmap = W.type_map(w)
    Ad = lattice.assemble_from_tables(Lt, Kt, COEF, Z, tmap, idx, sgn, nu, w.nx, w.ny)
    xy, _ = precond.unknown_positions(box, idx, w.nx, w.ny, A, A)
    R = 8
    b = W.random_vectors(R, nu, 5)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED,
                        max_rhs=R, unknown_xy=xy, cell=(A, A), precond_overlap=0.6 * A / w.n,
                        tensor_cores=True)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    st, info = B.emsurf_solve(h, bd, xd, rtol=1e-10, restart=30, max_iters=6000, max_refine=30)
    assert st == B.EMSURF_OK
    x = xd.cpu().numpy()
    for r in range(R):
        xs = solve.dense_solve(Ad, b[r])
        assert np.linalg.norm(x[r] - xs) <= 1e-7 * np.linalg.norm(xs)
    h.close()
