"""Result-level accuracy of the precision modes at the bench's size, on the
product path (GPU tables, patch-on-slab macromodels, excitation, solves,
far field):

* MIXED (FP32 operator inside FP64 residual refinement) solved to the
  16 x 16 / K = 576 configuration's rtol 1e-8 against the FP64-operator GMRES
  solved to 1e-11, both right-preconditioned: currents within rel-L2 1e-6
  and bistatic RCS within 0.05 dB wherever sigma > sigma_max - 40 dB (nulls
  left out), on a 3 x 6 degree grid of the whole sphere.
* The tensor-core bin multiply (BF16x3) at that size with 32 rhs (1024
  bins, the persistent CTAs' full tile schedule) against the oracle's
  FFT-free direct product on sampled rows, within its split-precision bar
  3 * 2^-18 * sqrt(2E).
"""
import numpy as np
import pytest

from oracle import lattice
from oracle.mesh import box_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A, H, K0 = W.PERIOD, W.BOX_H, W.K0
COEF = (1j * K0, 1.0, -1.0, 1j * K0)
PC_OVERLAP = 0.6


def _product_problem(B, torch, w, precision, max_rhs=1, tensor_cores=False):
    zl = B.emsurf_setup_slab_zlevels(H, w.n, W.SLAB_T)
    idx, sgn, nu = B.emsurf_setup_overlap(w.n, w.nx, w.ny)
    xy = B.emsurf_setup_unknown_xy(A, A, H, w.n, w.nx, w.ny, idx, nu)
    L = torch.empty((2 * w.ny - 1, 2 * w.nx - 1, w.E, w.E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, w.n, w.nx, w.ny, K0, L, K, zlevels=zl)
    Z = torch.empty((w.n_types, w.K, w.K), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_slab_patch(A, A, H, w.n, zl, W.patch_sides(w), w.patch_n, W.RING_LAYERS,
                                   W.EPS_SLAB, K0, Z)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, W.type_map(w), Z, L, K, COEF, idx, sgn, precision=precision,
                        max_rhs=max_rhs, tables_on_device=True, unknown_xy=xy, cell=(A, A),
                        precond_overlap=PC_OVERLAP * A / w.n, tensor_cores=tensor_cores)
    del L, K, Z
    torch.cuda.empty_cache()
    return h, zl, nu


def _rcs_db(B, torch, h, zl, w, X, rhat):
    F = torch.empty((X.shape[0], len(rhat), 3), dtype=torch.complex128, device="cuda")
    rcs = torch.empty((X.shape[0], len(rhat)), dtype=torch.float64, device="cuda")
    B.emsurf_far_field(h, A, A, H, w.n, K0, X, rhat, F, rcs, zlevels=zl)
    return 10 * np.log10(rcs.cpu().numpy())


def test_mixed_currents_and_rcs_match_fp64_solve(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    h, zl, nu = _product_problem(B, torch, w, B.MIXED)
    waves = W.plane_waves(w)
    V = torch.empty((1, nu), dtype=torch.complex128, device="cuda")
    B.emsurf_excitation(h, A, A, H, w.n, K0, [waves[0][0]], [waves[0][1]], V, zlevels=zl)
    X64 = torch.zeros_like(V)
    st, info = B.emsurf_solve(h, V, X64, rtol=1e-11, restart=30, max_iters=20000, solver=B.SOLVER_FP64)
    assert st == B.EMSURF_OK and info[0]["rel_residual"] <= 1e-11
    XM = torch.zeros_like(V)
    st, info = B.emsurf_solve(h, V, XM, rtol=1e-8, restart=30, max_iters=20000, max_refine=20,
                              solver=B.SOLVER_MIXED)
    assert st == B.EMSURF_OK and info[0]["rel_residual"] <= 1e-8
    x64, xm = X64.cpu().numpy(), XM.cpu().numpy()
    assert np.linalg.norm(xm - x64) <= 1e-6 * np.linalg.norm(x64)
    th = np.radians(np.arange(0.0, 180.01, 3.0))
    ph = np.radians(np.arange(0.0, 360.0, 6.0))
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    rhat = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    s64 = _rcs_db(B, torch, h, zl, w, X64, rhat)[0]
    sm = _rcs_db(B, torch, h, zl, w, XM, rhat)[0]
    keep = s64 > s64.max() - 40.0
    assert keep.sum() > 100
    assert np.abs(sm[keep] - s64[keep]).max() <= 0.05
    B.emsurf_check(h)
    h.close()


def test_tensor_core_product_full_size_sampled(emsurf_lib):
    """16 x 16, K = 576, 32 rhs: every bin of the 32 x 32 grid through the
    persistent tensor-core kernel; 24 sampled outputs of every rhs."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    R = 32
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = W.random_tables(w.nx, w.ny, w.E, 2600)
    Z = W.random_macromodels(w.n_types, w.K, 2601)
    tmap = W.type_map(w)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.FP32, max_rhs=R,
                        tensor_cores=True)
    assert B.emsurf_operator_info(h)[1]
    x = W.random_vectors(R, nu, 2602)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, B.FP32)
    y = yd.cpu().numpy()
    rows = np.sort(np.random.default_rng(2603).choice(nu, 24, replace=False))
    rows[0], rows[-1] = 0, nu - 1
    bar = 3 * 2.0 ** -18 * np.sqrt(2 * w.E)
    for r in range(R):
        yref = lattice.matvec_direct_rows(x[r], rows, Lt, Kt, COEF, Z, tmap, idx, sgn, w.nx, w.ny)
        assert np.linalg.norm(y[r, rows] - yref) <= bar * np.linalg.norm(yref), r
    # repeated products are bit-identical (fixed accumulation order)
    B.emsurf_matvec(h, xd, yd, B.FP32)
    assert np.array_equal(yd.cpu().numpy(), y)
    B.emsurf_check(h)
    h.close()


def test_batched_tensor_core_solve_accuracy(emsurf_lib):
    """48 x 48 lattice, K = 576, 32 plane waves on the tensor-core path (BF16x3
    bin multiply, macromodel product and preconditioner apply inside the
    MIXED refinement): every rhs solved to 1e-8 is within rel-L2 1e-6 of the
    same solve taken to 1e-10 (the FP64-residual-verified reference; the
    FP64-operator GMRES of 32 rhs at this size would take minutes), and its
    bistatic RCS within 0.05 dB on a 6-degree grid."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice48x48_k576_r32"]
    h, zl, nu = _product_problem(B, torch, w, B.MIXED, max_rhs=w.n_rhs, tensor_cores=True)
    assert B.emsurf_operator_info(h)[1]
    waves = W.plane_waves(w)
    V = torch.empty((w.n_rhs, nu), dtype=torch.complex128, device="cuda")
    B.emsurf_excitation(h, A, A, H, w.n, K0, [k for k, _ in waves], [e for _, e in waves], V, zlevels=zl)
    Xr = torch.zeros_like(V)
    st, info = B.emsurf_solve(h, V, Xr, rtol=1e-10, restart=30, max_iters=60000, max_refine=80,
                              solver=B.SOLVER_MIXED)
    worst = max(i["rel_residual"] for i in info)
    assert st == B.EMSURF_OK and worst <= 1e-10, (st, worst, info[0])
    X = torch.zeros_like(V)
    st, info = B.emsurf_solve(h, V, X, rtol=1e-8, restart=30, max_iters=40000, max_refine=40,
                              solver=B.SOLVER_MIXED)
    assert st == B.EMSURF_OK and max(i["rel_residual"] for i in info) <= 1e-8
    xr, x = Xr.cpu().numpy(), X.cpu().numpy()
    for r in range(w.n_rhs):
        assert np.linalg.norm(x[r] - xr[r]) <= 1e-6 * np.linalg.norm(xr[r]), r
    th = np.radians(np.arange(0.0, 180.01, 6.0))
    ph = np.radians(np.arange(0.0, 360.0, 6.0))
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    rhat = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    sr = _rcs_db(B, torch, h, zl, w, Xr, rhat)
    sx = _rcs_db(B, torch, h, zl, w, X, rhat)
    for r in range(w.n_rhs):
        keep = sr[r] > sr[r].max() - 40.0
        assert np.abs(sx[r][keep] - sr[r][keep]).max() <= 0.05, r
    B.emsurf_check(h)
    h.close()
