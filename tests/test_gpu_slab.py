"""GPU parity of the configurations' cell (patch on a lossy slab, Secs.
II-A..D) against the oracle, through the C ABI:

* macromodels Z~ (two regions with k_v = k0 sqrt(eps_v), U rules 1-3 and the
  junction with S_eq, Schur complement) -- same quadrature on both sides, so
  the bar is the setup tests' 1e-10 in norm;
* offset tables of boxes whose rows end at the slab top (1e-11 of the
  largest entry);
* the whole product path on the 3 x 3 / K = 324 lattice of slab cells
  (GPU tables, GPU macromodels, GPU excitation, FP64 GMRES to 1e-12)
  against the oracle's dense assembly solved by LU: currents within 1e-8.
"""
import numpy as np
import pytest

from oracle import lattice, macromodel, operators, solve
from oracle.mesh import box_mesh, slab_zlevels
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A, H, K0, T = W.PERIOD, W.BOX_H, W.K0, W.SLAB_T
COEF = (1j * K0, 1.0, -1.0, 1j * K0)


@pytest.mark.parametrize("n,patch_n,layers,eps", [(2, 3, 2, 3.0 * (1 - 0.001j)), (3, 4, 3, 3.0 * (1 - 0.001j)),
                                                   (2, 3, 1, 1.0)])
def test_slab_macromodels_match_oracle(emsurf_lib, n, patch_n, layers, eps):
    import torch
    from paper_1911_04576_gb300 import binding as B
    sides = np.array([0.2 * W.LAMBDA, 0.0, 0.42 * W.LAMBDA])
    z = B.emsurf_setup_slab_zlevels(H, n, T)
    K = 36 * n * n
    Z = torch.empty((len(sides), K, K), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_slab_patch(A, A, H, n, z, sides, patch_n, layers, eps, K0, Z)
    Z = Z.cpu().numpy()
    box = box_mesh(A, A, H, n, slab_zlevels(H, n, T))
    for t, s in enumerate(sides):
        ref = macromodel.slab_patch(box, n, s, patch_n, eps, K0, T, ring_layers=layers)
        assert np.linalg.norm(Z[t] - ref) <= 1e-10 * np.linalg.norm(ref), t


def test_slab_macromodel_rejects_bad_arguments(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    z = B.emsurf_setup_slab_zlevels(H, 2, T)
    Z = torch.empty((1, 144, 144), dtype=torch.complex128, device="cuda")
    for sides, eps in (([0.6 * W.LAMBDA], 3.0), ([0.2 * W.LAMBDA], 3.0 + 0.1j), ([0.2 * W.LAMBDA], -2.0)):
        with pytest.raises(B.EmsurfError) as e:
            B.emsurf_macromodel_slab_patch(A, A, H, 2, z, sides, 3, 2, eps, K0, Z)
        assert e.value.status == B.EMSURF_EINVAL


def test_offset_tables_with_slab_rows(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 3, 3, 2
    z = B.emsurf_setup_slab_zlevels(H, n, T)
    E = 18 * n * n
    L = torch.empty((2 * ny - 1, 2 * nx - 1, E, E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, n, nx, ny, K0, L, K, zlevels=z)
    Lo, Ko = lattice.offset_tables(box_mesh(A, A, H, n, slab_zlevels(H, n, T)), nx, ny, A, A, K0)
    L, K = L.cpu().numpy(), K.cpu().numpy()
    for dy in range(2 * ny - 1):
        for dx in range(2 * nx - 1):
            assert np.abs(L[dy, dx] - Lo[dy, dx]).max() <= 1e-11 * np.abs(Lo[dy, dx]).max()
            assert np.abs(K[dy, dx] - Ko[dy, dx]).max() <= 1e-11 * np.abs(Ko[dy, dx]).max()


def test_slab_lattice_product_path_matches_dense_lu(emsurf_lib):
    """3 x 3 lattice, K = 324, 9 patch-on-slab types: every setup step and the
    FP64 solve on the GPU, against the oracle's box-pair dense assembly."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice3x3_k324"]
    zb = B.emsurf_setup_slab_zlevels(H, w.n, T)
    idx, sgn, nu = B.emsurf_setup_overlap(w.n, w.nx, w.ny)
    L = torch.empty((2 * w.ny - 1, 2 * w.nx - 1, w.E, w.E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, w.n, w.nx, w.ny, K0, L, K, zlevels=zb)
    sides = W.patch_sides(w)
    Z = torch.empty((w.n_types, w.K, w.K), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_slab_patch(A, A, H, w.n, zb, sides, w.patch_n, W.RING_LAYERS, W.EPS_SLAB, K0, Z)
    tmap = W.type_map(w)
    # the slab makes the plain GMRES slow (thousands of iterations): the
    # near-field preconditioner (flexible GMRES) keeps the FP64 bars
    xy = B.emsurf_setup_unknown_xy(A, A, H, w.n, w.nx, w.ny, idx, nu)
    hd = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, L, K, COEF, idx, sgn, tables_on_device=True,
                         unknown_xy=xy, cell=(A, A), precond_overlap=0.6 * A / w.n)
    khat, ehat = W.plane_waves(w)[0]
    V = torch.empty((1, nu), dtype=torch.complex128, device="cuda")
    B.emsurf_excitation(hd, A, A, H, w.n, K0, [khat], [ehat], V, zlevels=zb)
    X = torch.zeros_like(V)
    st, info = B.emsurf_solve(hd, V, X, rtol=1e-12, restart=40, max_iters=6000)
    assert st == B.EMSURF_OK, info
    hd.close()
    # oracle: its own mesh, tables, macromodels, excitation and dense LU
    box = box_mesh(A, A, H, w.n, slab_zlevels(H, w.n, T))
    oi, os_, onu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    assert onu == nu and np.array_equal(oi, idx) and np.array_equal(os_, sgn)
    Zo = np.stack([macromodel.slab_patch(box, w.n, s, w.patch_n, W.EPS_SLAB, K0, T, W.RING_LAYERS)
                   for s in sides])
    Ad = lattice.assemble_dense(box, w.nx, w.ny, A, A, K0, COEF, Zo, tmap, oi, os_, onu)
    Vl = np.concatenate([operators.excitation(box, lattice.cell_shift(m % w.nx, m // w.nx, A, A), K0, khat, ehat)
                         for m in range(w.M)])
    Vo = lattice.scatter(Vl, oi, os_, onu)
    assert np.linalg.norm(V[0].cpu().numpy() - Vo) <= 1e-12 * np.linalg.norm(Vo)
    xo = solve.dense_solve(Ad, Vo)
    x = X[0].cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
