"""GPU parity of the setup and post-processing rows against the oracle:
offset tables (Eqs. out, blockZo), PEC-patch macromodels (Eq.
Zmacromodel), plane-wave excitation (Eq. out) and far field, all through
the C ABI; plus the empty-lattice physics pin run entirely on the product
path (GPU tables, GPU macromodels, GPU excitation, GPU solve, GPU far field).

Tolerances: same quadrature and closed forms on both sides, so only
rounding differs; entries are compared relative to the largest entry of
their block (1e-11), the macromodels (LU with different pivot tie-breaks)
relative to their norm (1e-10).
"""
import numpy as np
import pytest

from oracle import lattice, macromodel, operators
from oracle.mesh import box_mesh, patch_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.PERIOD
H = W.BOX_H
K0 = W.K0
COEF = (1j * K0, 1.0, -1.0, 1j * K0)


def _tables_gpu(B, n, nx, ny):
    import torch
    E = 18 * n * n
    L = torch.empty((2 * ny - 1, 2 * nx - 1, E, E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, n, nx, ny, K0, L, K)
    return L, K


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_offset_tables_small_lattice(emsurf_lib):
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 3, 3
    L, K = _tables_gpu(B, n, nx, ny)
    Lo, Ko = lattice.offset_tables(box_mesh(A, A, H, n), nx, ny, A, A, K0)
    L, K = L.cpu().numpy(), K.cpu().numpy()
    for dy in range(2 * ny - 1):
        for dx in range(2 * nx - 1):
            assert _maxrel(L[dy, dx], Lo[dy, dx]) <= 1e-11, (dx, dy)
            assert _maxrel(K[dy, dx], Ko[dy, dx]) <= 1e-11, (dx, dy)


def test_offset_tables_full_size_sampled(emsurf_lib):
    """16 x 16 lattice, boxes meshed 4 x 4 per face (K = 576): the whole table
    on the GPU, sampled offsets (near, touching, far, extreme) by the oracle."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 4, 16, 16
    L, K = _tables_gpu(B, n, nx, ny)
    offs = [(0, 0), (1, 0), (-1, 1), (1, -1), (2, -3), (-15, 15), (15, -7)]
    ref = lattice.offset_tables(box_mesh(A, A, H, n), nx, ny, A, A, K0, offsets=offs)
    for (dx, dy), (Lo, Ko) in ref.items():
        Lg = L[dy + ny - 1, dx + nx - 1].cpu().numpy()
        Kg = K[dy + ny - 1, dx + nx - 1].cpu().numpy()
        assert _maxrel(Lg, Lo) <= 1e-11, (dx, dy)
        assert _maxrel(Kg, Ko) <= 1e-11, (dx, dy)
    del L, K
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,patch_n", [(2, 3), (3, 4)])
def test_macromodels_match_oracle(emsurf_lib, n, patch_n):
    import torch
    from paper_1911_04576_gb300 import binding as B
    sides = np.array([0.2 * W.LAMBDA, 0.0, 0.42 * W.LAMBDA])
    K = 36 * n * n
    Z = torch.empty((len(sides), K, K), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_pec_patch(A, A, H, n, sides, W.PATCH_Z, patch_n, K0, Z)
    Z = Z.cpu().numpy()
    box = box_mesh(A, A, H, n)
    for t, s in enumerate(sides):
        ref = macromodel.empty_box(box, K0) if s <= 0 else \
            macromodel.pec_patch(box, patch_mesh(s, W.PATCH_Z, patch_n), K0)
        assert np.linalg.norm(Z[t] - ref) <= 1e-10 * np.linalg.norm(ref), t


def test_excitation_and_far_field(emsurf_lib):
    import torch
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 3, 2
    box = box_mesh(A, A, H, n)
    idx, sgn, nu = B.emsurf_setup_overlap(n, nx, ny)
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, 3)
    Z = W.random_macromodels(1, 2 * E, 4)
    hd = B.emsurf_create(nx, ny, E, nu, np.zeros(nx * ny, np.int32), Z, Lt, Kt, COEF, idx, sgn,
                         max_rhs=2)
    waves = [W.plane_waves(W.Workload("x", 1, 1, 1, 1, 0, 0, angles=[(th, ph, pol)]))[0]
             for th, ph, pol in [(0.0, 0.0, "theta"), (37.0, 120.0, "phi")]]
    khat = np.array([w[0] for w in waves])
    ehat = np.array([w[1] for w in waves])
    V = torch.empty((2, nu), dtype=torch.complex128, device="cuda")
    B.emsurf_excitation(hd, A, A, H, n, K0, khat, ehat, V)
    for r in range(2):
        Vl = np.concatenate([operators.excitation(box, lattice.cell_shift(m % nx, m // nx, A, A), K0,
                                                  khat[r], ehat[r]) for m in range(nx * ny)])
        ref = lattice.scatter(Vl, idx, sgn, nu)
        assert np.linalg.norm(V[r].cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    # far field of arbitrary currents
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((2, nu)) + 1j * rng.standard_normal((2, nu))
    th = rng.uniform(0, np.pi, 40)
    ph = rng.uniform(0, 2 * np.pi, 40)
    rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    F = torch.empty((2, 40, 3), dtype=torch.complex128, device="cuda")
    rcs = torch.empty((2, 40), dtype=torch.float64, device="cuda")
    B.emsurf_far_field(hd, A, A, H, n, K0, torch.from_numpy(Y).cuda(), rhat, F, rcs)
    F = F.cpu().numpy()
    for r in range(2):
        Yl = lattice.gather(Y[r], idx, sgn, nx * ny, 2 * E)
        ref = 0
        for m in range(nx * ny):
            rad = operators.radiation_vectors(box, lattice.cell_shift(m % nx, m // nx, A, A), K0, rhat)
            ref = ref + operators.far_field(rad, rhat, K0, Yl[m, :E], Yl[m, E:])
        assert np.abs(F[r] - ref).max() <= 1e-11 * np.abs(ref).max()
        assert np.allclose(rcs[r].cpu().numpy(), 4 * np.pi * np.sum(np.abs(ref) ** 2, -1), rtol=1e-10)
    hd.close()


def test_empty_lattice_on_product_path(emsurf_lib):
    """Tables, macromodels, excitation, FP64 solve and far field all on the
    GPU: an empty 2 x 2 lattice scatters (almost) nothing."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 2, 2
    E = 18 * n * n
    idx, sgn, nu = B.emsurf_setup_overlap(n, nx, ny)
    L, K = _tables_gpu(B, n, nx, ny)
    Z = torch.empty((1, 2 * E, 2 * E), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_pec_patch(A, A, H, n, [0.0], W.PATCH_Z, 3, K0, Z)
    hd = B.emsurf_create(nx, ny, E, nu, np.zeros(4, np.int32), Z, L, K, COEF, idx, sgn,
                         tables_on_device=True)
    V = torch.empty((1, nu), dtype=torch.complex128, device="cuda")
    B.emsurf_excitation(hd, A, A, H, n, K0, [[0, 0, -1.0]], [[1.0, 0, 0]], V)
    X = torch.zeros_like(V)
    st, info = B.emsurf_solve(hd, V, X, rtol=1e-10, restart=40, max_iters=3000)
    assert st == B.EMSURF_OK
    th = np.linspace(0, np.pi, 19)
    ph = np.linspace(0, 2 * np.pi, 37)
    TH, PH = np.meshgrid(th, ph)
    rhat = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    F = torch.empty((1, len(rhat), 3), dtype=torch.complex128, device="cuda")
    B.emsurf_far_field(hd, A, A, H, n, K0, X, rhat, F)
    # reference radiation: the J part alone
    XJ = X.clone()
    Xl = lattice.gather(X[0].cpu().numpy(), idx, sgn, 4, 2 * E)
    mask = np.zeros(nu, bool)
    mask[idx.reshape(4, 2 * E)[:, E:].ravel()] = True
    XJ[0, torch.from_numpy(mask).cuda()] = 0
    FJ = torch.empty_like(F)
    B.emsurf_far_field(hd, A, A, H, n, K0, XJ, rhat, FJ)
    ratio = F.abs().max().item() / FJ.abs().max().item()
    assert ratio < 0.03, ratio
    del Xl
    hd.close()
