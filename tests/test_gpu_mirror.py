"""GPU parity of the mirror-orbit form of the FP32 spectrum (one stored bin
per orbit of the box's mirror group, binmul_orbit_kernel) against the
oracle's FFT-free direct product, through the C ABI.

Inputs: tables that obey the mirror relations exactly,
L(g d) = P_g L(d) P_g^T and K(g d) = det(g) P_g K(d) P_g^T, made from
seeded random tables by averaging over the group (small lattices), and the
bench's own GPU-tabulated tables of the union-jack box (16 x 16, K = 576,
sampled rows).  Tolerances as in test_gpu_matvec: FP32 3e-5, FP64 1e-10.
"""
import numpy as np
import pytest

from oracle import lattice
from oracle.mesh import box_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A, H, K0 = W.PERIOD, W.BOX_H, W.K0
COEF = (1j * K0, 1.0, -1.0, 1j * K0)
TOL64 = 1e-10
TOL32 = 3e-5


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_matvec(B, h, x, prec):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, prec)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _compose(p1, p2):
    """P1 P2 for signed permutations (pi, sign) with P e_n = sign_n e_pi(n)."""
    (pi1, s1), (pi2, s2) = p1, p2
    return pi1[pi2], s2 * s1[pi2]


def _elements(perm, sign, mask):
    """Group elements e (bit 0: x mirror, 1: y mirror, 2: x <-> y) with their
    signed permutation P_e = Px^a Py^b Pd^c, det and offset map."""
    E = perm.shape[1]
    out = []
    n_el = 8 if mask & 4 else 4
    for e in range(n_el):
        P = (np.arange(E), np.ones(E, np.int64))
        det = 1
        for g in range(3):
            if e & (1 << g):
                P = _compose(P, (perm[g].astype(np.int64), sign[g].astype(np.int64)))
                det = -det

        def dmap(dx, dy, e=e):
            if e & 4:
                dx, dy = dy, dx
            if e & 2:
                dy = -dy
            if e & 1:
                dx = -dx
            return dx, dy
        out.append((P, det, dmap))
    return out


def mirror_average(T, perm, sign, mask, det_power):
    """T_s(d) = mean_e det_e^p P_e^T T(M_e d) P_e (p = 0 for L, 1 for K)."""
    ny2, nx2 = T.shape[:2]
    ny, nx = (ny2 + 1) // 2, (nx2 + 1) // 2
    out = np.zeros_like(T)
    els = _elements(perm, sign, mask)
    for (pi, sg), det, dmap in els:
        f = det ** det_power
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                gx, gy = dmap(dx, dy)
                M = T[gy + ny - 1, gx + nx - 1]
                out[dy + ny - 1, dx + nx - 1] += f * (sg[:, None] * sg[None, :]) * M[np.ix_(pi, pi)]
    return out / len(els)


def n_orbits(px, py, mask):
    seen, count = set(), 0
    for ky in range(py):
        for kx in range(px):
            if (kx, ky) in seen:
                continue
            count += 1
            for e in range(8 if mask & 4 else 4):
                x, y = kx, ky
                if e & 4:
                    x, y = y, x
                if e & 2:
                    y = (py - y) % py
                if e & 1:
                    x = (px - x) % px
                seen.add((x, y))
    return count


def symmetric_case(B, n, nx, ny, mask, seed, T=3):
    box = box_mesh(A, A, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    E = box.n_rwg
    perm, sign, m = B.emsurf_setup_box_mirrors(A, A, n)
    assert m == 7
    mask = mask if nx == ny else mask & 3
    Lt, Kt = W.random_tables(nx, ny, E, seed)
    Lt = mirror_average(Lt, perm, sign, mask, 0)
    Kt = mirror_average(Kt, perm, sign, mask, 1)
    Z = W.random_macromodels(T, 2 * E, seed + 1)
    tmap = np.random.default_rng(seed + 2).integers(0, T, nx * ny).astype(np.int32)
    return E, idx, sgn, nu, Lt, Kt, Z, tmap, (perm, sign, mask)


@pytest.mark.parametrize("n,nx,ny,mask,grid", [(2, 3, 3, 7, (0, 0)), (2, 3, 3, 3, (0, 0)), (2, 4, 4, 7, (8, 8)),
                                               (2, 3, 5, 3, (0, 0)), (2, 5, 2, 3, (10, 4)),
                                               (2, 4, 4, 7, (7, 7)), (2, 2, 2, 7, (0, 0))])
def test_orbit_spectrum_parity(emsurf_lib, n, nx, ny, mask, grid):
    from paper_1911_04576_gb300 import binding as B
    seed = 7000 + 100 * nx + 10 * ny + mask
    E, idx, sgn, nu, Lt, Kt, Z, tmap, mir = symmetric_case(B, n, nx, ny, mask, seed)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED, grid=grid,
                        mirrors=mir)
    px, py = B.emsurf_query(h)[:2]
    stored, tc = B.emsurf_operator_info(h)
    eff = mir[2] if px == py and nx == ny else mir[2] & 3
    assert stored == n_orbits(px, py, eff) and not tc
    x = W.random_vectors(1, nu, seed + 3)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    y32 = run_matvec(B, h, x, B.FP32)
    assert relerr(y32[0], yref[0]) <= TOL32
    assert relerr(run_matvec(B, h, x, B.FP64)[0], yref[0]) <= TOL64
    assert np.array_equal(run_matvec(B, h, x, B.FP32), y32)     # deterministic
    B.emsurf_check(h)
    h.close()


def test_orbit_falls_back_when_tables_are_not_mirror_symmetric(emsurf_lib):
    """Mirrors given, tables only reciprocal: the check at create rejects the
    orbit form and the handle keeps half of the bins."""
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 4, 4
    box = box_mesh(A, A, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, 91)
    Lt = 0.5 * (Lt + np.swapaxes(Lt[::-1, ::-1], 2, 3))
    Kt = 0.5 * (Kt + np.swapaxes(Kt[::-1, ::-1], 2, 3))
    Z = W.random_macromodels(2, 2 * E, 92)
    tmap = np.zeros(nx * ny, np.int32)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED,
                        mirrors=B.emsurf_setup_box_mirrors(A, A, n))
    assert B.emsurf_operator_info(h)[0] == 34          # (k, -k) pairs of the 8 x 8 grid
    x = W.random_vectors(1, nu, 93)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    assert relerr(run_matvec(B, h, x, B.FP32)[0], yref[0]) <= TOL32
    h.close()


def test_orbit_rejects_bad_permutation(emsurf_lib):
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 2, 2
    E, idx, sgn, nu, Lt, Kt, Z, tmap, (perm, sign, mask) = symmetric_case(B, n, nx, ny, 7, 95)
    bad = perm.copy()
    bad[1, 3] = bad[1, 4]
    with pytest.raises(B.EmsurfError):
        B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.MIXED,
                        mirrors=(bad, sign, mask))


def test_orbit_full_size_sampled(emsurf_lib):
    """The bench's configuration: 16 x 16 lattice, K = 576, GPU-tabulated
    tables of the union-jack box with the slab rows, one rhs; the eighth
    (153 of 1024 bins, x <-> y included) and the quarter (289 bins) forms,
    32 sampled outputs recomputed one by one by the oracle."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    zl = B.emsurf_setup_slab_zlevels(H, w.n, W.SLAB_T)
    idx, sgn, nu = B.emsurf_setup_overlap(w.n, w.nx, w.ny)
    L = torch.empty((2 * w.ny - 1, 2 * w.nx - 1, w.E, w.E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, w.n, w.nx, w.ny, K0, L, K, zlevels=zl)
    Z = W.random_macromodels(w.n_types, w.K, 1701)
    Zd = torch.from_numpy(Z).cuda()
    tmap = W.type_map(w)
    perm, sign, mask = B.emsurf_setup_box_mirrors(A, A, w.n)
    assert mask == 7
    x = W.random_vectors(1, nu, 1702)
    rows = np.sort(np.random.default_rng(1703).choice(nu, 32, replace=False))
    rows[0], rows[-1] = 0, nu - 1
    Lh, Kh = L.cpu().numpy(), K.cpu().numpy()
    yref = lattice.matvec_direct_rows(x[0], rows, Lh, Kh, COEF, Z, tmap, idx, sgn, w.nx, w.ny)
    del Lh, Kh
    for m, stored in ((7, 153), (3, 289)):
        h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Zd, L, K, COEF, idx, sgn, precision=B.MIXED,
                            tables_on_device=True, mirrors=(perm, sign, m))
        assert B.emsurf_operator_info(h) == (stored, False)
        y32 = run_matvec(B, h, x, B.FP32)[0]
        assert relerr(y32[rows], yref) <= TOL32
        assert relerr(run_matvec(B, h, x, B.FP64)[0][rows], yref) <= TOL64
        assert np.array_equal(run_matvec(B, h, x, B.FP32)[0], y32)
        B.emsurf_check(h)
        h.close()


def test_orbit_fp32_handle_and_shared_blocks(emsurf_lib):
    """An FP32-only handle derives the same orbit form from its temporary FP64
    blocks; a handle created like it (other macromodels and type map) reads
    its orbit blocks and gives the product of its own problem."""
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 4, 4
    E, idx, sgn, nu, Lt, Kt, Z, tmap, mir = symmetric_case(B, n, nx, ny, 7, 8100)
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.FP32, mirrors=mir)
    assert B.emsurf_operator_layout(h) == (2, 8)
    px, py = B.emsurf_query(h)[:2]
    assert B.emsurf_operator_info(h)[0] == n_orbits(px, py, 7)
    x = W.random_vectors(1, nu, 8101)
    yref = lattice.matvec_direct(x, Lt, Kt, COEF, Z, tmap, idx, sgn, nu, nx, ny)
    assert relerr(run_matvec(B, h, x, B.FP32)[0], yref[0]) <= TOL32
    Z2 = W.random_macromodels(2, 2 * E, 8102)
    t2 = np.random.default_rng(8103).integers(0, 2, nx * ny).astype(np.int32)
    like = B.emsurf_create(nx, ny, E, nu, t2, Z2, None, None, COEF, idx, sgn, precision=B.FP32, share=h,
                           mirrors=mir)
    assert B.emsurf_operator_layout(like) == (2, 8)
    y2 = lattice.matvec_direct(x, Lt, Kt, COEF, Z2, t2, idx, sgn, nu, nx, ny)
    assert relerr(run_matvec(B, like, x, B.FP32)[0], y2[0]) <= TOL32
    B.emsurf_check(like)
    like.close()
    h.close()
