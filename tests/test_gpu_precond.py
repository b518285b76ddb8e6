"""GPU parity of the near-field preconditioner (restricted additive Schwarz
by cells, Sec. IV-A / Eq. final_precond grouped by cell) and of the
preconditioned solves, against oracle/precond.py and the oracle's dense LU.

Tolerance of M^{-1} r: the device factors each subdomain block A_m in complex
FP32 with partial pivoting.  The computed solution of A_m z = b then solves
(A_m + dA) z = b with |dA| <= gamma_{3n} |L||U| (Higham, Thm. 9.4), so
||dz|| / ||z|| <= kappa(A_m) * 3 n u (growth ~ 1 for these blocks), with
u = 2^-24 and the FP32 rounding of r adding kappa * u.  The test uses
(3 n_max + 1) u max_m kappa(A_m), computed from the oracle's blocks.
Preconditioned solves use FGMRES (stored M^{-1} V_j), so their accuracy is
that of the unpreconditioned solves: FP64 1e-8, MIXED 1e-7 against dense LU.
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
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def phys():
    w = W.WORKLOADS["lattice3x3_k324"]
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = lattice.offset_tables(box, w.nx, w.ny, A, A, W.K0)
    Z = np.stack([macromodel.pec_patch(box, patch_mesh(s, W.PATCH_Z, w.patch_n), W.K0)
                  for s in W.patch_sides(w)])
    tmap = W.type_map(w)
    V = []
    for khat, ehat in W.plane_waves(w):
        Vl = np.concatenate([operators.excitation(box, lattice.cell_shift(m % w.nx, m // w.nx, A, A),
                                                  W.K0, khat, ehat) for m in range(w.M)])
        V.append(lattice.scatter(Vl, idx, sgn, nu))
    V = np.array(V)
    Ad = lattice.assemble_from_tables(Lt, Kt, COEF, Z, tmap, idx, sgn, nu, w.nx, w.ny)
    xy, owner = precond.unknown_positions(box, idx, w.nx, w.ny, A, A)
    delta = 0.6 * A / w.n
    subs = precond.subdomains(xy, owner, w.nx, w.ny, A, A, delta)
    return dict(w=w, box=box, idx=idx, sgn=sgn, nu=nu, Lt=Lt, Kt=Kt, Z=Z, tmap=tmap, V=V, Ad=Ad,
                xy=xy, delta=delta, subs=subs)


def _handle(B, d, prec, delta=None, max_rhs=2, xy=None, int8=False):
    w = d["w"]
    return B.emsurf_create(w.nx, w.ny, w.E, d["nu"], d["tmap"], d["Z"], d["Lt"], d["Kt"], COEF,
                           d["idx"], d["sgn"], precision=prec, max_rhs=max_rhs,
                           unknown_xy=d["xy"] if xy is None else xy, cell=(A, A),
                           precond_overlap=d["delta"] if delta is None else delta, precond_int8=int8)


def _bound(Ad, subs):
    """FP32 LU of each block ((3 n + 1) u kappa, see the module docstring) plus
    the FP16 storage of the owned inverse rows: relative error <= 2^-11 per
    entry, i.e. <= 2^-11 (sum |x_j||r_j|) / |sum x_j r_j| per output, about
    2^-11 sqrt(n) for random-phase r."""
    kap = max(np.linalg.cond(Ad[np.ix_(S, S)]) for S, _ in subs)
    nmax = max(len(S) for S, _ in subs)
    return (3 * nmax + 1) * U32 * kap + 2.0 ** -11 * np.sqrt(nmax)


@pytest.mark.parametrize("prec", ["FP64", "MIXED", "FP32"])
def test_precond_apply_matches_oracle(emsurf_lib, phys, prec):
    import torch
    from paper_1911_04576_gb300 import binding as B
    h = _handle(B, phys, getattr(B, prec))
    r = W.random_vectors(2, phys["nu"], 41)
    rd = torch.from_numpy(r).cuda()
    yd = torch.full_like(rd, float("nan"))
    B.emsurf_precond_apply(h, rd, yd)
    y = yd.cpu().numpy()
    tol = _bound(phys["Ad"], phys["subs"])
    for q in range(2):
        ref = precond.ras_apply(phys["Ad"], phys["subs"], r[q])
        assert np.all(np.isfinite(y[q]))
        assert np.linalg.norm(y[q] - ref) <= tol * np.linalg.norm(ref), (prec, q, tol)
    h.close()


def test_precond_apply_product_positions(emsurf_lib, phys):
    """The positions from the product's own setup call give the same result."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = phys["w"]
    xy = B.emsurf_setup_unknown_xy(A, A, H, w.n, w.nx, w.ny, phys["idx"], phys["nu"])
    h1 = _handle(B, phys, B.FP64)
    h2 = _handle(B, phys, B.FP64, xy=xy)
    rd = torch.from_numpy(W.random_vectors(1, phys["nu"], 5)).cuda()
    y1, y2 = torch.empty_like(rd), torch.empty_like(rd)
    B.emsurf_precond_apply(h1, rd, y1)
    B.emsurf_precond_apply(h2, rd, y2)
    assert torch.equal(y1, y2)
    h1.close()
    h2.close()


def _rhs(d, nrhs):
    """The plane-wave excitation, then seeded random right-hand sides."""
    extra = W.random_vectors(max(nrhs - len(d["V"]), 0), d["nu"], 77)
    return np.ascontiguousarray(np.concatenate([d["V"], extra])[:nrhs])


def _solve(B, d, prec, nrhs=1, **kw):
    import torch
    h = _handle(B, d, prec, max_rhs=nrhs)
    b = torch.from_numpy(_rhs(d, nrhs)).cuda()
    x = torch.zeros_like(b)
    st, info = B.emsurf_solve(h, b, x, **kw)
    st0, info0 = B.emsurf_solve(h, b, torch.zeros_like(b), precond=-1, **kw)
    h.close()
    return st, info, x.cpu().numpy(), st0, info0


def test_preconditioned_fp64_solve(emsurf_lib, phys):
    from paper_1911_04576_gb300 import binding as B
    st, info, x, st0, info0 = _solve(B, phys, B.FP64, rtol=1e-12, restart=30, max_iters=4000)
    assert st == B.EMSURF_OK and st0 == B.EMSURF_OK
    xs = solve.dense_solve(phys["Ad"], phys["V"][0])
    assert np.linalg.norm(x[0] - xs) <= 1e-8 * np.linalg.norm(xs)
    assert info[0]["rel_residual"] <= 1e-12
    # one mesh layer of overlap: far fewer iterations than without
    assert info[0]["iters"] * 5 <= info0[0]["iters"], (info[0]["iters"], info0[0]["iters"])


def test_preconditioned_mixed_solve_multi_rhs(emsurf_lib, phys):
    from paper_1911_04576_gb300 import binding as B
    st, info, x, st0, info0 = _solve(B, phys, B.MIXED, nrhs=2, rtol=1e-10, restart=30,
                                     max_iters=6000, max_refine=20)
    assert st == B.EMSURF_OK
    bs = _rhs(phys, 2)
    for q in range(2):
        xs = solve.dense_solve(phys["Ad"], bs[q])
        assert np.linalg.norm(x[q] - xs) <= 1e-7 * np.linalg.norm(xs)
        r = bs[q] - phys["Ad"] @ x[q]
        assert abs(np.linalg.norm(r) / np.linalg.norm(bs[q]) - info[q]["rel_residual"]) <= 1e-12
    assert info[0]["iters"] * 5 <= info0[0]["iters"]


def test_precond_invalid(emsurf_lib, phys):
    import torch
    from paper_1911_04576_gb300 import binding as B
    with pytest.raises(B.EmsurfError):
        _handle(B, phys, B.FP64, delta=0.5 * A)           # margin must stay below half a cell
    h = _handle(B, phys, B.FP64, delta=0.0)               # no preconditioner requested
    rd = torch.zeros((1, phys["nu"]), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.EmsurfError):
        B.emsurf_precond_apply(h, rd, torch.empty_like(rd))
    h.close()
    h = _handle(B, phys, B.FP64)
    with pytest.raises(B.EmsurfError):
        B.emsurf_precond_apply(h, rd, rd)                  # in place is not allowed
    h.close()


@pytest.mark.parametrize("R", [1, 2, 3, 11])
def test_precond_random_ragged_lattice(emsurf_lib, R):
    """A 4 x 3 lattice of n = 2 boxes with synthetic tables and strongly
    diagonal macromodels: cells at the edge and corners have smaller
    subdomains than interior ones (ragged sizes)."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    nx, ny, n = 4, 3, 2
    box = box_mesh(A, A, H, n)
    E = box.n_rwg
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    Lt, Kt = W.random_tables(nx, ny, E, 17, decay=2.0)
    Z = W.random_macromodels(3, 2 * E, 18, diag=60.0)
    tmap = np.arange(nx * ny, dtype=np.int32) % 3
    coef = (0.5j, 1.0, -1.0, 0.5j)
    Ad = lattice.assemble_from_tables(Lt, Kt, coef, Z, tmap, idx, sgn, nu, nx, ny)
    xy, owner = precond.unknown_positions(box, idx, nx, ny, A, A)
    delta = 0.6 * A / n
    subs = precond.subdomains(xy, owner, nx, ny, A, A, delta)
    assert len({len(S) for S, _ in subs}) >= 3
    h = B.emsurf_create(nx, ny, E, nu, tmap, Z, Lt, Kt, coef, idx, sgn, precision=B.FP64, max_rhs=R,
                        unknown_xy=xy, cell=(A, A), precond_overlap=delta)
    r = W.random_vectors(R, nu, 19)
    rd = torch.from_numpy(r).cuda()
    yd = torch.empty_like(rd)
    B.emsurf_precond_apply(h, rd, yd)
    y = yd.cpu().numpy()
    tol = _bound(Ad, subs)
    for q in range(R):
        ref = precond.ras_apply(Ad, subs, r[q])
        assert np.linalg.norm(y[q] - ref) <= tol * np.linalg.norm(ref)
    h.close()


@pytest.mark.parametrize("R", [8, 13])
def test_precond_apply_tensor_cores(emsurf_lib, phys, R):
    """With >= 8 rhs and the tensor-core option the apply runs as BF16x3
    GEMMs per cell: the FP32-LU bound plus the split's 3 * 2^-18 per term
    times sqrt(n_max) (random-phase sums), against the oracle."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = phys["w"]
    h = B.emsurf_create(w.nx, w.ny, w.E, phys["nu"], phys["tmap"], phys["Z"], phys["Lt"], phys["Kt"], COEF,
                        phys["idx"], phys["sgn"], precision=B.MIXED, max_rhs=R, unknown_xy=phys["xy"],
                        cell=(A, A), precond_overlap=phys["delta"], tensor_cores=True)
    r = W.random_vectors(R, phys["nu"], 61)
    rd = torch.from_numpy(r).cuda()
    yd = torch.full_like(rd, float("nan"))
    B.emsurf_precond_apply(h, rd, yd)
    y = yd.cpu().numpy()
    nmax = max(len(S) for S, _ in phys["subs"])
    tol = _bound(phys["Ad"], phys["subs"]) + 3 * 2.0 ** -18 * np.sqrt(nmax)
    for q in range(R):
        ref = precond.ras_apply(phys["Ad"], phys["subs"], r[q])
        assert np.all(np.isfinite(y[q]))
        assert np.linalg.norm(y[q] - ref) <= tol * np.linalg.norm(ref), (q, tol)
    h.close()


def test_precond_apply_full_size_sampled(emsurf_lib):
    """16 x 16 lattice, K = 576, one rhs: the single-rhs apply in the launch
    configuration of the bench (95,496 owned rows over the SMs, subdomains of
    up to ~850 unknowns).  The owned rows of a corner and an interior cell are
    recomputed by the oracle from their subdomain blocks A[S_m, S_m]; bar as
    above with kappa of those blocks."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = W.random_tables(w.nx, w.ny, w.E, 1700, decay=2.0)
    Z = W.random_macromodels(w.n_types, w.K, 1701, diag=200.0)
    tmap = W.type_map(w)
    coef = (0.5j, 1.0, -1.0, 0.5j)
    xy, owner = precond.unknown_positions(box, idx, w.nx, w.ny, A, A)
    delta = 0.6 * A / w.n
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, coef, idx, sgn, precision=B.MIXED,
                        max_rhs=1, unknown_xy=xy, cell=(A, A), precond_overlap=delta)
    r = W.random_vectors(1, nu, 1702)
    rd = torch.from_numpy(r).cuda()
    yd = torch.full_like(rd, float("nan"))
    B.emsurf_precond_apply(h, rd, yd)
    y = yd.cpu().numpy()[0]
    assert np.all(np.isfinite(y))
    subs = precond.subdomains(xy, owner, w.nx, w.ny, A, A, delta)
    for m in (0, 8 * w.nx + 7):
        S, own = subs[m]
        As = precond.subdomain_matrix(S, Lt, Kt, coef, Z, tmap, idx, sgn, w.nx, w.ny)
        ref = np.linalg.solve(As, r[0][S])[own]
        tol = (3 * len(S) + 1) * U32 * np.linalg.cond(As) + 2.0 ** -11 * np.sqrt(len(S))
        assert np.linalg.norm(y[S[own]] - ref) <= tol * np.linalg.norm(ref), (m, tol)
    B.emsurf_check(h)
    h.close()


def test_precond_apply_int8_rows(emsurf_lib, phys):
    """8-bit owned inverse rows (one FP32 scale per row): each entry within
    1/254 of its row's largest component, so an output's error is at most
    sqrt(n)/254 of the row's scale times |r| for random-phase r; the apply
    stays within that of the oracle, and the preconditioned solves keep
    their FP64 accuracy (flexible GMRES: the preconditioner only steers)."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    nmax = max(len(S) for S, _ in phys["subs"])
    kap = max(np.linalg.cond(phys["Ad"][np.ix_(S, S)]) for S, _ in phys["subs"])
    tol = (3 * nmax + 1) * U32 * kap + np.sqrt(nmax) / 254.0
    for prec in ("MIXED", "FP64"):
        h = _handle(B, phys, getattr(B, prec), int8=True)
        r = W.random_vectors(2, phys["nu"], 43)
        rd = torch.from_numpy(r).cuda()
        yd = torch.full_like(rd, float("nan"))
        B.emsurf_precond_apply(h, rd, yd)
        y = yd.cpu().numpy()
        h16 = _handle(B, phys, getattr(B, prec))
        y16d = torch.full_like(rd, float("nan"))
        B.emsurf_precond_apply(h16, rd, y16d)
        y16 = y16d.cpu().numpy()
        for q in range(2):
            ref = precond.ras_apply(phys["Ad"], phys["subs"], r[q])
            assert np.all(np.isfinite(y[q]))
            e8 = np.linalg.norm(y[q] - ref) / np.linalg.norm(ref)
            e16 = np.linalg.norm(y16[q] - ref) / np.linalg.norm(ref)
            assert e8 <= tol, (prec, q, e8, tol)
            assert e8 > e16          # the 8-bit rows are the coarser storage
        h.close()
        h16.close()
    # solves with the 8-bit preconditioner reach the dense-LU solution
    hs = _handle(B, phys, B.MIXED, max_rhs=1, int8=True)
    b = torch.from_numpy(_rhs(phys, 1)).cuda()
    x = torch.zeros_like(b)
    st, info = B.emsurf_solve(hs, b, x, rtol=1e-10, restart=30, max_iters=4000, max_refine=20)
    assert st == B.EMSURF_OK and info[0]["rel_residual"] <= 1e-10
    xs = solve.dense_solve(phys["Ad"], phys["V"][0])
    assert np.linalg.norm(x.cpu().numpy()[0] - xs) <= 1e-8 * np.linalg.norm(xs)
    hs.close()
