"""GPU parity of the GMRES solve of Eq. final against the oracle's dense LU,
on physical inputs: oracle-tabulated L(d), K(d) of a 3x3 lattice of boxes
meshed 3x3 per face (K = 324) and PEC-patch macromodels (Eq. Zmacromodel).

Bars: FP64 solve to rtol 1e-12, solution within rel-L2 1e-8 of dense LU;
MIXED (FP32 inner GMRES + FP64 refinement) to rtol 1e-10, within 1e-7.
"""
import numpy as np
import pytest

from oracle import lattice, macromodel, operators, solve
from oracle.mesh import box_mesh, patch_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.PERIOD
H = W.BOX_H
COEF = (1j * W.K0, 1.0, -1.0, 1j * W.K0)


@pytest.fixture(scope="module")
def physical_3x3():
    w = W.WORKLOADS["lattice3x3_k324"]
    box = box_mesh(A, A, H, w.n)
    idx, sgn, nu = lattice.overlap_map(box, w.nx, w.ny, A, A)
    Lt, Kt = lattice.offset_tables(box, w.nx, w.ny, A, A, W.K0)
    sides = W.patch_sides(w)
    Z = np.stack([macromodel.pec_patch(box, patch_mesh(s, W.PATCH_Z, w.patch_n), W.K0) for s in sides])
    tmap = W.type_map(w)
    V = []
    for khat, ehat in W.plane_waves(w):
        Vl = np.concatenate([operators.excitation(box, lattice.cell_shift(m % w.nx, m // w.nx, A, A),
                                                  W.K0, khat, ehat) for m in range(w.M)])
        V.append(lattice.scatter(Vl, idx, sgn, nu))
    V = np.array(V)
    Ad = lattice.assemble_from_tables(Lt, Kt, COEF, Z, tmap, idx, sgn, nu, w.nx, w.ny)
    xs = np.stack([solve.dense_solve(Ad, v) for v in V])
    return w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs


def _solve(B, w, idx, sgn, nu, Lt, Kt, Z, tmap, V, prec, **kw):
    import torch
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=prec,
                        max_rhs=len(V))
    b = torch.from_numpy(V).cuda()
    x = torch.zeros_like(b)
    st, info = B.emsurf_solve(h, b, x, **kw)
    h.close()
    return st, info, x.cpu().numpy()


def test_fp64_matvec_physical(emsurf_lib, physical_3x3):
    import torch
    from paper_1911_04576_gb300 import binding as B
    w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs = physical_3x3
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, tmap, Z, Lt, Kt, COEF, idx, sgn, precision=B.FP64)
    x = W.random_vectors(1, nu, 33)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, B.FP64)
    y = yd.cpu().numpy()[0]
    ref = Ad @ x[0]
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    h.close()


def test_fp64_solve_matches_dense_lu(emsurf_lib, physical_3x3):
    from paper_1911_04576_gb300 import binding as B
    w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs = physical_3x3
    st, info, x = _solve(B, w, idx, sgn, nu, Lt, Kt, Z, tmap, V, B.FP64, rtol=1e-12, restart=30,
                         max_iters=4000)
    assert st == B.EMSURF_OK and info[0]["converged"] == 1
    assert info[0]["rel_residual"] <= 1e-12
    assert np.linalg.norm(x[0] - xs[0]) <= 1e-8 * np.linalg.norm(xs[0])


def test_mixed_solve_matches_dense_lu(emsurf_lib, physical_3x3):
    from paper_1911_04576_gb300 import binding as B
    w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs = physical_3x3
    st, info, x = _solve(B, w, idx, sgn, nu, Lt, Kt, Z, tmap, V, B.MIXED, rtol=1e-10, restart=30,
                         max_iters=6000, max_refine=20)
    assert st == B.EMSURF_OK and info[0]["refinements"] >= 1
    assert np.linalg.norm(x[0] - xs[0]) <= 1e-7 * np.linalg.norm(xs[0])
    # the reported residual is the true FP64 one
    r = V[0] - Ad @ x[0]
    assert abs(np.linalg.norm(r) / np.linalg.norm(V[0]) - info[0]["rel_residual"]) <= 1e-12


def test_multi_rhs_solve_independent(emsurf_lib, physical_3x3):
    """Several right-hand sides in one call give each one's single solution."""
    from paper_1911_04576_gb300 import binding as B
    w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs = physical_3x3
    rng = np.random.default_rng(9)
    Vm = np.stack([V[0], rng.standard_normal(nu) + 1j * rng.standard_normal(nu), 2.0 * V[0]])
    st, info, x = _solve(B, w, idx, sgn, nu, Lt, Kt, Z, tmap, Vm, B.FP64, rtol=1e-12, restart=25,
                         max_iters=6000)
    assert st == B.EMSURF_OK
    for r in range(3):
        ref = solve.dense_solve(Ad, Vm[r])
        assert np.linalg.norm(x[r] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_not_converged_reports_best_iterate(emsurf_lib, physical_3x3):
    from paper_1911_04576_gb300 import binding as B
    w, idx, sgn, nu, Lt, Kt, Z, tmap, V, Ad, xs = physical_3x3
    st, info, x = _solve(B, w, idx, sgn, nu, Lt, Kt, Z, tmap, V, B.FP64, rtol=1e-12, restart=10,
                         max_iters=5)
    assert st == B.EMSURF_ENOTCONV and info[0]["converged"] == 0 and info[0]["iters"] == 5
    r = V[0] - Ad @ x[0]
    assert abs(np.linalg.norm(r) / np.linalg.norm(V[0]) - info[0]["rel_residual"]) <= 1e-10
    assert info[0]["rel_residual"] < 1.0
