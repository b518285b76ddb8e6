"""Handles that share another handle's Fourier-domain blocks
(emsurf_create_like, used by the serving cache): with the same lattice and
tables but their own macromodels, type map and preconditioner they give
bit-identical products and solves to a handle built from the tables, for the
half FP32 spectrum (one rhs), the full one (several rhs) and the tensor-core
planes; mismatched shapes are refused."""
import numpy as np
import pytest

from oracle import lattice
from oracle.mesh import box_mesh
from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A, H = W.PERIOD, W.BOX_H
# weak coupling against diagonally dominant macromodels: a well-conditioned
# synthetic system, so the solves below converge in a few dozen iterations
COEF = (0.01j, 0.01, -0.01, 0.01j)


def _case(n, nx, ny, seed):
    box = box_mesh(A, A, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, A)
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, seed)
    # reciprocal part, as the product's tabulation returns
    Lt = 0.5 * (Lt + np.swapaxes(Lt[::-1, ::-1], 2, 3))
    Kt = 0.5 * (Kt + np.swapaxes(Kt[::-1, ::-1], 2, 3))
    Z1 = W.random_macromodels(3, 2 * E, seed + 1, diag=40.0)
    Z2 = W.random_macromodels(4, 2 * E, seed + 2, diag=40.0)
    rng = np.random.default_rng(seed + 3)
    t1 = rng.integers(0, 3, nx * ny).astype(np.int32)
    t2 = rng.integers(0, 4, nx * ny).astype(np.int32)
    return E, idx, sgn, nu, Lt, Kt, Z1, Z2, t1, t2


def _run(B, torch, h, x, prec):
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    B.emsurf_matvec(h, xd, yd, prec)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("R,tc", [(1, False), (3, False), (8, True)])
def test_shared_spectrum_matches_own(emsurf_lib, R, tc):
    import torch
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 4, 3
    E, idx, sgn, nu, Lt, Kt, Z1, Z2, t1, t2 = _case(n, nx, ny, 40 + R)
    xy = B.emsurf_setup_unknown_xy(A, A, H, n, nx, ny, idx, nu)
    kw = dict(precision=B.MIXED, max_rhs=R, unknown_xy=xy, cell=(A, A), precond_overlap=0.6 * A / n,
              tensor_cores=tc)
    base = B.emsurf_create(nx, ny, E, nu, t1, Z1, Lt, Kt, COEF, idx, sgn, **kw)
    like = B.emsurf_create(nx, ny, E, nu, t2, Z2, None, None, COEF, idx, sgn, share=base, **kw)
    own = B.emsurf_create(nx, ny, E, nu, t2, Z2, Lt, Kt, COEF, idx, sgn, **kw)
    assert B.emsurf_operator_info(like) == B.emsurf_operator_info(own)
    # the shared handle holds less: no spectra of its own
    assert B.emsurf_query(like)[2] < B.emsurf_query(own)[2]
    x = W.random_vectors(R, nu, 50 + R)
    for prec in (B.FP32, B.FP64):
        assert np.array_equal(_run(B, torch, like, x, prec), _run(B, torch, own, x, prec))
    b = torch.from_numpy(x).cuda()
    xs = []
    for h in (like, own):
        X = torch.zeros_like(b)
        st, info = B.emsurf_solve(h, b, X, rtol=1e-9, restart=30, max_iters=4000, max_refine=10)
        assert st == B.EMSURF_OK
        xs.append(X.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])
    # the base still serves its own problem (its macromodels are untouched)
    yb = _run(B, torch, base, x, B.FP64)
    ref = lattice.matvec_direct(x, Lt, Kt, COEF, Z1, t1, idx, sgn, nu, nx, ny)
    assert np.linalg.norm(yb - ref) <= 1e-10 * np.linalg.norm(ref)
    for h in (like, own, base):
        B.emsurf_check(h)
    like.close()
    own.close()
    base.close()


def test_shared_spectrum_mismatch_refused(emsurf_lib):
    from paper_1911_04576_gb300 import binding as B
    n, nx, ny = 2, 4, 3
    E, idx, sgn, nu, Lt, Kt, Z1, Z2, t1, t2 = _case(n, nx, ny, 60)
    half = B.emsurf_create(nx, ny, E, nu, t1, Z1, Lt, Kt, COEF, idx, sgn, precision=B.MIXED)
    assert B.emsurf_operator_info(half)[0] < B.emsurf_query(half)[0] * B.emsurf_query(half)[1]
    with pytest.raises(B.EmsurfError) as e:        # several rhs need the full FP32 spectrum
        B.emsurf_create(nx, ny, E, nu, t2, Z2, None, None, COEF, idx, sgn, precision=B.MIXED, max_rhs=4,
                        share=half)
    assert e.value.status == B.EMSURF_EINVAL
    i2, s2, nu2 = lattice.overlap_map(box_mesh(A, A, H, n), nx + 1, ny, A, A)
    with pytest.raises(B.EmsurfError):             # another lattice
        B.emsurf_create(nx + 1, ny, E, nu2, np.zeros((nx + 1) * ny, np.int32), Z2, None, None, COEF, i2, s2,
                        precision=B.MIXED, share=half)
    half.close()
