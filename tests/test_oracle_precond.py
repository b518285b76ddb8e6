"""Pins for oracle/precond.py (the cell-grouped near-field preconditioner
of Sec. IV-A as restricted additive Schwarz).

* positions: every copy of a unique unknown (all RWGs merged by U_o) has its
  edge midpoint at the same point, so the first-copy position is the edge's;
* ownership partitions the unknowns and each unknown lies in its owner's
  subdomain for any margin >= 0;
* exactness cases that reduce to a plain inverse: one cell (S = everything),
  a margin so large that every subdomain is everything, and a matrix that is
  block diagonal on the ownership partition (then A[S,S]^{-1} restricted to
  the owned rows is the owned block's inverse).
A plausible mistake (a wrong owner, adding overlapped rows instead of keeping
only the owned ones, a transposed solve) breaks one of these.
"""
import numpy as np
import pytest

from oracle import lattice, precond
from oracle.mesh import box_mesh

LAM = 0.03
A = B = 0.5 * LAM
H = 0.25 * LAM


@pytest.fixture(scope="module")
def lat():
    box = box_mesh(A, B, H, 2)
    nx, ny = 3, 2
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, B)
    xy, owner = precond.unknown_positions(box, idx, nx, ny, A, B)
    return box, nx, ny, idx, sgn, nu, xy, owner


def test_all_copies_share_the_position(lat):
    box, nx, ny, idx, sgn, nu, xy, owner = lat
    E = box.n_rwg
    mid = 0.5 * (box.verts[box.edges[:, 0]] + box.verts[box.edges[:, 1]])
    for m in range(nx * ny):
        s = lattice.cell_shift(m % nx, m // nx, A, B)
        for k in range(2 * E):
            u = idx[m * 2 * E + k]
            assert np.allclose(xy[u], (mid[k % E] + s)[:2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("delta", [0.0, 0.3 * A / 2, 0.49 * A])
def test_ownership_partitions_and_owner_contains(lat, delta):
    box, nx, ny, idx, sgn, nu, xy, owner = lat
    subs = precond.subdomains(xy, owner, nx, ny, A, B, delta)
    count = np.zeros(nu, int)
    for m, (S, own) in enumerate(subs):
        count[S[own]] += 1
        assert np.all(owner[S[own]] == m)
    assert np.all(count == 1)
    # a larger margin only grows the subdomains
    big = precond.subdomains(xy, owner, nx, ny, A, B, delta + 0.1 * A)
    for (S, _), (S2, _) in zip(subs, big):
        assert set(S) <= set(S2)


def _rand(n, rng):
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * n ** 0.5 * np.eye(n)


def test_one_cell_is_the_exact_inverse():
    box = box_mesh(A, B, H, 2)
    idx, sgn, nu = lattice.overlap_map(box, 1, 1, A, B)
    xy, owner = precond.unknown_positions(box, idx, 1, 1, A, B)
    subs = precond.subdomains(xy, owner, 1, 1, A, B, 0.0)
    rng = np.random.default_rng(1)
    M = _rand(nu, rng)
    x = rng.standard_normal(nu) + 1j * rng.standard_normal(nu)
    assert np.linalg.norm(precond.ras_apply(M, subs, M @ x) - x) <= 1e-10 * np.linalg.norm(x)


def test_whole_lattice_margin_is_the_exact_inverse(lat):
    box, nx, ny, idx, sgn, nu, xy, owner = lat
    subs = precond.subdomains(xy, owner, nx, ny, A, B, 4 * A)
    assert all(len(S) == nu for S, _ in subs)
    rng = np.random.default_rng(2)
    M = _rand(nu, rng)
    x = rng.standard_normal(nu) + 1j * rng.standard_normal(nu)
    assert np.linalg.norm(precond.ras_apply(M, subs, M @ x) - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("delta", [0.0, 0.2 * A])
def test_block_diagonal_on_owners_is_exact(lat, delta):
    box, nx, ny, idx, sgn, nu, xy, owner = lat
    subs = precond.subdomains(xy, owner, nx, ny, A, B, delta)
    rng = np.random.default_rng(3)
    M = np.zeros((nu, nu), complex)
    for m in range(nx * ny):
        ids = np.nonzero(owner == m)[0]
        M[np.ix_(ids, ids)] = _rand(len(ids), rng)
    x = rng.standard_normal(nu) + 1j * rng.standard_normal(nu)
    assert np.linalg.norm(precond.ras_apply(M, subs, M @ x) - x) <= 1e-10 * np.linalg.norm(x)
    # with coupling added it is no longer exact, but still a contraction of
    # the error for this diagonally dominant case
    C = M + 0.05 * (rng.standard_normal((nu, nu)) + 1j * rng.standard_normal((nu, nu)))
    e = x - precond.ras_apply(C, subs, C @ x)
    assert 0 < np.linalg.norm(e) < 0.5 * np.linalg.norm(x)


@pytest.mark.parametrize("delta", [0.0, 0.3 * A])
def test_subdomain_matrix_is_the_dense_block(lat, delta):
    """The restricted assembly of A[S, S] equals the same block of the dense
    U_o^T [Z_eq + Z_o] U_o, for the cell subdomains and for an arbitrary
    scattered set of unknowns (copies in several non-adjacent cells)."""
    from paper_1911_04576_gb300 import workloads as W
    box, nx, ny, idx, sgn, nu, xy, owner = lat
    E = box.n_rwg
    Lt, Kt = W.random_tables(nx, ny, E, 31)
    Z = W.random_macromodels(2, 2 * E, 32)
    tmap = np.array([0, 1, 1, 0, 1, 0], dtype=np.int32)
    coef = (0.3j, 1.0, -1.0, 0.7j)
    Ad = lattice.assemble_from_tables(Lt, Kt, coef, Z, tmap, idx, sgn, nu, nx, ny)
    sets = [S for S, _ in precond.subdomains(xy, owner, nx, ny, A, B, delta)]
    sets.append(np.sort(np.random.default_rng(33).choice(nu, 40, replace=False)))
    for S in sets:
        As = precond.subdomain_matrix(S, Lt, Kt, coef, Z, tmap, idx, sgn, nx, ny)
        assert np.abs(As - Ad[np.ix_(S, S)]).max() <= 1e-12 * np.abs(Ad).max()
