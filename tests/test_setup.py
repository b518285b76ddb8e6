"""The product's setup library (C++, integer index arithmetic) reproduces
the oracle's meshes and its geometric U_o map exactly (host only)."""
import os

import numpy as np
import pytest

from oracle import lattice
from oracle.mesh import box_mesh, patch_mesh


@pytest.fixture(scope="module")
def B():
    from paper_1911_04576_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


def _same_mesh(p, o):
    assert np.array_equal(p["tris"], o.tris)
    assert np.array_equal(p["edges"], o.edges)
    assert np.array_equal(p["tplus"], o.tplus) and np.array_equal(p["tminus"], o.tminus)
    assert np.array_equal(p["slot_rwg"], o.slot_rwg) and np.array_equal(p["slot_sgn"], o.slot_sgn)
    assert np.allclose(p["verts"], o.verts, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_box_mesh_matches_oracle(B, n):
    _same_mesh(B.emsurf_setup_box_mesh(0.015, 0.012, 0.0075, n), box_mesh(0.015, 0.012, 0.0075, n))


def test_box_mesh_with_z_levels(B):
    z = [0.0, 0.00076, 0.004, 0.0075]
    _same_mesh(B.emsurf_setup_box_mesh(0.015, 0.015, 0.0075, 3, z), box_mesh(0.015, 0.015, 0.0075, 3, z))


@pytest.mark.parametrize("n", [1, 3, 4])
def test_patch_mesh_matches_oracle(B, n):
    _same_mesh(B.emsurf_setup_patch_mesh(0.009, 0.00076, n), patch_mesh(0.009, 0.00076, n))


@pytest.mark.parametrize("n,nx,ny", [(1, 1, 1), (2, 2, 1), (2, 1, 3), (2, 3, 3), (3, 4, 2), (4, 3, 2), (1, 6, 5)])
def test_overlap_matches_geometric_oracle(B, n, nx, ny):
    a = 0.015
    idx, sgn, nu = B.emsurf_setup_overlap(n, nx, ny)
    oi, osg, onu = lattice.overlap_map(box_mesh(a, a, 0.0075, n), nx, ny, a, a)
    assert nu == onu
    assert np.array_equal(idx, oi) and np.array_equal(sgn, osg)


def test_setup_rejects_bad_sizes(B):
    for call in (lambda: B.emsurf_setup_box_mesh(1.0, 1.0, 1.0, 0),
                 lambda: B.emsurf_setup_patch_mesh(-1.0, 0.0, 2),
                 lambda: B.emsurf_setup_overlap(2, 0, 3)):
        with pytest.raises(B.EmsurfError) as e:
            call()
        assert e.value.status == B.EMSURF_EINVAL


@pytest.mark.parametrize("n,nx,ny", [(1, 2, 3), (2, 3, 2), (3, 1, 1)])
def test_unknown_positions_match_oracle(B, n, nx, ny):
    """Edge-midpoint positions of the unique unknowns (host, for the
    near-field preconditioner) equal the oracle's first-copy positions."""
    from oracle import precond
    a, b, h = 0.015, 0.012, 0.0075
    box = box_mesh(a, b, h, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, a, b)
    xy = B.emsurf_setup_unknown_xy(a, b, h, n, nx, ny, idx, nu)
    ref, _ = precond.unknown_positions(box, idx, nx, ny, a, b)
    assert np.allclose(xy, ref, rtol=0, atol=1e-15)


def test_unknown_positions_reject_bad_index(B):
    idx, sgn, nu = B.emsurf_setup_overlap(1, 2, 2)
    bad = idx.copy()
    bad[5] = nu
    with pytest.raises(B.EmsurfError):
        B.emsurf_setup_unknown_xy(0.015, 0.015, 0.0075, 1, 2, 2, bad, nu)


@pytest.mark.parametrize("n,side,pn,layers", [(2, 0.009, 3, 1), (3, 0.009, 4, 3), (4, 0.0135, 4, 3),
                                              (4, 0.0045, 3, 2), (3, 0.0, 4, 3), (4, -1.0, 4, 3)])
def test_slab_top_mesh_matches_oracle(B, n, side, pn, layers):
    """The slab-top interface (patch grid, graded rings, zipped band onto the
    footprint boundary; or the bare footprint grid) and its patch flags."""
    from oracle.macromodel import _bare_top
    from oracle.mesh import slab_top_mesh
    a, b, z = 0.015, 0.015, 0.00076
    p = B.emsurf_setup_slab_top_mesh(a, b, z, n, side, pn, layers)
    o, pec = slab_top_mesh(a, b, z, n, side, pn, layers) if side > 0 else _bare_top(a, b, z, n)
    _same_mesh(p, o)
    assert np.array_equal(p["on_patch"].astype(bool), pec)


def test_slab_zlevels_match_oracle(B):
    from oracle.mesh import slab_zlevels
    for n in (2, 3, 4, 6):
        assert np.allclose(B.emsurf_setup_slab_zlevels(0.0075, n, 0.00076), slab_zlevels(0.0075, n, 0.00076),
                           rtol=0, atol=1e-18)
    for bad in ((0.0075, 1, 0.00076), (0.0075, 3, 0.0), (0.0075, 3, 0.008)):
        with pytest.raises(B.EmsurfError):
            B.emsurf_setup_slab_zlevels(*bad)


@pytest.mark.parametrize("n,side,pn,layers", [(2, 0.009, 3, 2), (3, 0.0, 4, 3), (4, 0.0135, 4, 3)])
def test_slab_cell_unknown_counts_match_oracle(B, n, side, pn, layers):
    """The product's U plan eliminates as many interior unknowns as the
    oracle's U of Eq. incidence1 (rules 1-3 count J and M per edge kind)."""
    from oracle.macromodel import _bare_top
    from oracle.mesh import slab_region_meshes, slab_top_mesh, slab_zlevels
    a, h, t = 0.015, 0.0075, 0.00076
    z = slab_zlevels(h, n, t)
    box = box_mesh(a, a, h, n, z)
    top, pec = slab_top_mesh(a, a, t, n, side, pn, layers) if side > 0 else _bare_top(a, a, t, n)
    (air, _), (slab, _) = slab_region_meshes(box, n, top)
    # interior unknowns by the rules: rule 1 edges J + M, rule 3 edges J, rule 2 edges J per side
    npec = np.array([int(pec[top.tplus[e]]) + int(pec[top.tminus[e]]) for e in range(top.n_rwg)])
    expect = 2 * np.sum(npec == 0) + np.sum(npec == 1) + 2 * np.sum(npec == 2)
    ni, (ea, es) = B.emsurf_setup_slab_cell_counts(a, a, h, n, z, side, pn, layers)
    assert ni == expect and ea == air.n_rwg and es == slab.n_rwg


@pytest.mark.parametrize("a,b,n", [(0.015, 0.015, 2), (0.015, 0.012, 4), (0.015, 0.015, 3), (0.015, 0.015, 4)])
def test_box_mirrors_match_oracle(B, a, b, n):
    from oracle.mesh import box_mirrors
    perm, sign, mask = B.emsurf_setup_box_mirrors(a, b, n)
    ref = box_mirrors(box_mesh(a, b, 0.0075, n), a, b)
    assert sorted("xyd"[g] for g in range(3) if mask & (1 << g)) == sorted(ref)
    for g, name in enumerate("xyd"):
        if name in ref:
            assert np.array_equal(perm[g], ref[name][0]) and np.array_equal(sign[g], ref[name][1]), name


def _image(e, kx, ky, px, py):
    if e & 4:
        kx, ky = ky, kx
    if e & 2:
        ky = (py - ky) % py
    if e & 1:
        kx = (px - kx) % px
    return ky * px + kx


@pytest.mark.parametrize("px,py,G", [(5, 5, 8), (8, 8, 8), (32, 32, 8), (7, 9, 4), (10, 4, 4), (32, 32, 4),
                                     (1, 1, 8), (2, 3, 4)])
def test_mirror_orbits_partition_the_bins(B, px, py, G):
    rep, sb, se = B.emsurf_setup_mirror_orbits(px, py, G)
    seen = np.zeros(px * py, int)
    for s, r in enumerate(rep):
        ky, kx = divmod(int(r), px)
        orbit = {_image(e, kx, ky, px, py) for e in range(G)}
        assert min(orbit) == r                                  # the smallest bin represents
        got = [b for b in sb[s] if b >= 0]
        assert sorted(got) == sorted(orbit) and len(got) == len(orbit)
        for j, b in enumerate(sb[s]):
            if b >= 0:
                assert _image(int(se[s, j]), kx, ky, px, py) == b
                seen[b] += 1
    assert np.all(seen == 1)


def test_mirror_group_relation_on_the_oracle_spectrum(B):
    """The library's T_e of every group element, applied to the spectrum of
    the oracle's own tables (union-jack box, 3 x 3 lattice, 5 x 5 grid),
    gives the spectrum at the mirrored bin: B^(e k) = T_e B^(k) T_e^T."""
    from oracle import lattice
    a, h, n, nx = 0.015, 0.0075, 2, 3
    k0 = 2 * np.pi / 0.03
    box = box_mesh(a, a, h, n)
    E = box.n_rwg
    Lt, Kt = lattice.offset_tables(box, nx, nx, a, a, k0)
    perm, sign, mask = B.emsurf_setup_box_mirrors(a, a, n)
    assert mask == 7
    P = 5
    coef = (1j * k0, 1.0, -1.0, 1j * k0)

    def spec(T):
        S = np.zeros((P, P, E, E), complex)
        for dy in range(-(nx - 1), nx):
            for dx in range(-(nx - 1), nx):
                S[dy % P, dx % P] += T[dy + nx - 1, dx + nx - 1]
        return np.fft.fft2(S, axes=(0, 1))
    Ls, Ks = spec(Lt), spec(Kt)

    def full(ky, kx):
        return np.block([[coef[0] * Ls[ky, kx], coef[1] * Ks[ky, kx]], [coef[2] * Ks[ky, kx], coef[3] * Ls[ky, kx]]])
    idx, sg = B.emsurf_setup_mirror_group(perm, sign, 8)
    scale = max(np.abs(Ls).max(), np.abs(Ks).max())
    for e in range(8):
        T = np.zeros((2 * E, 2 * E))
        T[idx[e], np.arange(2 * E)] = sg[e]                    # T e_n = sign_n e_idx(n)
        for ky in range(P):
            for kx in range(P):
                b = _image(e, kx, ky, P, P)
                lhs = full(b // P, b % P)
                rhs = T @ full(ky, kx) @ T.T
                assert np.abs(lhs - rhs).max() <= 1e-12 * scale * max(abs(c) for c in coef), (e, kx, ky)
