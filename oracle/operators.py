"""Galerkin L and K operators, plane-wave excitation and far field (oracle).

Readings of the paper used here:

* time convention e^{jwt}, Green's function G = e^{-jkR} / (4 pi R); in a
  lossy region k = k0 sqrt(eps_r) is complex with Im k < 0 (Sec. II-B:
  every operator of region v takes k_v = w sqrt(mu0 eps_v)), so G decays;
* L[m,n] = int int [Lam_m . Lam_n - (div Lam_m)(div' Lam_n)/k^2] G dS' dS,
  the RWG-tested form of Eq. SIE_LOperator1;
* K[m,n] = int int Lam_m(r) . [grad_r G(r,r') x Lam_n(r')] dS' dS, the
  principal-value part of Eq. SIE_KOperator1.  The +X/2 term and the
  left-hand sides n x M, n x J of Eqs. SIE_TEFIE1_Composite/_Outer cancel
  pairwise when U^T Z U (Eq. mmm_mult) and Z_eq + Z_o (Eq. out3) add the two
  sides of each interface, so only p.v. operators are tabulated;
* with unknowns x_J = eta0*J and x_M = M, every homogeneous region v with
  relative permittivity eps_v contributes the block
      [[ j k0 L_v ,  K_v ], [ -K_v , j k0 eps_v L_v ]]
  to the tested EFIE (rows 1) and eta0-scaled MFIE (rows 2), so the outer
  coupling block of Eq. blockZo is B(d) = [[a L, b K], [g K, d L]] with
  (a, b, g, d) = (j k0, 1, -1, j k0);
* excitation V (Eq. out): rows 1 test E_inc, rows 2 test eta0*H_inc.

Pins: tests/test_oracle_operators.py (reciprocity, coplanar K = 0) and the
physics tests in tests/test_oracle_physics.py (empty box, optical theorem).
"""
import numpy as np

from .quadrature import potential_integrals, radon7, tri_area, tri_points

FOUR_PI = 4.0 * np.pi
_EPS3 = np.zeros((3, 3, 3))
_EPS3[0, 1, 2] = _EPS3[1, 2, 0] = _EPS3[2, 0, 1] = 1.0
_EPS3[0, 2, 1] = _EPS3[2, 1, 0] = _EPS3[1, 0, 2] = -1.0


def _green_far(R, k):
    e = np.exp(-1j * k * R)
    G = e / (FOUR_PI * R)
    gfac = -(1.0 + 1j * k * R) * e / (FOUR_PI * R ** 3)   # grad_r G = (r-r') * gfac
    return G, gfac


def _green_smooth(R, k):
    """Remainder after removing 1/(4 pi R): G_s and grad_r G_s = (r-r') * gfac."""
    kR = k * R
    small = np.abs(k) * R < 0.1
    Rs = np.where(small, 1.0, R)
    e = np.exp(-1j * k * Rs)
    Gs_closed = (e - 1.0) / (FOUR_PI * Rs)
    h_closed = (1.0 - (1.0 + 1j * k * Rs) * e) / Rs ** 2
    # series: (e^{-jkR}-1)/R = sum_{n>=1} (-jk)^n R^{n-1}/n!
    #         its d/dR        = sum_{n>=2} (-jk)^n (n-1) R^{n-2}/n!
    Gs_ser = np.zeros(R.shape, dtype=complex)
    h_ser = np.zeros(R.shape, dtype=complex)
    fact = 1.0
    for n in range(1, 12):
        fact *= n
        c = (-1j * k) ** n / fact
        Gs_ser = Gs_ser + c * R ** (n - 1)
        if n >= 2:
            h_ser = h_ser + c * (n - 1) * R ** (n - 2)
    Gs = np.where(small, Gs_ser / FOUR_PI, Gs_closed)
    h = np.where(small, h_ser, h_closed)
    with np.errstate(divide="ignore", invalid="ignore"):
        gfac = np.where(R > 0.0, h / (FOUR_PI * np.where(R > 0.0, R, 1.0)), 0.0)
    return Gs, gfac


def _slot_coef(mesh, tri):
    """RWG amplitude sgn*len/(2A) per (triangle, slot)."""
    A = tri_area(tri)
    return mesh.slot_sgn * mesh.slot_len() / (2.0 * A[:, None]), A


def _projector(mesh, coef):
    """Dense (E, 3T) matrix mapping slot integrals to RWG integrals."""
    T = len(mesh.tris)
    P = np.zeros((mesh.n_rwg, 3 * T))
    for t in range(T):
        for i in range(3):
            m = mesh.slot_rwg[t, i]
            if m >= 0:
                P[m, 3 * t + i] += coef[t, i]
    return P


def galerkin_LK(test, test_shift, src, src_shift, k, singular, chunk=8):
    """Galerkin blocks L, K (E_test x E_src) between two meshes.

    test/src: Mesh; *_shift: translation (3,) of each mesh; k: wavenumber of
    the homogeneous region; singular: if True the 1/R and grad(1/R) parts are
    integrated in closed form over every source triangle (used for touching
    boxes and inside a cell), else plain 7x7-point quadrature.  In the
    singular case point pairs closer than 1e-9 of the source triangle size
    count as coincident (remainder at its R -> 0 limit, no gradient term).
    """
    _, w = radon7()
    tt = test.tri_coords(test_shift)
    ts = src.tri_coords(src_shift)
    ct, At = _slot_coef(test, tt)
    cs, As = _slot_coef(src, ts)
    rq = tri_points(tt)                                   # (Tt,7,3)
    rs = tri_points(ts)                                   # (Ts,7,3)
    a = rq[:, :, None, :] - tt[:, None, :, :]             # (Tt,7,3slot,3)
    b = rs[:, :, None, :] - ts[:, None, :, :]             # (Ts,7,3slot,3)
    Wt = w[None, :] * At[:, None]                         # (Tt,7)
    Ws = w[None, :] * As[:, None]                         # (Ts,7)
    Tt, Ts = len(tt), len(ts)
    CL = np.zeros((Tt, 3, Ts, 3), dtype=complex)
    CK = np.zeros((Tt, 3, Ts, 3), dtype=complex)
    if singular:
        v0 = ts[:, 0, :]
        nrm = np.cross(ts[:, 1, :] - v0, ts[:, 2, :] - v0)
        ns = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
        sscale = np.maximum(np.linalg.norm(ts[:, 1] - v0, axis=-1),
                            np.linalg.norm(ts[:, 2] - v0, axis=-1))
    for t0 in range(0, Tt, chunk):
        sl = slice(t0, min(Tt, t0 + chunk))
        diff = rq[sl, None, :, None, :] - rs[None, :, None, :, :]   # (c,Ts,7,7,3)
        R = np.linalg.norm(diff, axis=-1)
        if singular:
            # coincident points (up to rounding) take the R -> 0 limit: G_s = -jk/(4 pi)
            # and no gradient term (its direction is undefined there)
            R = np.where(R <= 1e-9 * sscale[None, :, None, None], 0.0, R)
            G, gfac = _green_smooth(R, k)
        else:
            G, gfac = _green_far(R, k)
        WG = Wt[sl, None, :, None] * Ws[None, :, None, :] * G       # (c,Ts,7,7)
        Wg = (Wt[sl, None, :, None] * Ws[None, :, None, :] * gfac)[..., None] * diff
        # L: sum_qp W G [(a_qi . b_pj) - 4/k^2]
        ab = np.einsum("cqix,cspq,spjx->cisj", a[sl], WG.transpose(0, 1, 3, 2), b,
                       optimize=True)
        CL[sl] += ab - (4.0 / k ** 2) * WG.sum(axis=(2, 3))[:, None, :, None]
        # K: sum_qp W a_qi . (gradG x b_pj)
        CK[sl] += np.einsum("cqix,csqpy,spjz,xyz->cisj", a[sl], Wg, b, _EPS3,
                            optimize=True)
        if singular:
            r = rq[sl][:, :, None, :]                                  # (c,7,1,3)
            I0, I1, Ig = potential_integrals(r, ts[None, None, :, :, :])  # (c,7,Ts)
            d = np.sum(ns[None, None] * (r - v0[None, None]), axis=-1)
            d = np.where(np.abs(d) <= 1e-9 * sscale[None, None], 0.0, d)
            rho = r - d[..., None] * ns[None, None]                   # (c,7,Ts,3)
            # int (r'-p_j)/R = I1 + (rho - p_j) I0
            vecL = I1[:, :, :, None, :] + (rho[:, :, :, None, :] - ts[None, None, :, :, :]) \
                * I0[..., None, None]                                  # (c,7,Ts,3j,3)
            sL = np.einsum("cqix,cqsjx,cq->cisj", a[sl], vecL, Wt[sl]) \
                - (4.0 / k ** 2) * np.einsum("cqs,cq->cs", I0, Wt[sl])[:, None, :, None]
            CL[sl] += sL / FOUR_PI
            # int grad(1/R) x (r'-p_j) = Ig x (r - p_j)
            rp = r[:, :, :, None, :] - ts[None, None, :, :, :]        # (c,7,Ts,3j,3)
            cr = np.cross(Ig[:, :, :, None, :], rp)
            sK = np.einsum("cqix,cqsjx,cq->cisj", a[sl], cr, Wt[sl])
            CK[sl] += sK / FOUR_PI
    Pt = _projector(test, ct)
    Ps = _projector(src, cs)
    L = Pt @ CL.reshape(3 * Tt, 3 * Ts) @ Ps.T
    K = Pt @ CK.reshape(3 * Tt, 3 * Ts) @ Ps.T
    return L, K


def plane_wave(khat, ehat):
    khat = np.asarray(khat, float)
    ehat = np.asarray(ehat, float)
    return khat / np.linalg.norm(khat), ehat


def excitation(mesh, shift, k, khat, ehat):
    """V = [<Lam, E_inc>; <Lam, eta0 H_inc>] for E_inc = ehat e^{-jk khat.r}
    (Eq. out), |E_inc| = 1 V/m; returns (2E,) complex."""
    _, w = radon7()
    tri = mesh.tri_coords(shift)
    c, A = _slot_coef(mesh, tri)
    rq = tri_points(tri)
    ph = np.exp(-1j * k * (rq @ np.asarray(khat)))                  # (T,7)
    a = rq[:, :, None, :] - tri[:, None, :, :]                      # (T,7,3,3)
    hvec = np.cross(khat, ehat)
    sE = np.einsum("tqix,x,tq,q,t->ti", a, np.asarray(ehat), ph, w, A)
    sH = np.einsum("tqix,x,tq,q,t->ti", a, hvec, ph, w, A)
    P = _projector(mesh, c)
    return np.concatenate([P @ sE.reshape(-1), P @ sH.reshape(-1)])


def radiation_vectors(mesh, shift, k, rhat):
    """int Lam_m e^{jk rhat.r'} dS' for directions rhat (D,3) -> (D, E, 3)."""
    _, w = radon7()
    tri = mesh.tri_coords(shift)
    c, A = _slot_coef(mesh, tri)
    rq = tri_points(tri)
    ph = np.exp(1j * k * np.einsum("dx,tqx->dtq", rhat, rq))       # (D,T,7)
    a = rq[:, :, None, :] - tri[:, None, :, :]
    s = np.einsum("tqix,dtq,q,t->dtix", a, ph, w, A)               # (D,T,3,3)
    P = _projector(mesh, c)
    D = len(rhat)
    return np.einsum("mj,djx->dmx", P, s.reshape(D, -1, 3))


def far_field(rad, rhat, k, xJ, xM):
    """Far-field pattern F with E ~ F e^{-jkr}/r from currents x_J = eta0 J,
    x_M = M (Sec. III-D: fields radiated through the EFIE/MFIE operators).
    rad: (D,E,3) radiation vectors of one box already phased; xJ, xM: (E,)."""
    N = np.einsum("dmx,m->dx", rad, xJ)
    Lm = np.einsum("dmx,m->dx", rad, xM)
    Nperp = N - np.sum(rhat * N, axis=-1, keepdims=True) * rhat
    return -(1j * k / FOUR_PI) * (Nperp - np.cross(rhat, Lm))
