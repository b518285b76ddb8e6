"""Physics pins of the oracle (fixed points named by the method, Sec. II-III).

* Empty box / empty lattice: the exact solution of Eq. final is the pair of
  incident-field equivalent currents J = n x H_inc, M = -n x E_inc (Eqs.
  Heq, Eeq) and nothing is scattered; the discrete solution's scattered far
  field must be small and shrink as the mesh is refined.  A sign error in
  any block (L, K, coefficients, U_o, excitation) gives O(1) scattering.
* PEC patch: the Schur complement (Eq. Zmacromodel) equals solving the
  unreduced system; a lossless cell obeys the optical theorem
  (scattered power = extinguished power) and reciprocity.
* GMRES agrees with dense LU.
* PEC sphere in one box: the macromodel chain (interior EFIE on the sphere,
  Schur complement, outer block, excitation, far field) reproduces the
  textbook Mie series for the bistatic RCS of a PEC sphere, to within the
  discretisation error, which shrinks as the box mesh is refined.
"""
import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn

from oracle import lattice, macromodel, operators, solve
from oracle.mesh import box_mesh, patch_mesh, sphere_mesh

LAM = 0.03
K0 = 2 * np.pi / LAM
A = B = 0.5 * LAM
H = 0.25 * LAM
COEF = (1j * K0, 1.0, -1.0, 1j * K0)
KHAT = np.array([0.0, 0.0, -1.0])
EHAT = np.array([1.0, 0.0, 0.0])


def _dirs(nth=19, nph=37):
    th = np.linspace(0, np.pi, nth)
    ph = np.linspace(0, 2 * np.pi, nph)
    TH, PH = np.meshgrid(th, ph)
    return np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)


def _lattice_solution(n, nx, ny, Ztypes, tmap):
    box = box_mesh(A, B, H, n)
    idx, sgn, nu = lattice.overlap_map(box, nx, ny, A, B)
    Ad = lattice.assemble_dense(box, nx, ny, A, B, K0, COEF, Ztypes, tmap, idx, sgn, nu)
    V = np.concatenate([operators.excitation(box, lattice.cell_shift(m % nx, m // nx, A, B),
                                             K0, KHAT, EHAT) for m in range(nx * ny)])
    Vt = lattice.scatter(V, idx, sgn, nu)
    x = solve.dense_solve(Ad, Vt)
    return box, Ad, Vt, x, idx, sgn, nu


def _scatter_ratio(box, nx, ny, Y):
    E = box.n_rwg
    rh = _dirs()
    F = 0
    FJ = 0
    for m in range(nx * ny):
        rad = operators.radiation_vectors(box, lattice.cell_shift(m % nx, m // nx, A, B), K0, rh)
        F = F + operators.far_field(rad, rh, K0, Y[m, :E], Y[m, E:])
        FJ = FJ + operators.far_field(rad, rh, K0, Y[m, :E], 0 * Y[m, E:])
    return np.abs(F).max() / np.abs(FJ).max()


def test_empty_box_scatters_nothing_and_converges():
    ratios = []
    for n in (2, 3):
        box = box_mesh(A, B, H, n)
        Z = macromodel.empty_box(box, K0)
        _, _, Vt, x, idx, sgn, nu = _lattice_solution(n, 1, 1, Z[None], np.array([0]))
        ratios.append(_scatter_ratio(box, 1, 1, x.reshape(1, -1)))
    assert ratios[0] < 0.03 and ratios[1] < 0.01 and ratios[1] < 0.6 * ratios[0]


def test_empty_lattice_with_merged_faces_scatters_nothing():
    n, nx, ny = 2, 2, 2
    box = box_mesh(A, B, H, n)
    Z = macromodel.empty_box(box, K0)
    box, Ad, Vt, x, idx, sgn, nu = _lattice_solution(n, nx, ny, Z[None], np.zeros(4, int))
    Y = lattice.gather(x, idx, sgn, nx * ny, 2 * box.n_rwg)
    assert _scatter_ratio(box, nx, ny, Y) < 0.03
    # GMRES (plain, restarted) reaches the LU solution
    xg, it, hist = solve.gmres(lambda v: Ad @ v, Vt, rtol=1e-12, restart=30)
    assert np.linalg.norm(xg - x) <= 1e-9 * np.linalg.norm(x)
    assert np.linalg.norm(Ad @ xg - Vt) <= 2e-12 * np.linalg.norm(Vt)


@pytest.mark.parametrize("n,npatch,tol_energy", [(2, 3, 0.03), (3, 4, 0.01)])
def test_pec_patch_macromodel(n, npatch, tol_energy):
    # the discretised lossless problem balances extinction and scattering up
    # to its discretisation error, which falls with the mesh: about 2.0 %,
    # 0.41 % and 0.21 % for n = 2, 3 and 4 quads per box face
    box = box_mesh(A, B, H, n)
    E = box.n_rwg
    sheet = patch_mesh(0.3 * LAM, 0.76e-3, npatch)
    Zt = macromodel.pec_patch(box, sheet, K0)
    Z0 = macromodel.empty_box(box, K0)        # outer self block B(0) = free-space S_eq operator
    V = operators.excitation(box, (0, 0, 0), K0, KHAT, EHAT)
    x = np.linalg.solve(Zt + Z0, V)
    # Schur step equals the unreduced solve (brute force)
    Zf, neq = macromodel.pec_sheet_system(box, sheet, K0)
    Zf[:neq, :neq] += Z0
    xf = np.linalg.solve(Zf, np.concatenate([V, np.zeros(sheet.n_rwg)]))
    assert np.linalg.norm(xf[:neq] - x) <= 1e-12 * np.linalg.norm(x)
    # reciprocity Z~^T = S Z~ S to quadrature accuracy
    S = np.concatenate([np.ones(E), -np.ones(E)])
    assert np.linalg.norm(Zt.T - S[:, None] * Zt * S[None, :]) <= 0.03 * np.linalg.norm(Zt)
    # optical theorem (lossless): sigma_sca = -(4 pi/k) Im[F(khat) . e*]  (e^{jwt})
    nth, nph = 40, 80
    th = (np.arange(nth) + 0.5) * np.pi / nth
    ph = np.arange(nph) * 2 * np.pi / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    rh = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    dW = (np.pi / nth) * (2 * np.pi / nph) * np.sin(TH).reshape(-1)
    rad = operators.radiation_vectors(box, (0, 0, 0), K0, rh)
    F = operators.far_field(rad, rh, K0, x[:E], x[E:])
    sca = np.sum(np.sum(np.abs(F) ** 2, -1) * dW)
    Ff = operators.far_field(operators.radiation_vectors(box, (0, 0, 0), K0, KHAT[None]),
                             KHAT[None], K0, x[:E], x[E:])[0]
    ext = -(4 * np.pi / K0) * np.imag(Ff @ EHAT)
    assert ext > 0 and abs(sca - ext) <= tol_energy * ext


def _mie_pec(x, mu):
    """Scattering amplitudes S1, S2 of a PEC sphere of size parameter x at
    cos(scattering angle) mu: the perfectly conducting limit of the Mie
    series (Bohren & Huffman 1983, Sec. 4.4), a_n = psi_n'/xi_n',
    b_n = psi_n/xi_n, psi_n = x j_n, xi_n = x h_n^(1)."""
    nmax = int(x + 4 * x ** (1 / 3) + 8)
    S1 = np.zeros_like(mu, dtype=complex)
    S2 = np.zeros_like(mu, dtype=complex)
    pi_prev, pi_cur = np.zeros_like(mu), np.ones_like(mu)     # pi_0, pi_1
    for n in range(1, nmax + 1):
        jn, yn = spherical_jn(n, x), spherical_yn(n, x)
        jd, yd = spherical_jn(n, x, True), spherical_yn(n, x, True)
        hn, hd = jn + 1j * yn, jd + 1j * yd
        an = (jn + x * jd) / (hn + x * hd)
        bn = (x * jn) / (x * hn)
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        c = (2 * n + 1) / (n * (n + 1))
        S1 += c * (an * pi_cur + bn * tau)
        S2 += c * (an * tau + bn * pi_cur)
        pi_prev, pi_cur = pi_cur, ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
    return S1, S2


def _sphere_rcs_db_error(n, sub, r=3.0e-3):
    """10 log10(sigma / sigma_Mie) in the E and H planes at 7 angles."""
    box = box_mesh(A, B, H, n)
    E = box.n_rwg
    sph = sphere_mesh(r, (0.0, 0.0, 0.5 * H), sub)
    Zt = macromodel.pec_patch(box, sph, K0)           # any PEC surface: EFIE rows, J columns
    Z0 = macromodel.empty_box(box, K0)
    V = operators.excitation(box, (0, 0, 0), K0, KHAT, EHAT)
    x = np.linalg.solve(Zt + Z0, V)
    th = np.radians([0.0, 30.0, 60.0, 90.0, 120.0, 150.0, 180.0])
    # incidence along -z: the scattering angle is pi - theta
    S1, S2 = _mie_pec(K0 * r, np.cos(np.pi - th))
    err = []
    for ph, S in ((0.0, S2), (0.5 * np.pi, S1)):          # E plane (x-z), H plane (y-z)
        rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
        F = operators.far_field(operators.radiation_vectors(box, (0, 0, 0), K0, rh), rh, K0, x[:E], x[E:])
        sig = 4 * np.pi * np.sum(np.abs(F) ** 2, -1)
        err.append(10 * np.log10(sig / (4 * np.pi / K0 ** 2 * np.abs(S) ** 2)))
    return np.abs(np.concatenate(err))


def test_mie_series_small_sphere_limit():
    # Rayleigh limit of a PEC sphere: backscatter sigma = 9 pi a^2 (ka)^4
    x = 0.05
    S1, S2 = _mie_pec(x, np.array([-1.0]))
    sig = 4 * np.pi / K0 ** 2 * abs(S1[0]) ** 2
    a = x / K0
    assert abs(sig / (9 * np.pi * a * a * x ** 4) - 1) < 0.01


def test_pec_sphere_matches_mie_series():
    """Sphere of radius 3 mm (ka = 0.63) at the centre of a box meshed
    n x n per face: within 2 dB (n = 2) and 1 dB (n = 3) of the Mie series at
    every angle of both planes, and closer on the finer box."""
    e2 = _sphere_rcs_db_error(2, 2)
    e3 = _sphere_rcs_db_error(3, 2)
    assert e2.max() < 2.0 and e3.max() < 1.0
    assert e3.max() < 0.75 * e2.max() and e3.mean() < e2.mean()


def test_bistatic_reciprocity():
    """Reciprocity of the scattering amplitude: for a plane wave travelling
    along k with polarisation e and the far field observed along r on
    polarisation q, q . F(r; k, e) = e . F(-k; -r, q).  The Galerkin system
    is symmetric up to the one-sided singular quadrature, so the identity
    holds to a few percent, better on the finer box; a sign or conjugation
    error in the excitation or the far field breaks it at O(1)."""
    def sph(th, ph):
        th, ph = np.radians(th), np.radians(ph)
        return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])

    k1, r1 = -sph(30, 20), sph(50, 110)
    e1 = np.cross(k1, [0, 0, 1])
    e1 /= np.linalg.norm(e1)
    q = np.cross(r1, [1, 0.3, 0])
    q /= np.linalg.norm(q)
    errs = []
    for n in (2, 3):
        box = box_mesh(A, B, H, n)
        E = box.n_rwg
        Z = macromodel.pec_patch(box, patch_mesh(0.3 * LAM, 0.76e-3, 3), K0) + macromodel.empty_box(box, K0)

        def amp(khat, ehat, rhat, pol):
            x = np.linalg.solve(Z, operators.excitation(box, (0, 0, 0), K0, khat, ehat))
            F = operators.far_field(operators.radiation_vectors(box, (0, 0, 0), K0, rhat[None]), rhat[None],
                                    K0, x[:E], x[E:])[0]
            return pol @ F

        a, b = amp(k1, e1, r1, q), amp(-r1, q, -k1, e1)
        errs.append(abs(a - b) / abs(a))
    assert errs[0] < 0.04 and errs[1] < 0.02 and errs[1] < 0.7 * errs[0]
