"""Triangle quadrature and closed-form potential integrals (oracle).

The paper names no quadrature rule (Sec. II-B and III-B only say the
operators are discretised with RWG testing).  The reading used throughout:

* every regular integral over a flat triangle uses the 7-point, degree-5
  Radon rule (the rule Dunavant lists as degree 5);
* for triangle pairs of touching boxes (and inside one cell) the 1/R and
  grad(1/R) parts of the Green's function are integrated over the source
  triangle in closed form (Wilton et al., IEEE TAP 1984; Graglia, IEEE TAP
  1993), the smooth remainder by the same 7-point rule.

Pins (tests/test_oracle_quadrature.py): the rule integrates all monomials of
degree <= 5 exactly; the three closed forms match adaptive SciPy integration
and finite differences of one another.
"""
import numpy as np


def radon7():
    """Return (barycentric points (7,3), weights (7,)) with weights summing to 1."""
    s15 = np.sqrt(15.0)
    a1, b1 = (6.0 - s15) / 21.0, (9.0 + 2.0 * s15) / 21.0
    a2, b2 = (6.0 + s15) / 21.0, (9.0 - 2.0 * s15) / 21.0
    w1, w2 = (155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0
    bary = np.array([
        [1 / 3, 1 / 3, 1 / 3],
        [b1, a1, a1], [a1, b1, a1], [a1, a1, b1],
        [b2, a2, a2], [a2, b2, a2], [a2, a2, b2],
    ])
    w = np.array([9.0 / 40.0, w1, w1, w1, w2, w2, w2])
    return bary, w


def tri_points(tri):
    """Quadrature points of triangles ``tri`` (...,3,3) -> (...,7,3)."""
    bary, _ = radon7()
    return np.einsum("qv,...vx->...qx", bary, tri)


def tri_area(tri):
    e1 = tri[..., 1, :] - tri[..., 0, :]
    e2 = tri[..., 2, :] - tri[..., 0, :]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=-1)


def _edge_log(lp, lm, Rp, Rm, R02):
    """ln((R+ + l+)/(R- + l-)) = integral of 1/R along one edge, in the form
    that avoids cancellation for the position of the projected point."""
    with np.errstate(divide="ignore", invalid="ignore"):
        fa = np.log((Rp + lp) / (Rm + lm))
        fb = np.log((Rm - lm) / (Rp - lp))
        fc = np.log((Rp + lp) * (Rm - lm) / R02)
    return np.where(lm >= 0.0, fa, np.where(lp <= 0.0, fb, fc))


def potential_integrals(r, tri):
    """Closed-form integrals over a flat source triangle.

    r:   observation points (...,3); tri: source triangles (...,3,3), broadcast.
    Returns (I0, I1, Ig):
      I0 = int_T 1/R dS'                 (...)
      I1 = int_T (rho' - rho)/R dS'      (...,3)  rho = projection of r on T's plane
      Ig = int_T grad_r (1/R) dS'        (...,3)  principal value when r is in T's plane
    A point whose distance to the plane is below 1e-9 of the longer of the
    edges v0v1, v0v2 counts as in the plane.
    """
    v0, v1, v2 = tri[..., 0, :], tri[..., 1, :], tri[..., 2, :]
    nrm = np.cross(v1 - v0, v2 - v0)
    n = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
    d = np.sum(n * (r - v0), axis=-1)
    # points in the triangle's plane up to rounding take the principal value
    scale = np.maximum(np.linalg.norm(v1 - v0, axis=-1), np.linalg.norm(v2 - v0, axis=-1))
    d = np.where(np.abs(d) <= 1e-9 * scale, 0.0, d)
    rho = r - d[..., None] * n
    ad = np.abs(d)
    I0 = 0.0
    I1 = 0.0
    fsum_u = 0.0
    bsum = 0.0
    verts = (v0, v1, v2)
    for i in range(3):
        a, b = verts[i], verts[(i + 1) % 3]
        le = np.linalg.norm(b - a, axis=-1)
        lh = (b - a) / le[..., None]
        u = np.cross(lh, n)                      # in-plane outward edge normal
        lp = np.sum((b - rho) * lh, axis=-1)
        lm = np.sum((a - rho) * lh, axis=-1)
        t = np.sum((a - rho) * u, axis=-1)       # signed distance rho -> edge line
        R02 = t * t + d * d
        Rp = np.sqrt(R02 + lp * lp)
        Rm = np.sqrt(R02 + lm * lm)
        f = _edge_log(lp, lm, Rp, Rm, R02)
        beta = (np.arctan2(t * lp, R02 + ad * Rp)
                - np.arctan2(t * lm, R02 + ad * Rm))
        I0 = I0 + t * f - ad * beta
        I1 = I1 + 0.5 * u * (R02 * f + lp * Rp - lm * Rm)[..., None]
        fsum_u = fsum_u + u * f[..., None]
        bsum = bsum + beta
    Ig = -n * (np.sign(d) * bsum)[..., None] - fsum_u
    return I0, I1, Ig
