"""Pins for oracle/quadrature.py against mathematics independent of it."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.quadrature import potential_integrals, radon7, tri_area


def test_radon7_exact_to_degree_5():
    # int over the unit right triangle of x^p y^q = p! q! / (p+q+2)!
    bary, w = radon7()
    x, y = bary[:, 1], bary[:, 2]
    for p in range(6):
        for q in range(6 - p):
            exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            got = 0.5 * np.sum(w * x ** p * y ** q)
            assert abs(got - exact) < 1e-15, (p, q)
    # degree 6 is NOT exact: the rule is not over-claimed
    assert abs(0.5 * np.sum(w * x ** 6) - math.factorial(6) / math.factorial(8)) > 1e-8


TRI = np.array([[0.1, 0.0, 0.0], [1.0, 0.2, 0.0], [0.3, 0.9, 0.0]])


def _num(fn):
    v0, v1, v2 = TRI
    A = tri_area(TRI)

    def f(t, s):
        return fn(v0 + s * (v1 - v0) + t * (v2 - v0))
    return 2 * A * integrate.dblquad(f, 0, 1, 0, lambda s: 1 - s, epsabs=1e-13, epsrel=1e-12)[0]


@pytest.mark.parametrize("r", [(0.4, 0.3, 0.5), (2.0, -0.5, 0.2), (1.5, 1.5, 0.0),
                               (0.4, 0.3, -0.05), (-0.3, 0.45, 0.0)])
def test_potential_integrals_match_adaptive_quadrature(r):
    r = np.array(r)
    I0, I1, Ig = potential_integrals(r, TRI)
    R = lambda p: np.linalg.norm(r - p)
    assert abs(I0 - _num(lambda p: 1 / R(p))) < 1e-11
    for c in range(2):
        assert abs(I1[c] - _num(lambda p: (p - r)[c] / R(p))) < 1e-11
    assert abs(I1[2]) < 1e-15                     # in-plane vector
    for c in range(3):
        assert abs(Ig[c] - _num(lambda p: -(r - p)[c] / R(p) ** 3)) < 1e-10


def test_gradient_is_derivative_of_potential():
    r = np.array([0.35, 0.25, 0.12])
    _, _, Ig = potential_integrals(r, TRI)
    hstep = 1e-5
    for c in range(3):
        e = np.zeros(3)
        e[c] = hstep
        fd = (potential_integrals(r + e, TRI)[0] - potential_integrals(r - e, TRI)[0]) / (2 * hstep)
        assert abs(fd - Ig[c]) < 1e-7


def test_normal_gradient_jumps_by_solid_angle():
    # above/below an interior point the normal component -> -/+ 2 pi, and the
    # in-plane point itself takes the principal value (normal part 0)
    rho = np.array([0.4, 0.3, 0.0])
    up = potential_integrals(rho + [0, 0, 1e-7], TRI)[2][2]
    dn = potential_integrals(rho - [0, 0, 1e-7], TRI)[2][2]
    pv = potential_integrals(rho, TRI)[2][2]
    assert abs(up + 2 * np.pi) < 1e-5 and abs(dn - 2 * np.pi) < 1e-5 and pv == 0.0
