"""Pins of the oracle's basis and quadrature rules.

The integrated Legendre modes (Sec. 2.1) are checked against exact rational
polynomial algebra written here from the Legendre recurrence, and the Gauss
rule against monomial integrals and numpy's independent Gauss-Legendre
routine."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.basis import basis_1d, element_1d_matrices, gauss_legendre


# ---- exact polynomial helpers (coefficient lists, lowest degree first) ----
def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pscale(a, s):
    return [s * c for c in a]


def pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pder(a):
    return [i * a[i] for i in range(1, len(a))] or [Fraction(0)]


def pint11(a):
    """Exact integral over [-1, 1]."""
    return sum(Fraction(2, k + 1) * c for k, c in enumerate(a) if k % 2 == 0)


def legendre_exact(n):
    P = [[Fraction(1)], [Fraction(0), Fraction(1)]]
    for k in range(1, n):
        xPk = [Fraction(0)] + P[k]
        P.append(padd(pscale(xPk, Fraction(2 * k + 1, k + 1)), pscale(P[k - 1], Fraction(-k, k + 1))))
    return P


def modes_exact(p):
    """(rational polynomial, float scale) per mode: N_j = scale * poly."""
    P = legendre_exact(max(p, 2))
    out = [([Fraction(1, 2), Fraction(-1, 2)], 1.0), ([Fraction(1, 2), Fraction(1, 2)], 1.0)]
    for j in range(2, p + 1):
        out.append((padd(P[j], pscale(P[j - 2], -1)), 1.0 / math.sqrt(4 * j - 2)))
    return out


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_rule_exact_on_monomials(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14 * max(1, n)
    # and it is the Gauss rule numpy computes independently
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, rtol=0, atol=1e-15)
    assert np.allclose(w, wr, rtol=0, atol=1e-14)
    assert np.all(np.diff(x) > 0) and np.array_equal(x, -x[::-1])


@pytest.mark.parametrize("p", range(1, 9))
def test_modes_match_exact_polynomials(p):
    ex = modes_exact(p)
    xi = np.linspace(-1, 1, 13)
    N, dN = basis_1d(p, xi)
    for j, (poly, s) in enumerate(ex):
        val = np.array([float(sum(c * Fraction(t) ** k for k, c in enumerate(poly))) for t in xi]) * s
        dp = pder(poly)
        der = np.array([float(sum(c * Fraction(t) ** k for k, c in enumerate(dp))) for t in xi]) * s
        assert np.allclose(N[j], val, atol=1e-13)
        assert np.allclose(dN[j], der, atol=1e-12)
    # bubbles vanish at both ends
    Ne, _ = basis_1d(p, np.array([-1.0, 1.0]))
    assert np.allclose(Ne[2:], 0.0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("h", [2.0, 0.125, 1.0 / 3.0])
def test_1d_element_matrices_closed_form(p, h):
    """K1 = (2/h) (1/2 [[1,-1],[-1,1]] (+) I_{p-1}) and M1 = (h/2) int N N,
    computed exactly."""
    K1, M1 = element_1d_matrices(p, h)
    Kx = np.zeros((p + 1, p + 1))
    Kx[:2, :2] = [[0.5, -0.5], [-0.5, 0.5]]
    for j in range(2, p + 1):
        Kx[j, j] = 1.0
    assert np.allclose(K1, (2.0 / h) * Kx, rtol=0, atol=1e-13 / h)
    ex = modes_exact(p)
    Mx = np.array([[float(pint11(pmul(a, b))) * sa * sb for (b, sb) in ex] for (a, sa) in ex])
    Kx2 = np.array([[float(pint11(pmul(pder(a), pder(b)))) * sa * sb for (b, sb) in ex] for (a, sa) in ex])
    assert np.allclose(Kx2, Kx, atol=1e-14)
    assert np.allclose(M1, (h / 2.0) * Mx, rtol=0, atol=1e-14 * h)
    # known entries: int N_0 N_2 = -1/sqrt(6), int N_0 N_3 = 1/(3 sqrt(10))
    if p >= 3:
        assert abs(Mx[0, 2] + 1 / math.sqrt(6)) < 1e-15
        assert abs(Mx[0, 3] - 1 / (3 * math.sqrt(10))) < 1e-15
        assert abs(Mx[1, 3] + 1 / (3 * math.sqrt(10))) < 1e-15
