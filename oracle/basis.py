"""Integrated Legendre basis and Gauss-Legendre rules (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

The paper discretises with the hierarchical p-FEM basis of integrated
Legendre polynomials (Sec. 2.1, Sec. 3.2): the degree-p basis contains every
mode of degree 1..p, which is what makes the coarse spaces nested
(Eq. hierarchicalFunctions).  The 1D modes on the reference interval
[-1, 1], in the local order used everywhere in this project, are

    N_0 = (1 - xi) / 2,   N_1 = (1 + xi) / 2                  (nodal modes)
    N_j = (P_j(xi) - P_{j-2}(xi)) / sqrt(4 j - 2),  j = 2..p  (bubble modes)

with P_j the Legendre polynomials.  With this scaling the bubble derivatives
are N_j' = sqrt((2j - 1) / 2) P_{j-1}, so the bubble block of the 1D
stiffness matrix is the identity (pinned in the tests against exact rational
polynomial integration).
"""
from __future__ import annotations

import functools
import math

import numpy as np


def legendre_all(n: int, x):
    """P_0..P_n at x (array), by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((n + 1,) + x.shape)
    out[0] = 1.0
    if n >= 1:
        out[1] = x
    for k in range(1, n):
        out[k + 1] = ((2 * k + 1) * x * out[k] - k * out[k - 1]) / (k + 1)
    return out


def basis_1d(p: int, xi):
    """Values and derivatives (d/dxi) of the p+1 modes at xi.
    Returns (N, dN), each of shape (p+1,) + xi.shape."""
    xi = np.asarray(xi, dtype=np.float64)
    P = legendre_all(max(p, 1), xi)
    N = np.empty((p + 1,) + xi.shape)
    dN = np.empty((p + 1,) + xi.shape)
    N[0] = 0.5 * (1.0 - xi)
    N[1] = 0.5 * (1.0 + xi)
    dN[0] = -0.5
    dN[1] = 0.5
    for j in range(2, p + 1):
        N[j] = (P[j] - P[j - 2]) / math.sqrt(4.0 * j - 2.0)
        dN[j] = math.sqrt((2.0 * j - 1.0) / 2.0) * P[j - 1]
    return N, dN


@functools.lru_cache(maxsize=None)
def _gauss_legendre(n: int):
    """Nodes are the roots of P_n, found by Newton's method from the classical
    initial guess cos(pi (i - 1/4) / (n + 1/2)); the positive half is
    computed and mirrored so the rule is exactly symmetric.  Weights are
    w = 2 / ((1 - x^2) P_n'(x)^2)."""
    if n < 1:
        raise ValueError("n >= 1")
    pos = []
    for i in range(1, n // 2 + 1):
        x = math.cos(math.pi * (i - 0.25) / (n + 0.5))
        for _ in range(100):
            p0, p1 = 1.0, x          # P_{k-1}, P_k, k = 1
            for k in range(1, n):
                p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
            dp = n * (x * p1 - p0) / (x * x - 1.0)
            dx = p1 / dp
            x = x - dx
            if abs(dx) <= 1e-17:
                break
        p0, p1 = 1.0, x
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        pos.append((x, 2.0 / ((1.0 - x * x) * dp * dp)))
    nodes = [-x for x, _ in pos] + ([0.0] if n % 2 else []) + [x for x, _ in reversed(pos)]
    weights = [w for _, w in pos]
    if n % 2:
        # middle weight: P_n'(0) from the recurrence
        x = 0.0
        p0, p1 = 1.0, x
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        wmid = [2.0 / (dp * dp)]
    else:
        wmid = []
    weights = weights + wmid + list(reversed(weights))
    return tuple(nodes), tuple(weights)


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1]: (nodes ascending, weights)."""
    x, w = _gauss_legendre(n)
    return np.array(x), np.array(w)


def element_1d_matrices(p: int, h: float):
    """1D stiffness and mass matrices of one cell of length h, computed by
    (p+1)-point Gauss quadrature (exact for these polynomial integrands).
    Returns (K1, M1)."""
    xq, wq = gauss_legendre(p + 1)
    N, dN = basis_1d(p, xq)
    K1 = (dN * wq) @ dN.T * (2.0 / h)
    M1 = (N * wq) @ N.T * (h / 2.0)
    return K1, M1
