"""Double-Gauss quadrature (Sec. 2.B, Eq. 15).

The paper discretises the angular integral over [-1, 1] with Gauss nodes placed
separately on each hemisphere; every node mu_n is positive and the sign marks the
hemisphere. On [0, 1] the N Gauss-Legendre nodes are mu_n = (1 + x_n)/2 with
weights alpha_n = w_n / 2, so sum_n alpha_n = 1 and
  int_{-1}^{1} f(mu) dmu ~= sum_n alpha_n [f(mu_n) + f(-mu_n)],
exact for polynomials of degree <= 2N - 1.

Pinned by tests: agreement with numpy's leggauss, exact integration of
monomials up to degree 2N - 1.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre_01(N: int):
    """Nodes (ascending) and weights of the N-point Gauss-Legendre rule on [0, 1].

    Newton's method on P_N(x) from the Tricomi initial guess; P_N and P_N' by the
    three-term Legendre recurrence.
    """
    if N < 1:
        raise ValueError("N >= 1 required")
    x = np.empty(N)
    w = np.empty(N)
    for i in range(N):
        # i-th root counted from x = 1 downward
        z = math.cos(math.pi * (i + 0.75) / (N + 0.5))
        for _ in range(100):
            p0, p1 = 1.0, z
            for k in range(2, N + 1):
                p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
            dp = N * (z * p1 - p0) / (z * z - 1.0)
            dz = p1 / dp
            z -= dz
            if abs(dz) < 1e-16:
                break
        p0, p1 = 1.0, z
        for k in range(2, N + 1):
            p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
        dp = N * (z * p1 - p0) / (z * z - 1.0)
        x[i] = z
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp)
    order = np.argsort(x)
    x, w = x[order], w[order]
    return 0.5 * (1.0 + x), 0.5 * w
