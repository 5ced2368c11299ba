"""Generalized spherical functions for the order-m phase matrices (Sec. 2.B, Eqs. 9-10).

The paper defines A^m(mu, mu') = sum_{l=m}^{L-1} P_l^m(mu) B_l P_l^m(mu') with
4x4 "associated Legendre matrices" P_l^m but does not write them out (it cites
Siewert 1982). This module uses Siewert's form

    P_l^m(mu) = [[p, 0, 0, 0], [0, r, -t, 0], [0, -t, r, 0], [0, 0, 0, p]],
    p = d^l_{m,0}(theta),
    r = -(d^l_{m,2}(theta) + d^l_{m,-2}(theta)) / 2,
    t = -(d^l_{m,2}(theta) - d^l_{m,-2}(theta)) / 2,      mu = cos(theta),

with d^l_{mn} the Wigner d-functions (normalised generalized spherical
functions). They satisfy the parity relation of Eq. 10,
P_l^m(-mu) = (-1)^(l-m) D P_l^m(mu) D, D = diag(1, 1, -1, -1).

Two independent evaluations are provided:
  * `wigner_d_family`: upward three-term recurrence in l from the closed-form
    seed at l = max(|m|, |n|) (used by the A^m assembly);
  * `wigner_d_jacobi`: the Jacobi-polynomial closed form (scipy's Jacobi
    polynomials; used by the direct scattering matrix F(Theta)).

Pinned by tests: exact rational values from Wigner's factorial sum at small l,
scipy's associated Legendre functions (n = 0), the Jacobi closed form
(n = +-2), orthogonality under Gauss quadrature, the parity relation, and the
Fourier-synthesis check of the assembled phase matrix against the directly
rotated one.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_jacobi


def wigner_d_family(lmax: int, m: int, n: int, x) -> np.ndarray:
    """d^l_{mn}(arccos x) for l = 0..lmax (zeros for l < max(|m|, |n|)).

    Seed at l0 = max(|m|, |n|):
      d^{l0}_{mn}(x) = xi 2^{-l0} sqrt((2 l0)! / (|m-n|! |m+n|!))
                       (1 - x)^{|m-n|/2} (1 + x)^{|m+n|/2},
      xi = 1 if n >= m else (-1)^(m-n),
    computed in logarithms so that large m does not overflow.
    Recurrence for l >= l0 (with d^{l0-1} = 0):
      l sqrt((l+1)^2 - m^2) sqrt((l+1)^2 - n^2) d^{l+1}
        = (2l+1) (l(l+1) x - m n) d^l - (l+1) sqrt(l^2 - m^2) sqrt(l^2 - n^2) d^{l-1}.
    For m = n = 0 this is the Legendre recurrence, started from d^0 = 1, d^1 = x.
    """
    x = np.asarray(x, dtype=float)
    out = np.zeros((lmax + 1,) + x.shape)
    l0 = max(abs(m), abs(n))
    if l0 > lmax:
        return out
    if m == 0 and n == 0:
        out[0] = 1.0
        if lmax >= 1:
            out[1] = x
        for l in range(1, lmax):
            out[l + 1] = ((2 * l + 1) * x * out[l] - l * out[l - 1]) / (l + 1)
        return out
    xi = 1.0 if n >= m else (-1.0) ** (m - n)
    logc = -l0 * math.log(2.0) + 0.5 * (math.lgamma(2 * l0 + 1) - math.lgamma(abs(m - n) + 1)
                                        - math.lgamma(abs(m + n) + 1))
    # (1 - x)^0 = 1 at x = 1: add a logarithm only where its exponent is positive
    log_seed = np.full(x.shape, logc)
    with np.errstate(divide="ignore"):
        if m != n:
            log_seed = log_seed + 0.5 * abs(m - n) * np.log(np.clip(1.0 - x, 0.0, None))
        if m != -n:
            log_seed = log_seed + 0.5 * abs(m + n) * np.log(np.clip(1.0 + x, 0.0, None))
    out[l0] = xi * np.exp(log_seed)
    for l in range(l0, lmax):
        denom = l * math.sqrt((l + 1) ** 2 - m * m) * math.sqrt((l + 1) ** 2 - n * n)
        term = (2 * l + 1) * (l * (l + 1) * x - m * n) * out[l]
        if l > l0:
            term = term - (l + 1) * math.sqrt(l * l - m * m) * math.sqrt(l * l - n * n) * out[l - 1]
        out[l + 1] = term / denom
    return out


def wigner_d_jacobi(l: int, m: int, n: int, theta) -> np.ndarray:
    """d^l_{mn}(theta) from the Jacobi-polynomial closed form.

    With a = |n - m|, b = |n + m|, s = l - (a + b)/2 and xi = 1 if n >= m else (-1)^(m-n):
      d^l_{mn}(theta) = xi sqrt(s! (s+a+b)! / ((s+a)! (s+b)!))
                        sin(theta/2)^a cos(theta/2)^b P_s^{(a, b)}(cos theta).
    """
    theta = np.asarray(theta, dtype=float)
    if l < max(abs(m), abs(n)):
        return np.zeros_like(theta)
    a, b = abs(n - m), abs(n + m)
    s = l - (a + b) // 2
    xi = 1.0 if n >= m else (-1.0) ** (m - n)
    pref = math.exp(0.5 * (math.lgamma(s + 1) + math.lgamma(s + a + b + 1)
                           - math.lgamma(s + a + 1) - math.lgamma(s + b + 1)))
    return (xi * pref * np.sin(theta / 2.0) ** a * np.cos(theta / 2.0) ** b
            * eval_jacobi(s, a, b, np.cos(theta)))


def gsf_tables(m: int, L: int, mu):
    """(p, r, t)[l, k] for l = 0..L-1 at the cosines mu[k]; rows l < m are zero."""
    mu = np.asarray(mu, dtype=float)
    lmax = L - 1
    p = wigner_d_family(lmax, m, 0, mu)
    dp2 = wigner_d_family(lmax, m, 2, mu)
    dm2 = wigner_d_family(lmax, m, -2, mu)
    r = -0.5 * (dp2 + dm2)
    t = -0.5 * (dp2 - dm2)
    return p, r, t
