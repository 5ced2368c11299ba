"""Lorenz-Mie scattering by homogeneous spheres and its expansion coefficients.

This is an input generator, not part of the DOM method. The paper obtains its
phase matrices from an external Mie code (Sec. 4); here the same kind of input is
produced from published Mie theory:

* Bohren & Huffman, "Absorption and Scattering of Light by Small Particles"
  (1983), Ch. 4: series coefficients a_n, b_n with the logarithmic derivative
  D_n(mx) from downward recurrence and the Riccati-Bessel functions from upward
  recurrence; amplitude functions S1, S2 from the angular functions pi_n, tau_n.
* Hansen & Travis (1974), Space Sci. Rev. 16: a lognormal size distribution
  parametrised by effective size r_eff and effective variance v_eff, with
  sigma_g^2 = ln(1 + v_eff) and r_g = r_eff / (1 + v_eff)^(5/2).
* The scattering matrix of randomly oriented spheres,
  F = [[a1, b1, 0, 0], [b1, a2, 0, 0], [0, 0, a3, b2], [0, 0, -b2, a4]],
  expanded in generalized spherical functions (Wigner d-functions d^l_{mn}):
  a1 = sum alpha1_l d^l_00, a4 = sum alpha4_l d^l_00,
  a2 + a3 = sum (alpha2 + alpha3)_l d^l_22, a2 - a3 = sum (alpha2 - alpha3)_l d^l_2,-2,
  b1 = -sum beta1_l d^l_02, b2 = -sum beta2_l d^l_02.
  The coefficients are projected by Gauss quadrature in cos(Theta) using the
  orthogonality  int d^l_mn d^l'_mn dx = 2/(2l+1) delta_ll'.

Stokes convention (shared with the rest of the project): for a beam with field
components (E1, E2) on a right-handed frame (e1, e2, k), I = |E1|^2 + |E2|^2,
Q = |E1|^2 - |E2|^2, U = 2 Re(E1 E2*), V = -2 Im(E1 E2*), time factor exp(-i w t).
In the scattering-plane frame the amplitude matrix is diag(S2, S1), which gives
a1 = a2 = (|S1|^2 + |S2|^2)/2, b1 = (|S2|^2 - |S1|^2)/2, a3 = a4 = Re(S2 S1*),
b2 = Im(S2 S1*).
"""
from __future__ import annotations

import math

import numpy as np


def n_terms(x: float) -> int:
    """Number of series terms, Wiscombe-style x + 4 x^(1/3) + 2 (Bohren & Huffman)."""
    return int(math.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))


def mie_coefficients_ab(m: complex, x: float, nmax: int | None = None):
    """Series coefficients a_n, b_n (n = 1..nmax) for refractive index m, size parameter x."""
    if nmax is None:
        nmax = n_terms(x)
    mx = m * x
    nmx = int(max(nmax, abs(mx))) + 16
    D = np.zeros(nmx + 1, dtype=complex)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    a = np.zeros(nmax, dtype=complex)
    b = np.zeros(nmax, dtype=complex)
    psi0, psi1 = math.cos(x), math.sin(x)
    chi0, chi1 = -math.sin(x), math.cos(x)
    xi1 = complex(psi1, -chi1)
    for n in range(1, nmax + 1):
        psi = (2 * n - 1) * psi1 / x - psi0
        chi = (2 * n - 1) * chi1 / x - chi0
        xi = complex(psi, -chi)
        ta = D[n] / m + n / x
        tb = m * D[n] + n / x
        a[n - 1] = (ta * psi - psi1) / (ta * xi - xi1)
        b[n - 1] = (tb * psi - psi1) / (tb * xi - xi1)
        psi0, psi1 = psi1, psi
        chi0, chi1 = chi1, chi
        xi1 = complex(psi1, -chi1)
    return a, b


def amplitude_functions(a, b, cos_theta):
    """S1, S2 at the given cos(Theta) values (Bohren & Huffman Sec. 4.4)."""
    mu = np.asarray(cos_theta, dtype=float)
    nmax = len(a)
    S1 = np.zeros(mu.shape, dtype=complex)
    S2 = np.zeros(mu.shape, dtype=complex)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    for n in range(1, nmax + 1):
        tau_cur = n * mu * pi_cur - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_cur + b[n - 1] * tau_cur)
        S2 += f * (a[n - 1] * tau_cur + b[n - 1] * pi_cur)
        pi_next = ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def efficiencies(a, b, x):
    """Extinction and scattering efficiencies from the series (Bohren & Huffman Eq. 4.61-4.62)."""
    n = np.arange(1, len(a) + 1)
    qext = 2.0 / x**2 * np.sum((2 * n + 1) * (a + b).real)
    qsca = 2.0 / x**2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return float(qext), float(qsca)


def scattering_matrix_elements(S1, S2):
    """(a1, a2, a3, a4, b1, b2) of one sphere from its amplitude functions (unnormalised)."""
    s1 = np.abs(S1) ** 2
    s2 = np.abs(S2) ** 2
    a1 = 0.5 * (s1 + s2)
    b1 = 0.5 * (s2 - s1)
    a3 = (S2 * np.conj(S1)).real
    b2 = (S2 * np.conj(S1)).imag
    return np.stack([a1, a1.copy(), a3, a3.copy(), b1, b2])


def _gauss_legendre(n: int):
    """Gauss-Legendre nodes/weights on [-1, 1] (numpy's routine; input-side only)."""
    return np.polynomial.legendre.leggauss(n)


def _wigner_d_family(lmax: int, m: int, n: int, x):
    """d^l_{mn}(arccos x) for l = 0..lmax by the three-term recurrence in l.

    Seed at l0 = max(|m|, |n|):
      d^{l0}_{mn} = xi 2^{-l0} sqrt((2 l0)! / (|m-n|! |m+n|!)) (1-x)^{|m-n|/2} (1+x)^{|m+n|/2},
      xi = 1 if n >= m else (-1)^(m-n);
    recurrence (l >= l0):
      l sqrt((l+1)^2-m^2) sqrt((l+1)^2-n^2) d^{l+1}
        = (2l+1)(l(l+1)x - mn) d^l - (l+1) sqrt(l^2-m^2) sqrt(l^2-n^2) d^{l-1}.
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
    logc = (-l0 * math.log(2.0) + 0.5 * (math.lgamma(2 * l0 + 1) - math.lgamma(abs(m - n) + 1)
                                          - math.lgamma(abs(m + n) + 1)))
    lg = np.full(x.shape, logc)
    with np.errstate(divide="ignore"):
        if m != n:
            lg = lg + 0.5 * abs(m - n) * np.log(np.maximum(1.0 - x, 0.0))
        if m != -n:
            lg = lg + 0.5 * abs(m + n) * np.log(np.maximum(1.0 + x, 0.0))
    out[l0] = xi * np.exp(lg)
    for l in range(l0, lmax):
        c_prev = (l + 1) * math.sqrt(l * l - m * m) * math.sqrt(l * l - n * n) if l > l0 else 0.0
        denom = l * math.sqrt((l + 1) ** 2 - m * m) * math.sqrt((l + 1) ** 2 - n * n)
        prev = out[l - 1] if l > l0 else 0.0
        out[l + 1] = ((2 * l + 1) * (l * (l + 1) * x - m * n) * out[l] - c_prev * prev) / denom
    return out


def expansion_coefficients(elements, x_nodes, w_nodes, L: int):
    """Project (a1, a2, a3, a4, b1, b2)(Theta) onto L generalized-spherical-function terms.

    Returns coef[L, 6] = (alpha1, alpha2, alpha3, alpha4, beta1, beta2), normalised
    so that alpha1_0 = 1 (phase function averaged over the sphere equals one).
    """
    a1, a2, a3, a4, b1, b2 = elements
    lmax = L - 1
    d00 = _wigner_d_family(lmax, 0, 0, x_nodes)
    d22 = _wigner_d_family(lmax, 2, 2, x_nodes)
    d2m2 = _wigner_d_family(lmax, 2, -2, x_nodes)
    d02 = _wigner_d_family(lmax, 0, 2, x_nodes)
    norm = 0.5 * np.sum(w_nodes * a1)
    coef = np.zeros((L, 6))
    for l in range(L):
        f = (2 * l + 1) / 2.0
        coef[l, 0] = f * np.sum(w_nodes * a1 * d00[l])
        coef[l, 3] = f * np.sum(w_nodes * a4 * d00[l])
        if l >= 2:
            s = f * np.sum(w_nodes * (a2 + a3) * d22[l])
            d = f * np.sum(w_nodes * (a2 - a3) * d2m2[l])
            coef[l, 1] = 0.5 * (s + d)
            coef[l, 2] = 0.5 * (s - d)
            coef[l, 4] = -f * np.sum(w_nodes * b1 * d02[l])
            coef[l, 5] = -f * np.sum(w_nodes * b2 * d02[l])
    return coef / norm


def lognormal_size_nodes(x_eff: float, v_eff: float, n_nodes: int = 48, width: float = 5.0):
    """Quadrature in ln(x) for the Hansen-Travis lognormal number distribution.

    Returns (x_i, w_i) with sum w_i = 1 (number weights), truncated at +-width sigma_g.
    """
    s2 = math.log(1.0 + v_eff)
    s = math.sqrt(s2)
    x_g = x_eff / (1.0 + v_eff) ** 2.5
    t, w = _gauss_legendre(n_nodes)
    lnx = math.log(x_g) + width * s * t
    dens = np.exp(-0.5 * ((lnx - math.log(x_g)) / s) ** 2)
    w = w * dens
    return np.exp(lnx), w / w.sum()


def polydisperse_coefficients(m: complex, x_eff: float, v_eff: float, L: int,
                              n_size: int = 48, n_theta: int | None = None):
    """Expansion coefficients [L, 6] of a lognormal ensemble of spheres.

    The ensemble scattering matrix is the number-weighted sum of the single-sphere
    matrices (all at the same wavelength, so the 1/k^2 factor is common).
    """
    xs, ws = lognormal_size_nodes(x_eff, v_eff, n_size)
    nmax = n_terms(float(xs.max()))
    if n_theta is None:
        n_theta = nmax + L + 8
    xt, wt = _gauss_legendre(n_theta)
    acc = np.zeros((6, n_theta))
    for x, w in zip(xs, ws):
        a, b = mie_coefficients_ab(m, float(x))
        S1, S2 = amplitude_functions(a, b, xt)
        acc += w * scattering_matrix_elements(S1, S2)
    return expansion_coefficients(acc, xt, wt, L)


def monodisperse_coefficients(m: complex, x: float, L: int, n_theta: int | None = None):
    """Expansion coefficients [L, 6] of a single sphere (used by the tests)."""
    a, b = mie_coefficients_ab(m, x)
    if n_theta is None:
        n_theta = len(a) + L + 8
    xt, wt = _gauss_legendre(n_theta)
    S1, S2 = amplitude_functions(a, b, xt)
    return expansion_coefficients(scattering_matrix_elements(S1, S2), xt, wt, L)
