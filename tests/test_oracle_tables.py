"""Pins of the oracle's quadrature, generalized spherical functions and phase matrices.

Each test checks the oracle against something other than itself: exact rational
values, library routines for special cases, closed forms and geometric
invariants (Sec. 2.B, Eqs. 5-10, 15).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import lpmv

import oracle as O
from oracle.gsf import wigner_d_family, wigner_d_jacobi
from vrte_inputs import rayleigh_coefficients
from vrte_inputs.mie import monodisperse_coefficients


# ---------------------------------------------------------------- quadrature (Eq. 15)
@pytest.mark.parametrize("N", [1, 2, 3, 8, 32, 64])
def test_gauss_nodes_match_library_and_integrate_exactly(N):
    mu, a = O.gauss_legendre_01(N)
    x, w = np.polynomial.legendre.leggauss(N)
    assert np.allclose(mu, 0.5 * (1 + x), atol=1e-15, rtol=0)
    assert np.allclose(a, 0.5 * w, atol=5e-15, rtol=0)
    assert abs(a.sum() - 1.0) < 1e-14
    # exact for degree <= 2N - 1 on [0, 1]: int mu^k = 1/(k+1)
    for k in range(2 * N):
        assert abs(np.sum(a * mu**k) - 1.0 / (k + 1)) < 1e-13


# ---------------------------------------------------------------- Wigner d (Eqs. 9-10)
def _wigner_exact(j, mp, m):
    """d^j_{mp,m}(theta) from Wigner's factorial sum, evaluated exactly.

    theta is chosen with cos(theta/2) = 3/5, sin(theta/2) = 4/5 (a Pythagorean
    angle), so the alternating sum is an exact Fraction; only the common square
    root of the factorial product is taken in floating point.
    """
    c = Fraction(3, 5)
    s = Fraction(4, 5)
    total = Fraction(0)
    for k in range(0, 2 * j + 2):
        a, b, cc = j + m - k, j - k - mp, k - m + mp
        if a < 0 or b < 0 or cc < 0:
            continue
        den = math.factorial(a) * math.factorial(k) * math.factorial(b) * math.factorial(cc)
        total += Fraction((-1) ** (k - m + mp), den) * c ** (2 * j - 2 * k + m - mp) * s ** (2 * k - m + mp)
    # the square root of the factorial product is common to every term
    num2 = (math.factorial(j + mp) * math.factorial(j - mp) * math.factorial(j + m) * math.factorial(j - m))
    return float(total) * math.sqrt(num2)


@pytest.mark.parametrize("m,n", [(0, 0), (0, 2), (0, -2), (1, 2), (1, -2), (2, 2), (2, -2),
                                 (3, 0), (3, 2), (3, -2), (6, 2), (6, -2)])
def test_recurrence_matches_wigner_factorial_sum(m, n):
    theta = 2 * math.acos(3 / 5)
    x = math.cos(theta)
    fam = wigner_d_family(16, m, n, np.array([x]))[:, 0]
    for l in range(17):
        ref = _wigner_exact(l, m, n) if l >= max(abs(m), abs(n)) else 0.0
        assert abs(fam[l] - ref) < 1e-13 * max(1.0, abs(ref)), (l, fam[l], ref)
        assert abs(wigner_d_jacobi(l, m, n, theta) - ref) < 1e-13 * max(1.0, abs(ref))


def test_n0_family_is_normalised_associated_legendre():
    x = np.linspace(-0.999, 0.999, 37)
    for m in [0, 1, 4, 17, 60]:
        fam = wigner_d_family(127, m, 0, x)
        for l in range(m, 128, 7):
            norm = math.exp(0.5 * (math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
            ref = norm * lpmv(m, l, x)
            # d^l_{m0} = sqrt((l-m)!/(l+m)!) P_l^m with the Condon-Shortley phase, as in scipy's lpmv
            assert np.allclose(fam[l], ref, atol=1e-12, rtol=1e-9), (m, l)


@pytest.mark.parametrize("m", [0, 1, 2, 5, 40, 100])
def test_recurrence_matches_jacobi_form_high_degree(m):
    x = np.cos(np.linspace(0.01, 3.13, 23))
    th = np.arccos(x)
    for n in (2, -2):
        fam = wigner_d_family(127, m, n, x)
        for l in range(max(m, 2), 128, 9):
            ref = wigner_d_jacobi(l, m, n, th)
            assert np.allclose(fam[l], ref, atol=1e-11, rtol=1e-8), (m, n, l)


def test_orthogonality_under_gauss_quadrature():
    mu, a = O.gauss_legendre_01(64)
    x = np.concatenate([mu, -mu])
    w = np.concatenate([a, a])
    for (m, n) in [(0, 0), (3, 0), (0, 2), (5, 2), (7, -2)]:
        fam = wigner_d_family(60, m, n, x)
        G = (fam * w[None, :]) @ fam.T
        l0 = max(abs(m), abs(n))
        for l in range(l0, 61):
            for lp in range(l0, 61):
                ref = 2.0 / (2 * l + 1) if l == lp else 0.0
                assert abs(G[l, lp] - ref) < 1e-13


def test_parity_relation_eq10():
    mu = np.array([0.13, 0.5, 0.91])
    D = np.diag([1.0, 1.0, -1.0, -1.0])
    for m in [0, 1, 3, 8]:
        P = O.P_matrices(m, 20, mu)
        Pm = O.P_matrices(m, 20, -mu)
        for l in range(m, 20):
            for k in range(3):
                assert np.allclose(Pm[l, k], (-1) ** (l - m) * D @ P[l, k] @ D, atol=1e-14)


# ---------------------------------------------------------------- phase matrices (Eqs. 5-9)
def test_rayleigh_scattering_matrix_closed_form():
    c = rayleigh_coefficients()
    for ct in np.linspace(-1, 1, 9):
        F = O.scattering_matrix(c, ct)
        ref = np.array([[0.75 * (1 + ct**2), -0.75 * (1 - ct**2), 0, 0],
                        [-0.75 * (1 - ct**2), 0.75 * (1 + ct**2), 0, 0],
                        [0, 0, 1.5 * ct, 0], [0, 0, 0, 1.5 * ct]])
        assert np.allclose(F, ref, atol=1e-14)


def _random_coef(rng, L):
    c = rng.normal(size=(L, 6)) * 0.4
    c[0] = [1.0, 0.0, 0.0, rng.normal(), 0.0, 0.0]
    c[1, [1, 2, 4, 5]] = 0.0
    return c


def test_fourier_synthesis_equals_rotated_phase_matrix():
    """P2: sum_m sum_k Phi_k^m A^m D_k (Eqs. 6-9) equals L(beta) F L(alpha) built from vectors."""
    rng = np.random.default_rng(11)
    for coef in [rayleigh_coefficients(), _random_coef(rng, 9),
                 monodisperse_coefficients(1.5 + 0.01j, 2.5, 20)]:
        for _ in range(6):
            mu_s, mu_i = rng.uniform(-1, 1, 2)
            dphi = rng.uniform(0, 2 * math.pi)
            Zs = O.fourier_synthesis_phase(coef, mu_s, mu_i, dphi)
            Zd = O.phase_matrix_direct(coef, mu_s, dphi, mu_i, 0.0)
            assert np.abs(Zs - Zd).max() < 1e-12 * np.abs(Zd).max()


def test_direct_phase_matrix_invariants():
    """Reciprocity Z(-n_i <- -n_s) = Q Z^T Q (Q = diag(1,1,-1,1)), mirror symmetry, in-plane = F."""
    rng = np.random.default_rng(5)
    coef = _random_coef(rng, 7)
    Q = np.diag([1.0, 1.0, -1.0, 1.0])
    D34 = np.diag([1.0, 1.0, -1.0, -1.0])
    for _ in range(6):
        mu, mup = rng.uniform(-1, 1, 2)
        phi, phip = rng.uniform(0, 2 * math.pi, 2)
        Z = O.phase_matrix_direct(coef, mu, phi, mup, phip)
        Zr = O.phase_matrix_direct(coef, -mup, phip + math.pi, -mu, phi + math.pi)
        assert np.allclose(Zr, Q @ Z.T @ Q, atol=1e-13)
        Zm = O.phase_matrix_direct(coef, mu, -phi, mup, -phip)
        assert np.allclose(Zm, D34 @ Z @ D34, atol=1e-13)
    ct = 0.3 * -0.5 + math.sqrt(1 - 0.09) * math.sqrt(1 - 0.25)
    assert np.allclose(O.phase_matrix_direct(coef, 0.3, 0.0, -0.5, 0.0),
                       O.scattering_matrix(coef, ct), atol=1e-14)


def test_A_matrix_symmetries():
    """A^m(-mu, -mu') = D A^m D and A^m(-mu, mu') = D A^m(mu, -mu') D, from Eq. 10."""
    rng = np.random.default_rng(2)
    coef = _random_coef(rng, 12)
    mu = np.array([0.2, 0.7])
    mup = np.array([0.4, 0.95, 0.05])
    D = np.diag([1.0, 1.0, -1.0, -1.0])
    for m in [0, 2, 5]:
        A = O.A_matrix(m, coef, mu, mup)
        Amm = O.A_matrix(m, coef, -mu, -mup)
        Amp = O.A_matrix(m, coef, -mu, mup)
        Apm = O.A_matrix(m, coef, mu, -mup)
        assert np.allclose(Amm, D @ A @ D, atol=1e-13)
        assert np.allclose(Amp, D @ Apm @ D, atol=1e-13)


def test_tables_at_the_poles():
    """x = +-1 (normal incidence/exit): d^l_{mn}(0) = delta_mn, d^l_{mn}(pi) = (-1)^(l+m) delta_{m,-n}."""
    for m in range(0, 5):
        for n in (0, 2, -2):
            fam = wigner_d_family(12, m, n, np.array([1.0, -1.0]))
            assert np.all(np.isfinite(fam))
            for l in range(max(abs(m), abs(n)), 13):
                assert abs(fam[l, 0] - (1.0 if m == n else 0.0)) < 1e-14
                assert abs(fam[l, 1] - ((-1.0) ** (l + m) if m == -n else 0.0)) < 1e-14
    c = monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)
    A1 = O.A_matrix(0, c, [1.0], [0.4])
    A2 = O.A_matrix(0, c, [1.0 - 1e-12], [0.4])
    assert np.all(np.isfinite(A1)) and np.abs(A1 - A2).max() < 1e-9
