"""Pins of the oracle's per-order DOM solution and BRDF (Sec. 2.C-2.D, Eqs. 12-54).

Every check here is independent of the oracle's own eigen path: the ODE itself,
a matrix-exponential propagator, the exact discrete flux balance, the
single-scattering closed form built from the directly rotated phase matrix,
Chandrasekhar's H-function, reciprocity, and degenerate limits.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.optimize import brentq

import oracle as O
from oracle.dom import _stack_matrix
from vrte_inputs import angle_grids, rayleigh_coefficients
from vrte_inputs.mie import monodisperse_coefficients


@pytest.fixture(scope="module")
def mie_coef():
    return monodisperse_coefficients(1.5 + 0.01j, 3.0, 24)


def _solve(coef, omega, tau0, N, mu0_ext, n, m=0):
    nodes = O.gauss_legendre_01(N)
    beam = O.fresnel_beam_in(mu0_ext, n)
    R = O.fresnel_internal_reflection(nodes[0], n) if n > 1 else None
    return O.solve_order(m, coef, omega, tau0, N, O.snell_mu(mu0_ext, n), beam, R, nodes)


@pytest.mark.parametrize("n", [1.0, 1.5])
@pytest.mark.parametrize("m", [0, 1, 4])
def test_ode_and_boundary_residuals(mie_coef, n, m):
    """P3: the nodal field satisfies Eq. 15 (our sign reading) and both boundary conditions."""
    sol = _solve(mie_coef[:16], 0.93, 1.7, 6, np.array([0.35, 0.8]), n, m)
    rng = np.random.default_rng(m)
    for tau in rng.uniform(0, sol.tau0, 4):
        u = sol.nodal(tau)
        du = sol.nodal_derivative(tau)
        src = sol.q * np.exp(-tau / sol.rhs_mu0)[None, :]
        res = sol.m8[:, None] * du - (u - 0.5 * sol.omega * (sol.calA * sol.w8[None, :]) @ u - src)
        assert np.abs(res).max() < 1e-12 * max(1.0, np.abs(u).max())
    N4 = 4 * sol.N
    u0, u1 = sol.nodal(0.0), sol.nodal(sol.tau0)
    assert np.abs(u0[N4:] - sol.R @ u0[:N4]).max() < 1e-13
    assert np.abs(u1[:N4]).max() < 1e-13


@pytest.mark.parametrize("n", [1.0, 1.5])
def test_matrix_exponential_brute_force(mie_coef, n):
    """P9: nodal top radiance from expm of the augmented 8N+1 system (no eigen solve)."""
    coef = mie_coef[:8]
    for m in [0, 2]:
        sol = _solve(coef, 0.9, 1.3, 3, np.array([0.6]), n, m)
        N4 = 4 * sol.N
        for col in range(4):
            s = -(sol.q[:, col] / sol.m8)
            aug = np.zeros((8 * sol.N + 1, 8 * sol.N + 1))
            aug[:-1, :-1] = sol.T
            aug[:-1, -1] = s
            aug[-1, -1] = -1.0 / sol.rhs_mu0[col]
            P = expm(aug * sol.tau0)
            # u(0) = [x; R x], unknown x = u_up(0); bottom: (P11 u(0) + P12)_up = 0
            E = np.vstack([np.eye(N4), sol.R])
            Amat = P[:N4, :-1] @ E
            x = np.linalg.solve(Amat, -P[:N4, -1])
            assert np.abs(x - sol.nodal(0.0)[:N4, col]).max() < 1e-11 * max(1e-3, np.abs(x).max())


@pytest.mark.parametrize("n", [1.0, 1.5])
@pytest.mark.parametrize("omega", [0.9, 1 - 1e-6, 1 - 1e-9])
def test_flux_balance_exact(mie_coef, n, omega):
    """P4: discrete energy balance of the m = 0 I-row, beam + diffuse, for any omega.

    mu0 I0' (1 - e^{-tau0/mu0}) + F_net(tau0) - F_net(0)
        = (1 - omega) int_0^tau0 [pi sum alpha I_0 + I0' e^{-tau/mu0}] dtau,
    F_net = pi sum_{s,i} alpha_i (s mu_i) I^0_0. At omega -> 1 both sides vanish:
    reflection + transmission = 1 (requires L <= 2N, satisfied here).
    """
    coef = mie_coef[:16]
    sol = _solve(coef, omega, 2.0, 8, np.array([0.3, 0.77]), n)
    comp0 = np.arange(0, 8 * sol.N, 4)
    mus, w = sol.m8, sol.w8

    def fnet(u):
        return math.pi * np.sum((w * mus)[comp0, None] * u[comp0], axis=0)

    I0 = np.concatenate([sol.beam[i][0] for i in range(sol.mu0.size)])
    mu0 = sol.rhs_mu0
    beam_abs = mu0 * I0 * -np.expm1(-sol.tau0 / mu0)
    lhs = beam_abs + fnet(sol.nodal(sol.tau0)) - fnet(sol.nodal(0.0))
    ui = sol.nodal_integral()
    rhs = (1 - omega) * (math.pi * np.sum(w[comp0, None] * ui[comp0], axis=0) + I0 * mu0 * -np.expm1(-sol.tau0 / mu0))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(beam_abs).max()
    if omega > 1 - 1e-8:
        # conservation: what entered leaves through top or bottom
        assert np.abs(lhs).max() < 1e-8 * np.abs(beam_abs).max()


@pytest.mark.parametrize("n", [1.0, 1.5])
def test_single_scattering_limit(mie_coef, n):
    """P1: tau0 -> 0 reproduces omega tau0 Z / (4 pi mu mu0) from the rotated phase matrix.

    The DOM result minus the exact single-scatter term is O(tau0) relative; the
    ratio at two thicknesses a decade apart checks that the difference is that
    physical correction and not a convention error.
    """
    mu_in, mu_out, dphi = angle_grids(3, 4, 5)
    errs = []
    for t0 in (1e-6, 1e-7):
        F = O.brdf(mie_coef, 0.9, t0, n, 8, 24, mu_in, mu_out, dphi)
        Fs = O.single_scatter_brdf(mie_coef, 0.9, t0, n, mu_in, mu_out, dphi)
        errs.append(np.abs(F - Fs).max() / np.abs(Fs).max())
    assert errs[0] < 2e-5
    assert 8.0 < errs[0] / errs[1] < 12.0


def _chandrasekhar_H(omega, mu_nodes, alpha, mu):
    """H-function of the N-th approximation, isotropic scattering (product form).

    Characteristic roots: omega sum_j alpha_j / (1 - k^2 mu_j^2) = 1 (N positive roots k).
    H(mu) = prod_i (mu + mu_i) / (prod_i mu_i prod_a (1 + k_a mu)).
    """
    s_poles = np.sort(1.0 / mu_nodes**2)

    def f(s):
        return omega * np.sum(alpha / (1.0 - s * mu_nodes**2)) - 1.0

    roots = []
    lo = 0.0
    for p in s_poles:
        eps = 1e-14 * p
        roots.append(brentq(f, lo + (eps if lo > 0 else 0.0), p - eps, xtol=1e-300, rtol=1e-15, maxiter=500))
        lo = p
    k = np.sqrt(np.array(roots))
    mu = np.atleast_1d(mu)
    num = np.prod(mu[:, None] + mu_nodes[None, :], axis=1)
    den = np.prod(mu_nodes) * np.prod(1.0 + k[None, :] * mu[:, None], axis=1)
    return num / den


@pytest.mark.parametrize("N", [4, 16])
def test_semi_infinite_isotropic_H_function(N):
    """P6: scalar isotropic, tau0 -> infinity: F = omega H(mu) H(mu0) / (4 pi (mu + mu0))."""
    coef = np.zeros((1, 6))
    coef[0, 0] = 1.0
    omega = 0.9
    mu = np.array([0.11, 0.42, 0.87])
    F = O.brdf(coef, omega, 200.0, 1.0, N, 1, mu, mu, np.array([0.0, 1.0]))
    nodes, alpha = O.gauss_legendre_01(N)
    H = _chandrasekhar_H(omega, nodes, alpha, mu)
    ref = omega * H[:, None] * H[None, :] / (4 * math.pi * (mu[:, None] + mu[None, :]))
    assert np.allclose(F[:, :, 0, 0, 0], ref.T, rtol=1e-12, atol=0)
    assert np.allclose(F[:, :, 1, 0, 0], ref.T, rtol=1e-12, atol=0)
    # polarization never appears for a scalar isotropic layer
    F2 = F.copy()
    F2[..., 0, 0] = 0.0
    assert np.abs(F2).max() == 0.0


def test_nodal_consistency_of_reconstruction(mie_coef):
    """P8: source-function integration at a node reproduces the nodal solution."""
    for n in (1.0, 1.5):
        sol = _solve(mie_coef[:16], 0.95, 3.0, 6, np.array([0.25, 0.66]), n, m=1)
        Irec = sol.reconstruct_top(sol.mu_nodes)  # [n_beam, N, 4, 4]
        u0 = sol.nodal(0.0)[:4 * sol.N]           # up directions
        for b in range(2):
            for k in range(sol.N):
                assert np.allclose(Irec[b, k], u0[4 * k:4 * k + 4, 4 * b:4 * b + 4], rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [1.0, 1.5])
def test_reciprocity_and_mirror_symmetry(mie_coef, n):
    """P5: F(mu', mu, -dphi) = Q F(mu, mu', dphi)^T Q, Q = diag(1,1,-1,1); F(-dphi) = D34 F D34."""
    mu = np.array([0.2, 0.5, 0.9])
    dphi = np.array([0.3, 1.7, 4.0])
    F = O.brdf(mie_coef, 0.95, 3.0, n, 12, 24, mu, mu, np.concatenate([dphi, 2 * math.pi - dphi]))
    Q = np.diag([1.0, 1.0, -1.0, 1.0])
    D34 = np.diag([1.0, 1.0, -1.0, -1.0])
    scale = np.abs(F).max()
    for j in range(3):
        jm = j + 3
        for i in range(3):
            for o in range(3):
                assert np.abs(F[o, i, jm] - Q @ F[i, o, j].T @ Q).max() < 1e-12 * scale
                assert np.abs(F[i, o, jm] - D34 @ F[i, o, j] @ D34).max() < 1e-12 * scale


def test_degenerate_limits(mie_coef):
    """P7: omega = 0 gives no subsurface light; n = 1 equals the bare layer exactly."""
    mu_in, mu_out, dphi = angle_grids(3, 3, 4)
    F0 = O.brdf(mie_coef, 0.0, 1.0, 1.5, 6, 24, mu_in, mu_out, dphi)
    assert np.abs(F0).max() == 0.0
    Fa = O.brdf(mie_coef, 0.8, 1.0, 1.0, 6, 24, mu_in, mu_out, dphi)
    Fb = O.brdf(mie_coef, 0.8, 1.0, 0.5, 6, 24, mu_in, mu_out, dphi)
    assert np.array_equal(Fa, Fb)
    Fc = O.brdf(mie_coef, 0.8, 1.0, 1.0 + 1e-9, 6, 24, mu_in, mu_out, dphi)
    assert np.abs(Fc - Fa).max() < 1e-7 * np.abs(Fa).max()


def test_orders_beyond_expansion_vanish():
    """Orders m > l_max carry no source and contribute nothing (A^m = 0)."""
    c = rayleigh_coefficients()
    mu_in, mu_out, dphi = angle_grids(2, 3, 5)
    Fa = O.brdf(c, 0.9, 1.0, 1.0, 8, 3, mu_in, mu_out, dphi)
    Fb = O.brdf(c, 0.9, 1.0, 1.0, 8, 6, mu_in, mu_out, dphi)
    assert np.array_equal(Fa, Fb)


def test_fresnel_energy_and_limits():
    mu = np.linspace(0.02, 1.0, 25)
    from oracle.fresnel import energy_transmittance
    for n in (1.3, 1.5, 1.7):
        Tp, Ts, Rp, Rs = energy_transmittance(mu, 1.0, n)
        assert np.allclose(Tp + Rp, 1.0, atol=1e-14) and np.allclose(Ts + Rs, 1.0, atol=1e-14)
        Tp, Ts, Rp, Rs = energy_transmittance(mu, n, 1.0)
        assert np.allclose(Tp + Rp, 1.0, atol=1e-14) and np.allclose(Ts + Rs, 1.0, atol=1e-14)
        mu_c = math.sqrt(1 - 1 / n**2)
        tir = mu < mu_c
        R = O.fresnel_internal_reflection(mu, n)
        assert np.allclose(R[tir, 0, 0], 1.0, atol=1e-14)
        # total internal reflection keeps the degree of polarization (unitary UV block)
        uv = R[tir][:, 2:, 2:]
        assert np.allclose(np.einsum("kab,kcb->kac", uv, uv), np.eye(2)[None], atol=1e-14)
        # normal incidence: r_p = -r_s gives U -> -r^2 U on meridian frames
        R1 = O.fresnel_internal_reflection(np.array([1.0]), n)[0]
        r = (n - 1) / (n + 1)
        assert np.allclose(R1, np.diag([r * r, r * r, -r * r, -r * r]), atol=1e-15)
    assert np.allclose(O.fresnel_beam_in(mu, 1.0), np.eye(4)) and np.allclose(O.fresnel_exit(mu, 1.0), np.eye(4))


def test_fresnel_tir_retardance_magnitude():
    """Beyond the critical angle |r_p| = |r_s| = 1 and the p-s phase difference delta obeys
    the closed form of total internal reflection (Born & Wolf, Sec. 1.5.4):
        tan(delta/2) = cos(theta) sqrt(sin^2(theta) - 1/n^2) / sin^2(theta).
    The internal-reflection Mueller matrix carries delta in its U/V block as the rotation
    [[cos delta, sin delta], [-sin delta, cos delta]]; its magnitude is independent of the
    p-axis convention (r_p = -r_s at normal incidence) and of the time convention."""
    for n in (1.3, 1.5, 1.7):
        mu_c = math.sqrt(1 - 1 / n**2)
        mu = np.linspace(0.01, mu_c - 1e-6, 40)
        R = O.fresnel_internal_reflection(mu, n)
        # unit reflectance of both polarizations: R = diag(1, 1, .) and no I-Q coupling
        assert np.allclose(R[:, 0, 0], 1.0, atol=1e-14) and np.allclose(R[:, 0, 1], 0.0, atol=1e-14)
        delta = np.arctan2(R[:, 2, 3], R[:, 2, 2])
        assert np.allclose(R[:, 3, 3], R[:, 2, 2], atol=1e-15)
        assert np.allclose(R[:, 3, 2], -R[:, 2, 3], atol=1e-15)
        sin2 = 1.0 - mu**2
        closed = mu * np.sqrt(sin2 - 1.0 / n**2) / sin2
        # 1e-10: the closed form itself loses digits in sin^2 - 1/n^2 next to critical
        assert np.allclose(np.abs(np.tan(0.5 * delta)), closed, rtol=1e-10, atol=1e-15)


def test_fresnel_tir_retardance_sign_follows_time_convention():
    """The sign of the TIR retardance is fixed by the branch of the transmitted-side
    cosine c2 = +-i sqrt(n^2 sin^2 - 1). Under the exp(-i w t) time factor of the Mie code
    the transmitted field is exp(i k0 c2 z) for z > 0 away from the interface, which decays
    only for Im c2 > 0. With that branch r_s = exp(-2i atan(beta/(n c1))) and
    r_p = exp(-2i atan(n beta/c1)), so delta = arg(r_p r_s*) is negative: the U -> V
    element of the Mueller matrix, sin(delta) = Im(r_p r_s*), is negative at every cosine
    below critical. The Mueller matrix itself follows the project's Stokes definition
    (U = 2 Re(E1 E2*), V = -2 Im(E1 E2*)), checked here on explicit fields, and it is the
    same map from a diagonal Jones matrix that the Mie code uses for its amplitude
    matrix diag(S2, S1) (b2 = Im(S2 S1*))."""
    from oracle.fresnel import _fresnel_amplitudes, _mueller_diag_jones
    from vrte_inputs.mie import amplitude_functions, mie_coefficients_ab, scattering_matrix_elements
    for n in (1.3, 1.5, 1.7):
        mu_c = math.sqrt(1 - 1 / n**2)
        mu = np.linspace(0.01, mu_c - 1e-6, 40)
        rp, rs, _, _, c2 = _fresnel_amplitudes(mu, n, 1.0)
        k0z = np.linspace(0.0, 5.0, 11)
        field = np.exp(1j * np.outer(c2, k0z))   # exp(i k0 c2 z) at z >= 0
        assert np.all(c2.imag > 0.0)
        assert np.all(np.diff(np.abs(field), axis=1) < 0.0)   # evanescent: decays away
        R = O.fresnel_internal_reflection(mu, n)
        assert np.all(R[:, 2, 3] < 0.0)
        assert np.allclose(R[:, 2, 3], (rp * np.conj(rs)).imag, atol=1e-15)
    # Mueller map of a diagonal Jones matrix against Stokes vectors formed from fields
    rng = np.random.default_rng(5)
    jp, js = rng.normal(size=2) + 1j * rng.normal(size=2)
    M = _mueller_diag_jones(np.array([jp]), np.array([js]))[0]
    for _ in range(4):
        E1, E2 = rng.normal(size=2) + 1j * rng.normal(size=2)

        def stokes(a, b):
            return np.array([abs(a)**2 + abs(b)**2, abs(a)**2 - abs(b)**2,
                             2 * (a * np.conj(b)).real, -2 * (a * np.conj(b)).imag])
        assert np.allclose(M @ stokes(E1, E2), stokes(jp * E1, js * E2), atol=1e-13)
    # the Mie code's scattering matrix is the same map from its amplitude matrix diag(S2, S1)
    a, b = mie_coefficients_ab(1.5 + 0.01j, 3.0)
    S1, S2 = amplitude_functions(a, b, np.array([0.3, -0.5]))
    el = scattering_matrix_elements(S1, S2)
    Mm = _mueller_diag_jones(S2, S1)
    assert np.allclose(Mm[:, 0, 0], el[0]) and np.allclose(Mm[:, 0, 1], el[4])
    assert np.allclose(Mm[:, 2, 2], el[2]) and np.allclose(Mm[:, 2, 3], el[5])
