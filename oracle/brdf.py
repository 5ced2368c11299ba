"""Polarized subsurface BRDF from the per-order solutions (Sec. 2.D, Eqs. 1, 12, 39).

For incident basis Stokes vectors e_s (s = I, Q, U, V) the Mueller BRDF is the
matrix whose column s is the exiting radiance divided by the incident
irradiance (Eq. 39 with the four unit vectors, so the matrix inverse is the
identity). The exiting radiance is the Fourier sum of Eq. 12,

    I(0, mu, phi) = 1/2 sum_m Phi_{k(s)}^m(phi - phi_p) I^m(0, mu),

k(s) = 1 for s in {I, Q} and 2 for s in {U, V} (the D_k of Eq. 14 selects it),
phi_p the azimuth of the beam's propagation direction.

Table conventions: F[i_in, i_out, j, r, s] with mu_in the cosine of the direction
towards the source, mu_out the cosine towards the viewer, dphi_j = phi_out - phi_in
(both directions pointing away from the surface, as for the paper's (mu0, phi0) in
Eq. 4). The beam propagates at azimuth phi_in + pi, so the Fourier argument is
dphi - pi. Incident Stokes vectors are given on the meridian frame of the beam's
propagation direction, exiting ones on the meridian frame of the viewing direction.
F = I_out / (mu_in I0) in 1/sr (the irradiance on the horizontal surface is
mu_in I0; the paper's Eq. 1 names it without fixing the cosine).

With a dielectric top (n > 1) the external cosines are refracted (Snell), the
beam is transmitted with M_in, internal radiance leaves with M_out; the external
specular reflection is not part of the subsurface BRDF.
"""
from __future__ import annotations

import numpy as np

from .dom import solve_order
from .fresnel import fresnel_beam_in, fresnel_exit, fresnel_internal_reflection, snell_mu
from .phase import phase_matrix_direct
from .quadrature import gauss_legendre_01


def synthesis_weights(m: int, dphi):
    """w[j, r, s] = (Phi_{k(s)}^m(dphi_j - pi))_rr of Eq. 7."""
    dphi = np.atleast_1d(np.asarray(dphi, dtype=float))
    f = 1.0 if m == 0 else 2.0
    arg = m * (dphi - np.pi)
    c = f * np.cos(arg)
    s = f * np.sin(arg)
    w = np.zeros((dphi.size, 4, 4))
    for r in range(4):
        for col in range(4):
            iq_row = r < 2
            iq_col = col < 2
            if iq_col:     # Phi_1: (cos, cos, sin, sin)
                w[:, r, col] = c if iq_row else s
            else:          # Phi_2: (-sin, -sin, cos, cos)
                w[:, r, col] = -s if iq_row else c
    return w


def brdf_orders(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, rho=0.0, base=None):
    """Per-order internal exiting radiance I^m [M, n_in, n_out, 4, 4] plus interface data."""
    coef = np.asarray(coef, dtype=float)
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    nodes = gauss_legendre_01(N)
    mu0_int = snell_mu(mu_in, n_interface)
    mu_out_int = snell_mu(mu_out, n_interface)
    beam = fresnel_beam_in(mu_in, n_interface)
    R_top = fresnel_internal_reflection(nodes[0], n_interface) if n_interface > 1.0 else None
    L = coef.shape[0]
    Im = np.zeros((M, mu_in.size, mu_out.size, 4, 4))
    for m in range(min(M, L)):
        sol = solve_order(m, coef, omega, tau0, N, mu0_int, beam, R_top, nodes, rho, base)
        Im[m] = sol.reconstruct_top(mu_out_int)
    return Im


def synthesize(Im, mu_in, mu_out, dphi, n_interface):
    """F[i_in, i_out, j, r, s] from per-order radiances (Eq. 12) and the interface exit."""
    M = Im.shape[0]
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    dphi = np.atleast_1d(np.asarray(dphi, dtype=float))
    F = np.zeros((Im.shape[1], Im.shape[2], dphi.size, 4, 4))
    for m in range(M):
        w = synthesis_weights(m, dphi)
        F += 0.5 * Im[m][:, :, None, :, :] * w[None, None, :, :, :]
    Mout = fresnel_exit(mu_out, n_interface)
    F = np.einsum("oab,iojbc->iojac", Mout, F)
    return F / mu_in[:, None, None, None, None]


def brdf(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, dphi, rho=0.0, base=None):
    """Mueller BRDF table F[n_in, n_out, n_phi, 4, 4] of one layer (FP64); rho is the albedo
    of a Lambertian base (0: black base), base a direction-independent 4x4 Mueller BRDF of a
    reflecting base added to it (R_00 = 2 rho)."""
    Im = brdf_orders(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, rho, base)
    return synthesize(Im, mu_in, mu_out, dphi, n_interface)


def btdf_orders(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, rho=0.0, base=None):
    """Per-order downward radiance at the bottom I^m(tau0, -mu_out) [M, n_in, n_out, 4, 4].

    mu_out are cosines of downward directions below the layer, which has no interface at the
    bottom (black base or free space below): they are internal cosines as they are. The beam
    enters through the top interface as for the BRDF.
    """
    coef = np.asarray(coef, dtype=float)
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    nodes = gauss_legendre_01(N)
    mu0_int = snell_mu(mu_in, n_interface)
    beam = fresnel_beam_in(mu_in, n_interface)
    iface = n_interface > 1.0
    R_top = fresnel_internal_reflection(nodes[0], n_interface) if iface else None
    R_out = fresnel_internal_reflection(mu_out, n_interface) if iface else None
    L = coef.shape[0]
    Im = np.zeros((M, mu_in.size, mu_out.size, 4, 4))
    for m in range(min(M, L)):
        sol = solve_order(m, coef, omega, tau0, N, mu0_int, beam, R_top, nodes, rho, base)
        Im[m] = sol.reconstruct_bottom(mu_out, R_out)
    return Im


def btdf(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, dphi, rho=0.0, base=None):
    """Mueller BTDF table T[n_in, n_out, n_phi, 4, 4] of one layer (FP64): the diffuse
    radiance leaving the bottom in direction (-mu_out, phi_out) per unit irradiance mu_in I0
    of the beam from (mu_in, phi_in) above, dphi = phi_out - phi_in, Stokes vectors on the
    meridian frames of the propagation directions (Eq. 12 with the same Fourier factors as
    the BRDF; no exit interface)."""
    Im = btdf_orders(coef, omega, tau0, n_interface, N, M, mu_in, mu_out, rho, base)
    return synthesize(Im, mu_in, mu_out, dphi, 1.0)


def radiance_orders(coef, omega, tau0, n_interface, N, M, mu_in, tau, mu_up, mu_down, rho=0.0,
                    base=None):
    """Per-order internal radiance at depth tau for incident beams mu_in (external, through the
    top): (up [M, n_in, n_up, 4, 4], down [M, n_in, n_down, 4, 4]) at the internal cosines
    mu_up (upward) and mu_down (downward)."""
    coef = np.asarray(coef, dtype=float)
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_up = np.atleast_1d(np.asarray(mu_up, dtype=float))
    mu_down = np.atleast_1d(np.asarray(mu_down, dtype=float))
    nodes = gauss_legendre_01(N)
    iface = n_interface > 1.0
    R_top = fresnel_internal_reflection(nodes[0], n_interface) if iface else None
    R_dn = fresnel_internal_reflection(mu_down, n_interface) if iface else None
    L = coef.shape[0]
    up = np.zeros((M, mu_in.size, mu_up.size, 4, 4))
    dn = np.zeros((M, mu_in.size, mu_down.size, 4, 4))
    for m in range(min(M, L)):
        sol = solve_order(m, coef, omega, tau0, N, snell_mu(mu_in, n_interface),
                          fresnel_beam_in(mu_in, n_interface), R_top, nodes, rho, base)
        up[m], dn[m] = sol.reconstruct_depth(tau, mu_up, mu_down, R_dn)
    return up, dn


def radiance(coef, omega, tau0, n_interface, N, M, mu_in, tau, mu_up, mu_down, dphi, rho=0.0,
             base=None):
    """Radiance field inside the layer at depth tau per unit irradiance mu_in I0 of the beam:
    (up [n_in, n_up, n_phi, 4, 4], down [n_in, n_down, n_phi, 4, 4]), directions (+-mu, phi)
    with dphi = phi - phi_in and Stokes vectors on their meridian frames (Eq. 12)."""
    up, dn = radiance_orders(coef, omega, tau0, n_interface, N, M, mu_in, tau, mu_up, mu_down, rho,
                             base)
    return (synthesize(up, mu_in, mu_up, dphi, 1.0), synthesize(dn, mu_in, mu_down, dphi, 1.0))


def single_scatter_btdf(coef, omega, tau0, n_interface, mu_in, mu_out, dphi):
    """Exact once-scattered BTDF from the directly rotated phase matrix, independent of the
    Fourier machinery: the beam scattered once downward,
        (omega / 4 pi) Z(-mu, phi; -mu0, phi_in + pi) I0' int_0^tau0 e^{-t/mu0} e^{-(tau0-t)/mu} dt / mu,
    plus, under a dielectric top, the light scattered once upward and specularly reflected
    back down at the top (it crosses the layer once more),
        exp(-tau0/mu) R_F(mu) (omega / 4 pi) Z(mu, phi; -mu0, phi_in + pi) I0' int_0^tau0 e^{-t/mu0} e^{-t/mu} dt / mu,
    both divided by mu_in."""
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    dphi = np.atleast_1d(np.asarray(dphi, dtype=float))
    mi = snell_mu(mu_in, n_interface)
    Min = fresnel_beam_in(mu_in, n_interface)
    Rf = fresnel_internal_reflection(mu_out, n_interface)
    F = np.zeros((mu_in.size, mu_out.size, dphi.size, 4, 4))
    for i in range(mu_in.size):
        for o in range(mu_out.size):
            x, y = 1.0 / mu_out[o], 1.0 / mi[i]
            if abs(x - y) * tau0 < 1e-8:
                depth = tau0 * np.exp(-x * tau0)
            else:
                depth = (np.exp(-y * tau0) - np.exp(-x * tau0)) / (x - y)
            up = -np.expm1(-tau0 * (x + y)) / (x + y)
            for j, dp in enumerate(dphi):
                Zd = phase_matrix_direct(coef, -mu_out[o], dp, -mi[i], np.pi)
                Zu = phase_matrix_direct(coef, mu_out[o], dp, -mi[i], np.pi)
                I = depth * Zd + np.exp(-x * tau0) * up * Rf[o] @ Zu
                F[i, o, j] = omega / (4 * np.pi) / mu_out[o] * I @ Min[i] / mu_in[i]
    return F


def single_scatter_brdf(coef, omega, tau0, n_interface, mu_in, mu_out, dphi):
    """Exact once-scattered BRDF, computed from the directly rotated phase matrix.

    I_ss(0, mu) = (omega / 4 pi) Z(mu, phi; -mu0, phi_in + pi) I0' mu0 (1 - exp(-tau0 (1/mu + 1/mu0))) / (mu + mu0)
    (Eq. 4 integrated along the exit path), then the interface and the 1/mu_in of
    the BRDF normalisation. Independent of the Fourier machinery.
    """
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    dphi = np.atleast_1d(np.asarray(dphi, dtype=float))
    mi = snell_mu(mu_in, n_interface)
    mo = snell_mu(mu_out, n_interface)
    Min = fresnel_beam_in(mu_in, n_interface)
    Mout = fresnel_exit(mu_out, n_interface)
    F = np.zeros((mu_in.size, mu_out.size, dphi.size, 4, 4))
    for i in range(mu_in.size):
        for o in range(mu_out.size):
            depth = mi[i] * -np.expm1(-tau0 * (1.0 / mo[o] + 1.0 / mi[i])) / (mo[o] + mi[i])
            for j, dp in enumerate(dphi):
                Z = phase_matrix_direct(coef, mo[o], dp, -mi[i], np.pi)
                F[i, o, j] = Mout[o] @ (omega / (4 * np.pi) * depth * Z @ Min[i]) / mu_in[i]
    return F
