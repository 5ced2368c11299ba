"""Pins of the oracle's interior radiance field (OrderSolution.reconstruct_depth, radiance):

* at the node cosines and any depth it equals the nodal solution u(tau) of the order, upward
  and downward, with and without a dielectric top and a Lambertian base;
* at tau = 0 its upward part equals the top reconstruction (the BRDF's internal radiance) and
  at tau = tau0 its downward part the bottom reconstruction (the transmission table);
* in azimuth-integrated form at the Gauss nodes it gives the net flux, which for a
  conservative layer is the same at every depth (the divergence of the flux is the
  absorption).
"""
import math

import numpy as np
import pytest

import oracle as O
from vrte_inputs import rayleigh_coefficients
from vrte_inputs.mie import monodisperse_coefficients


@pytest.mark.parametrize("n_if,rho", [(1.0, 0.0), (1.4, 0.0), (1.4, 0.5)])
def test_depth_reconstruction_at_nodes_is_the_nodal_solution(n_if, rho):
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 8)
    N = 4
    nodes = O.gauss_legendre_01(N)
    mi = np.array([0.8, 0.35])
    beam = O.fresnel_beam_in(mi, n_if)
    R = O.fresnel_internal_reflection(nodes[0], n_if) if n_if > 1 else None
    for m in (0, 2):
        sol = O.solve_order(m, coef, 0.9, 1.3, N, O.snell_mu(mi, n_if), beam, R, nodes, rho)
        for tau in (0.0, 0.4, 1.3):
            up, dn = sol.reconstruct_depth(tau, nodes[0], nodes[0], R)
            u = sol.nodal(tau)
            upn = u[:4 * N].reshape(N, 4, mi.size, 4).transpose(2, 0, 1, 3)
            dnn = u[4 * N:].reshape(N, 4, mi.size, 4).transpose(2, 0, 1, 3)
            scale = np.abs(u).max()
            assert np.abs(up - upn).max() <= 1e-12 * scale, (m, tau)
            assert np.abs(dn - dnn).max() <= 1e-12 * scale, (m, tau)
        mo = np.array([0.27, 0.66])
        Rd = O.fresnel_internal_reflection(mo, n_if) if n_if > 1 else None
        up0, _ = sol.reconstruct_depth(0.0, mo, mo, Rd)
        _, dnb = sol.reconstruct_depth(1.3, mo, mo, Rd)
        assert np.allclose(up0, sol.reconstruct_top(mo), rtol=0, atol=1e-15)
        assert np.allclose(dnb, sol.reconstruct_bottom(mo, Rd), rtol=0, atol=1e-15)


def test_net_flux_is_constant_in_a_conservative_layer():
    N, tau0 = 8, 2.0
    coef = rayleigh_coefficients()
    mu_n, al = O.gauss_legendre_01(N)
    mu_in = np.array([0.9, 0.4])
    dphi = 2 * math.pi * np.arange(8) / 8
    omega = 1.0 - 1e-12
    net = []
    for tau in (0.0, 0.5, 1.3, 2.0):
        up, dn = O.radiance(coef, omega, tau0, 1.0, N, 3, mu_in, tau, mu_n, mu_n, dphi)
        fu = (al * mu_n) @ up[..., 0, 0].mean(axis=2).T * 2 * math.pi
        fd = (al * mu_n) @ dn[..., 0, 0].mean(axis=2).T * 2 * math.pi
        net.append(fd + np.exp(-tau / mu_in) - fu)     # downward minus upward, beam included
    net = np.array(net)
    assert np.allclose(net, net[0][None, :], atol=1e-10)
