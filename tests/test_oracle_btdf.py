"""Pins of the oracle's transmission table (oracle.btdf, the downward radiance at the bottom).

* at the node cosines the bottom reconstruction equals the nodal solution u(tau0, -mu_i)
  (with and without a dielectric top, whose internal reflection sends the upward radiance
  back down);
* in the thin-layer limit it equals the closed-form once-scattered transmission built from
  the directly rotated phase matrix (the downward scattering, plus under a dielectric top the
  upward scattering reflected at the top), with a residual that falls as tau0;
* at the table level, for a conservative layer (omega -> 1) without interface, the reflected
  and diffusely transmitted fluxes (tables at the Gauss nodes, integrated over azimuth and
  cosine) plus the uncollided beam exp(-tau0/mu0) equal the incident flux.
"""
import math

import numpy as np
import pytest

import oracle as O
from vrte_inputs import angle_grids, rayleigh_coefficients
from vrte_inputs.mie import monodisperse_coefficients


@pytest.fixture(scope="module")
def mie():
    return monodisperse_coefficients(1.5 + 0.01j, 2.0, 8)


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_bottom_reconstruction_at_nodes_is_the_nodal_solution(mie, n_if):
    N = 4
    nodes = O.gauss_legendre_01(N)
    mi = np.array([0.8, 0.35])
    beam = O.fresnel_beam_in(mi, n_if)
    R = O.fresnel_internal_reflection(nodes[0], n_if) if n_if > 1 else None
    for m in (0, 1, 3):
        sol = O.solve_order(m, mie, 0.9, 1.3, N, O.snell_mu(mi, n_if), beam, R, nodes)
        bot = sol.reconstruct_bottom(nodes[0], R)
        down = sol.nodal(1.3)[4 * N:].reshape(N, 4, mi.size, 4).transpose(2, 0, 1, 3)
        assert np.abs(bot - down).max() <= 1e-13 * np.abs(down).max(), m


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_thin_layer_transmission_is_single_scattering(mie, n_if):
    grids = angle_grids(3, 4, 5)
    res = []
    for tau0 in (1e-5, 1e-6):
        T = O.btdf(mie, 0.8, tau0, n_if, 4, 8, *grids)
        Ts = O.single_scatter_btdf(mie, 0.8, tau0, n_if, *grids)
        res.append(np.abs(T - Ts).max() / np.abs(Ts).max())
    assert res[1] < 5e-5
    assert 7.0 < res[0] / res[1] < 13.0   # O(tau0) multiple-scattering residual


def test_table_flux_balance_with_transmission():
    """omega = 1 - 1e-12, Rayleigh (L = 3 <= 2N), tables at the N Gauss nodes and a uniform
    azimuth grid: R + T_diffuse + exp(-tau0/mu0) = 1 to the absorbed 1e-12."""
    N, tau0 = 8, 1.0
    coef = rayleigh_coefficients()
    mu_n, al = O.gauss_legendre_01(N)
    mu_in = np.array([0.95, 0.6, 0.2])
    dphi = 2 * math.pi * np.arange(8) / 8
    omega = 1.0 - 1e-12
    Fr = O.brdf(coef, omega, tau0, 1.0, N, 3, mu_in, mu_n, dphi)
    Ft = O.btdf(coef, omega, tau0, 1.0, N, 3, mu_in, mu_n, dphi)

    def flux(F):
        return np.einsum("o,iojq->i", al * mu_n, F[..., 0, 0][..., None]) * 2 * math.pi / dphi.size

    total = flux(Fr) + flux(Ft) + np.exp(-tau0 / mu_in)
    assert np.allclose(total, 1.0, atol=1e-10)
