"""Pins of the oracle's Lambertian base (Sec. 3.C, base reflection, R_00 = 2 rho).

At the table level (tables at the Gauss nodes, uniform azimuth grid, Rayleigh with L <= 2N):
* a conservative layer (omega -> 1) on a white base (rho = 1) reflects all the incident flux;
* on a grey base (rho < 1) the reflected flux plus the part (1 - rho) of the flux reaching the
  base (diffuse transmission plus the uncollided beam) equals the incident flux;
* a vanishing layer leaves the bare base: F_00 = rho / pi, every polarized element zero;
* rho = 0 is the black base exactly.
"""
import math

import numpy as np
import pytest

import oracle as O
from vrte_inputs import rayleigh_coefficients

N, TAU = 8, 1.0
MU_N, AL = O.gauss_legendre_01(N)
MU_IN = np.array([0.95, 0.6, 0.2])
DPHI = 2 * math.pi * np.arange(8) / 8


def _flux(F):
    return (AL * MU_N) @ F[..., 0, 0].mean(axis=2).T * 2 * math.pi


@pytest.mark.parametrize("rho", [1.0, 0.4])
def test_lambertian_base_flux_balance(rho):
    coef = rayleigh_coefficients()
    omega = 1.0 - 1e-12
    Fr = O.brdf(coef, omega, TAU, 1.0, N, 3, MU_IN, MU_N, DPHI, rho)
    Ft = O.btdf(coef, omega, TAU, 1.0, N, 3, MU_IN, MU_N, DPHI, rho)
    R = _flux(Fr)
    T = _flux(Ft) + np.exp(-TAU / MU_IN)
    assert np.allclose(R + (1.0 - rho) * T, 1.0, atol=1e-10)


def test_vanishing_layer_leaves_the_lambertian_base():
    coef = rayleigh_coefficients()
    F = O.brdf(coef, 0.9, 1e-10, 1.0, N, 3, MU_IN, MU_N[:3], DPHI, 0.5)
    # residual: single scattering of order tau0 / mu (mu down to 0.02 at the first node)
    assert np.allclose(F[..., 0, 0], 0.5 / math.pi, rtol=1e-7)
    F[..., 0, 0] = 0.0
    assert np.abs(F).max() < 1e-8


def test_black_base_is_rho_zero():
    coef = rayleigh_coefficients()
    a = O.brdf(coef, 0.9, TAU, 1.4, N, 3, MU_IN, MU_N[:3], DPHI)
    b = O.brdf(coef, 0.9, TAU, 1.4, N, 3, MU_IN, MU_N[:3], DPHI, 0.0)
    assert np.array_equal(a, b)


# A base with a direction-independent Mueller BRDF R (the paper's base reflection with R constant;
# the Lambertian base is R_00 = 2 rho): azimuth independence leaves the (I, Q) x (U, V) blocks zero.
def _mueller_base(a, b, c, d, e, g):
    return np.array([[a, b, 0, 0], [b, c, 0, 0], [0, 0, d, e], [0, 0, -e, g]], dtype=float)


def test_mueller_base_of_a_vanishing_layer_is_R_over_2pi():
    R = _mueller_base(0.7, -0.2, 0.5, 0.3, 0.1, 0.25)
    dphi = np.array([0.0, 1.1, 3.7])
    for n_if in (1.0,):
        F = O.brdf(rayleigh_coefficients(), 0.9, 1e-10, n_if, N, 3, MU_IN, MU_N[:3], dphi, base=R)
        # residual: single scattering of order tau0 / mu (mu down to 0.02 at the first node)
        assert np.allclose(F, (R / (2 * math.pi))[None, None, None], rtol=1e-7, atol=1e-8)


def test_lambertian_is_the_mueller_base_with_R00_2rho():
    coef = rayleigh_coefficients()
    a = O.brdf(coef, 0.9, TAU, 1.4, N, 3, MU_IN, MU_N[:3], DPHI, 0.3)
    b = O.brdf(coef, 0.9, TAU, 1.4, N, 3, MU_IN, MU_N[:3], DPHI, base=np.diag([0.6, 0, 0, 0]))
    assert np.allclose(a, b, rtol=1e-13, atol=1e-16)


def test_reciprocal_mueller_base_keeps_the_table_reciprocal():
    # Q R^T Q = R for the base (Q = diag(1, 1, -1, 1)) makes layer + base reciprocal
    R = _mueller_base(0.8, 0.15, 0.4, 0.35, 0.12, 0.3)
    Q = np.diag([1.0, 1.0, -1.0, 1.0])
    assert np.allclose(Q @ R.T @ Q, R)
    from vrte_inputs.mie import monodisperse_coefficients
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)
    mu = np.array([0.2, 0.5, 0.9])
    dphi = np.array([0.3, 1.7, 4.0])
    for n_if in (1.0, 1.5):
        F = O.brdf(coef, 0.95, 1.5, n_if, 8, 12, mu, mu,
                   np.concatenate([dphi, 2 * math.pi - dphi]), base=R)
        scale = np.abs(F).max()
        for j in range(3):
            for i in range(3):
                for o in range(3):
                    assert np.abs(F[o, i, j + 3] - Q @ F[i, o, j].T @ Q).max() < 1e-12 * scale


def test_polarizing_rows_of_a_white_base_keep_the_flux_balance():
    # first row (2, 0, 0, 0): the base returns all the flux it receives, whatever it does to
    # the polarization; a conservative layer over it then reflects all the incident flux
    R = _mueller_base(2.0, 0.0, 0.6, 0.4, 0.3, -0.2)
    R[1, 0] = 0.5
    coef = rayleigh_coefficients()
    Fr = O.brdf(coef, 1.0 - 1e-12, TAU, 1.0, N, 3, MU_IN, MU_N, DPHI, base=R)
    assert np.allclose(_flux(Fr), 1.0, atol=1e-10)
    # and a change of those rows does change the polarized part of the table
    F0 = O.brdf(coef, 1.0 - 1e-12, TAU, 1.0, N, 3, MU_IN, MU_N, DPHI, base=np.diag([2.0, 0, 0, 0]))
    assert np.abs(Fr[..., 1, :] - F0[..., 1, :]).max() > 1e-3
