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
