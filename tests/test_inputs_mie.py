"""Pins of the Mie input generator (P11): optical theorem, Rayleigh limit, expansion fidelity.

The Mie series is an input generator (the paper used an external Mie code), but
wrong coefficients would silently change every downstream value, so it is
checked against identities of Mie theory and against the oracle's independent
evaluation of the scattering matrix from coefficients.
"""
import math

import numpy as np
import pytest

import oracle as O
from vrte_inputs import make_config, rayleigh_coefficients, uniform_zenith_grid
from vrte_inputs import mie


@pytest.mark.parametrize("m,x", [(1.5 + 0.0j, 0.7), (1.5 + 0.001j, 5.0), (1.33 + 0.1j, 12.0), (1.7 + 0.01j, 40.0)])
def test_optical_theorem(m, x):
    a, b = mie.mie_coefficients_ab(m, x)
    qext, qsca = mie.efficiencies(a, b, x)
    S1, S2 = mie.amplitude_functions(a, b, np.array([1.0]))
    assert abs(S1[0] - S2[0]) < 1e-10 * abs(S1[0])
    assert abs(qext - 4.0 / x**2 * S1[0].real) < 1e-10 * qext
    assert qsca <= qext * (1 + 1e-12)
    if m.imag == 0:
        assert abs(qsca - qext) < 1e-9 * qext


def test_small_particle_tends_to_rayleigh():
    c = mie.monodisperse_coefficients(1.5 + 0.0j, 1e-3, 6)
    ref = np.zeros((6, 6))
    ref[:3] = rayleigh_coefficients()
    assert np.allclose(c, ref, atol=1e-5)


@pytest.mark.parametrize("x", [0.5, 3.0, 8.0])
def test_expansion_reproduces_scattering_matrix(x):
    """Coefficients with L large enough reproduce F(Theta) off the projection grid."""
    m = 1.5 + 0.01j
    a, b = mie.mie_coefficients_ab(m, x)
    L = 2 * len(a) + 2
    c = mie.monodisperse_coefficients(m, x, L)
    th = np.linspace(0.0, math.pi, 17) + 0.013
    ct = np.cos(th)
    S1, S2 = mie.amplitude_functions(a, b, ct)
    el = mie.scattering_matrix_elements(S1, S2)
    xt, wt = np.polynomial.legendre.leggauss(len(a) + L + 8)
    S1g, S2g = mie.amplitude_functions(a, b, xt)
    norm = 0.5 * np.sum(wt * mie.scattering_matrix_elements(S1g, S2g)[0])
    F = O.scattering_matrix(c, ct)
    assert np.allclose(F[:, 0, 0], el[0] / norm, rtol=1e-9, atol=1e-10 * el[0].max() / norm)
    assert np.allclose(F[:, 0, 1], el[4] / norm, atol=1e-9 * el[0].max() / norm)
    assert np.allclose(F[:, 2, 2], el[2] / norm, atol=1e-9 * el[0].max() / norm)
    assert np.allclose(F[:, 2, 3], el[5] / norm, atol=1e-9 * el[0].max() / norm)
    assert np.allclose(F[:, 1, 1], el[0] / norm, atol=1e-9 * el[0].max() / norm)


def test_normalisation_and_asymmetry():
    """alpha1_0 = 1 and alpha1_1 / 3 = <cos Theta> from the amplitude functions."""
    m, x = 1.5 + 0.001j, 4.0
    c = mie.monodisperse_coefficients(m, x, 40)
    assert abs(c[0, 0] - 1.0) < 1e-14
    a, b = mie.mie_coefficients_ab(m, x)
    xt, wt = np.polynomial.legendre.leggauss(200)
    S1, S2 = mie.amplitude_functions(a, b, xt)
    f11 = mie.scattering_matrix_elements(S1, S2)[0]
    g = np.sum(wt * f11 * xt) / np.sum(wt * f11)
    assert abs(c[1, 0] / 3.0 - g) < 1e-12


def test_grids_and_rayleigh_workload():
    mu = uniform_zenith_grid(8)
    assert np.all(np.diff(mu) < 0) and mu.min() > 0 and mu.max() < 1
    cfg = make_config(1)
    assert cfg["layers"][0]["n_orders"] == 3 and cfg["mu_in"].size == 8 and cfg["dphi"].size == 16
