"""Pins of the oracle's multi-layer slab (Sec. 2.C: one homogeneous solution per sub-layer,
8N continuity equations at each common boundary).

* a stack of identical sub-layers is the single layer of their total thickness (any interface,
  black or Lambertian base);
* a purely absorbing top sub-layer (omega = 0) under no interface only attenuates the light that
  crosses it: F = exp(-tau_a (1/mu_in + 1/mu_out)) F_below;
* a purely absorbing bottom sub-layer over a black base is invisible: F = F_above;
* reciprocity and mirror symmetry hold for an inhomogeneous stack;
* a conservative inhomogeneous stack on a white base reflects all the incident flux (table level);
* the nodal field is continuous across the inner boundaries and meets both boundary conditions.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.slab import slab_brdf, solve_slab_order
from oracle.fresnel import fresnel_beam_in, fresnel_internal_reflection, snell_mu
from vrte_inputs import angle_grids, rayleigh_coefficients
from vrte_inputs.mie import monodisperse_coefficients


@pytest.fixture(scope="module")
def mie():
    return monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("nif,rho", [(1.0, 0.0), (1.4, 0.0), (1.4, 0.3)])
def test_identical_sublayers_equal_one_layer(mie, nif, rho):
    grids = angle_grids(3, 4, 5)
    F1 = O.brdf(mie, 0.9, 1.5, nif, 5, 12, *grids, rho=rho)
    F3 = slab_brdf([dict(coef=mie, omega=0.9, tau=t) for t in (0.2, 0.9, 0.4)], nif, 5, 12,
                   *grids, rho=rho)
    assert _rel(F3, F1) < 1e-12
    F1b = slab_brdf([dict(coef=mie, omega=0.9, tau=1.5)], nif, 5, 12, *grids, rho=rho)
    assert np.array_equal(F1b, F1)


def test_absorbing_top_sublayer_attenuates(mie):
    mu_in, mu_out, dphi = angle_grids(3, 4, 5)
    ta = 0.3
    below = dict(coef=mie, omega=0.95, tau=2.0)
    Fb = O.brdf(mie, 0.95, 2.0, 1.0, 6, 12, mu_in, mu_out, dphi)
    Fs = slab_brdf([dict(coef=mie, omega=0.0, tau=ta), below], 1.0, 6, 12, mu_in, mu_out, dphi)
    att = np.exp(-ta * (1.0 / mu_in[:, None] + 1.0 / mu_out[None, :]))
    assert _rel(Fs, att[:, :, None, None, None] * Fb) < 1e-12


@pytest.mark.parametrize("nif", [1.0, 1.5])
def test_absorbing_bottom_sublayer_is_invisible(mie, nif):
    grids = angle_grids(3, 4, 5)
    Fa = O.brdf(mie, 0.9, 1.0, nif, 6, 12, *grids)
    Fs = slab_brdf([dict(coef=mie, omega=0.9, tau=1.0), dict(coef=mie, omega=0.0, tau=0.7)],
                   nif, 6, 12, *grids)
    assert _rel(Fs, Fa) < 1e-12


@pytest.mark.parametrize("nif", [1.0, 1.5])
def test_inhomogeneous_stack_reciprocity(mie, nif):
    mu = np.array([0.2, 0.5, 0.9])
    dphi = np.array([0.3, 1.7, 4.0])
    layers = [dict(coef=rayleigh_coefficients(), omega=0.99, tau=0.4),
              dict(coef=mie, omega=0.8, tau=1.2),
              dict(coef=mie[:6], omega=0.95, tau=0.5)]
    F = slab_brdf(layers, nif, 8, 12, mu, mu, np.concatenate([dphi, 2 * math.pi - dphi]))
    Q = np.diag([1.0, 1.0, -1.0, 1.0])
    D34 = np.diag([1.0, 1.0, -1.0, -1.0])
    scale = np.abs(F).max()
    for j in range(3):
        for i in range(3):
            for o in range(3):
                assert np.abs(F[o, i, j + 3] - Q @ F[i, o, j].T @ Q).max() < 1e-12 * scale
                assert np.abs(F[i, o, j + 3] - D34 @ F[i, o, j] @ D34).max() < 1e-12 * scale


def test_conservative_stack_on_white_base_reflects_all(mie):
    N = 8
    mu_n, al = O.gauss_legendre_01(N)
    mu_in = np.array([0.95, 0.6, 0.2])
    dphi = 2 * math.pi * np.arange(16) / 16
    w = 1.0 - 1e-12
    layers = [dict(coef=rayleigh_coefficients(), omega=w, tau=0.5),
              dict(coef=mie[:2 * N - 1], omega=w, tau=0.8),
              dict(coef=rayleigh_coefficients(), omega=w, tau=0.3)]
    F = slab_brdf(layers, 1.0, N, 2 * N, mu_in, mu_n, dphi, rho=1.0)
    R = (al * mu_n) @ F[..., 0, 0].mean(axis=2).T * 2 * math.pi
    assert np.allclose(R, 1.0, atol=1e-9)


def test_nodal_field_continuity_and_boundaries(mie):
    N, nif = 5, 1.4
    mu_n, al = O.gauss_legendre_01(N)
    mu_in = np.array([0.3, 0.8])
    mu0 = snell_mu(mu_in, nif)
    beam = fresnel_beam_in(mu_in, nif)
    Rt = fresnel_internal_reflection(mu_n, nif)
    layers = [dict(coef=mie, omega=0.9, tau=0.6), dict(coef=rayleigh_coefficients(), omega=0.7,
                                                         tau=0.4),
              dict(coef=mie[:5], omega=0.99, tau=1.1)]
    for m in (0, 2):
        sols, tops = solve_slab_order(m, layers, N, mu0, beam, Rt, rho=0.2)
        for a, b in zip(sols[:-1], sols[1:]):
            ua, ub = a.nodal(a.tau0), b.nodal(0.0)
            assert np.abs(ua - ub).max() < 1e-12 * np.abs(ua).max()
        u0 = sols[0].nodal(0.0)
        up, down = u0[:4 * N], u0[4 * N:]
        refl = np.concatenate([Rt[i] @ up[4 * i:4 * i + 4] for i in range(N)])
        assert np.abs(down - refl).max() < 1e-12 * np.abs(u0).max()
        last = sols[-1]
        u1 = last.nodal(last.tau0)
        target = np.zeros_like(u1[:4 * N])
        if m == 0:
            ttot = tops[-1] + last.tau0
            flux = 2 * 0.2 * (al * mu_n) @ u1[4 * N:][0::4]
            direct = (2 * 0.2 / math.pi) * np.repeat(mu0, 4) * np.exp(-ttot / np.repeat(mu0, 4)) \
                * beam[:, 0, :].reshape(-1)
            target[0::4] = flux + direct
        assert np.abs(u1[:4 * N] - target).max() < 1e-12 * np.abs(u1).max()


def test_identical_sublayers_over_a_mueller_base(mie):
    R = np.array([[0.8, 0.15, 0, 0], [0.15, 0.4, 0, 0], [0, 0, 0.35, 0.12], [0, 0, -0.12, 0.3]])
    grids = angle_grids(3, 4, 5)
    F1 = O.brdf(mie, 0.9, 1.5, 1.4, 5, 12, *grids, base=R)
    F3 = slab_brdf([dict(coef=mie, omega=0.9, tau=t) for t in (0.2, 0.9, 0.4)], 1.4, 5, 12,
                   *grids, base=R)
    assert _rel(F3, F1) < 1e-12
