"""Pins of the dual-number gradient oracle (oracle/tangent.py), the exact (non-difference)
reference of the adjoint.

* its derivative identity for the phase-matrix tables against central differences of the
  tables (d P_l^m / d mu);
* its Fresnel matrices in dual arithmetic: values equal oracle.fresnel, derivatives in n equal
  Richardson differences of oracle.fresnel (both sides of the critical angle);
* its propagator-form BRDF equals the eigen-form oracle BRDF (oracle.brdf), with and without
  an interface;
* its gradient of the loss equals the Richardson central differences of oracle.gradient;
* in the thin-layer limit its derivatives equal those of the closed-form single-scattering
  BRDF (linear in omega and in every coefficient).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import gradient as G
from oracle import tangent as T
from vrte_inputs import angle_grids
from vrte_inputs.mie import monodisperse_coefficients

N, L = 4, 8
GRID = angle_grids(3, 4, 5)


@pytest.fixture(scope="module")
def coef():
    return monodisperse_coefficients(1.5 + 0.01j, 2.0, L)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_table_derivative_identity():
    mu = np.array([-0.93, -0.4, 0.05, 0.31, 0.77, 0.99])
    for m in (0, 1, 2, 5):
        h = 1e-5
        num = (O.P_matrices(m, 9, mu + h) - O.P_matrices(m, 9, mu - h)) / (2 * h)
        num2 = (O.P_matrices(m, 9, mu + h / 2) - O.P_matrices(m, 9, mu - h / 2)) / h
        ref = (4 * num2 - num) / 3
        assert np.abs(T.dP_dmu(m, 9, mu) - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max()), m


@pytest.mark.parametrize("n", [1.33, 1.5])
def test_dual_fresnel_matches_oracle_and_its_differences(n):
    mu_in = np.array([0.97, 0.6, 0.15])
    mu_out = np.array([0.9, 0.45, 0.08])
    nodes = np.array([0.05, 0.3, 0.7, 0.95])   # below and above the critical cosine
    assert np.any(nodes < math.sqrt(1 - 1 / n**2)) and np.any(nodes > math.sqrt(1 - 1 / n**2))
    (mi, dmi), (mo, dmo), (Mi, dMi), (Mo, dMo), (R, dR) = T.interface_dual(mu_in, mu_out, nodes,
                                                                          n, 1.0)
    assert np.allclose(mi, O.snell_mu(mu_in, n), atol=1e-15)
    assert np.allclose(Mi, O.fresnel_beam_in(mu_in, n), atol=1e-14)
    assert np.allclose(Mo, O.fresnel_exit(mu_out, n), atol=1e-14)
    assert np.allclose(R, O.fresnel_internal_reflection(nodes, n), atol=1e-14)

    def rich(f, h=1e-4):
        d1 = (f(n + h) - f(n - h)) / (2 * h)
        d2 = (f(n + h / 2) - f(n - h / 2)) / h
        return (4 * d2 - d1) / 3
    assert np.allclose(dmi, rich(lambda x: O.snell_mu(mu_in, x)), atol=1e-10)
    assert np.allclose(dmo, rich(lambda x: O.snell_mu(mu_out, x)), atol=1e-10)
    assert np.allclose(dMi, rich(lambda x: O.fresnel_beam_in(mu_in, x)), atol=1e-9)
    assert np.allclose(dMo, rich(lambda x: O.fresnel_exit(mu_out, x)), atol=1e-9)
    assert np.allclose(dR, rich(lambda x: O.fresnel_internal_reflection(nodes, x)), atol=1e-9)


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_propagator_brdf_equals_eigen_oracle(coef, n_if):
    p = G.pack(0.9, 1.3, n_if, coef)
    F = O.brdf(coef, 0.9, 1.3, n_if, N, L, *GRID)
    Fd, dF = T.brdf_dual(p, np.zeros_like(p), L, N, L, *GRID)
    assert _rel(Fd, F) < 1e-9
    assert np.max(np.abs(dF)) == 0.0


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_dual_gradient_equals_central_differences(coef, n_if):
    p = G.pack(0.9, 1.3, n_if, coef)
    F = O.brdf(coef, 0.9, 1.3, n_if, N, L, *GRID)
    rng = np.random.default_rng(3)
    target = F * (1 + 0.03 * rng.normal(size=F.shape))
    idx = [0, 1] + ([2] if n_if > 1 else []) + [3, 4, 3 + 6 * 2 + 1, 3 + 6 * 3 + 2, 3 + 6 * 2 + 4,
                                                3 + 6 * 4 + 5, 3 + 6 * 7 + 0, 3 + 6 * 7 + 3]
    g = T.loss_gradient(p, target, L, N, L, *GRID, indices=idx)
    ref = G.loss_gradient(p, target, L, N, L, *GRID, indices=idx)
    big = np.abs(ref).max()
    for k in idx:
        assert abs(g[k] - ref[k]) <= 1e-5 * max(abs(ref[k]), 1e-3 * big), (k, g[k], ref[k])


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_dual_derivatives_in_the_thin_limit(coef, n_if):
    """dF/domega = F_ss/omega and dF/dcoef = F_ss of the unit coefficient at tau0 = 1e-7."""
    omega, tau0 = 0.8, 1e-7
    p = G.pack(omega, tau0, n_if, coef)
    Fss = O.single_scatter_brdf(coef, omega, tau0, n_if, *GRID)
    e = np.zeros_like(p)
    e[0] = 1.0
    _, d = T.brdf_dual(p, e, L, N, L, *GRID)
    assert _rel(d, Fss / omega) < 1e-5
    for (l, c) in [(0, 0), (2, 1), (3, 2), (5, 4)]:
        u = np.zeros_like(coef)
        u[l, c] = 1.0
        e = np.zeros_like(p)
        e[3 + 6 * l + c] = 1.0
        _, d = T.brdf_dual(p, e, L, N, L, *GRID)
        assert _rel(d, O.single_scatter_brdf(u, omega, tau0, n_if, *GRID)) < 1e-5, (l, c)
