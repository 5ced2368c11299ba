"""Pins of the gradient oracle (oracle/gradient.py), the target of the adjoint (row a9).

In the thin-layer limit the oracle's BRDF tends to the closed-form single-scattering BRDF
(oracle.single_scatter_brdf, computed from the directly rotated phase matrix, independent of
the Fourier machinery), which is linear in omega and in every expansion coefficient and has a
closed tau0 and interface dependence. So at tau0 = 1e-7 the oracle's central-difference
derivatives must equal
  * dF/domega     = F_ss / omega,
  * dF/dcoef[l,c] = F_ss evaluated with the unit coefficient vector e_{l,c},
  * dF/dtau0, dF/dn = the same differences taken on the closed form,
up to the O(tau0) multiple-scattering and depth corrections (relative ~1e-5 here). The chain
rule of the loss gradient is checked against a central difference of the loss itself on a
layer that is not thin.
"""
import numpy as np
import pytest

import oracle as O
from oracle import gradient as G
from vrte_inputs import angle_grids
from vrte_inputs.mie import monodisperse_coefficients

N, L = 4, 6
GRID = angle_grids(3, 3, 4)


@pytest.fixture(scope="module")
def coef():
    return monodisperse_coefficients(1.5 + 0.01j, 1.2, L)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("n_if", [1.0, 1.4])
def test_omega_and_coefficient_derivatives_in_the_thin_limit(coef, n_if):
    omega, tau0 = 0.8, 1e-7
    p = G.pack(omega, tau0, n_if, coef)
    Fss = O.single_scatter_brdf(coef, omega, tau0, n_if, *GRID)
    d_omega = G.table_derivative(p, 0, L, N, L, *GRID)
    assert _rel(d_omega, Fss / omega) < 1e-4
    scale = np.max(np.abs(Fss))
    for (l, c) in [(0, 0), (1, 0), (2, 1), (3, 2), (1, 3), (2, 4), (4, 5)]:
        e = np.zeros_like(coef)
        e[l, c] = 1.0
        ref = O.single_scatter_brdf(e, omega, tau0, n_if, *GRID)
        d = G.table_derivative(p, 3 + 6 * l + c, L, N, L, *GRID)
        assert _rel(d, ref) < 1e-4, (l, c, _rel(d, ref))
    # the polarization entries of degree l < 2 (alpha2, alpha3, beta1, beta2) do not enter:
    # generalized spherical functions of index 2 vanish there, in the closed form and the DOM
    for (l, c) in [(1, 1), (1, 2), (0, 4), (1, 5)]:
        e = np.zeros_like(coef)
        e[l, c] = 1.0
        assert np.max(np.abs(O.single_scatter_brdf(e, omega, tau0, n_if, *GRID))) == 0.0
        d = G.table_derivative(p, 3 + 6 * l + c, L, N, L, *GRID)
        assert np.max(np.abs(d)) <= 1e-9 * scale / omega, (l, c)


def test_tau_and_interface_derivatives_in_the_thin_limit(coef):
    omega, tau0, n_if = 0.8, 1e-7, 1.4

    def ss(t, n):
        return O.single_scatter_brdf(coef, omega, t, n, *GRID)

    p = G.pack(omega, tau0, n_if, coef)
    ht, hn = 1e-6 * tau0, 1e-6 * n_if
    ref_tau = (ss(tau0 + ht, n_if) - ss(tau0 - ht, n_if)) / (2 * ht)
    ref_n = (ss(tau0, n_if + hn) - ss(tau0, n_if - hn)) / (2 * hn)
    assert _rel(G.table_derivative(p, 1, L, N, L, *GRID), ref_tau) < 1e-4
    assert _rel(G.table_derivative(p, 2, L, N, L, *GRID), ref_n) < 1e-4


def test_richardson_is_in_the_asymptotic_regime(coef):
    """Plain central differences at h and h/2 agree with the extrapolated one to O(h^2)."""
    p = G.pack(0.9, 0.7, 1.3, coef)
    d_rich = G.table_derivative(p, 0, L, N, L, *GRID)
    d_h = G.table_derivative(p, 0, L, N, L, *GRID, richardson=False)
    d_h2 = G.table_derivative(p, 0, L, N, L, *GRID, h=5e-7, richardson=False)
    e_h, e_h2 = _rel(d_h, d_rich), _rel(d_h2, d_rich)
    assert e_h < 1e-7 and e_h2 < 1e-7


def test_loss_gradient_chain_rule_against_loss_difference(coef):
    """dL/dp_k = sum (F - T) dF/dp_k against (L(p + h e_k) - L(p - h e_k)) / 2h."""
    p = G.pack(0.9, 0.7, 1.3, coef)
    q = p.copy()
    q[0] *= 0.98
    q[3 + 6 * 1 + 0] *= 1.03
    target = G.table(q, L, N, L, *GRID)
    idx = [0, 1, 2, 3 + 6 * 1 + 0, 3 + 6 * 2 + 4]
    g = G.loss_gradient(p, target, L, N, L, *GRID, indices=idx)
    for k in idx:
        hk = 1e-5 * (abs(p[k]) if p[k] else 1.0)
        pp, pm = p.copy(), p.copy()
        pp[k] += hk
        pm[k] -= hk
        fd = (G.loss(G.table(pp, L, N, L, *GRID), target)
              - G.loss(G.table(pm, L, N, L, *GRID), target)) / (2 * hk)
        assert abs(g[k] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (k, g[k], fd)
    assert np.all(g[[k for k in range(p.size) if k not in idx]] == 0.0)


def test_pack_and_unpack_follow_the_gradient_layout(coef):
    p = G.pack(0.5, 2.0, 1.33, coef)
    assert p.size == 3 + 6 * L
    om, t, n, c = G.unpack(p, L)
    assert (om, t, n) == (0.5, 2.0, 1.33)
    assert np.array_equal(c, coef)
    assert p[3 + 6 * 2 + 4] == coef[2, 4]
