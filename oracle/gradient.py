"""Gradient of the BRDF loss with respect to the layer parameters (the target of the adjoint),
by central differences of the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never calls it.

Parameters, in the order of the plan's gradient layout [3 + 6 L]:
    p = (omega, tau0, n_interface, coef[0, 0..5], coef[1, 0..5], ..., coef[L-1, 0..5])
with the coefficients in input order (alpha1, alpha2, alpha3, alpha4, beta1, beta2) per l.
Loss L(p) = 1/2 sum over the table (F(p) - F_target)^2, so
    dL/dp_k = sum (F - F_target) dF/dp_k
(the chain rule through the table), with dF/dp_k a central difference of step
h_k = h max(1, |p_k|), Richardson-extrapolated from the steps h_k and h_k / 2,
(4 D(h_k / 2) - D(h_k)) / 3, so that the truncation error is O(h^4) and the rounding error
O(u / h) of the table. The floor of one keeps the step, and so the rounding error, bounded
for the small high-order coefficients (a step relative to a coefficient of 1e-5 would leave
only rounding); a thin layer (tau0 below h) takes h_k = h |tau0| instead so that tau0 - h_k
stays positive. The interface index must sit away from n = 1, where the interface switches
off.

Pinned by tests/test_oracle_gradient.py: in the thin-layer limit F tends to the closed-form
single-scattering BRDF, which is linear in omega and in every coefficient and has a closed
tau0 and n dependence; the chain rule is checked against a difference of the loss itself.
"""
from __future__ import annotations

import numpy as np

from .brdf import brdf


def pack(omega, tau0, n_interface, coef) -> np.ndarray:
    """Parameter vector [3 + 6 L] in the gradient layout."""
    return np.concatenate([[float(omega), float(tau0), float(n_interface)],
                           np.asarray(coef, dtype=float).ravel()])


def unpack(p, L: int):
    p = np.asarray(p, dtype=float)
    return p[0], p[1], p[2], p[3:3 + 6 * L].reshape(L, 6)


def table(p, L, N, M, mu_in, mu_out, dphi) -> np.ndarray:
    """F[n_in, n_out, n_phi, 4, 4] of the layer described by p."""
    omega, tau0, n_if, coef = unpack(p, L)
    return brdf(coef, omega, tau0, n_if, N, M, mu_in, mu_out, dphi)


def table_derivative(p, k: int, L, N, M, mu_in, mu_out, dphi, h: float = 1e-6,
                     richardson: bool = True) -> np.ndarray:
    """dF/dp_k by central differences (Richardson-extrapolated unless richardson=False)."""
    p = np.asarray(p, dtype=float)
    hk = h * max(1.0, abs(p[k]))
    if k == 1 and hk >= 0.5 * p[k]:   # thin layer: keep tau0 - h_k > 0
        hk = h * abs(p[k])

    def central(step):
        pp = p.copy()
        pm = p.copy()
        pp[k] += step
        pm[k] -= step
        return (table(pp, L, N, M, mu_in, mu_out, dphi)
                - table(pm, L, N, M, mu_in, mu_out, dphi)) / (2.0 * step)

    d1 = central(hk)
    if not richardson:
        return d1
    d2 = central(0.5 * hk)
    return (4.0 * d2 - d1) / 3.0


def loss(F, target) -> float:
    return 0.5 * float(np.sum((np.asarray(F) - np.asarray(target)) ** 2))


def loss_gradient(p, target, L, N, M, mu_in, mu_out, dphi, indices=None, h: float = 1e-6,
                  richardson: bool = True) -> np.ndarray:
    """dL/dp for the components in `indices` (all by default; the others stay 0)."""
    p = np.asarray(p, dtype=float)
    r = table(p, L, N, M, mu_in, mu_out, dphi) - np.asarray(target)
    g = np.zeros(p.size)
    for k in (range(p.size) if indices is None else indices):
        g[k] = float(np.sum(r * table_derivative(p, k, L, N, M, mu_in, mu_out, dphi, h,
                                                 richardson)))
    return g
