"""Seeded layer/grid recipes for the five workloads the solver is measured on.

Every workload is deterministic: the base seed is 1707 plus the workload index.
Coefficient arrays are [L, 6] in the order (alpha1, alpha2, alpha3, alpha4,
beta1, beta2); angle grids hold cosines of external zenith angles in (0, 1] and
azimuth differences in radians.
"""
from __future__ import annotations

import math

import numpy as np

from .mie import polydisperse_coefficients

BASE_SEED = 1707

CONFIG_NAMES = {
    1: "rayleigh-N8-M3-8x8x16",
    2: "mie-N32-M64-L64-64x64x90-n1.5",
    3: "mie-N64-M128-L128-1024x1024x360-n1.5",
    4: "batched-256-layers-mixed-N-64x64x90",
    5: "adjoint-64-layers-N48-M96-64x64x90",
}


def rayleigh_coefficients() -> np.ndarray:
    """Expansion coefficients of the Rayleigh scattering matrix (no depolarisation).

    F11 = F22 = 3/4 (1 + cos^2), F12 = -3/4 sin^2, F33 = F44 = 3/2 cos, F34 = 0,
    which expand as alpha1 = (1, 0, 1/2), alpha2 = (0, 0, 3), alpha3 = 0,
    alpha4 = (0, 3/2, 0), beta1 = (0, 0, sqrt(6)/2), beta2 = 0 (l = 0, 1, 2).
    """
    c = np.zeros((3, 6))
    c[0, 0] = 1.0
    c[2, 0] = 0.5
    c[2, 1] = 3.0
    c[1, 3] = 1.5
    c[2, 4] = math.sqrt(6.0) / 2.0
    return c


def uniform_zenith_grid(n: int) -> np.ndarray:
    """mu_k = cos((k + 1/2) pi / (2 n)), k = 0..n-1: uniform in zenith angle, avoids mu = 0."""
    k = np.arange(n, dtype=float)
    return np.cos((k + 0.5) * math.pi / (2.0 * n))


def angle_grids(n_in: int, n_out: int, n_phi: int):
    """(mu_in, mu_out, dphi) with dphi_j = 2 pi j / n_phi over the full circle."""
    dphi = 2.0 * math.pi * np.arange(n_phi, dtype=float) / n_phi
    return uniform_zenith_grid(n_in), uniform_zenith_grid(n_out), dphi


def _layer(tau, omega, n_interface, N, M, coef):
    return dict(tau=float(tau), omega=float(omega), n_interface=float(n_interface),
                n_nodes=int(N), n_orders=int(M), coef=np.ascontiguousarray(coef, dtype=float))


def make_config(index: int, small: bool = False) -> dict:
    """Workload `index` (1..5) as dict(name, layers=[...], mu_in, mu_out, dphi).

    `small=True` keeps the layer(s) but shrinks the angle grids and layer count so
    the oracle finishes in seconds (used by parity tests).
    """
    rng = np.random.default_rng(BASE_SEED + index)
    if index == 1:
        layers = [_layer(1.0, 0.9, 1.0, 8, 3, rayleigh_coefficients())]
        grids = angle_grids(8, 8, 16)
    elif index in (2, 3):
        # the N = 64 layer is the N = 32 particle layer with larger particles, L = 128
        x_eff = rng.uniform(2.0, 20.0) if index == 2 else rng.uniform(2.0, 40.0)
        omega = rng.uniform(0.8, 0.999)
        L = 64 if index == 2 else 128
        N = 32 if index == 2 else 64
        coef = polydisperse_coefficients(1.5 + 0.001j, x_eff, 0.1, L)
        layers = [_layer(10.0, omega, 1.5, N, L, coef)]
        if index == 2:
            grids = angle_grids(64, 64, 90)
        else:
            grids = angle_grids(1024, 1024, 360)
    elif index == 4:
        n_layers = 8 if small else 256
        layers = []
        n_choices = [16, 24, 32, 48, 64, 96]
        for mat in range(8):
            n_real = rng.uniform(1.3, 1.7)
            m_ref = complex(n_real, rng.uniform(1e-4, 1e-2))
            r_eff_um = rng.uniform(0.2, 0.8)
            n_wl = n_layers // 8
            for w in range(n_wl):
                lam_um = 0.400 + 0.010 * (w * (32 // n_wl))
                x_eff = 2.0 * math.pi * r_eff_um / lam_um
                L = int(rng.integers(16, 129))
                N = int(rng.choice(n_choices))
                tau = math.exp(rng.uniform(math.log(0.1), math.log(100.0)))
                omega = rng.uniform(0.5, 0.999)
                coef = polydisperse_coefficients(m_ref, x_eff, 0.1, L, n_size=24)
                layers.append(_layer(tau, omega, n_real, N, L, coef))
        grids = angle_grids(64, 64, 90)
    elif index == 5:
        n_layers = 4 if small else 64
        layers = []
        for i in range(n_layers):
            x_eff = rng.uniform(2.0, 20.0)
            m_ref = complex(rng.uniform(1.3, 1.7), rng.uniform(1e-4, 1e-2))
            coef = polydisperse_coefficients(m_ref, x_eff, 0.1, 96, n_size=24)
            layers.append(_layer(math.exp(rng.uniform(0.0, math.log(50.0))),
                                 rng.uniform(0.5, 0.999), m_ref.real, 48, 96, coef))
        grids = angle_grids(64, 64, 90)
    else:
        raise ValueError(f"unknown workload {index}")
    mu_in, mu_out, dphi = grids
    return dict(name=CONFIG_NAMES[index], layers=layers, mu_in=mu_in, mu_out=mu_out, dphi=dphi)
