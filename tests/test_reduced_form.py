"""P10: the reduced 4N formulation the CUDA path implements (Sec. 3.A-3.B, Eqs. 41-48:
F'E' eigenpairs, Phi+- from E'X / kappa, the eigenbasis particular solution, the
boundary matrix of scaled modes, the parity-split reconstruction operators) reproduces
the oracle's full 8N solution of every order."""
import numpy as np
import pytest

import oracle as O
from reduced_model import solve_order_reduced
from vrte_inputs.mie import polydisperse_coefficients


@pytest.mark.parametrize("n_if", [1.0, 1.5])
@pytest.mark.parametrize("m", [0, 1, 3, 10])
def test_reduced_matches_full(n_if, m):
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 24)
    mu_in = np.array([0.23, 0.61, 0.97])
    mu_out = np.array([0.15, 0.5, 0.88, 0.99])
    N, omega, tau0 = 8, 0.97, 2.5
    nodes = O.gauss_legendre_01(N)
    beam = O.fresnel_beam_in(mu_in, n_if)
    mu0i, muoi = O.snell_mu(mu_in, n_if), O.snell_mu(mu_out, n_if)
    Rt = O.fresnel_internal_reflection(nodes[0], n_if) if n_if > 1 else None
    sol = O.solve_order(m, coef, omega, tau0, N, mu0i, beam, Rt, nodes)
    mout = O.fresnel_exit(mu_out, n_if)
    full = np.einsum("oab,iobc->ioac", mout, sol.reconstruct_top(muoi)) / mu_in[:, None, None, None]
    red, lam = solve_order_reduced(m, coef, omega, tau0, N, mu0i, beam / mu_in[:, None, None], Rt,
                                   muoi, mout)
    # the reduced problem carries complex eigenpairs for this particle layer
    assert np.sum(np.abs(lam.imag) > 0) > 0
    assert np.abs(red - full).max() < 1e-11 * np.abs(full).max()
    # eigenvalues of F'E' are the squares of the full problem's growing rates (P10)
    k_full = sol.kappa[sol.kappa.real > 0]
    a = np.sort_complex(np.round(k_full**2, 8))
    b = np.sort_complex(np.round(lam, 8))
    assert np.allclose(np.sort(np.abs(a)), np.sort(np.abs(b)), rtol=1e-9)
