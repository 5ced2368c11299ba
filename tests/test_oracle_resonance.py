"""Pin of the oracle's particular solution across a resonance (Sec. 3.B, particular solution;
the beam term of Eqs. 28-33): where 1 + mu0 kappa_j = 0 for a decaying mode, the particular
solve (T + I / mu0) z = q is singular, but the radiance is not: the boundary solve answers
with a homogeneous coefficient that cancels the growing particular part, and the exiting
radiance is a smooth function of mu0 through the resonance. Over incident cosines within
2e-6 of a resonance, a low-degree polynomial in mu0 fits every element of the reconstructed
order radiance to within max(1e-10, 2 u / gap) of the order-0 radiance I^0_00 at the same
directions (u = 2^-52, gap = min_j |1 + mu0 kappa_j|): the rounding that the conditioning
1 / gap leaves is within the FP64 tolerance that the parity tests grant near a resonance.
A dropped or mis-signed term of the particular solution or of its boundary values leaves
the 1 / gap pole in the radiance and fails the fit by orders of magnitude.
"""
import numpy as np

import oracle as O
from vrte_inputs.mie import polydisperse_coefficients

U = 2.0 ** -52


def _layer():
    N, L, n_if = 16, 32, 1.33
    nodes = O.gauss_legendre_01(N)
    return dict(coef=polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, L), omega=0.95,
                tau=2.0, N=N, nodes=nodes, R_top=O.fresnel_internal_reflection(nodes[0], n_if))


def _solve(ly, m, mu0):
    beam = np.repeat(np.eye(4)[None], mu0.size, axis=0)
    return O.solve_order(m, ly["coef"], ly["omega"], ly["tau"], ly["N"], mu0, beam,
                         ly["R_top"], ly["nodes"])


def test_order_radiance_is_smooth_across_a_resonance():
    ly = _layer()
    m = 2
    probe = _solve(ly, m, np.array([0.5]))
    kap = probe.kappa[(probe.kappa.real < 0.0) & (np.abs(probe.kappa.imag) == 0.0)]
    mu_r = -1.0 / kap.real
    mu_r = mu_r[(mu_r > 0.3) & (mu_r < 0.95)]
    assert mu_r.size > 0
    mu_r = mu_r[0]
    # cosines on both sides of the resonance (none on it): gaps from ~1e-9 to ~2e-6
    half, n_pts = 2e-6, 200
    d = (np.arange(n_pts) - n_pts / 2 + 0.5) * (2 * half / n_pts)
    mu0 = mu_r + d
    mo = np.array([0.15, 0.55, 0.9])
    sol = _solve(ly, m, mu0)
    I = sol.reconstruct_top(mo)                                  # [n_mu0, n_out, 4, 4]
    assert np.all(np.isfinite(I))
    gap = np.abs(1.0 + mu0[:, None] * sol.kappa[None, sol.kappa.real < 0.0]).min(axis=1)
    assert gap.min() < 1e-7                                       # the sample spans the resonance
    # the particular part alone is singular there: |z| grows like 1 / gap
    z = np.abs(sol.z).reshape(sol.z.shape[0], n_pts, 4).max(axis=(0, 2))
    lo, hi = np.argmin(gap), np.argmax(gap)
    assert z[lo] / z[hi] > 0.3 * gap[hi] / gap[lo]
    I0 = _solve(ly, 0, mu0).reconstruct_top(mo)[..., 0, 0]       # [n_mu0, n_out]
    V = np.vander(d / half, 9)
    Y = I.reshape(n_pts, -1)
    fit, *_ = np.linalg.lstsq(V, Y, rcond=None)
    res = np.abs(Y - V @ fit).reshape(I.shape) / np.abs(I0)[:, :, None, None]
    bound = np.maximum(1e-10, 2.0 * U / gap)[:, None, None, None]
    assert np.all(res <= bound), float((res / bound).max())
    # and the fit itself is not swamped: away from the pole the residual is at rounding level
    far = gap > 1e-6
    assert far.any() and res[far].max() < 1e-10


def test_error_at_a_resonance_is_the_conditioning_1_over_gap():
    """Against a reference with no resonance at all: the top radiance from the matrix
    exponential of the augmented system d/dtau [u; s] = [[T, -M^-1 q], [0, -1/mu0]] [u; s]
    (the beam carried as an extra state, so nothing divides by 1 + mu0 kappa_j), with the
    top boundary condition and the black base imposed on the propagator (as in the brute-force
    pin of the per-order solution; N = 3 and tau0 = 0.8 keep the propagator well conditioned).
    The oracle's error grows as u / gap and no faster (measured ~3 u / gap of the largest
    component, from gap = 1e-3 to 1e-10): the rounding that the FP64 parity tolerance widens
    for, with the radiance itself finite and correct to that level."""
    from scipy.linalg import expm
    coef = polydisperse_coefficients(1.5 + 0.001j, 5.0, 0.1, 12)
    N, tau0, omega, m = 3, 0.8, 0.9, 2
    nodes = O.gauss_legendre_01(N)
    R = O.fresnel_internal_reflection(nodes[0], 1.33)
    N4 = 4 * N

    def solve(mu0):
        return O.solve_order(m, coef, omega, tau0, N, np.array([mu0]), np.eye(4)[None], R, nodes)

    kap = solve(0.5).kappa
    mu_r = -1.0 / kap[(kap.real < 0.0) & (kap.imag == 0.0)].real
    mu_r = mu_r[(mu_r > 0.3) & (mu_r < 0.95)][0]
    errs = {}
    for delta in (1e-3, 1e-6, 1e-8, 1e-10):
        mu0 = mu_r * (1.0 + delta)
        sol = solve(mu0)
        gap = np.abs(1.0 + mu0 * sol.kappa[sol.kappa.real < 0.0]).min()
        err = 0.0
        for col in range(4):
            aug = np.zeros((8 * N + 1, 8 * N + 1))
            aug[:-1, :-1] = sol.T
            aug[:-1, -1] = -sol.q[:, col] / sol.m8
            aug[-1, -1] = -1.0 / mu0
            P = expm(aug * tau0)
            # u(0) = [x; R x] with x = u_up(0); black base: the upward part of u(tau0) is zero
            x = np.linalg.solve(P[:N4, :-1] @ np.vstack([np.eye(N4), sol.R]), -P[:N4, -1])
            y = sol.nodal(0.0)[:N4, col]
            assert np.all(np.isfinite(y))
            err = max(err, np.abs(x - y).max() / np.abs(x).max())
        assert err <= 10.0 * U / gap + 1e-12, (delta, err, U / gap)
        errs[delta] = err
    assert errs[1e-3] < 1e-11
    assert errs[1e-10] > 100.0 * errs[1e-3]        # the 1 / gap growth is real
