"""Phase matrices: the order-m matrices A^m (Sec. 2.B, Eqs. 6-10) and the directly
rotated phase matrix they must add up to.

* `B_matrix`: the 4x4 coefficient block B_l of Eq. 9. The paper only says it
  "contains the expansion coefficients"; with the six coefficients
  (alpha1..alpha4, beta1, beta2) of the scattering matrix
  F = [[a1, b1, 0, 0], [b1, a2, 0, 0], [0, 0, a3, b2], [0, 0, -b2, a4]] it is
  B_l = [[alpha1, beta1, 0, 0], [beta1, alpha2, 0, 0], [0, 0, alpha3, beta2],
         [0, 0, -beta2, alpha4]].
* `A_matrix`: A^m(mu, mu') = sum_{l=m}^{L-1} P_l^m(mu) B_l P_l^m(mu')   (Eq. 9).
* `scattering_matrix`: F(Theta) from the coefficients,
  a1 = sum alpha1_l d^l_00, a4 = sum alpha4_l d^l_00, a2 + a3 = sum (alpha2+alpha3)_l d^l_22,
  a2 - a3 = sum (alpha2-alpha3)_l d^l_2,-2, b1 = -sum beta1_l d^l_02, b2 = -sum beta2_l d^l_02.
* `phase_matrix_direct`: Z(n_s <- n_i) = L(beta) F(Theta) L(alpha), built from the
  actual direction vectors: cos Theta = n_i . n_s (Eq. 5), alpha rotates the
  incident meridian frame into the scattering-plane frame, beta rotates the
  scattered scattering-plane frame into its meridian frame.
* `fourier_synthesis_phase`: sum_m sum_k Phi_k^m(phi_s - phi_i) A^m D_k with
  Phi_1^m = (2 - delta_m0) diag(cos, cos, sin, sin), Phi_2^m = (2 - delta_m0)
  diag(-sin, -sin, cos, cos), D_1 = diag(1,1,0,0), D_2 = diag(0,0,1,1) (Eqs. 6-8).
  The azimuth argument is (scattered - incident), the same order as the
  radiance expansion of Eq. 12; with the paper's printed (phi' - phi) the sine
  terms would change sign and the per-order equations would no longer carry
  the full A^m.

Pinned by tests: Rayleigh closed form of F, the Fourier synthesis equal to the
direct rotation at random directions (1e-13), reciprocity and mirror symmetry of
the direct phase matrix, and the parity relation of Eq. 10.
"""
from __future__ import annotations

import math

import numpy as np

from .gsf import gsf_tables, wigner_d_jacobi


def B_matrix(c) -> np.ndarray:
    """B_l from one coefficient row (alpha1, alpha2, alpha3, alpha4, beta1, beta2)."""
    a1, a2, a3, a4, b1, b2 = c
    return np.array([[a1, b1, 0.0, 0.0],
                     [b1, a2, 0.0, 0.0],
                     [0.0, 0.0, a3, b2],
                     [0.0, 0.0, -b2, a4]])


def P_matrices(m: int, L: int, mu) -> np.ndarray:
    """P_l^m(mu_k) as an array [L, K, 4, 4] (zero for l < m)."""
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    p, r, t = gsf_tables(m, L, mu)
    P = np.zeros((L, mu.size, 4, 4))
    P[:, :, 0, 0] = p
    P[:, :, 3, 3] = p
    P[:, :, 1, 1] = r
    P[:, :, 2, 2] = r
    P[:, :, 1, 2] = -t
    P[:, :, 2, 1] = -t
    return P


def A_matrix(m: int, coef, mu, mup) -> np.ndarray:
    """A^m(mu_i, mu'_j) as [len(mu), len(mu'), 4, 4] (Eq. 9), summing l = m..L-1."""
    coef = np.asarray(coef, dtype=float)
    L = coef.shape[0]
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    mup = np.atleast_1d(np.asarray(mup, dtype=float))
    if m >= L:
        return np.zeros((mu.size, mup.size, 4, 4))
    P1 = P_matrices(m, L, mu)
    P2 = P_matrices(m, L, mup)
    B = np.stack([B_matrix(c) for c in coef])
    PB = np.einsum("lxab,lbc->lxac", P1, B)
    return np.einsum("lxac,lycd->xyad", PB, P2)


def scattering_matrix(coef, cos_theta) -> np.ndarray:
    """F(Theta) [..., 4, 4] in the scattering-plane frame from the coefficients."""
    coef = np.asarray(coef, dtype=float)
    ct = np.clip(np.asarray(cos_theta, dtype=float), -1.0, 1.0)
    th = np.arccos(ct)
    a1 = np.zeros_like(th)
    a4 = np.zeros_like(th)
    s23 = np.zeros_like(th)
    d23 = np.zeros_like(th)
    b1 = np.zeros_like(th)
    b2 = np.zeros_like(th)
    for l, (al1, al2, al3, al4, be1, be2) in enumerate(coef):
        d00 = wigner_d_jacobi(l, 0, 0, th)
        a1 = a1 + al1 * d00
        a4 = a4 + al4 * d00
        if l >= 2:
            s23 = s23 + (al2 + al3) * wigner_d_jacobi(l, 2, 2, th)
            d23 = d23 + (al2 - al3) * wigner_d_jacobi(l, 2, -2, th)
            d02 = wigner_d_jacobi(l, 0, 2, th)
            b1 = b1 - be1 * d02
            b2 = b2 - be2 * d02
    a2 = 0.5 * (s23 + d23)
    a3 = 0.5 * (s23 - d23)
    F = np.zeros(th.shape + (4, 4))
    F[..., 0, 0] = a1
    F[..., 0, 1] = b1
    F[..., 1, 0] = b1
    F[..., 1, 1] = a2
    F[..., 2, 2] = a3
    F[..., 2, 3] = b2
    F[..., 3, 2] = -b2
    F[..., 3, 3] = a4
    return F


def direction(mu: float, phi: float) -> np.ndarray:
    """Unit propagation vector with z up: (sin(theta) cos(phi), sin(theta) sin(phi), mu)."""
    st = math.sqrt(max(0.0, 1.0 - mu * mu))
    return np.array([st * math.cos(phi), st * math.sin(phi), mu])


def meridian_frame(mu: float, phi: float):
    """(e_theta, e_phi) of a propagation direction; e_theta x e_phi = direction."""
    st = math.sqrt(max(0.0, 1.0 - mu * mu))
    e_th = np.array([mu * math.cos(phi), mu * math.sin(phi), -st])
    e_ph = np.array([-math.sin(phi), math.cos(phi), 0.0])
    return e_th, e_ph


def stokes_rotation(angle: float) -> np.ndarray:
    """Stokes transform for a frame rotated by `angle` about the propagation direction.

    With e1' = cos(a) e1 + sin(a) e2 and e2' = -sin(a) e1 + cos(a) e2:
    Q' = cos(2a) Q + sin(2a) U, U' = -sin(2a) Q + cos(2a) U, I and V unchanged.
    """
    c, s = math.cos(2.0 * angle), math.sin(2.0 * angle)
    return np.array([[1.0, 0.0, 0.0, 0.0],
                     [0.0, c, s, 0.0],
                     [0.0, -s, c, 0.0],
                     [0.0, 0.0, 0.0, 1.0]])


def phase_matrix_direct(coef, mu_s: float, phi_s: float, mu_i: float, phi_i: float) -> np.ndarray:
    """Phase matrix for incident propagation (mu_i, phi_i) scattered into (mu_s, phi_s).

    Both Stokes vectors are on their meridian frames. The scattering-plane frame of
    a beam along n is (q x n, q) with q = n_i x n_s / |n_i x n_s|; for exact forward
    or backward scattering q is taken as the incident e_phi.
    """
    n_s = direction(mu_s, phi_s)
    n_i = direction(mu_i, phi_i)
    cos_th = float(np.clip(n_s @ n_i, -1.0, 1.0))
    q = np.cross(n_i, n_s)
    qn = float(np.linalg.norm(q))
    e1_i, e2_i = meridian_frame(mu_i, phi_i)
    if qn < 1e-14:
        q = e2_i
    else:
        q = q / qn
    par_i = np.cross(q, n_i)
    alpha = math.atan2(float(par_i @ e2_i), float(par_i @ e1_i))
    e1_s, _ = meridian_frame(mu_s, phi_s)
    par_s = np.cross(q, n_s)
    beta = math.atan2(float(e1_s @ q), float(e1_s @ par_s))
    F = scattering_matrix(coef, cos_th)
    return stokes_rotation(beta) @ F @ stokes_rotation(alpha)


def fourier_weights(m: int, dphi: float):
    """(Phi_1^m, Phi_2^m) of Eq. 7 as diagonal 4-vectors at azimuth difference dphi."""
    f = 1.0 if m == 0 else 2.0
    c, s = math.cos(m * dphi), math.sin(m * dphi)
    return f * np.array([c, c, s, s]), f * np.array([-s, -s, c, c])


def fourier_synthesis_phase(coef, mu_s: float, mu_i: float, dphi: float, M: int | None = None):
    """sum_{m<M} sum_k Phi_k^m(dphi) A^m(mu_s, mu_i) D_k (Eq. 6), dphi = phi_s - phi_i."""
    coef = np.asarray(coef, dtype=float)
    if M is None:
        M = coef.shape[0]
    Z = np.zeros((4, 4))
    D1 = np.array([1.0, 1.0, 0.0, 0.0])
    D2 = np.array([0.0, 0.0, 1.0, 1.0])
    for m in range(M):
        A = A_matrix(m, coef, [mu_s], [mu_i])[0, 0]
        w1, w2 = fourier_weights(m, dphi)
        Z += (w1[:, None] * A) * D1[None, :] + (w2[:, None] * A) * D2[None, :]
    return Z
