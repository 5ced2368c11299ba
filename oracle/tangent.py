"""Exact derivative of the BRDF with respect to one layer parameter, by forward-mode dual
numbers (value, derivative) carried through a propagator form of every Fourier order.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never calls it.

This is the oracle's gradient that is not a finite difference. It does not use the
eigen-decomposition of oracle.dom (a library eigensolver does not carry dual parts); each
order's two-point problem of Sec. 2.C is solved instead through matrix exponentials, and a
dual matrix X + eps X' is exponentiated exactly by the block identity
    expm([[X, X'], [0, X]]) = [[expm(X), D], [0, expm(X)]],   D = d/deps expm(X + eps X'),
so the derivative is exact up to rounding. For order m, beam cosine mu0 (internal) and the
four incident Stokes basis vectors at once:

  * state y = [u; e] with u the 8N nodal radiances and e = exp(-tau/mu0) I4, so that Eq. 15
    (M du/dtau = u - (omega/2) calA W u - q exp(-tau/mu0), oracle.dom) becomes the autonomous
    y' = A y,  A = [[T, -M^-1 q], [0, -I4/mu0]],  T = M^-1 (I - (omega/2) calA W);
  * boundary conditions (Eqs. 49-50 with the dielectric top): u(0) = [a; R_F a] and
    u_up(tau0) = 0 give one 4N x 4N solve for a = u_up(0) through expm(A tau0);
  * reconstruction at an internal outgoing cosine mu (Eqs. 36, 38 with the 1/mu of the formal
    solution): with v = y exp(-t/mu), v' = (A - I/mu) v and J' = H v / mu,
    H = [(omega/2) G(mu) W, (omega/2pi) A^m(mu, -mu0) b], so I^m(0, mu) = J(tau0) is one more
    exponential of the augmented matrix [[A - I/mu, 0], [H/mu, 0]].

The propagator form loses accuracy as exp(kappa_max tau0) for the growing modes, so it serves
small layers (N <= 4, tau0 of a few units), where it agrees with oracle.brdf to ~1e-10.

Dual parts enter through: the coefficients (linear in B_l), omega, tau0 (the exponentials'
argument A tau0), and the interface index n, which moves the internal cosines (Snell), the
phase-matrix tables at those cosines (d P_l^m / d mu from the derivative identity of the
Wigner functions, d/dtheta d^l_{m,n} = (1/2)[c- d^l_{m,n-1} - c+ d^l_{m,n+1}],
c-+ = sqrt((l +- n)(l -+ n + 1))) and the Fresnel matrices (written here in dual arithmetic).

Pinned by tests/test_oracle_tangent.py: the value equals oracle.brdf, the derivative identity
against differences of wigner_d_family, the dual Fresnel matrices against oracle.fresnel and
its differences, and the whole gradient against the Richardson central differences of
oracle.gradient and against the thin-layer closed forms.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

from .gsf import wigner_d_family
from .phase import B_matrix, P_matrices
from .quadrature import gauss_legendre_01


# ----------------------------------------------------------------- scalar dual numbers
class Dual:
    """Scalar dual number v + eps d with complex v, d."""

    __slots__ = ("v", "d")

    def __init__(self, v, d=0.0):
        self.v = complex(v)
        self.d = complex(d)

    @staticmethod
    def _c(x):
        return x if isinstance(x, Dual) else Dual(x, 0.0)

    def __add__(self, o):
        o = Dual._c(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual._c(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return Dual._c(o) - self

    def __mul__(self, o):
        o = Dual._c(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual._c(o)
        return Dual(self.v / o.v, (self.d * o.v - self.v * o.d) / (o.v * o.v))

    def __rtruediv__(self, o):
        return Dual._c(o) / self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def conj(self):
        return Dual(self.v.conjugate(), self.d.conjugate())

    def sqrt(self):
        r = np.sqrt(self.v)
        return Dual(r, self.d / (2.0 * r) if r != 0 else 0.0)

    @property
    def real(self):
        return Dual(self.v.real, self.d.real)


def _abs2(z: Dual) -> Dual:
    return (z * z.conj()).real


def _mueller(jp: Dual, js: Dual):
    """(value, derivative) 4x4 Mueller matrices of diag(jp, js) on meridian frames
    (the map of oracle.fresnel, written in dual arithmetic)."""
    a = 0.5 * (_abs2(jp) + _abs2(js))
    b = 0.5 * (_abs2(jp) - _abs2(js))
    z = jp * js.conj()
    M = np.zeros((4, 4))
    dM = np.zeros((4, 4))
    for (i, j), e in {(0, 0): a, (1, 1): a, (0, 1): b, (1, 0): b}.items():
        M[i, j], dM[i, j] = e.v.real, e.d.real
    M[2, 2] = M[3, 3] = z.v.real
    dM[2, 2] = dM[3, 3] = z.d.real
    M[2, 3], dM[2, 3] = z.v.imag, z.d.imag
    M[3, 2], dM[3, 2] = -z.v.imag, -z.d.imag
    return M, dM


def _amplitudes(c1, n1, n2):
    """(rp, rs, tp, ts) in dual arithmetic; beyond the critical angle the transmitted cosine
    is +i sqrt(.) (evanescent under exp(-i w t))."""
    c1, n1, n2 = Dual._c(c1), Dual._c(n1), Dual._c(n2)
    s2sq = (n1 / n2) * (n1 / n2) * (1.0 - c1 * c1)
    if s2sq.v.real <= 1.0:
        c2 = (1.0 - s2sq).sqrt()
    else:
        c2 = Dual(1j, 0.0) * (s2sq - 1.0).sqrt()
    rs = (n1 * c1 - n2 * c2) / (n1 * c1 + n2 * c2)
    rp = (n2 * c1 - n1 * c2) / (n2 * c1 + n1 * c2)
    ts = 2.0 * n1 * c1 / (n1 * c1 + n2 * c2)
    tp = 2.0 * n1 * c1 / (n2 * c1 + n1 * c2)
    return rp, rs, tp, ts


def interface_dual(mu_in, mu_out, mu_nodes, n: float, dn: float):
    """Internal cosines, beam, exit and reflection matrices with their derivatives along dn:
    (mu0, dmu0), (mu_o, dmu_o), (Min, dMin), (Mout, dMout), (R, dR); R None without interface."""
    mu_in = np.atleast_1d(np.asarray(mu_in, float))
    mu_out = np.atleast_1d(np.asarray(mu_out, float))
    if n <= 1.0:
        eye = np.broadcast_to(np.eye(4), (mu_in.size, 4, 4)).copy()
        eyo = np.broadcast_to(np.eye(4), (mu_out.size, 4, 4)).copy()
        return ((mu_in.copy(), np.zeros(mu_in.size)), (mu_out.copy(), np.zeros(mu_out.size)),
                (eye, np.zeros_like(eye)), (eyo, np.zeros_like(eyo)), (None, None))
    nd = Dual(n, dn)

    def snell(me):
        return (1.0 - (1.0 - me * me) / (nd * nd)).sqrt()

    mi = [snell(x) for x in mu_in]
    mo = [snell(x) for x in mu_out]
    Min = np.zeros((mu_in.size, 4, 4))
    dMin = np.zeros_like(Min)
    for k, me in enumerate(mu_in):
        _, _, tp, ts = _amplitudes(me, 1.0, nd)
        M, dM = _mueller(tp, ts)
        Min[k] = n * M
        dMin[k] = dn * M + n * dM
    Mout = np.zeros((mu_out.size, 4, 4))
    dMout = np.zeros_like(Mout)
    for o, me in enumerate(mu_out):
        _, _, tp, ts = _amplitudes(mo[o], nd, 1.0)
        M, dM = _mueller(tp, ts)
        f = me / (nd * nd * nd * mo[o])   # Re(c2) / (n^3 mu_int) with c2 = mu_ext
        Mout[o] = f.v.real * M
        dMout[o] = f.d.real * M + f.v.real * dM
    R = np.zeros((mu_nodes.size, 4, 4))
    dR = np.zeros_like(R)
    for i, c1 in enumerate(mu_nodes):
        rp, rs, _, _ = _amplitudes(c1, nd, 1.0)
        R[i], dR[i] = _mueller(rp, rs)
    return ((np.array([x.v.real for x in mi]), np.array([x.d.real for x in mi])),
            (np.array([x.v.real for x in mo]), np.array([x.d.real for x in mo])),
            (Min, dMin), (Mout, dMout), (R, dR))


# ----------------------------------------------------------------- tables and their mu-derivative
def dP_dmu(m: int, L: int, mu) -> np.ndarray:
    """d P_l^m / d mu [L, K, 4, 4] from d/dtheta d^l_{m,n} = (1/2)[c- d^l_{m,n-1} - c+ d^l_{m,n+1}]
    with c-+ = sqrt((l +- n)(l -+ n + 1)) and d mu = -sin(theta) d theta (interior cosines)."""
    mu = np.atleast_1d(np.asarray(mu, dtype=float))
    lmax = L - 1
    ls = np.arange(L, dtype=float)[:, None]

    def ddtheta(nn):
        cm = np.sqrt(np.clip((ls + nn) * (ls - nn + 1), 0.0, None))
        cp = np.sqrt(np.clip((ls - nn) * (ls + nn + 1), 0.0, None))
        return 0.5 * (cm * wigner_d_family(lmax, m, nn - 1, mu)
                      - cp * wigner_d_family(lmax, m, nn + 1, mu))

    sin_t = np.sqrt(1.0 - mu * mu)[None, :]
    dp = -ddtheta(0) / sin_t
    dp2 = -ddtheta(2) / sin_t
    dm2 = -ddtheta(-2) / sin_t
    dr, dt = -0.5 * (dp2 + dm2), -0.5 * (dp2 - dm2)
    D = np.zeros((L, mu.size, 4, 4))
    D[:, :, 0, 0] = D[:, :, 3, 3] = dp
    D[:, :, 1, 1] = D[:, :, 2, 2] = dr
    D[:, :, 1, 2] = D[:, :, 2, 1] = -dt
    return D


def _A_dual(m, coef, dcoef, x, dx, y, dy):
    """A^m(x_i, y_j) [nx, ny, 4, 4] and its derivative for moving points and coefficients."""
    L = coef.shape[0]
    x = np.atleast_1d(np.asarray(x, float))
    y = np.atleast_1d(np.asarray(y, float))
    if m >= L:
        z = np.zeros((x.size, y.size, 4, 4))
        return z, z.copy()
    Px, Py = P_matrices(m, L, x), P_matrices(m, L, y)
    B = np.stack([B_matrix(c) for c in coef])
    dB = np.stack([B_matrix(c) for c in dcoef])
    A = np.einsum("lxab,lbc,lycd->xyad", Px, B, Py)
    dA = np.einsum("lxab,lbc,lycd->xyad", Px, dB, Py)
    dx = np.broadcast_to(np.asarray(dx, float), x.shape)
    dy = np.broadcast_to(np.asarray(dy, float), y.shape)
    if np.any(dx != 0.0):
        dPx = dP_dmu(m, L, x) * dx[None, :, None, None]
        dA = dA + np.einsum("lxab,lbc,lycd->xyad", dPx, B, Py)
    if np.any(dy != 0.0):
        dPy = dP_dmu(m, L, y) * dy[None, :, None, None]
        dA = dA + np.einsum("lxab,lbc,lycd->xyad", Px, B, dPy)
    return A, dA


def _stack(A4):
    X, Y = A4.shape[0], A4.shape[1]
    return A4.transpose(0, 2, 1, 3).reshape(4 * X, 4 * Y)


def _dexpm(X, dX):
    n = X.shape[0]
    big = np.zeros((2 * n, 2 * n))
    big[:n, :n] = X
    big[n:, n:] = X
    big[:n, n:] = dX
    E = expm(big)
    return E[:n, :n], E[:n, n:]


# ----------------------------------------------------------------- one order, propagator form
def order_radiance_dual(m, coef, dcoef, omega, domega, tau0, dtau0, N, mu0, dmu0, beam, dbeam,
                        R, dR, mu_out, dmu_out):
    """I^m(0, mu_out) [n_in, n_out, 4, 4] (rows = exiting Stokes, columns = incident basis,
    beam included) and its derivative, from the propagator form of the module docstring."""
    mu_n, al = gauss_legendre_01(N)
    n4, n8 = 4 * N, 8 * N
    mus = np.concatenate([mu_n, -mu_n])
    m8 = np.repeat(mus, 4)
    w8 = np.repeat(np.concatenate([al, al]), 4)
    zero_n = np.zeros(mus.size)
    cA, dcA = _A_dual(m, coef, dcoef, mus, zero_n, mus, zero_n)
    calA, dcalA = _stack(cA), _stack(dcA)
    T = (np.eye(n8) - 0.5 * omega * calA * w8[None, :]) / m8[:, None]
    dT = (-0.5 * domega * calA - 0.5 * omega * dcalA) * w8[None, :] / m8[:, None]
    cQ, dcQ = omega / (2 * np.pi), domega / (2 * np.pi)
    Rb = np.zeros((n4, n4))
    dRb = np.zeros((n4, n4))
    if R is not None:
        for i in range(N):
            Rb[4 * i:4 * i + 4, 4 * i:4 * i + 4] = R[i]
            dRb[4 * i:4 * i + 4, 4 * i:4 * i + 4] = dR[i]
    n_in, n_out = len(mu0), len(mu_out)
    I = np.zeros((n_in, n_out, 4, 4))
    dI = np.zeros_like(I)
    na = n8 + 4
    for k in range(n_in):
        Aq, dAq = _A_dual(m, coef, dcoef, mus, zero_n, [-mu0[k]], [-dmu0[k]])
        Aq, dAq = _stack(Aq), _stack(dAq)                              # [8N, 4]
        q = cQ * Aq @ beam[k]
        dq = dcQ * Aq @ beam[k] + cQ * dAq @ beam[k] + cQ * Aq @ dbeam[k]
        Aa = np.zeros((na, na))
        dAa = np.zeros((na, na))
        Aa[:n8, :n8], dAa[:n8, :n8] = T, dT
        Aa[:n8, n8:], dAa[:n8, n8:] = -q / m8[:, None], -dq / m8[:, None]
        Aa[n8:, n8:] = -np.eye(4) / mu0[k]
        dAa[n8:, n8:] = np.eye(4) * dmu0[k] / mu0[k] ** 2
        Phi, dPhi = _dexpm(Aa * tau0, dAa * tau0 + Aa * dtau0)
        up, down, ee = slice(0, n4), slice(n4, n8), slice(n8, na)
        Kb = Phi[up, up] + Phi[up, down] @ Rb
        dKb = dPhi[up, up] + dPhi[up, down] @ Rb + Phi[up, down] @ dRb
        a = np.linalg.solve(Kb, -Phi[up, ee])
        da = np.linalg.solve(Kb, -dPhi[up, ee] - dKb @ a)
        y0 = np.concatenate([a, Rb @ a, np.eye(4)], axis=0)            # [na, 4]
        dy0 = np.concatenate([da, dRb @ a + Rb @ da, np.zeros((4, 4))], axis=0)
        for o in range(n_out):
            mo, dmo = mu_out[o], dmu_out[o]
            G, dG = _A_dual(m, coef, dcoef, [mo], [dmo], mus, zero_n)
            G, dG = _stack(G), _stack(dG)                              # [4, 8N]
            Ad, dAd = _A_dual(m, coef, dcoef, [mo], [dmo], [-mu0[k]], [-dmu0[k]])
            Ad, dAd = Ad[0, 0], dAd[0, 0]
            H = np.concatenate([0.5 * omega * G * w8[None, :], cQ * Ad @ beam[k]], axis=1)
            dH = np.concatenate([(0.5 * domega * G + 0.5 * omega * dG) * w8[None, :],
                                 dcQ * Ad @ beam[k] + cQ * dAd @ beam[k] + cQ * Ad @ dbeam[k]],
                                axis=1)
            nb = na + 4
            Bm = np.zeros((nb, nb))
            dBm = np.zeros((nb, nb))
            Bm[:na, :na] = Aa - np.eye(na) / mo
            dBm[:na, :na] = dAa + np.eye(na) * dmo / mo ** 2
            Bm[na:, :na] = H / mo
            dBm[na:, :na] = dH / mo - H * dmo / mo ** 2
            E, dE = _dexpm(Bm * tau0, dBm * tau0 + Bm * dtau0)
            I[k, o] = E[na:, :na] @ y0
            dI[k, o] = dE[na:, :na] @ y0 + E[na:, :na] @ dy0
    return I, dI


def _synthesis_weights(m, dphi):
    f = 1.0 if m == 0 else 2.0
    arg = m * (np.atleast_1d(dphi) - np.pi)
    c, s = f * np.cos(arg), f * np.sin(arg)
    w = np.zeros((c.size, 4, 4))
    for r in range(4):
        for col in range(4):
            if col < 2:
                w[:, r, col] = c if r < 2 else s
            else:
                w[:, r, col] = -s if r < 2 else c
    return w


def brdf_dual(p, dp, L, N, M, mu_in, mu_out, dphi):
    """F[n_in, n_out, n_phi, 4, 4] and dF along dp for the parameter vector
    p = (omega, tau0, n, coef[L, 6] flattened) of oracle.gradient."""
    p = np.asarray(p, float)
    dp = np.asarray(dp, float)
    omega, tau0, nif = p[0], p[1], p[2]
    domega, dtau0, dn = dp[0], dp[1], dp[2]
    coef = p[3:3 + 6 * L].reshape(L, 6)
    dcoef = dp[3:3 + 6 * L].reshape(L, 6)
    mu_in = np.atleast_1d(np.asarray(mu_in, float))
    mu_out = np.atleast_1d(np.asarray(mu_out, float))
    mu_n, _ = gauss_legendre_01(N)
    (mu0, dmu0), (mo, dmo), (Min, dMin), (Mout, dMout), (R, dR) = interface_dual(
        mu_in, mu_out, mu_n, nif, dn)
    F = np.zeros((mu_in.size, mu_out.size, np.size(dphi), 4, 4))
    dF = np.zeros_like(F)
    for m in range(min(M, L)):
        I, dI = order_radiance_dual(m, coef, dcoef, omega, domega, tau0, dtau0, N, mu0, dmu0,
                                    Min, dMin, R, dR, mo, dmo)
        w = _synthesis_weights(m, dphi)
        F += 0.5 * I[:, :, None] * w[None, None]
        dF += 0.5 * dI[:, :, None] * w[None, None]
    # exit through the interface and the 1/mu_in of F = I / (mu_in I0)
    dF = (np.einsum("oab,iojbc->iojac", dMout, F) + np.einsum("oab,iojbc->iojac", Mout, dF))
    F = np.einsum("oab,iojbc->iojac", Mout, F)
    return F / mu_in[:, None, None, None, None], dF / mu_in[:, None, None, None, None]


def loss_gradient(p, target, L, N, M, mu_in, mu_out, dphi, indices=None):
    """dL/dp for L = 1/2 |F - target|^2 along the unit directions in `indices` (all by
    default; the interface entry is skipped when there is no interface)."""
    p = np.asarray(p, float)
    g = np.zeros(p.size)
    for k in (range(p.size) if indices is None else indices):
        if k == 2 and p[2] <= 1.0:
            continue
        e = np.zeros(p.size)
        e[k] = 1.0
        F, dF = brdf_dual(p, e, L, N, M, mu_in, mu_out, dphi)
        g[k] = float(np.sum((F - np.asarray(target)) * dF))
    return g
