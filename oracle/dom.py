"""One Fourier order of the DOM solution in the full 8N formulation (Sec. 2.C).

For order m the radiance at the 2N double-Gauss directions +-mu_n is stacked as
u(tau) = [I(tau, +mu_1..+mu_N); I(tau, -mu_1..-mu_N)] (8N values, 4 Stokes
components per direction). With tau downward and mu > 0 upward, Eq. 15 reads

    M du/dtau = u - (omega/2) calA W u - q exp(-tau/mu0),                  (1)

M = diag(+-mu_n I4) (Eq. 20), W = diag(alpha_n I4) on both hemispheres (Eq. 21),
calA[(s,i),(s',n)] = A^m(s mu_i, s' mu_n) (Eqs. 22-23) and
q[(s,i)] = (omega / 2 pi) A^m(s mu_i, -mu0) I0' (Eq. 14 with the factor and beam
direction explained in the package docstring). The weights multiply the
integration (column) index, which is what the quadrature sum of Eq. 15 needs.

* Homogeneous part (Eqs. 16-19): u = v exp(kappa tau) with kappa, v the 8N
  eigenpairs of T = M^-1 (I - (omega/2) calA W). The basis function of a mode is
  exp(kappa tau) if Re kappa < 0 and exp(kappa (tau - tau0)) otherwise, the scaled
  form of Eqs. 24-25 (every basis function is bounded by 1 on [0, tau0]).
* Particular part (Eqs. 28-33): u = z exp(-tau/mu0) with
  (I - (omega/2) calA W + M/mu0) z = q, solved by LU for every mu0.
* Boundary conditions (Eqs. 49-54): no diffuse light enters at the top, or with a
  dielectric top the downward radiance equals the internally reflected upward
  radiance, u_down(0) = R_F u_up(0); black base u_up(tau0) = 0 (Eq. 35 with R = 0).
  The 8N coefficients c follow from one dense LU solve with all beams as
  right-hand sides.
* Reconstruction (Eqs. 36, 38): for an upward internal cosine mu at tau = 0,
    I^m(0, mu) = int_0^tau0 S(t, mu) exp(-t/mu) dt / mu,
    S(t, mu) = (omega/2) sum_{s,n} alpha_n A^m(mu, s mu_n) u_{s,n}(t)
               + (omega / 2 pi) A^m(mu, -mu0) I0' exp(-t/mu0),
  with the depth integral of every exponential in closed form. (The paper's
  Eq. 36 omits the 1/mu of the formal solution; it is restored here.)

Complex eigenpairs are kept complex; the physical field is the real part (its
imaginary part is zero to round-off because modes come in conjugate pairs).

Pinned by tests: every mode and the particular solution satisfy (1) at random
tau; boundary residuals; reconstruction at a node equals the nodal solution;
brute-force matrix-exponential propagation for tiny N; the exact discrete flux
balance; the single-scattering limit; the H-function limit; reciprocity.
"""
from __future__ import annotations

import numpy as np

from .phase import A_matrix
from .quadrature import gauss_legendre_01


def expm1_complex(z):
    """exp(z) - 1 for complex arrays, by its Taylor series where |z| is small."""
    z = np.asarray(z, dtype=complex)
    small = np.abs(z) < 1e-2
    with np.errstate(over="ignore", invalid="ignore"):
        out = np.exp(z) - 1.0
    zs = z[small]
    term = zs.copy()
    acc = zs.copy()
    for k in range(2, 10):
        term = term * zs / k
        acc = acc + term
    out[small] = acc
    return out


def _stack_matrix(A4):
    """[X, Y, 4, 4] block array -> [4X, 4Y] matrix with row (x, a), column (y, b)."""
    X, Y = A4.shape[0], A4.shape[1]
    return A4.transpose(0, 2, 1, 3).reshape(4 * X, 4 * Y)


class OrderSolution:
    """Nodal solution of one Fourier order for a set of collimated beams.

    Right-hand sides are indexed (beam i, incident Stokes column s) -> i*4 + s.
    """

    def __init__(self, m, coef, omega, tau0, mu_nodes, alpha, mu0, beam, R_top, rho=0.0,
                 base=None):
        self.m = m
        self.coef = np.asarray(coef, dtype=float)
        self.omega = float(omega)
        self.tau0 = float(tau0)
        self.mu_nodes = np.asarray(mu_nodes, dtype=float)
        self.alpha = np.asarray(alpha, dtype=float)
        self.mu0 = np.atleast_1d(np.asarray(mu0, dtype=float))
        self.beam = np.asarray(beam, dtype=float).reshape(self.mu0.size, 4, 4)
        N = self.mu_nodes.size
        self.N = N
        self.mus = np.concatenate([self.mu_nodes, -self.mu_nodes])
        n8 = 8 * N
        self.calA = _stack_matrix(A_matrix(m, self.coef, self.mus, self.mus))
        self.w8 = np.repeat(np.concatenate([self.alpha, self.alpha]), 4)
        self.m8 = np.repeat(self.mus, 4)
        self.cQ = self.omega / (2.0 * np.pi)
        lhs = np.eye(n8) - 0.5 * self.omega * self.calA * self.w8[None, :]
        self.T = lhs / self.m8[:, None]
        kappa, V = np.linalg.eig(self.T)
        self.kappa = kappa
        self.V = V
        self.growing = kappa.real >= 0.0
        # particular solutions, one LU per beam cosine
        n_rhs = 4 * self.mu0.size
        self.q = np.zeros((n8, n_rhs))
        self.z = np.zeros((n8, n_rhs))
        for i, mu0 in enumerate(self.mu0):
            Aq = _stack_matrix(A_matrix(m, self.coef, self.mus, [-mu0]))  # [8N, 4]
            qi = self.cQ * Aq @ self.beam[i]
            self.q[:, 4 * i:4 * i + 4] = qi
            self.z[:, 4 * i:4 * i + 4] = np.linalg.solve(lhs + np.diag(self.m8 / mu0), qi)
        self.rhs_mu0 = np.repeat(self.mu0, 4)
        # boundary conditions
        up = np.arange(4 * N)
        down = 4 * N + np.arange(4 * N)
        R = np.zeros((4 * N, 4 * N))
        if R_top is not None:
            for i in range(N):
                R[4 * i:4 * i + 4, 4 * i:4 * i + 4] = R_top[i]
        self.R = R
        f0 = self._basis(0.0)
        f1 = self._basis(self.tau0)
        K = np.zeros((n8, n8), dtype=complex)
        K[:4 * N] = (V[down] - R @ V[up]) * f0[None, :]
        K[4 * N:] = V[up] * f1[None, :]
        att = np.exp(-self.tau0 / self.rhs_mu0)
        rhs = np.zeros((n8, n_rhs))
        rhs[:4 * N] = -(self.z[down] - R @ self.z[up])
        rhs[4 * N:] = -self.z[up] * att[None, :]
        # Reflecting base (Sec. 3.C, base reflection) with a direction-independent Mueller BRDF
        # R of the base (R = base + 2 rho e0 e0^T; the Lambertian base of albedo rho is
        # R_00 = 2 rho): only order 0 sees it, as it has no azimuth dependence. The upward
        # radiance at the bottom is isotropic,
        #   I^0(tau0, +mu) = R sum_j alpha_j mu_j I^0(tau0, -mu_j) + (1/pi) mu0 R I0' e^{-tau0/mu0}
        # (the beam's order-0 Fourier part is I0'/pi in the Fourier convention of Eq. 12, the
        # same factor-2 reading as the source constant). An azimuth-independent R keeps its
        # (I, Q) x (U, V) blocks zero: those couple through the sine terms, which vanish at m = 0.
        self.rho = float(rho) if m == 0 else 0.0
        Rg = np.zeros((4, 4))
        if m == 0:
            Rg[0, 0] = 2.0 * float(rho)
            if base is not None:
                Rg = Rg + np.asarray(base, dtype=float).reshape(4, 4)
        self.Rbase = Rg if np.any(Rg != 0.0) else None
        if self.Rbase is not None:
            Rb = np.zeros((4 * N, 4 * N))
            for i in range(N):
                for j in range(N):
                    Rb[4 * i:4 * i + 4, 4 * j:4 * j + 4] = Rg * (self.alpha[j] * self.mu_nodes[j])
            self.Rb = Rb
            K[4 * N:] -= (Rb @ V[down]) * f1[None, :]
            rhs[4 * N:] += (Rb @ self.z[down]) * att[None, :]
            ls = np.einsum("ab,kbs->kas", Rg, self.beam.reshape(-1, 4, 4))   # [n_beams, a, s]
            ls = ls * (self.mu0 * np.exp(-self.tau0 / self.mu0) / np.pi)[:, None, None]
            ls = ls.transpose(1, 0, 2).reshape(4, -1)                         # [a, 4 k + s]
            for i in range(N):
                rhs[4 * N + 4 * i:4 * N + 4 * i + 4] += ls
        self.K = K
        self.c = np.linalg.solve(K, rhs.astype(complex))

    def _basis(self, tau):
        """Basis functions f_j(tau) of all 8N modes."""
        k = self.kappa
        with np.errstate(over="ignore", invalid="ignore"):
            return np.where(self.growing, np.exp(k * (tau - self.tau0)), np.exp(k * tau))

    def nodal(self, tau, real=True):
        """u(tau) [8N, n_rhs] at one depth."""
        u = self.V @ (self._basis(tau)[:, None] * self.c) \
            + self.z * np.exp(-tau / self.rhs_mu0)[None, :]
        return u.real if real else u

    def nodal_derivative(self, tau):
        """du/dtau [8N, n_rhs] at one depth."""
        du = self.V @ ((self.kappa * self._basis(tau))[:, None] * self.c) \
            - self.z * (np.exp(-tau / self.rhs_mu0) / self.rhs_mu0)[None, :]
        return du.real

    def nodal_integral(self):
        """int_0^tau0 u(tau) dtau [8N, n_rhs] in closed form."""
        k = self.kappa
        t0 = self.tau0
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(self.growing, -expm1_complex(-k * t0) / k, expm1_complex(k * t0) / k)
        g = np.where(np.abs(k) * t0 < 1e-300, t0, g)
        zint = self.z * (self.rhs_mu0 * -np.expm1(-t0 / self.rhs_mu0))[None, :]
        return (self.V @ (g[:, None] * self.c) + zint).real

    def reconstruct_top(self, mu_out):
        """I^m(0, mu) for upward internal cosines mu: array [n_beams, n_out, 4, 4] (row r, column s)."""
        mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
        n_out = mu_out.size
        t0 = self.tau0
        G = _stack_matrix(A_matrix(self.m, self.coef, mu_out, self.mus))  # [4 n_out, 8N]
        GW = 0.5 * self.omega * G * self.w8[None, :]
        H = GW @ self.V                                                   # [4 n_out, 8N]
        mu_rows = np.repeat(mu_out, 4)
        x = 1.0 / mu_rows[:, None]
        k = self.kappa[None, :]
        # decaying modes exp(k t): (1 - exp(-(x - k) t0)) / (mu (x - k))
        a = x - k
        with np.errstate(over="ignore", invalid="ignore"):
            g_dec = -expm1_complex(-a * t0) / (mu_rows[:, None] * a)
        # growing modes exp(k (t - t0)): exp(-x t0) (1 - exp(-(k - x) t0)) / (mu (k - x))
        b = k - x
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            g_gro = np.where(np.abs(b * t0) < 1e-2,
                             np.exp(-x * t0) * -expm1_complex(-b * t0) / (mu_rows[:, None] * b),
                             (np.exp(-x * t0) - np.exp(-k * t0)) / (mu_rows[:, None] * b))
        g_gro = np.where(np.abs(b) == 0.0, t0 * np.exp(-x * t0) / mu_rows[:, None], g_gro)
        g = np.where(self.growing[None, :], g_gro, g_dec)
        hom = (H * g) @ self.c                                            # [4 n_out, n_rhs]
        # particular + direct-beam source, both decaying as exp(-t/mu0)
        y = 1.0 / self.rhs_mu0[None, :]
        g0 = -np.expm1(-(x + y) * t0) / (mu_rows[:, None] * (x + y))      # [4 n_out, n_rhs]
        part = GW @ self.z
        n_b = self.mu0.size
        direct = np.zeros((4 * n_out, 4 * n_b))
        for i, mu0 in enumerate(self.mu0):
            Ad = _stack_matrix(A_matrix(self.m, self.coef, mu_out, [-mu0]))  # [4 n_out, 4]
            direct[:, 4 * i:4 * i + 4] = self.cQ * Ad @ self.beam[i]
        tot = hom + (part + direct) * g0
        if self.Rbase is not None:
            # the base's isotropic radiance I^0(tau0, +mu) attenuated along the exit path
            up = self.nodal(t0, real=False)[:4 * self.N]                   # u_up(tau0) [4N, n_rhs]
            for a in range(4):                                           # same at every node
                tot[a::4] += np.exp(-t0 / mu_rows[a::4])[:, None] * up[a][None, :]
        self.max_imag = float(np.max(np.abs(tot.imag))) if np.iscomplexobj(tot) else 0.0
        out = tot.real.reshape(n_out, 4, n_b, 4).transpose(2, 0, 1, 3)
        return out


def _reconstruct_bottom(self, mu_out, R_out=None):
    """I^m(tau0, -mu) for downward internal cosines mu at the bottom: [n_beams, n_out, 4, 4].

    Formal solution along the downward path (tau grows downward, -mu dI/dtau = -(I - S) for
    the direction -mu, i.e. dI/dtau = (S - I)/mu):
        I^m(tau0, -mu) = I^m(0, -mu) exp(-tau0/mu) + int_0^tau0 S(t, -mu) exp(-(tau0 - t)/mu) dt / mu,
        S(t, -mu) = (omega/2) sum_{s,n} alpha_n A^m(-mu, s mu_n) u_{s,n}(t)
                    + (omega / 2 pi) A^m(-mu, -mu0) I0' exp(-t/mu0),
    with the downward radiance entering at the top I^m(0, -mu) = R_F(mu) I^m(0, +mu) (the
    internal specular reflection of the upward radiance at the same cosine; zero for a bare
    top; R_out[k] the reflection matrix at mu_out[k]). With x = 1/mu the depth integrals are
        exp(kappa t)           (Re kappa < 0):  x (exp(kappa tau0) - exp(-x tau0)) / (kappa + x)
        exp(kappa (t - tau0))  (Re kappa >= 0): x (1 - exp(-(kappa + x) tau0)) / (kappa + x)
        exp(-t/mu0):                            x (exp(-tau0/mu0) - exp(-x tau0)) / (x - 1/mu0),
    each evaluated through expm1 where its denominator is small. The once-scattered beam is
    included; the uncollided beam (a delta in direction) is not part of the diffuse field.
    """
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    n_out = mu_out.size
    t0 = self.tau0
    G = _stack_matrix(A_matrix(self.m, self.coef, -mu_out, self.mus))     # [4 n_out, 8N]
    GW = 0.5 * self.omega * G * self.w8[None, :]
    H = GW @ self.V
    mu_rows = np.repeat(mu_out, 4)
    x = (1.0 / mu_rows)[:, None]
    k = self.kappa[None, :]
    a = k + x
    small = np.abs(a * t0) < 1e-2
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        g_dec = np.where(small, x * np.exp(-x * t0) * expm1_complex(a * t0) / a,
                         x * (np.exp(k * t0) - np.exp(-x * t0)) / a)
        g_gro = x * -expm1_complex(-a * t0) / a
    g_dec = np.where(np.abs(a) == 0.0, x * t0 * np.exp(-x * t0), g_dec)
    g = np.where(self.growing[None, :], g_gro, g_dec)
    hom = (H * g) @ self.c
    y = (1.0 / self.rhs_mu0)[None, :]
    d = x - y
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        g0 = np.where(np.abs(d * t0) < 1e-2, x * np.exp(-x * t0) * expm1_complex(d * t0).real / d,
                      x * (np.exp(-y * t0) - np.exp(-x * t0)) / d)
    g0 = np.where(d == 0.0, x * t0 * np.exp(-x * t0), g0)
    part = GW @ self.z
    n_b = self.mu0.size
    direct = np.zeros((4 * n_out, 4 * n_b))
    for i, mu0 in enumerate(self.mu0):
        Ad = _stack_matrix(A_matrix(self.m, self.coef, -mu_out, [-mu0]))
        direct[:, 4 * i:4 * i + 4] = self.cQ * Ad @ self.beam[i]
    tot = (hom + (part + direct) * g0).real
    out = tot.reshape(n_out, 4, n_b, 4).transpose(2, 0, 1, 3)
    if R_out is not None:
        top = self.reconstruct_top(mu_out)                               # [n_b, n_out, 4, 4]
        att = np.exp(-t0 / mu_out)
        out = out + np.einsum("oab,kobc->koac", np.asarray(R_out) * att[:, None, None], top)
    return out


OrderSolution.reconstruct_bottom = _reconstruct_bottom


def _dd_exp(a, b, T):
    """(exp(-a T) - exp(-b T)) / (b - a), through expm1 where |(b - a) T| is small."""
    a = np.asarray(a, dtype=complex)
    b = np.asarray(b, dtype=complex)
    a, b = np.broadcast_arrays(a, b)
    d = b - a
    out = np.empty(d.shape, dtype=complex)
    zero = d == 0
    near = (np.abs(d * T) < 1e-2) & ~zero
    far = ~near & ~zero
    out[zero] = T * np.exp(-a[zero] * T)
    out[near] = np.exp(-a[near] * T) * -expm1_complex(-d[near] * T) / d[near]
    out[far] = (np.exp(-a[far] * T) - np.exp(-b[far] * T)) / d[far]
    return out


def _reconstruct_depth(self, tau, mu_up, mu_down, R_down=None):
    """Radiance inside the layer at depth tau (0 <= tau <= tau0), Sec. 2.C reconstruction:
    upward directions +mu_up and downward directions -mu_down, each [n_beams, n, 4, 4].

        I^m(tau, +mu) = I^m(tau0, +mu) e^{-(tau0 - tau)/mu} + int_tau^tau0 S(t, mu) e^{-(t - tau)/mu} dt / mu
        I^m(tau, -mu) = I^m(0, -mu) e^{-tau/mu} + int_0^tau S(t, -mu) e^{-(tau - t)/mu} dt / mu

    with S as in reconstruct_top / reconstruct_bottom, I^m(tau0, +mu) the Lambertian base's
    isotropic radiance (zero for a black base) and I^m(0, -mu) = R_F(mu) I^m(0, +mu) under a
    dielectric top (R_down[k] at mu_down[k]). With x = 1/mu every depth integral is a divided
    difference D(a, b; T) = (e^{-aT} - e^{-bT})/(b - a):
        upward,   decaying e^{kappa t}:        x e^{kappa tau} D(0, x - kappa; tau0 - tau)
        upward,   growing e^{kappa (t-tau0)}:  x D(x, kappa; tau0 - tau)
        upward,   beam e^{-t/mu0}:             x e^{-tau/mu0} D(0, x + 1/mu0; tau0 - tau)
        downward, decaying:                    x D(x, -kappa; tau)
        downward, growing:                     x e^{-kappa (tau0 - tau)} D(0, kappa + x; tau)
        downward, beam:                        x D(1/mu0, x; tau)
    At tau = 0 (upward) and tau = tau0 (downward) these are the top and bottom reconstructions.
    """
    t0 = self.tau0
    tau = float(tau)
    n_b = self.mu0.size
    k = self.kappa[None, :]
    y = (1.0 / self.rhs_mu0)[None, :]
    out = []
    for sign, mus in ((1.0, mu_up), (-1.0, mu_down)):
        mus = np.atleast_1d(np.asarray(mus, dtype=float))
        G = _stack_matrix(A_matrix(self.m, self.coef, sign * mus, self.mus))
        GW = 0.5 * self.omega * G * self.w8[None, :]
        H = GW @ self.V
        x = (1.0 / np.repeat(mus, 4))[:, None]
        gro = self.growing
        kd, kg = k[:, ~gro], k[:, gro]
        g = np.zeros((x.shape[0], k.shape[1]), dtype=complex)
        if sign > 0:
            g[:, ~gro] = x * np.exp(kd * tau) * _dd_exp(0.0, x - kd, t0 - tau)
            g[:, gro] = x * _dd_exp(x, kg, t0 - tau)
            g0 = x * np.exp(-y * tau) * _dd_exp(0.0, x + y, t0 - tau)
        else:
            g[:, ~gro] = x * _dd_exp(x, -kd, tau)
            g[:, gro] = x * np.exp(-kg * (t0 - tau)) * _dd_exp(0.0, kg + x, tau)
            g0 = x * _dd_exp(y, x, tau)
        hom = (H * g) @ self.c
        direct = np.zeros((4 * mus.size, 4 * n_b))
        for i, mu0 in enumerate(self.mu0):
            Ad = _stack_matrix(A_matrix(self.m, self.coef, sign * mus, [-mu0]))
            direct[:, 4 * i:4 * i + 4] = self.cQ * Ad @ self.beam[i]
        tot = (hom + (GW @ self.z + direct) * g0).real
        if sign > 0 and self.Rbase is not None:
            base = self.nodal(t0)[:4]                      # the base's isotropic radiance
            for a in range(4):
                tot[a::4] += np.exp(-(t0 - tau) / mus)[:, None] * base[a][None, :]
        res = tot.reshape(mus.size, 4, n_b, 4).transpose(2, 0, 1, 3)
        if sign < 0 and R_down is not None:
            top = self.reconstruct_top(mus)
            att = np.exp(-tau / mus)
            res = res + np.einsum("oab,kobc->koac", np.asarray(R_down) * att[:, None, None], top)
        out.append(res)
    return out[0], out[1]


OrderSolution.reconstruct_depth = _reconstruct_depth


def solve_order(m, coef, omega, tau0, N, mu0_int, beam=None, R_top=None, nodes=None, rho=0.0,
                base=None):
    """Solve Fourier order m for internal beam cosines mu0_int.

    beam[i] is the 4x4 matrix whose column s is the internal beam Stokes vector
    produced by incident Stokes basis vector s (identity without an interface).
    R_top[n] is the 4x4 internal reflection at node n (None for a bare top); rho the albedo of
    a Lambertian base (0: black base); base a direction-independent 4x4 Mueller BRDF of the base
    added to the Lambertian one (R_00 = 2 rho).
    """
    mu0_int = np.atleast_1d(np.asarray(mu0_int, dtype=float))
    if beam is None:
        beam = np.broadcast_to(np.eye(4), (mu0_int.size, 4, 4))
    if nodes is None:
        nodes = gauss_legendre_01(N)
    mu_n, alpha = nodes
    return OrderSolution(m, coef, omega, tau0, mu_n, alpha, mu0_int, beam, R_top, rho, base)
