"""Multi-layer slabs: a stack of homogeneous sub-layers (Sec. 2.C's solution per sub-layer,
joined by continuity of the radiance at their common boundaries).

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never calls it.

Sub-layer k (k = 0 at the top) spans the total optical depths [t_k, t_k + tau_k]. In its local
depth s the order-m field is its own mode expansion plus its particular solution for the beam
attenuated to its top,
    u_k(s) = V_k diag(f_k(s)) c_k + z_k exp(-(t_k + s)/mu0),
(f_k the scaled basis of oracle.dom), and the 8N K coefficients solve one block-banded system:
    top:        u_0,down(0) - R_F u_0,up(0) = 0                         (4N rows)
    continuity: u_k(tau_k) - u_{k+1}(0) = 0 for every inner boundary    (8N rows each)
    bottom:     u_K-1,up(tau_K-1) = the Lambertian base's radiance      (4N rows; 0 black)
The radiance leaving the top at an internal cosine mu is the sum over sub-layers of their own
top reconstructions (oracle.dom, with the beam scaled by exp(-t_k/mu0)) attenuated by
exp(-t_k/mu), plus the base's radiance attenuated through the whole slab.

Pinned by tests/test_oracle_slab.py: a stack of identical sub-layers equals the single layer of
their total thickness; a one-sub-layer stack equals oracle.brdf; the nodal field is continuous
across the boundaries and satisfies each sub-layer's transfer equation; the table-level flux
balance of a conservative stack.
"""
from __future__ import annotations

import numpy as np

from .brdf import synthesize
from .dom import OrderSolution
from .fresnel import fresnel_beam_in, fresnel_internal_reflection, snell_mu
from .quadrature import gauss_legendre_01


def _base_matrix(m, rho, base):
    """The base's direction-independent Mueller BRDF R (R_00 = 2 rho for the Lambertian part)
    seen by order m (only order 0), or None."""
    if m != 0:
        return None
    Rg = np.zeros((4, 4))
    Rg[0, 0] = 2.0 * float(rho)
    if base is not None:
        Rg = Rg + np.asarray(base, dtype=float).reshape(4, 4)
    return Rg if np.any(Rg != 0.0) else None


def solve_slab_order(m, sublayers, N, mu0_int, beam, R_top, rho=0.0, nodes=None, base=None):
    """Order m of a stack: list of per-sub-layer OrderSolution objects whose `c` are the stack's
    coefficients (each built with the beam attenuated to its top). sublayers: dicts with coef,
    omega, tau."""
    if nodes is None:
        nodes = gauss_legendre_01(N)
    mu_n, alpha = nodes
    mu0_int = np.atleast_1d(np.asarray(mu0_int, dtype=float))
    beam = np.asarray(beam, dtype=float).reshape(mu0_int.size, 4, 4)
    K = len(sublayers)
    n8, n4 = 8 * N, 4 * N
    sols, tops = [], []
    t = 0.0
    for sl in sublayers:
        att = np.exp(-t / mu0_int)[:, None, None]
        sols.append(OrderSolution(m, sl["coef"], sl["omega"], sl["tau"], mu_n, alpha, mu0_int,
                                  beam * att, None))
        tops.append(t)
        t += sl["tau"]
    n_rhs = 4 * mu0_int.size
    A = np.zeros((n8 * K, n8 * K), dtype=complex)
    b = np.zeros((n8 * K, n_rhs), dtype=complex)
    up, down = np.arange(n4), n4 + np.arange(n4)
    R = np.zeros((n4, n4))
    if R_top is not None:
        for i in range(N):
            R[4 * i:4 * i + 4, 4 * i:4 * i + 4] = R_top[i]
    s0 = sols[0]
    f0 = s0._basis(0.0)
    A[:n4, :n8] = (s0.V[down] - R @ s0.V[up]) * f0[None, :]
    b[:n4] = -(s0.z[down] - R @ s0.z[up])
    row = n4
    for k in range(K - 1):
        a, c = sols[k], sols[k + 1]
        fa = a._basis(a.tau0)
        fb = c._basis(0.0)
        atte = np.exp(-a.tau0 / a.rhs_mu0)[None, :]
        A[row:row + n8, k * n8:(k + 1) * n8] = a.V * fa[None, :]
        A[row:row + n8, (k + 1) * n8:(k + 2) * n8] = -c.V * fb[None, :]
        b[row:row + n8] = -(a.z * atte - c.z)
        row += n8
    sl = sols[-1]
    f1 = sl._basis(sl.tau0)
    att = np.exp(-sl.tau0 / sl.rhs_mu0)[None, :]
    A[row:, (K - 1) * n8:] = sl.V[up] * f1[None, :]
    b[row:] = -sl.z[up] * att
    Rg = _base_matrix(m, rho, base)
    if Rg is not None:
        Rb = np.zeros((n4, n4))
        for i in range(N):
            for j in range(N):
                Rb[4 * i:4 * i + 4, 4 * j:4 * j + 4] = Rg * (alpha[j] * mu_n[j])
        A[row:, (K - 1) * n8:] -= (Rb @ sl.V[down]) * f1[None, :]
        b[row:] += (Rb @ sl.z[down]) * att
        ttot = tops[-1] + sl.tau0
        ls = np.einsum("ab,kbs->kas", Rg, beam.reshape(-1, 4, 4))
        ls = ls * (mu0_int * np.exp(-ttot / mu0_int) / np.pi)[:, None, None]
        ls = ls.transpose(1, 0, 2).reshape(4, -1)                 # [a, 4 k + s]
        for i in range(N):
            b[row + 4 * i:row + 4 * i + 4] += ls
    c = np.linalg.solve(A, b)
    for k, s in enumerate(sols):
        s.c = c[k * n8:(k + 1) * n8]
    return sols, tops


def slab_reconstruct_top(sols, tops, mu_out, rho=0.0, m=0, base=None):
    """I^m(0, mu) [n_beams, n_out, 4, 4] of the stack at internal upward cosines mu."""
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    out = 0.0
    for s, t in zip(sols, tops):
        out = out + np.exp(-t / mu_out)[None, :, None, None] * s.reconstruct_top(mu_out)
    if _base_matrix(m, rho, base) is not None:
        last = sols[-1]
        rad = last.nodal(last.tau0)[:4]                     # the base's isotropic radiance
        ttot = tops[-1] + last.tau0
        n_b = last.mu0.size
        add = np.zeros((n_b, mu_out.size, 4, 4))
        for a in range(4):
            add[:, :, a, :] = (np.exp(-ttot / mu_out)[None, :, None]
                               * rad[a].reshape(n_b, 4)[:, None, :])
        out = out + add
    return out


def slab_brdf(sublayers, n_interface, N, M, mu_in, mu_out, dphi, rho=0.0, base=None):
    """Mueller BRDF table F[n_in, n_out, n_phi, 4, 4] of a stack of sub-layers (top first; each
    a dict with coef [L_k, 6], omega, tau) under an optional dielectric top and over an
    optional reflecting base (Lambertian albedo rho and/or a direction-independent Mueller BRDF
    `base`, added). Orders beyond every sub-layer's expansion contribute nothing."""
    mu_in = np.atleast_1d(np.asarray(mu_in, dtype=float))
    mu_out = np.atleast_1d(np.asarray(mu_out, dtype=float))
    nodes = gauss_legendre_01(N)
    mu0_int = snell_mu(mu_in, n_interface)
    mu_out_int = snell_mu(mu_out, n_interface)
    beam = fresnel_beam_in(mu_in, n_interface)
    R_top = fresnel_internal_reflection(nodes[0], n_interface) if n_interface > 1.0 else None
    Lmax = max(np.asarray(s["coef"]).shape[0] for s in sublayers)
    Im = np.zeros((M, mu_in.size, mu_out.size, 4, 4))
    for m in range(min(M, Lmax)):
        sols, tops = solve_slab_order(m, sublayers, N, mu0_int, beam, R_top, rho, nodes, base)
        Im[m] = slab_reconstruct_top(sols, tops, mu_out_int, rho, m, base)
    return synthesize(Im, mu_in, mu_out, dphi, n_interface)
