"""A numpy model of the reduced (4N) formulation that the CUDA path implements.

Test support only: it restates, in plain numpy, the formulas the kernels use
(parity-split sums S+-, F'E' eigenpairs, eigenbasis particular solution, boundary
matrix with scaled modes, reconstruction operators) so that the tests can check the
reduced formulation of Sec. 3.A-3.B (Eqs. 41-48) against the oracle's full 8N
solution before trusting the kernels. It uses the oracle's generalized spherical
functions for the tables and numpy's eigensolver.
"""
import numpy as np

import oracle as O


def S_pm(m, coef, x, y):
    """S+-(x_i, y_j) [len(x), len(y), 4, 4] = sum_l P(x) B_l (I +- (-1)^(l-m) D) P(y)."""
    L = coef.shape[0]
    Px = O.P_matrices(m, L, x)
    Py = O.P_matrices(m, L, y)
    D = np.diag([1.0, 1.0, -1.0, -1.0])
    B = np.stack([O.B_matrix(c) for c in coef])
    par = np.array([(-1.0) ** (l - m) for l in range(L)])
    Ip = np.stack([np.eye(4) + par[l] * D for l in range(L)])
    Im = np.stack([np.eye(4) - par[l] * D for l in range(L)])
    Sp = np.einsum("lxab,lbc,lcd,lyde->xyae", Px, B, Ip, Py)
    Sm = np.einsum("lxab,lbc,lcd,lyde->xyae", Px, B, Im, Py)
    return Sp, Sm


def stack(A4):
    X, Y = A4.shape[:2]
    return A4.transpose(0, 2, 1, 3).reshape(4 * X, 4 * Y)


def solve_order_reduced(m, coef, omega, tau0, N, mu0, beam, R_top, mu_out, mout,
                        return_intermediates=False):
    """Per-order exiting radiance [n_in, n_out, 4, 4] (rows already multiplied by M_out).

    beam[k] includes the 1/mu_in factor, as in the kernels.
    """
    mu, al = O.gauss_legendre_01(N)
    n = 4 * N
    m4 = np.repeat(mu, 4)
    w4 = np.repeat(al, 4)
    Sp, Sm = S_pm(m, coef, mu, mu)
    E = (np.eye(n) - 0.5 * omega * stack(Sp) * w4[None, :]) / m4[:, None]
    F = (np.eye(n) - 0.5 * omega * stack(Sm) * w4[None, :]) / m4[:, None]
    lam, X = np.linalg.eig(F @ E)
    kap = np.sqrt(lam.astype(complex))
    Y = (E @ X) / kap[None, :]
    php, phm = 0.5 * (X + Y), 0.5 * (X - Y)
    Dl = np.tile([1.0, 1.0, -1.0, -1.0], N)
    R = np.zeros((n, n))
    if R_top is not None:
        for i in range(N):
            R[4 * i:4 * i + 4, 4 * i:4 * i + 4] = R_top[i]
    Ek = np.exp(-kap * tau0)
    K = np.zeros((2 * n, 2 * n), dtype=complex)
    K[:n, :n] = Dl[:, None] * php - R @ phm
    K[:n, n:] = (Dl[:, None] * phm - R @ php) * Ek[None, :]
    K[n:, :n] = phm * Ek[None, :]
    K[n:, n:] = php
    # beam vectors p, r and the eigenbasis particular solution
    n_in = mu0.size
    cq = omega / (2 * np.pi)
    Spb, Smb = S_pm(m, coef, mu, mu0)           # [N, n_in, 4, 4]
    Db = np.diag([1.0, 1.0, -1.0, -1.0])
    p = np.zeros((n, 4 * n_in))
    r = np.zeros((n, 4 * n_in))
    for k in range(n_in):
        blkp = np.concatenate([Spb[i, k] @ Db @ beam[k] for i in range(N)], axis=0)
        blkm = np.concatenate([Smb[i, k] @ Db @ beam[k] for i in range(N)], axis=0)
        p[:, 4 * k:4 * k + 4] = cq * blkp / m4[:, None]
        r[:, 4 * k:4 * k + 4] = -cq * blkm / m4[:, None]
    mu0c = np.repeat(mu0, 4)
    w = F @ p - r / mu0c[None, :]
    y = np.linalg.solve(X, w.astype(complex))
    y = y / (lam[:, None] - 1.0 / mu0c[None, :] ** 2)
    s = (X @ y).real
    d = mu0c[None, :] * (p - E @ s)
    zp = 0.5 * (s + d)
    zm = Dl[:, None] * 0.5 * (s - d)
    rhs = np.concatenate([-(zm - R @ zp), -zp * np.exp(-tau0 / mu0c)[None, :]], axis=0)
    C = np.linalg.solve(K, rhs.astype(complex))
    # reconstruction
    n_out = mu_out.size
    Spo, Smo = S_pm(m, coef, mu_out, mu)          # [n_out, N, 4, 4]
    Up = np.zeros((4 * n_out, n))
    Um = np.zeros((4 * n_out, n))
    for o in range(n_out):
        for j in range(N):
            Up[4 * o:4 * o + 4, 4 * j:4 * j + 4] = 0.25 * omega * al[j] * mout[o] @ Spo[o, j]
            Um[4 * o:4 * o + 4, 4 * j:4 * j + 4] = 0.25 * omega * al[j] * mout[o] @ Smo[o, j]
    P1, P2 = Up @ X, Um @ Y
    mur = np.repeat(mu_out, 4)[:, None]
    x = 1.0 / mur
    a = x + kap[None, :]
    gD = -np.expm1(-a * tau0) / (mur * a) if not np.iscomplexobj(a) else (1 - np.exp(-a * tau0)) / (mur * a)
    b = kap[None, :] - x
    gG = (np.exp(-x * tau0) - np.exp(-kap[None, :] * tau0)) / (mur * b)
    Hh = np.concatenate([(P1 - P2) * gD, (P1 + P2) * gG], axis=1)
    hom = Hh @ C
    SpD, SmD = S_pm(m, coef, mu_out, mu0)         # direct term
    direct = np.zeros((4 * n_out, 4 * n_in))
    for o in range(n_out):
        for k in range(n_in):
            A = 0.5 * (SpD[o, k] - SmD[o, k]) @ Db
            direct[4 * o:4 * o + 4, 4 * k:4 * k + 4] = cq * mout[o] @ A @ beam[k]
    y0 = 1.0 / mu0c[None, :]
    g0 = -np.expm1(-(x + y0) * tau0) / (mur * (x + y0))
    tot = hom + g0 * (Up @ s + Um @ d + direct)
    inter = dict(E=E, F=F, lam=lam, p=p, r=r, s=s, d=d, rhs=rhs, Up=Up, Um=Um,
                 T1=(hom + g0 * direct).real, tot=tot.real)
    out = tot.real.reshape(n_out, 4, n_in, 4).transpose(2, 0, 1, 3)
    if return_intermediates:
        return out, lam, inter
    return out, lam
