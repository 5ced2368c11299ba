"""Smooth dielectric top interface (not in the paper; a reading of its Sec. 2.C BCs).

The paper's layer has a bare top: the only top condition is "no diffuse light
enters from above" (Eq. 49). The workloads place the particles under a smooth
interface of relative index n > 1, which this module models with Fresnel's
equations:

* Snell: mu_int = sqrt(1 - (1 - mu_ext^2) / n^2).
* Amplitude coefficients in the (p, s) basis with p = s x k for every beam (so
  that r_p = -r_s at normal incidence):
    r_s = (n1 c1 - n2 c2)/(n1 c1 + n2 c2),   r_p = (n2 c1 - n1 c2)/(n2 c1 + n1 c2),
    t_s = 2 n1 c1/(n1 c1 + n2 c2),           t_p = 2 n1 c1/(n2 c1 + n1 c2),
  c1, c2 the cosines on the incident and transmitted sides. Beyond the critical
  angle c2 = +i sqrt(n1^2 (1 - c1^2)/n2^2 - 1) (evanescent under exp(-i w t)).
* On meridian frames (e1, e2) = (e_theta, e_phi) = (p, s) the Jones matrix is
  diag(j_p, j_s) and its Mueller matrix is
  [[(|jp|^2+|js|^2)/2, (|jp|^2-|js|^2)/2, 0, 0], [same, swapped, 0, 0],
   [0, 0, Re(jp js*), Im(jp js*)], [0, 0, -Im(jp js*), Re(jp js*)]].
* Collimated beam entering: its flux per unit area normal to the beam becomes
  n |t|^2 times the incident one (energy transmittance n c2/c1 |t|^2 over the beam
  compression c1/c2), so M_in = n * Mueller(t_p, t_s).
* Radiance leaving (inside -> outside): L_out = T L_in / n^2 with the energy
  transmittance T = (c2 / (n c1)) |t'|^2, so M_out = Mueller(t'_p, t'_s) c2 / (n^3 c1).
* Internal specular reflection of radiance: Mueller(r_p, r_s) at the node cosine,
  identical for every Fourier order since it keeps the azimuth.
For n <= 1 the interface is absent: M_in = M_out = identity, no reflection.

Pinned by tests: R + T = 1 per polarization on both sides, |r| = 1 beyond the
critical angle, the total-internal-reflection retardance against its closed form
tan(delta/2) = cos(theta) sqrt(sin^2(theta) - 1/n^2) / sin^2(theta) (Born & Wolf) and
its sign against the evanescent decay of the transmitted field under exp(-i w t), the
Mueller map against Stokes vectors formed from explicit fields, n -> 1 limits, and the
end-to-end invariants of the BRDF with an interface (energy balance inside,
reciprocity outside, n = 1 equals no interface).
"""
from __future__ import annotations

import numpy as np


def snell_mu(mu_ext, n: float):
    """Internal cosine of the refracted direction for external cosine mu_ext."""
    mu_ext = np.asarray(mu_ext, dtype=float)
    if n <= 1.0:
        return mu_ext.copy()
    return np.sqrt(1.0 - (1.0 - mu_ext**2) / n**2)


def _mueller_diag_jones(jp, js) -> np.ndarray:
    jp = np.asarray(jp, dtype=complex)
    js = np.asarray(js, dtype=complex)
    a = 0.5 * (np.abs(jp) ** 2 + np.abs(js) ** 2)
    b = 0.5 * (np.abs(jp) ** 2 - np.abs(js) ** 2)
    z = jp * np.conj(js)
    M = np.zeros(jp.shape + (4, 4))
    M[..., 0, 0] = a
    M[..., 1, 1] = a
    M[..., 0, 1] = b
    M[..., 1, 0] = b
    M[..., 2, 2] = z.real
    M[..., 3, 3] = z.real
    M[..., 2, 3] = z.imag
    M[..., 3, 2] = -z.imag
    return M


def _fresnel_amplitudes(c1, n1: float, n2: float):
    """(r_p, r_s, t_p, t_s, c2) for incidence cosine c1 from index n1 onto n2."""
    c1 = np.asarray(c1, dtype=complex)
    s2sq = (n1 / n2) ** 2 * (1.0 - c1**2)
    c2 = np.where(s2sq.real <= 1.0, np.sqrt(np.clip((1.0 - s2sq).real, 0.0, None)) + 0j,
                  1j * np.sqrt(np.clip((s2sq - 1.0).real, 0.0, None)))
    rs = (n1 * c1 - n2 * c2) / (n1 * c1 + n2 * c2)
    rp = (n2 * c1 - n1 * c2) / (n2 * c1 + n1 * c2)
    ts = 2 * n1 * c1 / (n1 * c1 + n2 * c2)
    tp = 2 * n1 * c1 / (n2 * c1 + n1 * c2)
    return rp, rs, tp, ts, c2


def fresnel_beam_in(mu_ext, n: float) -> np.ndarray:
    """M_in[k, 4, 4]: external beam Stokes (flux normal to beam) -> internal beam Stokes."""
    mu_ext = np.atleast_1d(np.asarray(mu_ext, dtype=float))
    if n <= 1.0:
        return np.broadcast_to(np.eye(4), mu_ext.shape + (4, 4)).copy()
    _, _, tp, ts, _ = _fresnel_amplitudes(mu_ext, 1.0, n)
    return n * _mueller_diag_jones(tp, ts)


def fresnel_exit(mu_ext, n: float) -> np.ndarray:
    """M_out[k, 4, 4]: internal radiance at mu_int = snell_mu(mu_ext) -> external radiance."""
    mu_ext = np.atleast_1d(np.asarray(mu_ext, dtype=float))
    if n <= 1.0:
        return np.broadcast_to(np.eye(4), mu_ext.shape + (4, 4)).copy()
    mu_int = snell_mu(mu_ext, n)
    _, _, tp, ts, c2 = _fresnel_amplitudes(mu_int, n, 1.0)
    scale = c2.real / (n**3 * mu_int)
    return scale[:, None, None] * _mueller_diag_jones(tp, ts)


def fresnel_internal_reflection(mu_int, n: float) -> np.ndarray:
    """R[k, 4, 4]: upward radiance at the top (inside, cosine mu_int) -> reflected downward."""
    mu_int = np.atleast_1d(np.asarray(mu_int, dtype=float))
    if n <= 1.0:
        return np.zeros(mu_int.shape + (4, 4))
    rp, rs, _, _, _ = _fresnel_amplitudes(mu_int, n, 1.0)
    return _mueller_diag_jones(rp, rs)


def fresnel_external_reflection(mu_ext, n: float) -> np.ndarray:
    """Specular reflection outside (not part of the subsurface BRDF; used for energy checks)."""
    mu_ext = np.atleast_1d(np.asarray(mu_ext, dtype=float))
    if n <= 1.0:
        return np.zeros(mu_ext.shape + (4, 4))
    rp, rs, _, _, _ = _fresnel_amplitudes(mu_ext, 1.0, n)
    return _mueller_diag_jones(rp, rs)


def energy_transmittance(c1, n1: float, n2: float):
    """(T_p, T_s) = (n2 Re(c2) / (n1 c1)) |t|^2 (zero beyond the critical angle)."""
    rp, rs, tp, ts, c2 = _fresnel_amplitudes(c1, n1, n2)
    f = n2 * c2.real / (n1 * np.asarray(c1, dtype=float))
    return f * np.abs(tp) ** 2, f * np.abs(ts) ** 2, np.abs(rp) ** 2, np.abs(rs) ** 2
