"""Plain FP64 CPU oracle for the discrete-ordinate (DOM) solution of the vector
radiative transfer equation and the polarized subsurface BRDF of a flat
particulate layer (Collin & Pattanaik, "GPU accelerated computation of
Polarized Subsurface BRDF for Flat Particulate Layers", arXiv 1707.05882).

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check in __graft_entry__ and
the CPU-baseline / reference legs of bench.py import this package. The CUDA
library never links, imports or calls it, and it imports nothing from the CUDA
library: the two share no code. Inputs common to both come from `vrte_inputs`.

It is written to be read against the paper, not to be fast: FP64 throughout
(complex128 where eigenvalues may be complex), the full 8N formulation of each
Fourier order (Sec. 2.C, Eqs. 15-33), dense LU solves and LAPACK's
nonsymmetric eigensolver (numpy.linalg) as library steps.

Conventions fixed here (the paper leaves them open or states them
inconsistently; each is pinned by the tests listed in the module docstrings):
  * Optical depth tau grows downward from the top (tau = 0) to the bottom (tau0);
    mu > 0 is an upward propagation direction; the transfer equation per
    Fourier order reads mu dI/dtau = I - J (the paper's Eq. 2 with this reading).
  * Directions in phase matrices and radiances are propagation directions. The
    collimated beam therefore enters as A^m(mu, -mu0).
  * Stokes (I, Q, U, V) on the meridian frame (e_theta, e_phi) of the
    propagation direction, with V = -2 Im(E1 E2*).
  * The Fourier factors of the phase matrix use the same azimuth order as the
    radiance expansion, Phi_k^m(phi - phi'), so the per-order equations keep the
    full A^m (Eqs. 6, 12, 13).
  * The order-m source constant is omega/(2 pi) (consistent with Eqs. 4, 6 and 12).
  * F_r = I_out / (mu0 I0): radiance per unit irradiance on the horizontal
    surface, in 1/sr, with Delta-phi = phi_out - phi_in and both directions
    pointing away from the surface.

Functions whose parity is not pinned by an invariant independent of the
oracle say "parity unpinned" in their docstring. None does at present.
"""
from .quadrature import gauss_legendre_01
from .gsf import gsf_tables, wigner_d_family, wigner_d_jacobi
from .phase import (A_matrix, B_matrix, P_matrices, fourier_synthesis_phase,
                    phase_matrix_direct, scattering_matrix)
from .fresnel import (fresnel_beam_in, fresnel_exit, fresnel_internal_reflection,
                      fresnel_external_reflection, snell_mu)
from .dom import OrderSolution, solve_order
from .brdf import (brdf, brdf_orders, btdf, btdf_orders, radiance, radiance_orders,
                   single_scatter_brdf, single_scatter_btdf)
from .slab import slab_brdf, slab_reconstruct_top, solve_slab_order

__all__ = [
    "gauss_legendre_01", "gsf_tables", "wigner_d_family", "wigner_d_jacobi",
    "A_matrix", "B_matrix", "P_matrices", "fourier_synthesis_phase",
    "phase_matrix_direct", "scattering_matrix",
    "fresnel_beam_in", "fresnel_exit", "fresnel_internal_reflection",
    "fresnel_external_reflection", "snell_mu",
    "OrderSolution", "solve_order", "brdf", "brdf_orders", "single_scatter_brdf",
    "btdf", "btdf_orders", "radiance", "radiance_orders", "single_scatter_btdf",
    "slab_brdf", "slab_reconstruct_top", "solve_slab_order",
]
