"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This package holds no arithmetic of the DOM method itself: it only produces the
inputs a user of the solver would supply (phase-matrix expansion coefficients,
layer parameters, angle grids). The paper computes its phase matrices with an
external Mie code and runs on measured refractive indices (Sec. 4); neither is
available, so seeded synthetic layers of the same kind stand in for them.
"""
from .configs import (CONFIG_NAMES, angle_grids, make_config, rayleigh_coefficients,
                      uniform_zenith_grid)
from . import mie

__all__ = ["CONFIG_NAMES", "angle_grids", "make_config", "rayleigh_coefficients",
           "uniform_zenith_grid", "mie"]
