"""Radiance field inside the layer (vrte_solve_radiance) against the oracle (oracle.radiance):
upward and downward tables at interior depths, with and without a dielectric top and a
Lambertian base, several layers at different depths in one call, and the end depths equal to
the internal top radiance and the transmission table. FP64, 1e-10 of the I->I element at the
same point; the radiance-field shape of the paper's experiment (11 zenith x 19 azimuth
directions per hemisphere) in the last case."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COEF = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)


def _err(F, G):
    scale = np.maximum(np.abs(G[..., 0, 0])[..., None, None], 1e-300)
    return float((np.abs(F - G) / scale).max())


def _gpu(lys, grids, taus):
    lys = [dict(l, n_coef=np.asarray(l["coef"]).shape[0]) for l in lys]
    coef = vr.pack_coefficients(lys)
    plan = vr.Plan(*grids, max(l["n_nodes"] for l in lys), max(l["n_orders"] for l in lys),
                   coef.shape[1], len(lys), vr.VRTE_FP64, transmission=True)
    try:
        plan.set_layers(lys, torch.from_numpy(coef).cuda())
        up = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        dn = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        plan.solve_radiance(taus, up, dn)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return up.cpu().numpy(), dn.cpu().numpy()
    finally:
        plan.close()


def _oracle(ly, grids, tau):
    mu_in, mu_out, dphi = grids
    return O.radiance(ly["coef"], ly["omega"], ly["tau"], ly.get("n_interface", 1.0),
                      ly["n_nodes"], ly["n_orders"], mu_in, tau, mu_out, mu_out, dphi,
                      rho=ly.get("base_albedo", 0.0))


@pytest.mark.parametrize("n_if,rho", [(1.0, 0.0), (1.5, 0.0), (1.33, 0.4)])
def test_interior_radiance(n_if, rho):
    ly = dict(tau=3.0, omega=0.97, n_interface=n_if, n_nodes=20, n_orders=40, coef=COEF,
              base_albedo=rho)
    grids = angle_grids(7, 9, 5)
    up, dn = _gpu([ly], grids, [1.1])
    gu, gd = _oracle(ly, grids, 1.1)
    assert _err(up[0], gu) < 1e-10 and _err(dn[0], gd) < 1e-10


def test_layers_at_different_depths_and_the_ends():
    lys = [dict(tau=2.0, omega=0.9, n_interface=1.4, n_nodes=10, n_orders=20, coef=COEF[:20]),
           dict(tau=0.5, omega=0.8, n_interface=1.0, n_nodes=6, n_orders=12, coef=COEF[:12],
                base_albedo=0.7),
           dict(tau=8.0, omega=0.99, n_interface=1.6, n_nodes=12, n_orders=16, coef=COEF[:16])]
    grids = angle_grids(4, 5, 6)
    taus = [0.0, 0.5, 3.3]
    up, dn = _gpu(lys, grids, taus)
    for i, ly in enumerate(lys):
        gu, gd = _oracle(ly, grids, taus[i])
        assert _err(up[i], gu) < 1e-10 and _err(dn[i], gd) < 1e-10, i
    # tau = 0 upward is the BRDF's internal radiance before the exit: the BRDF with n = 1
    # equals it for the bare-top layer; tau = tau0 downward is the transmission table
    bt = O.btdf(lys[1]["coef"], 0.8, 0.5, 1.0, 6, 12, *grids, rho=0.7)
    assert _err(dn[1], bt) < 1e-10


def test_radiance_field_experiment_shape():
    """The paper's radiance-field experiment: a thick layer (tau0 = 100), one incident cosine
    mu0 = 0.6, N = 40, 11 zenith x 19 azimuth directions per hemisphere, at mid-depth."""
    coef = polydisperse_coefficients(0.5 + 2.0j, 3.0, 0.1, 24)   # strongly absorbing particles
    ly = dict(tau=100.0, omega=0.7, n_interface=1.0, n_nodes=40, n_orders=24, coef=coef)
    mu_out = np.cos(np.radians(np.linspace(5.0, 85.0, 11)))
    dphi = np.radians(np.linspace(0.0, 180.0, 19))
    grids = (np.array([0.6]), mu_out, dphi)
    up, dn = _gpu([ly], grids, [1.0])
    gu, gd = _oracle(ly, grids, 1.0)
    assert _err(up[0], gu) < 1e-10 and _err(dn[0], gd) < 1e-10
