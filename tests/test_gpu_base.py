"""Lambertian base (vrte_layer.base_albedo; the paper's base reflection with R_00 = 2 rho) on the
GPU against the oracle: reflection and transmission tables, FP64 and mixed forms, with and
without a dielectric top, mixed with black-base layers in one call. Tolerances as for the
black base (1e-10 FP64; 1e-6 I row and 1e-5 Q, U, V rows mixed; normalised by F_00)."""
import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err_rows(F, G):
    scale = np.maximum(np.abs(G[..., 0, 0])[..., None, None], 1e-300)
    e = np.abs(F - G) / scale
    return float(e[..., 0, :].max()), float(e[..., 1:, :].max())


def _solve(lys, grids, precision=vr.VRTE_FP64, btdf=False, out_dtype=torch.float64):
    lys = [dict(l, n_coef=np.asarray(l["coef"]).shape[0]) for l in lys]
    coef = vr.pack_coefficients(lys)
    plan = vr.Plan(*grids, max(l["n_nodes"] for l in lys), max(l["n_orders"] for l in lys),
                   coef.shape[1], len(lys), precision, transmission=btdf)
    try:
        plan.set_layers(lys, torch.from_numpy(coef).cuda())
        out = torch.empty(plan.table_shape, dtype=out_dtype, device="cuda")
        (plan.solve_btdf if btdf else plan.solve)(out)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return out.double().cpu().numpy()
    finally:
        plan.close()


def _oracle(ly, grids, btdf=False):
    f = O.btdf if btdf else O.brdf
    return f(ly["coef"], ly["omega"], ly["tau"], ly.get("n_interface", 1.0), ly["n_nodes"],
             ly["n_orders"], *grids, rho=ly.get("base_albedo", 0.0))


COEF = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)


@pytest.mark.parametrize("n_if", [1.0, 1.5])
@pytest.mark.parametrize("btdf", [False, True])
def test_lambertian_base_fp64(n_if, btdf):
    ly = dict(tau=2.0, omega=0.95, n_interface=n_if, n_nodes=20, n_orders=40, coef=COEF,
              base_albedo=0.35)
    grids = angle_grids(17, 19, 11)
    F = _solve([ly], grids, btdf=btdf)[0]
    G = _oracle(ly, grids, btdf=btdf)
    assert max(_err_rows(F, G)) < 1e-10


def test_lambertian_base_mixed_fp32():
    ly = dict(tau=2.0, omega=0.95, n_interface=1.4, n_nodes=20, n_orders=40, coef=COEF,
              base_albedo=0.6)
    grids = angle_grids(17, 19, 11)
    F = _solve([ly], grids, precision=vr.VRTE_MIXED, out_dtype=torch.float32)[0]
    G = _oracle(ly, grids)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-6 and e_q < 1e-5


def test_white_and_black_bases_in_one_call():
    lys = [dict(tau=0.8, omega=0.9, n_interface=1.33, n_nodes=8, n_orders=12, coef=COEF[:12],
                base_albedo=1.0),
           dict(tau=0.8, omega=0.9, n_interface=1.33, n_nodes=8, n_orders=12, coef=COEF[:12]),
           dict(tau=5.0, omega=0.5, n_interface=1.0, n_nodes=6, n_orders=12, coef=COEF[:12],
                base_albedo=0.2)]
    grids = angle_grids(5, 6, 7)
    F = _solve(lys, grids)
    for i, ly in enumerate(lys):
        assert max(_err_rows(F[i], _oracle(ly, grids))) < 1e-10, i
    assert np.all(F[0][..., 0, 0] > F[1][..., 0, 0])    # the white base adds reflected light


def test_adjoint_declines_a_reflecting_base():
    ly = dict(tau=1.0, omega=0.9, n_interface=1.4, n_nodes=4, n_orders=8, n_coef=8,
              coef=COEF[:8], base_albedo=0.5)
    grids = angle_grids(2, 2, 3)
    plan = vr.Plan(*grids, 4, 8, 8, 1, vr.VRTE_FP64, adjoint=True)
    try:
        plan.set_layers([ly], torch.from_numpy(vr.pack_coefficients([ly])).cuda())
        G = torch.zeros(plan.table_shape, dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.backward(G)
        assert e.value.code == 8  # VRTE_ERR_UNSUPPORTED
    finally:
        plan.close()
