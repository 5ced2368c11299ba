"""Reflecting base on the GPU against the oracle (the paper's base reflection, Sec. 3.C): the
Lambertian base (vrte_layer.base_albedo, R_00 = 2 rho) and a polarizing base with a
direction-independent Mueller BRDF matrix (vrte_layer.base_mueller, alone and added to a
Lambertian one): reflection and transmission tables and the radiance at depth, FP64 and mixed
forms, with and without a dielectric top, mixed with black-base layers in one call; base
matrices the library must reject. Tolerances as for the black base (1e-10 FP64; 1e-6 I row and
1e-5 Q, U, V rows mixed; normalised by F_00)."""
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
             ly["n_orders"], *grids, rho=ly.get("base_albedo", 0.0), base=ly.get("base_mueller"))


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


# A polarizing base: direction-independent Mueller BRDF matrix with both diagonal blocks filled
# (the (I, Q) x (U, V) blocks stay zero, as an azimuth-independent base has them).
R_POL = np.array([[0.9, 0.25, 0.0, 0.0],
                  [0.18, 0.5, 0.0, 0.0],
                  [0.0, 0.0, 0.4, 0.15],
                  [0.0, 0.0, -0.1, 0.3]])


@pytest.mark.parametrize("n_if", [1.0, 1.5])
@pytest.mark.parametrize("btdf", [False, True])
def test_mueller_base_fp64(n_if, btdf):
    ly = dict(tau=1.5, omega=0.95, n_interface=n_if, n_nodes=20, n_orders=40, coef=COEF,
              base_mueller=R_POL)
    grids = angle_grids(17, 19, 11)
    F = _solve([ly], grids, btdf=btdf)[0]
    G = _oracle(ly, grids, btdf=btdf)
    assert max(_err_rows(F, G)) < 1e-10
    # the polarizing rows reach the table: it differs from the Lambertian base of equal R_00
    L = _solve([dict(ly, base_mueller=None, base_albedo=R_POL[0, 0] / 2)], grids, btdf=btdf)[0]
    assert np.abs(F[..., 1:, :] - L[..., 1:, :]).max() > 1e-4 * np.abs(F[..., 0, 0]).max()


def test_mueller_plus_lambertian_base_mixed_fp32():
    ly = dict(tau=2.0, omega=0.95, n_interface=1.4, n_nodes=20, n_orders=40, coef=COEF,
              base_albedo=0.3, base_mueller=0.5 * R_POL)
    grids = angle_grids(17, 19, 11)
    F = _solve([ly], grids, precision=vr.VRTE_MIXED, out_dtype=torch.float32)[0]
    G = _oracle(ly, grids)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-6 and e_q < 1e-5


def test_mueller_base_radiance_at_depth():
    ly = dict(tau=2.5, omega=0.97, n_interface=1.33, n_nodes=16, n_orders=32, coef=COEF[:32],
              n_coef=32, base_mueller=R_POL, base_albedo=0.1)
    grids = angle_grids(7, 9, 5)
    coef = vr.pack_coefficients([ly])
    plan = vr.Plan(*grids, 16, 32, 32, 1, vr.VRTE_FP64, transmission=True)
    try:
        plan.set_layers([ly], torch.from_numpy(coef).cuda())
        up = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        dn = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        plan.solve_radiance([0.9], up, dn)
        torch.cuda.synchronize()
        assert plan.status() == 0
        up, dn = up.cpu().numpy()[0], dn.cpu().numpy()[0]
    finally:
        plan.close()
    mu_in, mu_out, dphi = grids
    gu, gd = O.radiance(ly["coef"], ly["omega"], ly["tau"], 1.33, 16, 32, mu_in, 0.9, mu_out,
                        mu_out, dphi, rho=0.1, base=R_POL)
    assert max(_err_rows(up, gu)) < 1e-10 and max(_err_rows(dn, gd)) < 1e-10


def test_mueller_and_black_bases_in_one_call():
    lys = [dict(tau=0.8, omega=0.9, n_interface=1.33, n_nodes=8, n_orders=12, coef=COEF[:12],
                base_mueller=R_POL),
           dict(tau=0.8, omega=0.9, n_interface=1.33, n_nodes=8, n_orders=12, coef=COEF[:12]),
           dict(tau=5.0, omega=0.5, n_interface=1.0, n_nodes=6, n_orders=12, coef=COEF[:12],
                base_albedo=0.2, base_mueller=0.3 * R_POL)]
    grids = angle_grids(5, 6, 7)
    F = _solve(lys, grids)
    for i, ly in enumerate(lys):
        assert max(_err_rows(F[i], _oracle(ly, grids))) < 1e-10, i


@pytest.mark.parametrize("bad", ["cross_block", "r00_high", "r00_negative", "nonfinite"])
def test_invalid_base_matrix_is_rejected(bad):
    R = R_POL.copy()
    if bad == "cross_block":
        R[0, 2] = 0.1
    elif bad == "r00_high":
        R[0, 0] = 1.9          # with the Lambertian 2 rho = 0.4 below: R_00 = 2.3 > 2
    elif bad == "r00_negative":
        R[0, 0] = -0.5
    else:
        R[3, 3] = np.nan
    ly = dict(tau=1.0, omega=0.9, n_nodes=4, n_orders=4, n_coef=4, coef=COEF[:4],
              base_albedo=0.2, base_mueller=R)
    grids = angle_grids(2, 2, 3)
    plan = vr.Plan(*grids, 4, 4, 4, 1, vr.VRTE_FP64)
    try:
        with pytest.raises(vr.VrteError) as e:
            plan.set_layers([ly], torch.from_numpy(vr.pack_coefficients([ly])).cuda())
        assert e.value.code == 1  # VRTE_ERR_INVALID_ARG
    finally:
        plan.close()
