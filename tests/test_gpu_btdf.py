"""Parity of the transmission table (vrte_solve_btdf, the diffuse radiance leaving the bottom)
with the FP64 oracle (oracle.btdf), through the C ABI.

Tolerance as for the BRDF: every element normalised by the I->I element at the same point,
1e-10 in the FP64 form and 1e-6 (I row) / 1e-5 (Q, U, V rows) in the mixed form, whose
synthesis runs on the tensor cores.
"""
import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids, make_config
from vrte_inputs.mie import polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err_rows(F, G):
    scale = np.maximum(np.abs(G[..., 0, 0])[..., None, None], 1e-300)
    e = np.abs(F - G) / scale
    return float(e[..., 0, :].max()), float(e[..., 1:, :].max())


def gpu_btdf(layers, grids, precision=vr.VRTE_FP64, out_dtype=torch.float64):
    lys = [dict(l, n_coef=np.asarray(l["coef"]).shape[0]) for l in layers]
    coef = vr.pack_coefficients(lys)
    plan = vr.Plan(*grids, max(l["n_nodes"] for l in lys), max(l["n_orders"] for l in lys),
                   coef.shape[1], len(lys), precision, transmission=True)
    try:
        plan.set_layers(lys, torch.from_numpy(coef).cuda())
        out = torch.empty(plan.table_shape, dtype=out_dtype, device="cuda")
        plan.solve_btdf(out)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return out.double().cpu().numpy()
    finally:
        plan.close()


def oracle_btdf(ly, grids):
    return O.btdf(ly["coef"], ly["omega"], ly["tau"], ly.get("n_interface", 1.0), ly["n_nodes"],
                  ly["n_orders"], *grids)


@pytest.mark.parametrize("n_if", [1.0, 1.5])
def test_btdf_ragged_multi_tile_mie(n_if):
    """4N = 80, 4 n_in = 68, 4 n_out = 76: full tiles and ragged tails in every contraction."""
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    ly = dict(tau=3.0, omega=0.97, n_interface=n_if, n_nodes=20, n_orders=40, coef=coef)
    grids = angle_grids(17, 19, 11)
    F = gpu_btdf([ly], grids)[0]
    G = oracle_btdf(ly, grids)
    assert max(_err_rows(F, G)) < 1e-10


def test_btdf_mie_N32_M64_64x64x90():
    """The full 64 x 64 x 90 table on the GPU; the oracle on every fourth incident and outgoing
    cosine (all azimuths), which it solves for those directions only."""
    cfg = make_config(2)
    ly = cfg["layers"][0]
    grids = (cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    F = gpu_btdf([ly], grids)[0]
    sel = np.arange(1, 64, 4)
    G = oracle_btdf(ly, (cfg["mu_in"][sel], cfg["mu_out"][sel], cfg["dphi"]))
    assert max(_err_rows(F[np.ix_(sel, sel)], G)) < 1e-10


def test_btdf_mixed_form_and_fp32():
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    ly = dict(tau=3.0, omega=0.97, n_interface=1.4, n_nodes=20, n_orders=40, coef=coef)
    grids = angle_grids(17, 19, 11)
    G = oracle_btdf(ly, grids)
    F = gpu_btdf([ly], grids, precision=vr.VRTE_MIXED, out_dtype=torch.float32)[0]
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-6 and e_q < 1e-5


def test_btdf_several_layers_and_edge_cases():
    """Uneven layers in one call (concurrent streams): thin, thick, no scattering, one node."""
    c40 = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    c8 = polydisperse_coefficients(1.4 + 0.001j, 2.0, 0.1, 8)
    lys = [dict(tau=1e-4, omega=0.9, n_interface=1.5, n_nodes=8, n_orders=8, coef=c8),
           dict(tau=40.0, omega=0.99, n_interface=1.3, n_nodes=12, n_orders=20, coef=c40[:20]),
           dict(tau=2.0, omega=0.0, n_interface=1.5, n_nodes=6, n_orders=8, coef=c8),
           dict(tau=0.5, omega=0.8, n_interface=1.0, n_nodes=1, n_orders=8, coef=c8)]
    grids = angle_grids(5, 6, 7)
    F = gpu_btdf(lys, grids)
    for i, ly in enumerate(lys):
        G = oracle_btdf(ly, grids)
        if ly["omega"] == 0.0:
            assert np.all(F[i] == 0.0)
        else:
            assert max(_err_rows(F[i], G)) < 1e-10, i


def test_btdf_requires_its_workspace():
    grids = angle_grids(2, 2, 3)
    c8 = polydisperse_coefficients(1.4 + 0.001j, 2.0, 0.1, 8)
    ly = dict(tau=1.0, omega=0.9, n_interface=1.4, n_nodes=4, n_orders=8, n_coef=8, coef=c8)
    plan = vr.Plan(*grids, 4, 8, 8)
    try:
        plan.set_layers([ly], torch.from_numpy(vr.pack_coefficients([ly])).cuda())
        out = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.solve_btdf(out)
        assert e.value.code == 2
    finally:
        plan.close()
