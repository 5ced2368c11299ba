"""Parity of the CUDA path (FP64 form, through the C ABI) with the FP64 CPU oracle.

Tolerance: every element of the 4x4 Mueller matrix, normalised by the I->I element
F_00 at the same (incident, outgoing, azimuth) point, agrees within 1e-10.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids, make_config
from vrte_inputs.mie import monodisperse_coefficients, polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def normalised_error(F, G):
    """max |F - G| / |G_00| over all points and elements."""
    scale = np.abs(G[..., 0, 0])[..., None, None]
    return float(np.max(np.abs(F - G) / np.maximum(scale, 1e-300)))


def gpu_brdf(layer, mu_in, mu_out, dphi, out_dtype=None):
    out = vr.brdf([layer], mu_in, mu_out, dphi, precision=vr.VRTE_FP64,
                  out_dtype=out_dtype or torch.float64)
    torch.cuda.synchronize()
    return out[0].cpu().numpy()


def oracle_brdf(layer, mu_in, mu_out, dphi):
    return O.brdf(layer["coef"], layer["omega"], layer["tau"], layer.get("n_interface", 1.0),
                  layer["n_nodes"], layer["n_orders"], mu_in, mu_out, dphi)


def test_rayleigh_N8_M3_8x8x16():
    cfg = make_config(1)
    ly = cfg["layers"][0]
    F = gpu_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    G = oracle_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    assert F.shape == G.shape == (8, 8, 16, 4, 4)
    assert normalised_error(F, G) < TOL_FP64


@pytest.mark.parametrize("n_if", [1.0, 1.5])
def test_ragged_multi_tile_mie(n_if):
    """4N = 80, 4 n_in = 68, 4 n_out = 76: every GEMM has a full tile and a ragged tail."""
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    ly = dict(tau=3.0, omega=0.97, n_interface=n_if, n_nodes=20, n_orders=40, coef=coef)
    mu_in, mu_out, dphi = angle_grids(17, 19, 11)
    F = gpu_brdf(ly, mu_in, mu_out, dphi)
    G = oracle_brdf(ly, mu_in, mu_out, dphi)
    assert normalised_error(F, G) < TOL_FP64


def test_mie_N32_M64_64x64x90():
    cfg = make_config(2)
    ly = cfg["layers"][0]
    F = gpu_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    G = oracle_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    assert normalised_error(F, G) < TOL_FP64


def test_fp32_output_rounds_the_fp64_result():
    cfg = make_config(1)
    ly = cfg["layers"][0]
    F64 = gpu_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    F32 = gpu_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"], out_dtype=torch.float32)
    assert np.array_equal(F32, F64.astype(np.float32))


@pytest.mark.parametrize("case", ["omega0", "thin", "thick", "N1", "orders_beyond_L", "mu_one",
                                  "one_direction"])
def test_edge_cases(case):
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)
    ly = dict(tau=1.0, omega=0.9, n_interface=1.33, n_nodes=6, n_orders=12, coef=coef)
    mu_in, mu_out, dphi = angle_grids(5, 6, 7)
    if case == "omega0":
        ly["omega"] = 0.0
    elif case == "thin":
        ly["tau"] = 1e-4
    elif case == "thick":
        ly["tau"] = 100.0
    elif case == "N1":
        ly["n_nodes"] = 1
        ly["coef"] = coef[:2]
        ly["n_orders"] = 2
    elif case == "orders_beyond_L":
        ly["n_orders"] = 20
    elif case == "mu_one":
        mu_in = np.array([1.0, 0.5])
        mu_out = np.array([1.0, 0.3])
    elif case == "one_direction":
        mu_in, mu_out, dphi = np.array([0.7]), np.array([0.4]), np.array([1.0])
    F = gpu_brdf(ly, mu_in, mu_out, dphi)
    G = oracle_brdf(ly, mu_in, mu_out, dphi)
    if case == "omega0":
        assert np.abs(F).max() == 0.0
    else:
        assert normalised_error(F, G) < TOL_FP64


def test_invalid_arguments_rejected():
    mu = np.array([0.5])
    with pytest.raises(vr.VrteError) as e:
        vr.Plan(np.array([1.5]), mu, mu, 4, 4, 4)
    assert e.value.code == 1
    plan = vr.Plan(mu, mu, mu, 4, 4, 4)
    coef = torch.zeros((1, 4, 6), dtype=torch.float64, device="cuda")
    for bad in [dict(tau=0.0), dict(omega=1.0), dict(omega=-0.1), dict(n_nodes=5),
                dict(n_coef=9), dict(n_interface=3.5)]:
        ly = dict(tau=1.0, omega=0.5, n_interface=1.0, n_nodes=2, n_orders=2, n_coef=2)
        ly.update(bad)
        with pytest.raises(vr.VrteError) as e:
            plan.set_layers([ly], coef)
        assert e.value.code == 1
    out = torch.empty((1, 1, 1, 1, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(vr.VrteError) as e:
        plan.solve(out)
    assert e.value.code == 2
    plan.close()


def test_nonfinite_coefficients_reported():
    mu = np.array([0.5, 0.8])
    coef = np.zeros((1, 3, 6))
    coef[0, 0, 0] = 1.0
    coef[0, 2, 0] = float("nan")
    plan = vr.Plan(mu, mu, np.array([0.0]), 4, 3, 3)
    plan.set_layers([dict(tau=1.0, omega=0.5, n_interface=1.0, n_nodes=4, n_orders=3, n_coef=3)],
                    torch.from_numpy(coef).cuda())
    out = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
    plan.solve(out)
    assert plan.status() != 0
    plan.close()


def test_host_buffer_entry_point_matches_device_entry_point():
    cfg = make_config(1)
    ly = dict(cfg["layers"][0])
    ly["n_coef"] = ly["coef"].shape[0]
    coef = vr.pack_coefficients([ly])
    plan = vr.Plan(cfg["mu_in"], cfg["mu_out"], cfg["dphi"], 8, 3, coef.shape[1])
    d_coef = torch.from_numpy(coef).cuda()
    plan.set_layers([ly], d_coef)
    dev = torch.empty(plan.table_shape, dtype=torch.float32, device="cuda")
    plan.solve(dev)
    torch.cuda.synchronize()
    # pinned and pageable host buffers
    h_coef = torch.from_numpy(coef).pin_memory()
    h_out = torch.empty(plan.table_shape, dtype=torch.float32).pin_memory()
    plan.solve_host(h_coef, h_out)
    assert plan.status() == 0
    assert torch.equal(h_out, dev.cpu())
    h_page = torch.full(plan.table_shape, float("nan"), dtype=torch.float32)
    plan.solve_host(torch.from_numpy(coef.copy()), h_page)
    assert plan.status() == 0
    assert torch.equal(h_page, dev.cpu())
    plan.close()
