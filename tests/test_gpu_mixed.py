"""Parity of the mixed-precision form (tensor-core contractions, through the C ABI) with
the FP64 CPU oracle.

Tolerance of the mixed form: every element of the I row of the 4x4 Mueller matrix
(I -> I, Q, U, V coupling) agrees within 1e-6 of F_00 at the same (incident, outgoing,
azimuth) point, and every element of the Q, U, V rows within 1e-5 of F_00.
"""
import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids, make_config
from vrte_inputs.mie import monodisperse_coefficients, polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_I = 1e-6
TOL_QUV = 1e-5


def row_errors(F, G):
    """(I-row error, QUV-row error), each max |F - G| / |G_00| over points."""
    scale = np.maximum(np.abs(G[..., 0, 0]), 1e-300)[..., None]
    e = np.abs(F - G)
    return float(np.max(e[..., 0, :] / scale)), float(np.max(e[..., 1:, :] / scale[..., None]))


def mixed_brdf(layer, mu_in, mu_out, dphi, out_dtype=None):
    out = vr.brdf([layer], mu_in, mu_out, dphi, precision=vr.VRTE_MIXED,
                  out_dtype=out_dtype or torch.float64)
    torch.cuda.synchronize()
    return out[0].cpu().numpy()


def oracle_brdf(layer, mu_in, mu_out, dphi):
    return O.brdf(layer["coef"], layer["omega"], layer["tau"], layer.get("n_interface", 1.0),
                  layer["n_nodes"], layer["n_orders"], mu_in, mu_out, dphi)


def check(layer, mu_in, mu_out, dphi):
    F = mixed_brdf(layer, mu_in, mu_out, dphi)
    G = oracle_brdf(layer, mu_in, mu_out, dphi)
    assert F.shape == G.shape
    assert np.all(np.isfinite(F))
    ei, eq = row_errors(F, G)
    assert ei < TOL_I, (ei, eq)
    assert eq < TOL_QUV, (ei, eq)
    return ei, eq


def test_mixed_rayleigh_N8_M3_8x8x16():
    cfg = make_config(1)
    check(cfg["layers"][0], cfg["mu_in"], cfg["mu_out"], cfg["dphi"])


@pytest.mark.parametrize("n_if", [1.0, 1.5])
def test_mixed_ragged_multi_tile_mie(n_if):
    """4N = 80, 4 n_in = 68, 4 n_out = 76, 4L = 160: ragged tails on every tensor-core tile."""
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    ly = dict(tau=3.0, omega=0.97, n_interface=n_if, n_nodes=20, n_orders=40, coef=coef)
    check(ly, *angle_grids(17, 19, 11))


def test_mixed_mie_N32_M64_64x64x90():
    cfg = make_config(2)
    check(cfg["layers"][0], cfg["mu_in"], cfg["mu_out"], cfg["dphi"])


def test_mixed_synthesis_spans_several_incident_blocks():
    """n_in = 150 > 64 incident cosines per synthesis block: three blocks, the last ragged."""
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 16)
    ly = dict(tau=2.0, omega=0.95, n_interface=1.33, n_nodes=8, n_orders=16, coef=coef)
    check(ly, *angle_grids(150, 5, 9))


@pytest.mark.parametrize("case", ["thin", "thick", "N1", "orders_beyond_L", "mu_one",
                                  "one_direction", "albedo_near_one"])
def test_mixed_edge_cases(case):
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)
    ly = dict(tau=1.0, omega=0.9, n_interface=1.33, n_nodes=6, n_orders=12, coef=coef)
    mu_in, mu_out, dphi = angle_grids(5, 6, 7)
    if case == "thin":
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
    elif case == "albedo_near_one":
        ly["omega"] = 0.999
        ly["tau"] = 10.0
    check(ly, mu_in, mu_out, dphi)


def test_mixed_zero_albedo_is_exactly_zero():
    coef = monodisperse_coefficients(1.5 + 0.01j, 2.0, 12)
    ly = dict(tau=1.0, omega=0.0, n_interface=1.33, n_nodes=6, n_orders=12, coef=coef)
    F = mixed_brdf(ly, *angle_grids(5, 6, 7))
    assert np.abs(F).max() == 0.0


def test_mixed_fp32_output_rounds_the_mixed_result():
    """The FP32 table is the mixed result rounded to FP32 (summed error-free in FP32
    pairs, so within one unit in the last place of the rounded FP64-output value)."""
    cfg = make_config(1)
    ly = cfg["layers"][0]
    F64 = mixed_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"])
    F32 = mixed_brdf(ly, cfg["mu_in"], cfg["mu_out"], cfg["dphi"], out_dtype=torch.float32)
    R = F64.astype(np.float32)
    assert np.all(np.abs(F32 - R) <= np.spacing(np.abs(R)))
    assert np.mean(F32 == R) > 0.9


def test_mixed_rejects_contraction_beyond_exact_limit():
    """4L > 1024 leaves the exact-accumulation range of the sliced product."""
    mu = np.array([0.5])
    plan = vr.Plan(mu, mu, mu, 8, 300, 300, precision=vr.VRTE_MIXED)
    coef = torch.zeros((1, 300, 6), dtype=torch.float64, device="cuda")
    ly = dict(tau=1.0, omega=0.5, n_interface=1.0, n_nodes=8, n_orders=8, n_coef=300)
    with pytest.raises(vr.VrteError) as e:
        plan.set_layers([ly], coef)
    assert e.value.code == 8
    plan.close()


def test_mixed_reconstruction_split_in_k():
    """2 * 4N + 4L = 320 + 800 > 1024: the reconstruction contraction runs in two parts."""
    coef = polydisperse_coefficients(1.5 + 0.001j, 25.0, 0.1, 200)
    ly = dict(tau=2.0, omega=0.95, n_interface=1.5, n_nodes=40, n_orders=5, coef=coef)
    check(ly, *angle_grids(7, 6, 9))


def test_mixed_matches_fp64_form_on_the_same_plan_shape():
    """The two forms differ only by the sliced-product rounding of the contractions."""
    coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
    ly = dict(tau=3.0, omega=0.97, n_interface=1.5, n_nodes=20, n_orders=40, coef=coef)
    mu_in, mu_out, dphi = angle_grids(17, 19, 11)
    F = mixed_brdf(ly, mu_in, mu_out, dphi)
    G = vr.brdf([ly], mu_in, mu_out, dphi, precision=vr.VRTE_FP64,
                out_dtype=torch.float64)[0].cpu().numpy()
    ei, eq = row_errors(F, G)
    assert ei < TOL_I and eq < TOL_QUV
    assert ei > 0.0  # the mixed form really ran the sliced contractions


@pytest.mark.parametrize("grid", ["uniform_odd", "irregular"])
def test_mixed_synthesis_azimuth_mirrors(grid):
    """The tensor-core synthesis computes one azimuth of every pair (phi, -phi mod 2 pi) on the
    grid and stores the mirror from it (cosine class even, sine class odd): a uniform grid of
    odd length (0 unpaired), and an irregular grid with paired, unpaired, self-paired (0, pi),
    repeated and out-of-range azimuths (-0.3 = 2 pi - 0.3; 7.0 paired with 4 pi - 7.0)."""
    if grid == "uniform_odd":
        dphi = 2 * np.pi * np.arange(13) / 13
    else:
        dphi = np.array([0.3, 1.7, 4.0, 2 * np.pi - 0.3, np.pi, 0.0, 2 * np.pi - 1.7, 5.1,
                         1.7, -0.3, 7.0, 4 * np.pi - 7.0, 2.2])
    layer = dict(tau=1.3, omega=0.93, n_interface=1.5, n_nodes=12, n_orders=24,
                 coef=polydisperse_coefficients(1.5 + 0.001j, 5.0, 0.1, 24))
    mu_in, mu_out, _ = angle_grids(5, 6, 4)
    F = mixed_brdf(layer, mu_in, mu_out, dphi, out_dtype=torch.float32)
    G = oracle_brdf(layer, mu_in, mu_out, dphi)
    ei, eq = row_errors(F, G)
    assert ei < TOL_I and eq < TOL_QUV, (ei, eq)


@pytest.mark.parametrize("case", ["ragged_blocks", "mie_N64_L128"])
def test_mixed_host_buffer_blockwise_matches_device(case):
    """The host-buffer solve reconstructs a one-batch mixed layer and synthesizes its table in
    blocks of 64 incident cosines (the copy of each finished block overlaps the next block's
    work): the same column tiles, FP64 column fixes and synthesis as the device-buffer solve,
    so the tables are equal bit for bit, and so are the counts of fixed column blocks."""
    if case == "ragged_blocks":
        coef = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)
        ly = dict(tau=2.0, omega=0.95, n_interface=1.33, n_nodes=20, n_orders=40, coef=coef)
        grids = angle_grids(150, 37, 24)      # blocks of 64, 64 and 22 incident cosines
    else:
        ly = dict(make_config(3)["layers"][0])
        grids = angle_grids(256, 96, 36)
    ly["n_coef"] = np.asarray(ly["coef"]).shape[0]
    coef = vr.pack_coefficients([ly])
    plan = vr.Plan(*grids, ly["n_nodes"], ly["n_orders"], coef.shape[1], 1, vr.VRTE_MIXED)
    try:
        plan.set_layers([ly], torch.from_numpy(coef).cuda())
        blocks = -(-grids[0].size // 64)
        for dt in (torch.float32, torch.float64):
            dev = torch.empty(plan.table_shape, dtype=dt, device="cuda")
            plan.solve(dev)
            torch.cuda.synchronize()
            assert plan.status() == 0
            fixed_dev = plan.debug_buffer("refined")[0]
            h_out = torch.full(plan.table_shape, float("nan"), dtype=dt).pin_memory()
            plan.reset_stages()
            plan.solve_host(torch.from_numpy(coef).pin_memory(), h_out)
            assert plan.status() == 0
            refine = next(st for st in plan.stages() if st["name"] == "refine")
            assert refine["launches"] == 4 + 4 * blocks      # the block-wise path ran
            assert plan.debug_buffer("refined")[0] == fixed_dev
            assert torch.equal(h_out, dev.cpu())
    finally:
        plan.close()
