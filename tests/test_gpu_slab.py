"""Multi-layer slabs (vrte_solve_slab_brdf; Sec. 2.C, one solution per sub-layer joined by the
continuity of the radiance) on the GPU against the oracle's block-banded solve: sub-layers with
different expansions, albedos and thicknesses under a dielectric top and over a Lambertian base;
a stack of identical sub-layers against the single-layer solve; the mixed plan's synthesis; the
argument checks. Tolerances as for one layer (1e-10 FP64; 1e-6 I row and 1e-5 Q, U, V rows of
the mixed synthesis; normalised by F_00)."""
import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids, rayleigh_coefficients
from vrte_inputs.mie import polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COEF = polydisperse_coefficients(1.5 + 0.001j, 6.0, 0.1, 40)


def _err_rows(F, G):
    scale = np.maximum(np.abs(G[..., 0, 0])[..., None, None], 1e-300)
    e = np.abs(F - G) / scale
    return float(e[..., 0, :].max()), float(e[..., 1:, :].max())


def _plan(lys, grids, precision=vr.VRTE_FP64, slab=True):
    lys = [dict(l, n_coef=np.asarray(l["coef"]).shape[0]) for l in lys]
    coef = vr.pack_coefficients(lys)
    plan = vr.Plan(*grids, max(l["n_nodes"] for l in lys), max(l["n_orders"] for l in lys),
                   coef.shape[1], len(lys), precision, slab=slab)
    plan.set_layers(lys, torch.from_numpy(coef).cuda())
    return plan


def _solve_slab(lys, grids, precision=vr.VRTE_FP64, out_dtype=torch.float64):
    plan = _plan(lys, grids, precision)
    try:
        out = torch.empty(plan.table_shape[1:], dtype=out_dtype, device="cuda")
        plan.solve_slab(out)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return out.double().cpu().numpy()
    finally:
        plan.close()


def _oracle(lys, grids, N, M):
    return O.slab_brdf([dict(coef=l["coef"], omega=l["omega"], tau=l["tau"]) for l in lys],
                       lys[0].get("n_interface", 1.0), N, M, *grids,
                       rho=lys[-1].get("base_albedo", 0.0), base=lys[-1].get("base_mueller"))


def _stack(N, M, n_if=1.4, rho=0.3):
    return [dict(tau=0.5, omega=0.97, n_interface=n_if, n_nodes=N, n_orders=M, coef=COEF[:M]),
            dict(tau=0.3, omega=0.6, n_nodes=N, n_orders=M, coef=rayleigh_coefficients()),
            dict(tau=1.2, omega=0.9, n_nodes=N, n_orders=M, coef=COEF[:M // 2],
                 base_albedo=rho)]


@pytest.mark.parametrize("n_if,rho", [(1.0, 0.0), (1.4, 0.3)])
def test_slab_fp64_against_oracle(n_if, rho):
    N, M = 12, 24
    lys = _stack(N, M, n_if, rho)
    grids = angle_grids(9, 11, 7)
    F = _solve_slab(lys, grids)
    G = _oracle(lys, grids, N, M)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-10 and e_q < 1e-10, (e_i, e_q)


def test_identical_sublayers_equal_the_single_layer():
    N, M = 10, 20
    one = dict(tau=1.7, omega=0.93, n_interface=1.5, n_nodes=N, n_orders=M, coef=COEF[:M],
               base_albedo=0.2)
    parts = [dict(one, tau=0.4, base_albedo=0.0), dict(one, tau=0.9, n_interface=1.0,
                                                       base_albedo=0.0),
             dict(one, tau=0.4, n_interface=1.0)]
    grids = angle_grids(7, 8, 5)
    F = _solve_slab(parts, grids)
    plan = _plan([one], grids, slab=False)
    try:
        out = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        plan.solve(out)
        torch.cuda.synchronize()
        G = out[0].cpu().numpy()
    finally:
        plan.close()
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-10 and e_q < 1e-10, (e_i, e_q)


def test_slab_larger_case_against_oracle():
    N, M = 24, 48
    lys = _stack(N, M)
    grids = angle_grids(16, 16, 12)
    F = _solve_slab(lys, grids)
    G = _oracle(lys, grids, N, M)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-10 and e_q < 1e-10, (e_i, e_q)


def test_slab_mixed_synthesis_fp32():
    N, M = 12, 24
    lys = _stack(N, M)
    grids = angle_grids(9, 11, 7)
    F = _solve_slab(lys, grids, precision=vr.VRTE_MIXED, out_dtype=torch.float32)
    G = _oracle(lys, grids, N, M)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-6 and e_q < 1e-5, (e_i, e_q)


def test_slab_argument_checks():
    N, M = 4, 8
    grids = angle_grids(2, 2, 3)
    lys = _stack(N, M)
    bad = [dict(lys[0]), dict(lys[1], n_interface=1.3), dict(lys[2])]
    plan = _plan(bad, grids)
    try:
        out = torch.empty(plan.table_shape[1:], dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.solve_slab(out)
        assert e.value.code == 1  # VRTE_ERR_INVALID_ARG: a smooth top inside the slab
    finally:
        plan.close()
    plan = _plan(lys, grids, slab=False)
    try:
        out = torch.empty(plan.table_shape[1:], dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.solve_slab(out)
        assert e.value.code == 2  # VRTE_ERR_STATE: no slab workspace
    finally:
        plan.close()


def test_slab_more_sublayers_than_slots():
    # six sub-layers on the plan's four workspace slots: slots are reused within an order
    # batch, each sub-layer's modes waiting until the elimination has used the slot's last ones
    N, M = 8, 16
    base = _stack(N, M)
    lys = [dict(base[k % 3], n_interface=(1.4 if k == 0 else 1.0),
                base_albedo=(0.25 if k == 5 else 0.0), tau=0.2 + 0.15 * k) for k in range(6)]
    grids = angle_grids(6, 7, 5)
    F = _solve_slab(lys, grids)
    G = _oracle(lys, grids, N, M)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-10 and e_q < 1e-10, (e_i, e_q)


def test_slab_over_a_polarizing_base():
    # a direction-independent Mueller BRDF matrix under the last sub-layer (with a Lambertian
    # part added), and the same matrix under an inner sub-layer rejected
    R = np.array([[0.9, 0.25, 0.0, 0.0], [0.18, 0.5, 0.0, 0.0],
                  [0.0, 0.0, 0.4, 0.15], [0.0, 0.0, -0.1, 0.3]])
    N, M = 12, 24
    lys = _stack(N, M, 1.4, 0.1)
    lys[-1]["base_mueller"] = R
    grids = angle_grids(9, 11, 7)
    F = _solve_slab(lys, grids)
    G = _oracle(lys, grids, N, M)
    e_i, e_q = _err_rows(F, G)
    assert e_i < 1e-10 and e_q < 1e-10, (e_i, e_q)
    bad = [dict(lys[0]), dict(lys[1], base_mueller=R), dict(lys[2])]
    plan = _plan(bad, angle_grids(2, 2, 3))
    try:
        out = torch.empty(plan.table_shape[1:], dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.solve_slab(out)
        assert e.value.code == 1  # VRTE_ERR_INVALID_ARG: a reflecting base inside the slab
    finally:
        plan.close()
