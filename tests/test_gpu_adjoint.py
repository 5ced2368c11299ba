"""The adjoint (vrte_brdf_backward and the autograd binding) against the FP64 oracle.

dL/dp for L = 1/2 |F - F_target|^2 over the whole table, p = (omega, tau0, n, every
coefficient), from the GPU's FP64 form, element by element against the oracle's two
gradients on small layers with and without a dielectric top: the exact one of
oracle/tangent.py (dual numbers through the propagator form of each order) and the
Richardson-extrapolated central differences of oracle/gradient.py. Tolerance: 1e-5 relative
for every entry at least 1e-3 of the largest; smaller entries (whose differences the
difference oracle resolves less well) to 1e-8 of the largest. The FP32-table path is checked against the FP64 gradient at the 1e-3
relative bound that FP32 rounding of the table allows.
"""
import numpy as np
import pytest

import oracle as O
import oracle.gradient as OG
import oracle.tangent as OT
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import monodisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _layer(nif, L=8, x=2.0, omega=0.9, tau=1.3, N=4):
    coef = monodisperse_coefficients(1.5 + 0.01j, x, L)
    return dict(tau=tau, omega=omega, n_interface=nif, n_nodes=N, n_orders=L, n_coef=L,
                coef=coef)


def _target(ly, grids, seed=11):
    """Oracle table of the layer with every parameter perturbed by a seeded 1-5 %."""
    rng = np.random.default_rng(seed)
    L = ly["n_coef"]
    p = OG.pack(ly["omega"], ly["tau"], ly["n_interface"], ly["coef"])
    p = p * (1.0 + rng.uniform(0.01, 0.05, p.size) * rng.choice([-1.0, 1.0], p.size))
    if ly["n_interface"] <= 1.0:
        p[2] = ly["n_interface"]
    return OG.table(p, L, ly["n_nodes"], ly["n_orders"], *grids)


def _gpu_grad(ly, grids, target, out_dtype=torch.float64):
    L = ly["n_coef"]
    plan = vr.Plan(*grids, ly["n_nodes"], ly["n_orders"], L, 1, vr.VRTE_FP64, adjoint=True)
    try:
        d_coef = torch.from_numpy(vr.pack_coefficients([ly])).cuda()
        plan.set_layers([ly], d_coef)
        F = torch.empty(plan.table_shape, dtype=out_dtype, device="cuda")
        plan.solve(F)
        G = F - torch.from_numpy(target[None]).to(F.device, out_dtype)
        g = plan.backward(G)
        torch.cuda.synchronize()
        assert plan.status() == 0
        return g[0].cpu().numpy(), F[0].double().cpu().numpy()
    finally:
        plan.close()


def _compare(g, ref, rel=1e-5, floor=1e-3, tiny=1e-8):
    big = np.abs(ref).max()
    err = np.abs(g - ref)
    lim = np.where(np.abs(ref) >= floor * big, rel * np.abs(ref), tiny * big)
    bad = np.nonzero(err > lim)[0]
    if bad.size:
        lines = [f"  p[{k}] gpu {g[k]: .12e} ref {ref[k]: .12e} err {err[k]:.2e}" for k in bad[:20]]
        raise AssertionError(f"{bad.size} gradient entries off (max |ref| {big:.3e}):\n" +
                             "\n".join(lines))


@pytest.mark.parametrize("nif", [1.4, 1.0])
def test_adjoint_matches_oracle_gradient(nif):
    ly = _layer(nif)
    grids = angle_grids(3, 4, 5)
    target = _target(ly, grids)
    g, F = _gpu_grad(ly, grids, target)
    L = ly["n_coef"]
    p = OG.pack(ly["omega"], ly["tau"], nif, ly["coef"])
    idx = [k for k in range(p.size) if not (k == 2 and nif <= 1.0)]
    ref = OG.loss_gradient(p, target, L, ly["n_nodes"], ly["n_orders"], *grids, indices=idx)
    exact = OT.loss_gradient(p, target, L, ly["n_nodes"], ly["n_orders"], *grids, indices=idx)
    if nif <= 1.0:
        assert g[2] == 0.0
    _compare(g, exact)
    _compare(g, ref)
    big = np.abs(exact).max()
    print(f"max |gpu - exact| / max|g| = {np.abs(g - exact).max() / big:.2e}")


def test_adjoint_thick_layer_resolves_every_order():
    """A thicker, more absorbing-free layer (tau0 = 6, omega = 0.97) with a larger expansion,
    where high orders carry clusters of equal eigenvalues of F'E' and complex pairs."""
    ly = _layer(1.33, L=10, x=3.0, omega=0.97, tau=6.0, N=4)
    grids = angle_grids(2, 3, 4)
    target = _target(ly, grids, seed=5)
    g, _ = _gpu_grad(ly, grids, target)
    p = OG.pack(ly["omega"], ly["tau"], ly["n_interface"], ly["coef"])
    ref = OG.loss_gradient(p, target, ly["n_coef"], ly["n_nodes"], ly["n_orders"], *grids)
    _compare(g, ref)


def test_adjoint_optically_thick_layer_stays_finite():
    """tau0 = 40 with N = 8 (kappa up to ~50): the mode integrals of the adjoint two-point problem
    pair modes whose exponentials e^{-kappa tau0} differ by far more than the FP64 range; each is
    taken in the form whose Phi1 argument has a non-negative real part, so the gradient is finite
    and matches the oracle's difference gradient (the eigen-form oracle keeps its exponentials
    scaled; the propagator form of the exact one overflows at this thickness)."""
    ly = _layer(1.33, L=8, x=2.0, omega=0.95, tau=40.0, N=8)
    grids = angle_grids(2, 3, 4)
    target = _target(ly, grids, seed=7)
    g, _ = _gpu_grad(ly, grids, target)
    assert np.all(np.isfinite(g))
    p = OG.pack(ly["omega"], ly["tau"], ly["n_interface"], ly["coef"])
    ref = OG.loss_gradient(p, target, ly["n_coef"], ly["n_nodes"], ly["n_orders"], *grids)
    _compare(g, ref)


def test_adjoint_fp32_table():
    """The gradient of the loss of an FP32 table (FP32 table gradient in, grad_dtype F32)
    equals the FP64 path's on the same values, and the FP64 gradient to 1e-3 relative."""
    ly = _layer(1.5)
    grids = angle_grids(3, 4, 5)
    target = _target(ly, grids)
    g64, _ = _gpu_grad(ly, grids, target)
    g32, _ = _gpu_grad(ly, grids, target, out_dtype=torch.float32)
    big = np.abs(g64).max()
    assert np.abs(g32 - g64).max() <= 1e-3 * big


def test_adjoint_autograd_matches_backward():
    """torch.autograd through brdf_autograd gives plan.backward's gradient, and a directional
    difference of the loss in omega agrees with it."""
    ly = _layer(1.4)
    grids = angle_grids(3, 4, 5)
    target = torch.from_numpy(_target(ly, grids)[None]).cuda()
    L = ly["n_coef"]
    plan = vr.Plan(*grids, ly["n_nodes"], ly["n_orders"], L, 1, vr.VRTE_FP64, adjoint=True)
    try:
        params = torch.tensor([[ly["omega"], ly["tau"], ly["n_interface"]]], dtype=torch.float64,
                              requires_grad=True)
        coeffs = torch.from_numpy(vr.pack_coefficients([ly])).cuda().requires_grad_(True)
        sizes = [(ly["n_nodes"], ly["n_orders"], L)]

        def loss(pp, cc):
            F = vr.brdf_autograd(pp, cc, sizes, plan)
            return 0.5 * ((F - target) ** 2).sum()

        lo = loss(params, coeffs)
        lo.backward()
        g_auto = np.concatenate([params.grad[0].numpy(), coeffs.grad[0].cpu().numpy().ravel()])
        g_ref, _ = _gpu_grad(ly, grids, target[0].cpu().numpy())
        assert np.allclose(g_auto, g_ref, rtol=1e-12, atol=1e-14 * np.abs(g_ref).max())
        with torch.no_grad():
            h = 1e-5
            dp = torch.tensor([[h, 0.0, 0.0]], dtype=torch.float64)
            fd = (loss(params + dp, coeffs) - loss(params - dp, coeffs)).item() / (2 * h)
        assert abs(fd - g_auto[0]) <= 1e-6 * abs(g_auto[0])
    finally:
        plan.close()


def test_adjoint_several_layers_in_one_call():
    """Three uneven layers in one plan (they run on the plan's concurrent streams): each
    layer's gradient row equals the single-layer gradient."""
    lys = [_layer(1.4), _layer(1.0, L=6, x=1.5, omega=0.8, tau=0.7, N=3),
           _layer(1.6, L=9, x=2.5, omega=0.95, tau=2.5, N=5)]
    grids = angle_grids(3, 4, 5)
    targets = [_target(ly, grids, seed=3 + i) for i, ly in enumerate(lys)]
    Lmax = max(ly["n_coef"] for ly in lys)
    plan = vr.Plan(*grids, max(ly["n_nodes"] for ly in lys), max(ly["n_orders"] for ly in lys),
                   Lmax, len(lys), vr.VRTE_FP64, adjoint=True)
    try:
        d_coef = torch.from_numpy(vr.pack_coefficients(lys)).cuda()
        plan.set_layers(lys, d_coef)
        F = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
        plan.solve(F)
        G = F - torch.from_numpy(np.stack(targets)).cuda()
        g = plan.backward(G).cpu().numpy()
        assert plan.status() == 0
    finally:
        plan.close()
    for i, ly in enumerate(lys):
        gi, _ = _gpu_grad(ly, grids, targets[i])
        L = ly["n_coef"]
        assert np.allclose(g[i, :3 + 6 * L], gi, rtol=1e-10, atol=1e-13 * np.abs(gi).max())
        assert np.all(g[i, 3 + 6 * L:] == 0.0)


def test_adjoint_argument_checks():
    grids = angle_grids(2, 2, 3)
    ly = _layer(1.4)
    plan = vr.Plan(*grids, 4, 8, 8, 1, vr.VRTE_FP64)  # no adjoint workspace
    try:
        plan.set_layers([ly], torch.from_numpy(vr.pack_coefficients([ly])).cuda())
        G = torch.zeros(plan.table_shape, dtype=torch.float64, device="cuda")
        with pytest.raises(vr.VrteError) as e:
            plan.backward(G)
        assert e.value.code == 2  # VRTE_ERR_STATE
        lib = vr.load_library()
        assert lib.vrte_brdf_backward(plan.handle, None, 1, None, None) == 1
    finally:
        plan.close()
