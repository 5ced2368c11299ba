"""A solve captured into a CUDA graph from the caller's stream and replayed writes the same
table as a direct solve: `vrte_solve_brdf` allocates nothing and does not synchronize the
host, and the layers of a multi-layer plan fork onto the plan's own streams and join back
into the caller's stream with events."""
import numpy as np
import pytest

import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import monodisperse_coefficients, polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _layers():
    out = []
    for N, L, x, tau in [(6, 10, 2.0, 0.7), (10, 20, 4.0, 5.0), (8, 16, 3.0, 2.0)]:
        coef = polydisperse_coefficients(1.5 + 0.001j, x, 0.1, L) if x > 3 else \
            monodisperse_coefficients(1.4 + 0.002j, x, L)
        out.append(dict(tau=tau, omega=0.9, n_interface=1.4, n_nodes=N, n_orders=L, coef=coef,
                        n_coef=coef.shape[0]))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_direct_solve(precision):
    layers = _layers()
    mu_in, mu_out, dphi = angle_grids(7, 9, 11)
    prec = vr.VRTE_FP64 if precision == "fp64" else vr.VRTE_MIXED
    coef = vr.pack_coefficients(layers)
    plan = vr.Plan(mu_in, mu_out, dphi, max(l["n_nodes"] for l in layers),
                   max(l["n_orders"] for l in layers), coef.shape[1], len(layers), prec)
    plan.set_layers(layers, torch.from_numpy(coef).cuda())
    ref = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
    plan.solve(ref)
    torch.cuda.synchronize()
    assert plan.status() == 0

    s = torch.cuda.Stream()
    out = torch.zeros_like(ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        plan.solve(out, s)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    a, b = ref.cpu().numpy(), out.cpu().numpy()
    assert np.all(np.isfinite(b))
    scale = np.abs(a[..., 0, 0])[..., None, None] + 1e-300
    assert float(np.max(np.abs(a - b) / scale)) < 1e-13
    plan.close()
