"""Several layers of uneven size in one plan and one solve (the batched form).

Layers differ in N, M, L, tau, omega and interface index, as in the batched workload
(materials x wavelengths); every layer's table is checked against the oracle run on that
layer alone. Tolerances as in the single-layer parity tests (FP64: 1e-10 of F_00; mixed:
1e-6 on the I row, 1e-5 on the Q, U, V rows).
"""
import numpy as np
import pytest

import oracle as O
import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import monodisperse_coefficients, polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _layers():
    rng = np.random.default_rng(17070004)
    out = []
    for N, L, x in [(6, 10, 2.0), (12, 24, 4.0), (8, 16, 3.0), (16, 32, 6.0)]:
        coef = polydisperse_coefficients(1.5 + 0.001j, x, 0.1, L) if x > 3 else \
            monodisperse_coefficients(1.4 + 0.002j, x, L)
        out.append(dict(tau=float(10 ** rng.uniform(-1, 2)), omega=float(rng.uniform(0.5, 0.999)),
                        n_interface=float(rng.uniform(1.3, 1.7)), n_nodes=N, n_orders=L,
                        coef=coef))
    return out


def _errors(F, G):
    scale = np.abs(G[..., 0, 0])[..., None]
    e = np.abs(F - G)
    return float(np.max(e[..., 0, :] / scale)), float(np.max(e[..., 1:, :] / scale[..., None]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_layers_in_one_solve(precision):
    layers = _layers()
    mu_in, mu_out, dphi = angle_grids(9, 11, 13)
    prec = vr.VRTE_FP64 if precision == "fp64" else vr.VRTE_MIXED
    F = vr.brdf(layers, mu_in, mu_out, dphi, precision=prec, out_dtype=torch.float64)
    torch.cuda.synchronize()
    F = F.cpu().numpy()
    assert F.shape == (len(layers), 9, 11, 13, 4, 4)
    for b, ly in enumerate(layers):
        G = O.brdf(ly["coef"], ly["omega"], ly["tau"], ly["n_interface"], ly["n_nodes"],
                   ly["n_orders"], mu_in, mu_out, dphi)
        ei, eq = _errors(F[b], G)
        if precision == "fp64":
            assert max(ei, eq) < 1e-10, (b, ei, eq)
        else:
            assert ei < 1e-6 and eq < 1e-5, (b, ei, eq)
