"""The allocation-free eigen entry point (vrte_eigen_noalloc) against the solver's own.

Callers that cannot allocate device memory use vrte_eigen_noalloc, which keeps its
scratch in a static device array. This test feeds it the reduced homogeneous matrices
F'E' that a plan solve produced, twice in a row, and checks eigenvalues and
eigenvectors against what the plan's eigen stage computed from the same matrices.
(Order 0 is left out: the FP64 plan re-solves it in the block form.) It lives in a file
collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import paper_1707_05882_gb300 as vr
from vrte_inputs import angle_grids
from vrte_inputs.mie import polydisperse_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_eigen_matches_solver_eigen_stage():
    lib = vr.load_library()
    N, M, L = 8, 16, 16
    n = 4 * N
    coef = polydisperse_coefficients(1.5 + 0.001j, 5.0, 0.1, L)
    mu_in, mu_out, dphi = angle_grids(4, 5, 6)
    plan = vr.Plan(mu_in, mu_out, dphi, N, M, L)
    plan.set_layers([dict(tau=2.0, omega=0.95, n_interface=1.5, n_nodes=N, n_orders=M, n_coef=L)],
                    torch.from_numpy(vr.pack_coefficients([dict(coef=coef)])).cuda())
    out = torch.empty(plan.table_shape, dtype=torch.float64, device="cuda")
    plan.solve(out)
    assert plan.status() == 0
    FE = plan.debug_buffer("FE")[:M * n * n].reshape(M, n, n)
    ref_re = plan.debug_buffer("lam_re")[:M * n].reshape(M, n)
    ref_im = plan.debug_buffer("lam_im")[:M * n].reshape(M, n)
    ref_X = plan.debug_buffer("X")[:M * n * n].reshape(M, n, n)
    plan.close()

    d_A = torch.from_numpy(np.ascontiguousarray(FE)).cuda()
    for call in range(2):
        lr = torch.full((M, n), float("nan"), dtype=torch.float64, device="cuda")
        li = torch.full((M, n), float("nan"), dtype=torch.float64, device="cuda")
        X = torch.full((M, n, n), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        code = lib.vrte_eigen_noalloc(_ptr(d_A), n, M, _ptr(lr), _ptr(li), _ptr(X), _ptr(st),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        lr, li, X = lr.cpu().numpy(), li.cpu().numpy(), X.cpu().numpy()
        for m in range(1, M):
            scale = np.abs(ref_re[m] + 1j * ref_im[m]).max()
            assert np.abs(lr[m] - ref_re[m]).max() <= 1e-11 * scale, (call, m)
            assert np.abs(li[m] - ref_im[m]).max() <= 1e-11 * scale, (call, m)
            assert np.abs(X[m] - ref_X[m]).max() <= 1e-11, (call, m)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = vr.load_library()
    n, batch = 768, 2  # (3 n^2 + n) * batch exceeds 2^21 - 8 doubles
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = lib.vrte_eigen_noalloc(_ptr(d), n, batch, _ptr(d), _ptr(d), _ptr(d), None, None)
    assert code == 1  # VRTE_ERR_INVALID_ARG, before any launch
