"""The tensor-core GEMM with exact fixed-point slicing (vrte_gemm_sliced) against FP64.

Sizes span several 128 x 64 output tiles and 32-wide K blocks with ragged tails; rows of A
and columns of B carry widely different scales (the slicing is per row / per column).
Error bound: |C - A B| <= c 2^(-7S) max|A_i| max|B_j| K (measured in a CPU simulation of
the same arithmetic: 2.1e-3, 3.1e-5, 3.5e-7, 3.2e-9 for S = 1..4; on the GPU 9.1e-10,
7.7e-12, 7.2e-14, 6.0e-16, 1.4e-16 for S = 4..8).
"""
import numpy as np
import pytest

import paper_1707_05882_gb300 as vr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {1: 1e-2, 2: 1.5e-4, 3: 2e-6, 4: 2e-8, 5: 2e-10, 6: 2e-12, 7: 4e-15, 8: 1e-15}


def _case(rng, b, M, K, N):
    A = rng.normal(size=(b, M, K)) * np.exp(rng.normal(size=(b, M, 1)) * 3)
    B = rng.normal(size=(b, K, N)) * np.exp(rng.normal(size=(b, 1, N)) * 3)
    return A, B


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("shape", [(1, 128, 64, 64), (3, 200, 300, 100), (2, 257, 1000, 130)])
def test_sliced_gemm_accuracy(S, shape):
    rng = np.random.default_rng(7 + S)
    b, M, K, N = shape
    A, B = _case(rng, b, M, K, N)
    C, st = vr.gemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), slices=S)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    C = C.cpu().numpy()
    ref = A @ B
    scale = np.abs(A).max(axis=2)[:, :, None] * np.abs(B).max(axis=1)[:, None, :] * K
    err = np.max(np.abs(C - ref) / scale)
    assert err < BOUND[S], err


def test_sliced_gemm_zero_rows_and_columns():
    A = np.zeros((1, 130, 70))
    B = np.random.default_rng(1).normal(size=(1, 70, 65))
    A[0, 5] = np.arange(70)
    C, st = vr.gemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), slices=4)
    C = C.cpu().numpy()
    assert int(st.item()) == 0
    assert np.abs(C[0, :5]).max() == 0.0 and np.abs(C[0, 6:]).max() == 0.0
    bound = 2e-8 * np.abs(A[0, 5]).max() * np.abs(B[0]).max(axis=0) * 70
    assert np.all(np.abs(C[0, 5] - A[0, 5] @ B[0]) < bound)


def test_sliced_gemm_rejects_bad_sizes():
    lib = vr.load_library()
    assert lib.vrte_gemm_sliced_workspace(10, 10, 2000, 1, 4) == 0
    assert lib.vrte_gemm_sliced_workspace(10, 10, 100, 1, 9) == 0
    assert lib.vrte_gemm_sliced_workspace(10, 10, 100, 1, 0) == 0
    assert lib.vrte_gemm_sliced_workspace(10, 10, 100, 1, 4) > 0
