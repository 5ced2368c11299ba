"""The allocation-free eigen entry point (vrte_eigen_noalloc).

Callers that cannot allocate device memory (memory owned by another allocator or a
fixed pool, paths where an allocation would synchronize or is forbidden) use
vrte_eigen_noalloc, which keeps its scratch in a static device array. The tests check
it three ways: against the solver's own eigen stage on the reduced homogeneous matrices
F'E' of a plan solve, on two calls in a row; independently of the solver, by the
eigen-residual |A X - X Lambda| / (|A| |X|) of every matrix and by its eigenvalues as a
sorted set against numpy's; at the size limit n = 768 that the scratch admits for
one matrix; and replayed from a captured CUDA graph. The file is collected last so that a run stopping at the first failure has
run every other test.
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


def _call(lib, A, with_status=True):
    """Runs vrte_eigen_noalloc on host matrices A [batch, n, n]; returns (lr, li, X, status)."""
    batch, n, _ = A.shape
    d_A = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    lr = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
    li = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
    X = torch.full((batch, n, n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.vrte_eigen_noalloc(_ptr(d_A), n, batch, _ptr(lr), _ptr(li), _ptr(X),
                                  _ptr(st) if with_status else None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    return lr.cpu().numpy(), li.cpu().numpy(), X.cpu().numpy(), int(st.item())


def _complex_eigvecs(lr, li, X):
    """Columns of the real-packed eigenvector matrix as complex eigenvectors, with their
    eigenvalues: a pair (j, j+1) with li[j] > 0 holds the real and imaginary parts."""
    n = lr.size
    V = X.astype(complex).copy()
    lam = lr + 1j * li
    j = 0
    while j < n:
        if li[j] > 0.0:
            V[:, j] = X[:, j] + 1j * X[:, j + 1]
            V[:, j + 1] = X[:, j] - 1j * X[:, j + 1]
            j += 2
        else:
            j += 1
    return lam, V


def _check_independent(A, lr, li, X, tol=1e-12):
    for b in range(A.shape[0]):
        lam, V = _complex_eigvecs(lr[b], li[b], X[b])
        res = np.abs(A[b] @ V - V * lam[None, :]).max()
        assert res <= tol * np.abs(A[b]).max() * np.abs(V).max() * A.shape[1], b
        ref = np.linalg.eigvals(A[b])
        key = lambda z: (np.round(z.real, 9), np.round(z.imag, 9))
        a = np.array(sorted(lam, key=key))
        r = np.array(sorted(ref, key=key))
        assert np.abs(a - r).max() <= 1e-10 * np.abs(ref).max(), b


@pytest.fixture(scope="module")
def fe_matrices():
    """F'E' of every order of a small Mie layer with an interface, and the plan's own
    eigenpairs of the same matrices."""
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
    ref = (plan.debug_buffer("lam_re")[:M * n].reshape(M, n),
           plan.debug_buffer("lam_im")[:M * n].reshape(M, n),
           plan.debug_buffer("X")[:M * n * n].reshape(M, n, n))
    plan.close()
    return FE, ref


def test_noalloc_eigen_matches_solver_eigen_stage(fe_matrices):
    lib = vr.load_library()
    FE, (ref_re, ref_im, ref_X) = fe_matrices
    M = FE.shape[0]
    for call in range(2):
        lr, li, X, st = _call(lib, FE)
        assert st == 0
        # order 0 is left out: the FP64 plan re-solves it in the block form
        for m in range(1, M):
            scale = np.abs(ref_re[m] + 1j * ref_im[m]).max()
            assert np.abs(lr[m] - ref_re[m]).max() <= 1e-11 * scale, (call, m)
            assert np.abs(li[m] - ref_im[m]).max() <= 1e-11 * scale, (call, m)
            assert np.abs(X[m] - ref_X[m]).max() <= 1e-11, (call, m)


def test_noalloc_eigen_residual_and_eigenvalues(fe_matrices):
    """Independent of the solver: every order's eigenpairs satisfy A x = lambda x and the
    eigenvalues equal numpy's as sorted sets; once without a status word."""
    lib = vr.load_library()
    FE, _ = fe_matrices
    lr, li, X, st = _call(lib, FE)
    assert st == 0
    _check_independent(FE, lr, li, X)
    lr2, li2, X2, _ = _call(lib, FE, with_status=False)
    assert np.array_equal(lr, lr2) and np.array_equal(li, li2) and np.array_equal(X, X2)


def test_noalloc_eigen_at_its_size_limit():
    """n = 768, batch = 1 fills the scratch array to (3 n^2 + n) doubles of 2^21 - 8. The
    matrix has well-separated real eigenvalues and two complex pairs."""
    lib = vr.load_library()
    n = 768
    rng = np.random.default_rng(768)
    D = np.diag(np.linspace(1.0, 40.0, n))
    D[10:12, 10:12] = [[5.0, 2.0], [-2.0, 5.0]]
    D[400:402, 400:402] = [[20.0, 0.5], [-0.5, 20.0]]
    Q = np.eye(n) + 0.2 * rng.normal(size=(n, n)) / np.sqrt(n)
    A = (Q @ D @ np.linalg.inv(Q))[None]
    lr, li, X, st = _call(lib, A)
    assert st == 0
    assert np.sum(li[0] > 0) == 2
    _check_independent(A, lr, li, X)


def test_noalloc_eigen_replayed_from_a_captured_graph(fe_matrices):
    """Allocating nothing, the call can be captured into a CUDA graph once a first call has
    resolved the scratch address on the device: two replays give the direct call's
    eigenpairs bit for bit, with the status word clear."""
    lib = vr.load_library()
    FE, _ = fe_matrices
    lr0, li0, X0, st0 = _call(lib, FE)
    assert st0 == 0
    batch, n, _ = FE.shape
    d_A = torch.from_numpy(np.ascontiguousarray(FE)).cuda()
    lr = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
    li = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
    X = torch.full((batch, n, n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        code = lib.vrte_eigen_noalloc(_ptr(d_A), n, batch, _ptr(lr), _ptr(li), _ptr(X), _ptr(st),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(lr.cpu().numpy(), lr0) and np.array_equal(li.cpu().numpy(), li0)
        assert np.array_equal(X.cpu().numpy(), X0)
        lr.fill_(float("nan"))
        X.fill_(float("nan"))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = vr.load_library()
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (3 n^2 + n) * batch exceeds 2^21 - 8 doubles
    assert lib.vrte_eigen_noalloc(_ptr(d), 768, 2, _ptr(d), _ptr(d), _ptr(d), None, None) == 1
    # small matrices, but more than the 65535 a launch grid dimension takes
    assert lib.vrte_eigen_noalloc(_ptr(d), 2, 70000, _ptr(d), _ptr(d), _ptr(d), None, None) == 1
