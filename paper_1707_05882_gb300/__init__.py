"""GB300 DOM solver for the polarized subsurface BRDF of flat particulate layers.

Thin Python binding over the C ABI in include/vrte.h (libvrte.so, built in-tree by
paper_1707_05882_gb300.build). Argument marshalling only: every step of the solve
runs in the library's CUDA kernels. PyTorch supplies device memory and streams.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VRTE_FP64, VRTE_MIXED = 0, 1
VRTE_OUT_F32, VRTE_OUT_F64 = 0, 1

STATUS_NAMES = {
    0: "VRTE_OK", 1: "VRTE_ERR_INVALID_ARG", 2: "VRTE_ERR_STATE", 3: "VRTE_ERR_CUDA",
    4: "VRTE_ERR_OOM", 5: "VRTE_ERR_NO_CONVERGENCE", 6: "VRTE_ERR_SINGULAR",
    7: "VRTE_ERR_NONFINITE", 8: "VRTE_ERR_UNSUPPORTED",
}

EXPORTED = ["vrte_plan_create", "vrte_set_layer", "vrte_solve_brdf", "vrte_solve_brdf_host",
            "vrte_solve_btdf", "vrte_solve_radiance", "vrte_solve_slab_brdf",
            "vrte_brdf_backward", "vrte_plan_status", "vrte_profile_stages", "vrte_profile_reset",
            "vrte_debug_copy", "vrte_eigen_noalloc", "vrte_gemm_sliced", "vrte_gemm_sliced_workspace",
            "vrte_workspace_bytes", "vrte_destroy", "vrte_status_string"]


class VrteError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


class PlanDesc(ctypes.Structure):
    _fields_ = [("n_nodes_max", ctypes.c_int), ("n_orders_max", ctypes.c_int),
                ("n_coef_max", ctypes.c_int), ("n_layers_max", ctypes.c_int),
                ("n_mu_in", ctypes.c_int), ("n_mu_out", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("mu_in", ctypes.POINTER(ctypes.c_double)),
                ("mu_out", ctypes.POINTER(ctypes.c_double)),
                ("phi", ctypes.POINTER(ctypes.c_double)),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint)]


VRTE_FLAG_PROFILE = 1
VRTE_FLAG_ADJOINT = 2
VRTE_FLAG_TRANSMISSION = 4
VRTE_FLAG_SLAB = 8


class StageStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("tc_flops", ctypes.c_double)]


class Layer(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("omega", ctypes.c_double),
                ("n_interface", ctypes.c_double), ("n_nodes", ctypes.c_int),
                ("n_orders", ctypes.c_int), ("n_coef", ctypes.c_int),
                ("base_albedo", ctypes.c_double), ("base_mueller", ctypes.c_double * 16)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libvrte.so (building it first if asked); raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libvrte.so not found at {path}; run paper_1707_05882_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.vrte_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]
    lib.vrte_set_layer.argtypes = [P, ctypes.c_int, ctypes.POINTER(Layer), P]
    lib.vrte_solve_brdf.argtypes = [P, P, ctypes.c_int, P]
    lib.vrte_solve_brdf_host.argtypes = [P, P, P, ctypes.c_int, P]
    lib.vrte_solve_btdf.argtypes = [P, P, ctypes.c_int, P]
    lib.vrte_solve_radiance.argtypes = [P, P, P, P, ctypes.c_int, P]
    lib.vrte_solve_slab_brdf.argtypes = [P, P, ctypes.c_int, P]
    lib.vrte_brdf_backward.argtypes = [P, P, ctypes.c_int, P, P]
    lib.vrte_plan_status.argtypes = [P]
    lib.vrte_profile_stages.argtypes = [P, ctypes.POINTER(StageStat), ctypes.c_int]
    lib.vrte_profile_stages.restype = ctypes.c_int
    lib.vrte_profile_reset.argtypes = [P]
    lib.vrte_profile_reset.restype = None
    lib.vrte_debug_copy.argtypes = [P, ctypes.c_char_p, P, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_size_t)]
    lib.vrte_debug_copy.restype = ctypes.c_int
    lib.vrte_eigen_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
    lib.vrte_eigen_noalloc.restype = ctypes.c_int
    lib.vrte_gemm_sliced_workspace.argtypes = [ctypes.c_int] * 5
    lib.vrte_gemm_sliced_workspace.restype = ctypes.c_size_t
    I, LL = ctypes.c_int, ctypes.c_longlong
    lib.vrte_gemm_sliced.argtypes = [I, I, I, P, I, LL, P, I, LL, P, I, LL, I, I, P,
                                     ctypes.c_size_t, P, P]
    lib.vrte_gemm_sliced.restype = ctypes.c_int
    lib.vrte_workspace_bytes.argtypes = [P]
    lib.vrte_workspace_bytes.restype = ctypes.c_size_t
    lib.vrte_destroy.argtypes = [P]
    lib.vrte_destroy.restype = None
    lib.vrte_status_string.argtypes = [ctypes.c_int]
    lib.vrte_status_string.restype = ctypes.c_char_p
    lib.vrte_azimuth_mirrors.argtypes = [ctypes.c_int, P, P, P]
    lib.vrte_azimuth_mirrors.restype = ctypes.c_int
    for name in ["vrte_plan_create", "vrte_set_layer", "vrte_solve_brdf", "vrte_solve_brdf_host",
                 "vrte_solve_btdf", "vrte_solve_radiance", "vrte_solve_slab_brdf",
                 "vrte_brdf_backward", "vrte_plan_status"]:
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(code, where):
    if code != 0:
        raise VrteError(code, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Plan:
    """A solver plan (vrte_plan_create / vrte_set_layer / vrte_solve_brdf / vrte_destroy)."""

    def __init__(self, mu_in, mu_out, dphi, n_nodes_max, n_orders_max, n_coef_max,
                 n_layers_max=1, precision=VRTE_FP64, profile=False, adjoint=False,
                 transmission=False, slab=False):
        self.lib = load_library()
        self._mu_in = np.ascontiguousarray(mu_in, dtype=np.float64)
        self._mu_out = np.ascontiguousarray(mu_out, dtype=np.float64)
        self._phi = np.ascontiguousarray(dphi, dtype=np.float64)
        d = PlanDesc(int(n_nodes_max), int(n_orders_max), int(n_coef_max), int(n_layers_max),
                     self._mu_in.size, self._mu_out.size, self._phi.size, _dptr(self._mu_in),
                     _dptr(self._mu_out), _dptr(self._phi), int(precision),
                     (VRTE_FLAG_PROFILE if profile else 0) | (VRTE_FLAG_ADJOINT if adjoint else 0)
                     | (VRTE_FLAG_TRANSMISSION if transmission else 0)
                     | (VRTE_FLAG_SLAB if slab else 0))
        h = ctypes.c_void_p()
        _check(self.lib.vrte_plan_create(ctypes.byref(d), ctypes.byref(h)), "vrte_plan_create")
        self.handle = h
        self.n_coef_max = int(n_coef_max)
        self.n_layers = 0
        self._coeffs = None

    @property
    def table_shape(self):
        return (self.n_layers, self._mu_in.size, self._mu_out.size, self._phi.size, 4, 4)

    def set_layers(self, layers, d_coeffs):
        """layers: list of dict(tau, omega, n_interface, n_nodes, n_orders, n_coef[, base_albedo]
        [, base_mueller]) with base_mueller a 4x4 Mueller matrix of a reflecting base
        (row-major; the Lambertian base is base_albedo, R_00 = 2 rho);
        d_coeffs: CUDA float64 tensor [n_layers, n_coef_max, 6] (kept alive by the plan)."""
        arr = (Layer * len(layers))()
        for i, l in enumerate(layers):
            bm = l.get("base_mueller")
            bm = [0.0] * 16 if bm is None else [float(v) for v in np.asarray(bm, float).reshape(16)]
            arr[i] = Layer(float(l["tau"]), float(l["omega"]), float(l.get("n_interface", 1.0)),
                           int(l["n_nodes"]), int(l["n_orders"]), int(l["n_coef"]),
                           float(l.get("base_albedo", 0.0)), (ctypes.c_double * 16)(*bm))
        self._coeffs = d_coeffs
        _check(self.lib.vrte_set_layer(self.handle, len(layers), arr,
                                       ctypes.c_void_p(d_coeffs.data_ptr())), "vrte_set_layer")
        self.n_layers = len(layers)

    def solve(self, out, stream=None):
        """Writes the table into the CUDA tensor `out` (float32 or float64) on `stream`."""
        import torch
        dt = VRTE_OUT_F64 if out.dtype == torch.float64 else VRTE_OUT_F32
        _check(self.lib.vrte_solve_brdf(self.handle, ctypes.c_void_p(out.data_ptr()), dt,
                                        _stream_handle(stream)), "vrte_solve_brdf")
        return out

    def solve_btdf(self, out, stream=None):
        """Writes the transmission table (vrte_solve_btdf) into the CUDA tensor `out`."""
        import torch
        dt = VRTE_OUT_F64 if out.dtype == torch.float64 else VRTE_OUT_F32
        _check(self.lib.vrte_solve_btdf(self.handle, ctypes.c_void_p(out.data_ptr()), dt,
                                        _stream_handle(stream)), "vrte_solve_btdf")
        return out

    def solve_slab(self, out, stream=None):
        """Writes the BRDF table of the slab made of the set layers, top first
        (vrte_solve_slab_brdf), into the CUDA tensor `out` [n_in, n_out, n_phi, 4, 4]."""
        import torch
        dt = VRTE_OUT_F64 if out.dtype == torch.float64 else VRTE_OUT_F32
        _check(self.lib.vrte_solve_slab_brdf(self.handle, ctypes.c_void_p(out.data_ptr()), dt,
                                             _stream_handle(stream)), "vrte_solve_slab_brdf")
        return out

    def solve_radiance(self, taus, up=None, down=None, stream=None):
        """Radiance tables at depths `taus` (one per layer) into the CUDA tensors `up` and/or
        `down` (vrte_solve_radiance)."""
        import torch
        ref = up if up is not None else down
        dt = VRTE_OUT_F64 if ref.dtype == torch.float64 else VRTE_OUT_F32
        h = np.ascontiguousarray(taus, dtype=np.float64)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(self.lib.vrte_solve_radiance(self.handle, h.ctypes.data_as(ctypes.c_void_p),
                                            ptr(up), ptr(down), dt, _stream_handle(stream)),
               "vrte_solve_radiance")
        return up, down

    def solve_host(self, h_coeffs, h_out, stream=None):
        """Host-buffer solve (copies in, solves, copies out, synchronizes)."""
        import torch
        dt = VRTE_OUT_F64 if h_out.dtype == torch.float64 else VRTE_OUT_F32
        _check(self.lib.vrte_solve_brdf_host(self.handle, ctypes.c_void_p(h_coeffs.data_ptr()),
                                             ctypes.c_void_p(h_out.data_ptr()), dt,
                                             _stream_handle(stream)), "vrte_solve_brdf_host")
        return h_out

    def backward(self, grad_table, out=None, stream=None):
        """dL/d(omega, tau0, n, coefficients) for the table gradient `grad_table` (CUDA float32
        or float64, the table's shape) through vrte_brdf_backward: CUDA float64 tensor
        [n_layers, 3 + 6 n_coef_max]. Needs a plan created with adjoint=True."""
        import torch
        g = grad_table.contiguous()
        dt = VRTE_OUT_F64 if g.dtype == torch.float64 else VRTE_OUT_F32
        if out is None:
            out = torch.empty((self.n_layers, 3 + 6 * self.n_coef_max), dtype=torch.float64,
                              device=g.device)
        _check(self.lib.vrte_brdf_backward(self.handle, ctypes.c_void_p(g.data_ptr()), dt,
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "vrte_brdf_backward")
        return out

    def status(self):
        return self.lib.vrte_plan_status(self.handle)

    def stages(self):
        """Per-stage statistics since the last reset: list of dicts (synchronizes)."""
        arr = (StageStat * 32)()
        n = self.lib.vrte_profile_stages(self.handle, arr, 32)
        return [dict(name=arr[i].name.decode(), launches=int(arr[i].launches), ms=arr[i].ms,
                     flops=arr[i].flops, bytes=arr[i].bytes, tc_flops=arr[i].tc_flops)
                for i in range(max(n, 0))]

    def debug_buffer(self, name):
        """float64 copy of an internal buffer of the most recent order batch."""
        size = ctypes.c_size_t()
        _check(self.lib.vrte_debug_copy(self.handle, name.encode(), None, 0, ctypes.byref(size)),
               "vrte_debug_copy")
        out = np.empty(size.value // 8, dtype=np.float64)
        _check(self.lib.vrte_debug_copy(self.handle, name.encode(),
                                        out.ctypes.data_as(ctypes.c_void_p), size.value, None),
               "vrte_debug_copy")
        return out

    def reset_stages(self):
        self.lib.vrte_profile_reset(self.handle)

    def workspace_bytes(self):
        return int(self.lib.vrte_workspace_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.vrte_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def azimuth_mirrors(dphi):
    """vrte_azimuth_mirrors: (computed, mirror) index arrays of the azimuth pairing the
    tensor-core synthesis uses (mirror[r] = -1 where azimuth computed[r] has no partner)."""
    lib = load_library()
    phi = np.ascontiguousarray(dphi, dtype=np.float64)
    out = np.empty(2 * phi.size, dtype=np.int32)
    n_rep = ctypes.c_int()
    _check(lib.vrte_azimuth_mirrors(phi.size, phi.ctypes.data_as(ctypes.c_void_p),
                                    out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n_rep)),
           "vrte_azimuth_mirrors")
    r = n_rep.value
    return out[:r].copy(), out[phi.size:phi.size + r].copy()


def pack_coefficients(layers, n_coef_max=None):
    """[n_layers, n_coef_max, 6] float64 array from each layer's 'coef' [L, 6] (zero padded)."""
    if n_coef_max is None:
        n_coef_max = max(np.asarray(l["coef"]).shape[0] for l in layers)
    out = np.zeros((len(layers), n_coef_max, 6))
    for i, l in enumerate(layers):
        c = np.asarray(l["coef"], dtype=np.float64)
        out[i, :c.shape[0]] = c
    return out


def gemm_sliced(A, B, slices=4, stream=None):
    """C = A @ B (CUDA float64 tensors [batch, M, K] x [batch, K, N]) on the tensor cores
    through vrte_gemm_sliced (exact 7-bit slicing, relative accuracy ~2^(-7 slices))."""
    import torch
    lib = load_library()
    b, M, K = A.shape
    N = B.shape[2]
    A = A.contiguous()
    B = B.contiguous()
    C = torch.empty((b, M, N), dtype=torch.float64, device=A.device)
    nbytes = lib.vrte_gemm_sliced_workspace(M, N, K, b, slices)
    if nbytes == 0:
        raise VrteError(1, "vrte_gemm_sliced_workspace")
    work = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.vrte_gemm_sliced(M, N, K, ctypes.c_void_p(A.data_ptr()), K, M * K,
                                ctypes.c_void_p(B.data_ptr()), N, K * N,
                                ctypes.c_void_p(C.data_ptr()), N, M * N, b, slices,
                                ctypes.c_void_p(work.data_ptr()), nbytes,
                                ctypes.c_void_p(status.data_ptr()), _stream_handle(stream)),
           "vrte_gemm_sliced")
    return C, status


def brdf(layers, mu_in, mu_out, dphi, precision=VRTE_FP64, out_dtype=None, stream=None):
    """Solve the BRDF tables of `layers` on the current CUDA device.

    layers: list of dict(tau, omega, n_interface, n_nodes, n_orders, coef[L, 6]).
    Returns a CUDA tensor [n_layers, n_in, n_out, n_phi, 4, 4].
    """
    import torch
    if out_dtype is None:
        out_dtype = torch.float64
    coef = pack_coefficients(layers)
    d_coef = torch.from_numpy(coef).cuda()
    lay = [dict(l, n_coef=np.asarray(l["coef"]).shape[0]) for l in layers]
    plan = Plan(mu_in, mu_out, dphi, max(l["n_nodes"] for l in lay),
                max(l["n_orders"] for l in lay), coef.shape[1], len(lay), precision)
    try:
        plan.set_layers(lay, d_coef)
        out = torch.empty(plan.table_shape, dtype=out_dtype, device="cuda")
        plan.solve(out, stream)
        code = plan.status()
        _check(code, "solve status")
        return out
    finally:
        plan.close()


def _autograd_function():
    import torch

    class BRDFFunction(torch.autograd.Function):
        """The BRDF table as a differentiable function of the layer parameters: forward is
        vrte_solve_brdf, backward is vrte_brdf_backward (argument marshalling only)."""

        @staticmethod
        def forward(ctx, params, coeffs, plan, sizes, out_dtype):
            # params [n_layers, 3] = (omega, tau0, n_interface); coeffs [n_layers, L, 6]
            host = params.detach().double().cpu().tolist()
            layers = [dict(omega=h[0], tau=h[1], n_interface=h[2], n_nodes=sz[0],
                           n_orders=sz[1], n_coef=sz[2]) for h, sz in zip(host, sizes)]
            d_coef = coeffs.detach().double().contiguous()
            plan.set_layers(layers, d_coef)
            out = torch.empty(plan.table_shape, dtype=out_dtype, device=d_coef.device)
            plan.solve(out)
            _check(plan.status(), "vrte_solve_brdf status")
            ctx.plan, ctx.layers, ctx.d_coef = plan, layers, d_coef
            ctx.params_dtype, ctx.params_device = params.dtype, params.device
            return out

        @staticmethod
        def backward(ctx, grad_out):
            plan = ctx.plan
            plan.set_layers(ctx.layers, ctx.d_coef)
            g = plan.backward(grad_out.contiguous())
            _check(plan.status(), "vrte_brdf_backward status")
            n_layers = len(ctx.layers)
            gp = g[:, :3].to(ctx.params_device, ctx.params_dtype)
            gc = g[:, 3:].reshape(n_layers, -1, 6)
            return gp, gc, None, None, None

    return BRDFFunction


def brdf_autograd(params, coeffs, sizes, plan, out_dtype=None):
    """Differentiable BRDF table [n_layers, n_in, n_out, n_phi, 4, 4] of the layers described
    by params [n_layers, 3] = (omega, tau0, n_interface) and coeffs (CUDA float64
    [n_layers, n_coef_max, 6]); sizes: per layer (n_nodes, n_orders, n_coef); plan: a Plan
    created with adjoint=True for these grids. Gradients flow to params and coeffs through
    torch.autograd (vrte_brdf_backward)."""
    import torch
    if out_dtype is None:
        out_dtype = torch.float64
    return _autograd_function().apply(params, coeffs, plan, [tuple(int(v) for v in z) for z in sizes],
                                      out_dtype)
