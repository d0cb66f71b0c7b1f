"""GB300-native mixed-precision covariance factorisation for spherical-harmonic
climate emulators (arXiv 2408.04440): Python binding of ``libemucov``.

This module only marshals arguments into the C ABI declared in
``include/emucov.h`` (same function names); every step of the computation runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.
Importing works without a GPU; calling anything that needs the library fails
loudly if ``libemucov.so`` has not been built (``build.build()``).
"""
from __future__ import annotations

import ctypes
import weakref
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libemucov.so")

EMU_OK, EMU_EINVAL, EMU_ENOMEM, EMU_ENOTPD, EMU_ENOCONV, EMU_ETIMEOUT, EMU_ECUDA, EMU_ESTATE = range(8)
STATUS_NAMES = {0: "EMU_OK", 1: "EMU_EINVAL", 2: "EMU_ENOMEM", 3: "EMU_ENOTPD", 4: "EMU_ENOCONV",
                5: "EMU_ETIMEOUT", 6: "EMU_ECUDA", 7: "EMU_ESTATE"}
CLASS_FP64, CLASS_FP32, CLASS_TF32, CLASS_BF16, CLASS_E4M3 = range(5)
NCLASS = 5
CLASS_NAMES = ("fp64", "fp32", "tf32", "bf16", "e4m3")
# u[c] <= 0 asks the library for its default unit roundoff of class c
DEFAULT_U = (0.0,) * 5
# precision maps: the norm rule, or the paper's band variants (DP/SP, DP/SP/HP, DP/HP)
MAP_NORM, MAP_DP_SP, MAP_DP_SP_HP, MAP_DP_HP = range(4)
MAP_NAMES = ("norm", "dp_sp", "dp_sp_hp", "dp_hp")

# Every symbol the header declares (checked by the CPU test suite).
EXPORTED = (
    "emu_create", "emu_destroy", "emu_set_stream", "emu_status_str", "emu_last_error",
    "emu_launch_count", "emu_host_launch_count", "emu_prof_enable", "emu_prof_read", "emu_prof_timeline", "emu_trace_enable", "emu_trace_read", "emu_potrf_task_list", "emu_test_wait_hook", "emu_schedule", "emu_schedule_info", "emu_measure_alu_peaks", "emu_cov_build", "emu_mat_import",
    "emu_mat_import_host", "emu_cov_from_residuals", "emu_var_recursion", "emu_isht", "emu_sht", "emu_emulate_grid", "emu_cov_build_classfmt",
    "emu_backward_error_est", "emu_mat_clone", "emu_mat_export", "emu_mat_tile_info", "emu_mat_shape",
    "emu_mat_free", "emu_potrf_mp", "emu_sample", "emu_sample_host", "emu_potrs", "emu_solve_refine",
    "emu_batch_potrf_sample", "emu_batch_release", "emu_cov_build_dense_noalloc",
)
PROF_GROUPS = ("cov", "map", "potrf", "trsm64", "trsm32", "update64", "tc_factor", "tc_sample", "trmm64",
               "rng", "split", "solve")


class EmuError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class emu_cov_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("beta", ctypes.c_double), ("sigma_exp", ctypes.c_double),
                ("nugget_rel", ctypes.c_double)]


class emu_trend(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("tau", ctypes.c_double), ("beta0", ctypes.c_void_p),
                ("beta1", ctypes.c_void_p), ("beta2", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("nyears", ctypes.c_int)]


class emu_mp_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("prec_mask", ctypes.c_uint), ("diag_fp64", ctypes.c_int),
                ("u", ctypes.c_double * NCLASS), ("band", ctypes.c_int), ("sp_frac", ctypes.c_double)]


class emu_factor_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nb", ctypes.c_int), ("nt", ctypes.c_int), ("pivot", ctypes.c_int),
                ("tiles", ctypes.c_int * NCLASS), ("update_flops", ctypes.c_double * NCLASS),
                ("frob", ctypes.c_double), ("ms", ctypes.c_double)]


class emu_refine_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double), ("ms", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libemucov.so; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2408_04440_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, lg, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    st = ctypes.c_int
    L.emu_create.argtypes = [ctypes.POINTER(vp), i, vp]
    L.emu_destroy.argtypes = [vp]
    L.emu_set_stream.argtypes = [vp, vp]
    L.emu_status_str.argtypes = [st]
    L.emu_status_str.restype = ctypes.c_char_p
    L.emu_last_error.argtypes = [vp]
    L.emu_last_error.restype = ctypes.c_char_p
    L.emu_launch_count.argtypes = [vp]
    L.emu_launch_count.restype = ctypes.c_uint64
    L.emu_host_launch_count.argtypes = [vp]
    L.emu_host_launch_count.restype = ctypes.c_uint64
    dpp = ctypes.POINTER(ctypes.c_double)
    L.emu_prof_enable.argtypes = [vp, i]
    L.emu_trace_enable.argtypes = [vp, i]
    L.emu_test_wait_hook.argtypes = [vp, ctypes.c_longlong, i]
    L.emu_schedule.argtypes = [vp, i, i]
    L.emu_measure_alu_peaks.argtypes = [vp, dpp, dpp]
    L.emu_schedule_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.emu_prof_timeline.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.emu_trace_read.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.emu_prof_read.argtypes = [vp, i, ctypes.POINTER(i), dpp, dpp, dpp, dpp]
    L.emu_cov_build.argtypes = [vp, ctypes.POINTER(emu_cov_params), i, ctypes.POINTER(vp)]
    L.emu_mat_import_host.argtypes = [vp, vp, i, lg, i, ctypes.POINTER(vp)]
    L.emu_mat_import.argtypes = [vp, vp, i, lg, i, ctypes.POINTER(vp)]
    L.emu_cov_from_residuals.argtypes = [vp, vp, i, lg, lg, ctypes.c_double, i, ctypes.POINTER(vp)]
    L.emu_var_recursion.argtypes = [vp, vp, i, i, lg, vp, i, vp, lg]
    L.emu_isht.argtypes = [vp, vp, i, i, lg, i, i, vp, lg]
    L.emu_sht.argtypes = [vp, vp, i, i, i, lg, i, vp, lg]
    L.emu_cov_build_classfmt.argtypes = [vp, ctypes.POINTER(emu_cov_params), i, ctypes.POINTER(emu_mp_opts),
                                         ctypes.POINTER(vp)]
    L.emu_backward_error_est.argtypes = [vp, vp, ctypes.POINTER(emu_cov_params), i, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_double)]
    L.emu_emulate_grid.argtypes = [vp, vp, lg, i, lg, ctypes.POINTER(emu_trend), vp, vp, ctypes.c_uint64,
                                   ctypes.c_uint32, vp, lg]
    L.emu_potrf_task_list.argtypes = [i, i, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.emu_mat_clone.argtypes = [vp, vp, ctypes.POINTER(vp)]
    L.emu_mat_export.argtypes = [vp, vp, vp, lg]
    L.emu_mat_tile_info.argtypes = [vp, vp, vp, vp]
    L.emu_mat_shape.argtypes = [vp] + [ctypes.POINTER(i)] * 4
    L.emu_mat_free.argtypes = [vp]
    L.emu_potrf_mp.argtypes = [vp, vp, ctypes.POINTER(emu_mp_opts), ctypes.POINTER(emu_factor_info)]
    L.emu_sample.argtypes = [vp, vp, i, ctypes.c_uint64, ctypes.c_uint32, vp, lg, vp]
    L.emu_sample_host.argtypes = [vp, vp, i, ctypes.c_uint64, ctypes.c_uint32, vp, lg]
    L.emu_potrs.argtypes = [vp, vp, vp, lg, vp, lg, i]
    L.emu_solve_refine.argtypes = [vp, vp, vp, vp, lg, vp, lg, i, d, i, ctypes.POINTER(emu_refine_info)]
    L.emu_cov_build_dense_noalloc.argtypes = [i, d, d, d, vp, lg, vp]
    L.emu_batch_potrf_sample.argtypes = [vp, i, ctypes.POINTER(emu_cov_params), i, ctypes.POINTER(emu_mp_opts), i,
                                         ctypes.c_uint64, vp, vp, ctypes.POINTER(emu_factor_info)]
    L.emu_batch_release.argtypes = [vp]
    for name in ("emu_create", "emu_destroy", "emu_set_stream", "emu_prof_enable", "emu_prof_read",
                 "emu_trace_enable", "emu_trace_read", "emu_potrf_task_list", "emu_prof_timeline",
                 "emu_test_wait_hook",
                 "emu_schedule", "emu_schedule_info", "emu_measure_alu_peaks",
                 "emu_mat_import_host", "emu_cov_build", "emu_mat_import", "emu_emulate_grid",
                 "emu_cov_build_classfmt", "emu_backward_error_est",
                 "emu_mat_clone", "emu_mat_export", "emu_mat_tile_info", "emu_mat_shape", "emu_mat_free",
                 "emu_potrf_mp", "emu_sample", "emu_sample_host", "emu_potrs", "emu_solve_refine",
                 "emu_cov_build_dense_noalloc", "emu_batch_potrf_sample", "emu_batch_release"):
        getattr(L, name).restype = st
    _lib = L
    return L


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _colmajor_empty(rows: int, cols: int, device):
    """(rows x cols) FP64 tensor whose storage is column-major with ld = rows."""
    import torch

    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.lib = load()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        h = ctypes.c_void_p()
        self._check(self.lib.emu_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)),
                    "emu_create", with_ctx=False)
        self.h = h
        # matrices still alive: a matrix must be freed before its context
        self._mats = weakref.WeakSet()

    def _check(self, status: int, where: str, with_ctx: bool = True):
        if status != EMU_OK:
            detail = ""
            if with_ctx and getattr(self, "h", None):
                detail = (self.lib.emu_last_error(self.h) or b"").decode()
            raise EmuError(status, where, detail)

    @property
    def launch_count(self) -> int:
        return int(self.lib.emu_launch_count(self.h))

    @property
    def host_launch_count(self) -> int:
        return int(self.lib.emu_host_launch_count(self.h))

    def prof_enable(self, on: bool = True):
        self._check(self.lib.emu_prof_enable(self.h, int(on)), "emu_prof_enable")

    def prof_read(self) -> dict:
        """Per kernel group: launches, total ms, algorithmic flops/bytes, tensor-core flops."""
        out = {}
        for g, name in enumerate(PROF_GROUPS):
            n = ctypes.c_int()
            ms, fl, by, mm = (ctypes.c_double() for _ in range(4))
            self._check(self.lib.emu_prof_read(self.h, g, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                               ctypes.byref(by), ctypes.byref(mm)), "emu_prof_read")
            out[name] = {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value,
                         "mma_flops": mm.value}
        return out

    def prof_timeline(self):
        """(N, 4) array: group index, stream (0 ctx, 1 critical, 2 panel, 3 bulk), start ms, end ms."""
        n = ctypes.c_size_t()
        self._check(self.lib.emu_prof_timeline(self.h, None, 0, ctypes.byref(n)), "emu_prof_timeline")
        out = np.zeros((n.value, 4), dtype=np.float64)
        if n.value:
            self._check(self.lib.emu_prof_timeline(self.h, ctypes.c_void_p(out.ctypes.data), n.value,
                                                   ctypes.byref(n)), "emu_prof_timeline")
        return out

    def alu_peaks(self):
        """(FP64, FP32) FMA rates of the device in TFLOP/s, measured with FMA loops."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.emu_measure_alu_peaks(self.h, ctypes.byref(a), ctypes.byref(b)), "emu_measure_alu_peaks")
        return a.value, b.value

    def schedule(self, graphs: bool = True, tuning: bool = True):
        """Graph replay and reserved-SM tuning of the single-matrix mixed factor (both on by default)."""
        self._check(self.lib.emu_schedule(self.h, int(graphs), int(tuning)), "emu_schedule")

    def schedule_info(self):
        """(choices timed, SMs left free, SMs left free near FP64-class panel work) of the tuner."""
        t, r, r64 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.emu_schedule_info(self.h, ctypes.byref(t), ctypes.byref(r), ctypes.byref(r64)),
                    "emu_schedule_info")
        return t.value, r.value, r64.value

    def test_wait_hook(self, wait_cycles: int = 0, withhold_index: int = -1):
        """Bound of the diagonal POTRF's flag waits (cycles, 0 = default) and one flag index they never see set."""
        self._check(self.lib.emu_test_wait_hook(self.h, int(wait_cycles), int(withhold_index)), "emu_test_wait_hook")

    def trace_enable(self, on: bool = True):
        self._check(self.lib.emu_trace_enable(self.h, int(on)), "emu_trace_enable")

    def trace_read(self):
        """Task records of the dataflow POTRF: numpy (N, 5) uint64 array."""
        n = ctypes.c_size_t()
        self._check(self.lib.emu_trace_read(self.h, None, 0, ctypes.byref(n)), "emu_trace_read")
        out = np.zeros((n.value, 5), dtype=np.uint64)
        if n.value:
            self._check(self.lib.emu_trace_read(self.h, ctypes.c_void_p(out.ctypes.data), n.value, ctypes.byref(n)),
                        "emu_trace_read")
        return out

    def close(self):
        if getattr(self, "h", None):
            for m in list(self._mats):
                m.free()
            self.lib.emu_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mat:
    """A tiled matrix owned by the library (covariance or factor)."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p):
        self.ctx = ctx
        self.h = handle
        ctx._mats.add(self)

    def shape_info(self):
        n, nb, nt, st = (ctypes.c_int() for _ in range(4))
        self.ctx._check(self.ctx.lib.emu_mat_shape(self.h, ctypes.byref(n), ctypes.byref(nb), ctypes.byref(nt),
                                                   ctypes.byref(st)), "emu_mat_shape")
        return n.value, nb.value, nt.value, st.value

    @property
    def n(self):
        return self.shape_info()[0]

    def free(self):
        # after the context is closed its matrices are already freed
        if self.h and getattr(self.ctx, "h", None):
            self.ctx.lib.emu_mat_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def emu_cov_build(ctx: Context, L: int, beta: float, nb: int, sigma_exp: float = 1.5,
                  nugget_rel: float = 1e-8) -> Mat:
    p = emu_cov_params(L, beta, sigma_exp, nugget_rel)
    h = ctypes.c_void_p()
    ctx._check(ctx.lib.emu_cov_build(ctx.h, ctypes.byref(p), nb, ctypes.byref(h)), "emu_cov_build")
    return Mat(ctx, h)


def emu_cov_build_classfmt(ctx: Context, L: int, beta: float, nb: int, eps: float = 1e-6, prec_mask: int = 0b11011,
                           band: int = MAP_NORM, sigma_exp: float = 1.5, nugget_rel: float = 1e-8, u=None,
                           sp_frac: float = 0.0) -> Mat:
    """The covariance stored tile by tile in the format of its precision class (map of the norm rule at eps, or
    a band map); factor it with emu_potrf_mp."""
    p = emu_cov_params(L, beta, sigma_exp, nugget_rel)
    o = mp_opts(eps, prec_mask, True, u, band, sp_frac)
    h = ctypes.c_void_p()
    ctx._check(ctx.lib.emu_cov_build_classfmt(ctx.h, ctypes.byref(p), nb, ctypes.byref(o), ctypes.byref(h)),
               "emu_cov_build_classfmt")
    return Mat(ctx, h)


def emu_backward_error_est(ctx: Context, A: Mat, L: int, beta: float, nprobes: int = 32, seed: int = 0,
                           sigma_exp: float = 1.5, nugget_rel: float = 1e-8) -> float:
    """Hutchinson estimate of ||A A^T - S||_F / ||S||_F for the factor A of the covariance (L, beta, ...)."""
    p = emu_cov_params(L, beta, sigma_exp, nugget_rel)
    est = ctypes.c_double()
    ctx._check(ctx.lib.emu_backward_error_est(ctx.h, A.h, ctypes.byref(p), nprobes, seed, ctypes.byref(est)),
               "emu_backward_error_est")
    return est.value


def emu_mat_import(ctx: Context, A, nb: int) -> Mat:
    """A: (n x n) float64 CUDA tensor; its lower triangle is read."""
    n = A.shape[0]
    if A.stride() != (1, n):
        A = A.t().contiguous().t()  # column-major storage
    h = ctypes.c_void_p()
    ctx._check(ctx.lib.emu_mat_import(ctx.h, ctypes.c_void_p(_ptr(A)), n, n, nb, ctypes.byref(h)),
               "emu_mat_import")
    m = Mat(ctx, h)
    m._keep = A
    return m


def emu_cov_from_residuals(ctx: Context, Xi, nb: int = 256, nugget_rel=None, raise_on_error: bool = True):
    """Empirical covariance U = Xi Xi^T / m (+ nugget_rel * max diag on the
    diagonal) of the m columns of Xi, an (n x m) float64 CUDA tensor.  By
    default the perturbation is 1e-8 when m < n (fewer residuals than
    coefficients, as the paper does) and 0 otherwise.  Returns (Mat, status)."""
    n, m = Xi.shape
    if Xi.stride(0) != 1:
        Xi = Xi.t().contiguous().t()  # column-major storage
    ld = Xi.stride(1) if m > 1 else n
    if nugget_rel is None:
        nugget_rel = 1e-8 if m < n else 0.0
    h = ctypes.c_void_p()
    st = ctx.lib.emu_cov_from_residuals(ctx.h, ctypes.c_void_p(_ptr(Xi)), n, m, ld, float(nugget_rel), nb,
                                        ctypes.byref(h))
    if st != EMU_OK:
        if raise_on_error:
            ctx._check(st, "emu_cov_from_residuals")
        return None, st
    return Mat(ctx, h), st


def emu_var_recursion(ctx: Context, Xi, Phi):
    """f_t = sum_p Phi[:, p-1] * f_{t-p} + Xi[:, t] (f before t = 0 zero): Xi (n x T),
    Phi (n x P) float64 CUDA tensors; returns F (n x T, column-major)."""
    n, T = Xi.shape
    Xi = Xi if Xi.stride(0) == 1 else Xi.t().contiguous().t()
    P = 0 if Phi is None else Phi.shape[1]
    if P:
        Phi = Phi if Phi.stride(0) == 1 and Phi.stride(1) == n else Phi.t().contiguous().t()
    F = _colmajor_empty(n, T, ctx.device)
    ctx._check(ctx.lib.emu_var_recursion(ctx.h, ctypes.c_void_p(_ptr(Xi)), n, T, Xi.stride(1) if T > 1 else n,
                                         ctypes.c_void_p(_ptr(Phi)) if P else None, P, ctypes.c_void_p(_ptr(F)), n),
               "emu_var_recursion")
    return F


def emu_isht(ctx: Context, F, L: int, ntheta: int, nphi: int):
    """Inverse SHT of each column of F (L^2 x T) to an (ntheta x nphi) grid per
    time step: returns Z as a (ntheta*nphi x T) column-major tensor, grid point
    (i, j) at row i + j*ntheta."""
    n, T = F.shape
    F = F if F.stride(0) == 1 else F.t().contiguous().t()
    Z = _colmajor_empty(ntheta * nphi, T, ctx.device)
    ctx._check(ctx.lib.emu_isht(ctx.h, ctypes.c_void_p(_ptr(F)), L, T, F.stride(1) if T > 1 else n, ntheta, nphi,
                                ctypes.c_void_p(_ptr(Z)), ntheta * nphi), "emu_isht")
    return Z


def emu_sht(ctx: Context, Z, L: int, ntheta: int, nphi: int):
    """Forward SHT of each column of Z ((ntheta*nphi) x T, grid point (i, j) at row
    i + j*ntheta) to real-form coefficients: returns F (L^2 x T, column-major)."""
    npts, T = Z.shape
    Z = Z if Z.stride(0) == 1 else Z.t().contiguous().t()
    F = _colmajor_empty(L * L, T, ctx.device)
    ctx._check(ctx.lib.emu_sht(ctx.h, ctypes.c_void_p(_ptr(Z)), ntheta, nphi, T, Z.stride(1) if T > 1 else npts, L,
                               ctypes.c_void_p(_ptr(F)), L * L), "emu_sht")
    return F


def emu_emulate_grid(ctx: Context, Zs, tau: float, beta0, beta1, beta2, rho, A, B, x, sigma, v, seed: int,
                     stream_id: int = 0, out=None):
    """Emulations y_t = m_t + sigma (Zs_t + v e_t), t = 1..T (Eq. decouple): Zs (G x T) from emu_isht,
    per-point beta0/beta1/beta2/rho/sigma/v (G), harmonic amplitudes A, B (K x G, or None), forcing x[0..Y];
    all float64 CUDA tensors.  Returns Y (G x T, column-major)."""
    G, T = Zs.shape
    Zs = Zs if Zs.stride(0) == 1 else Zs.t().contiguous().t()
    K = 0 if A is None else A.shape[0]
    vecs = [q.contiguous() for q in (beta0, beta1, beta2, rho, sigma, v, x)]
    AB = [q.t().contiguous() for q in (A, B)] if K else [None, None]  # amplitude k of point g at [k + g K]
    m = emu_trend(K, tau, _ptr(vecs[0]), _ptr(vecs[1]), _ptr(vecs[2]), _ptr(vecs[3]),
                  _ptr(AB[0]) if K else None, _ptr(AB[1]) if K else None, _ptr(vecs[6]), x.numel() - 1)
    Y = _colmajor_empty(G, T, ctx.device) if out is None else out
    ctx._check(ctx.lib.emu_emulate_grid(ctx.h, ctypes.c_void_p(_ptr(Zs)), G, T, Zs.stride(1) if T > 1 else G,
                                        ctypes.byref(m), ctypes.c_void_p(_ptr(vecs[4])),
                                        ctypes.c_void_p(_ptr(vecs[5])), seed, stream_id,
                                        ctypes.c_void_p(_ptr(Y)), Y.stride(1) if T > 1 else G),
               "emu_emulate_grid")
    return Y


def emu_mat_import_host(ctx: Context, A, nb: int) -> Mat:
    """A: (n x n) float64 host array (numpy or CPU tensor, ideally pinned), Fortran
    (column-major) storage; its lower triangle is copied and read."""
    import torch

    if isinstance(A, torch.Tensor):
        n = A.shape[0]
        if A.stride() != (1, n):
            raise ValueError("host matrix must be column-major (stride (1, n))")
        ptr = A.data_ptr()
    else:
        if not A.flags.f_contiguous:
            raise ValueError("host matrix must be Fortran-ordered")
        n = A.shape[0]
        ptr = A.ctypes.data
    h = ctypes.c_void_p()
    ctx._check(ctx.lib.emu_mat_import_host(ctx.h, ctypes.c_void_p(ptr), n, n, nb, ctypes.byref(h)),
               "emu_mat_import_host")
    return Mat(ctx, h)


def emu_mat_clone(ctx: Context, A: Mat) -> Mat:
    h = ctypes.c_void_p()
    ctx._check(ctx.lib.emu_mat_clone(ctx.h, A.h, ctypes.byref(h)), "emu_mat_clone")
    return Mat(ctx, h)


def emu_mat_export(ctx: Context, A: Mat, out=None):
    n = A.n
    if out is None:
        out = _colmajor_empty(n, n, ctx.device)
    ctx._check(ctx.lib.emu_mat_export(ctx.h, A.h, ctypes.c_void_p(_ptr(out)), out.stride(1)), "emu_mat_export")
    return out


def emu_potrf_task_list(nb: int, single_tile: int = 1) -> np.ndarray:
    """Task list of the dataflow POTRF of one nb x nb diagonal tile, rows
    (kind, r, c, s) in fetch order (host only; see emucov.h): single_tile 1
    (chain on one CTA), 2 (chain on a cluster of three CTAs) or 0 (batch)."""
    L = load()
    n = ctypes.c_size_t(0)
    st = L.emu_potrf_task_list(int(nb), int(single_tile), None, 0, ctypes.byref(n))
    if st != 0:
        raise EmuError(st, "emu_potrf_task_list")
    out = np.zeros((n.value, 4), dtype=np.int16)
    st = L.emu_potrf_task_list(int(nb), int(single_tile), out.ctypes.data, n.value, ctypes.byref(n))
    if st != 0:
        raise EmuError(st, "emu_potrf_task_list")
    return out


def emu_mat_tile_info(ctx: Context, A: Mat):
    nt = A.shape_info()[2]
    cls = np.zeros((nt, nt), dtype=np.uint8, order="F")
    tn = np.zeros((nt, nt), dtype=np.float64, order="F")
    ctx._check(ctx.lib.emu_mat_tile_info(ctx.h, A.h, ctypes.c_void_p(cls.ctypes.data),
                                         ctypes.c_void_p(tn.ctypes.data)), "emu_mat_tile_info")
    return cls, tn


@dataclass
class FactorInfo:
    status: int
    n: int
    nb: int
    nt: int
    pivot: int
    tiles: list = field(default_factory=list)
    update_flops: list = field(default_factory=list)
    frob: float = 0.0
    ms: float = 0.0


def mp_opts(eps: float = 0.0, prec_mask: int = 0b01011, diag_fp64: bool = False, u=None, band: int = MAP_NORM,
            sp_frac: float = 0.0) -> emu_mp_opts:
    uu = (ctypes.c_double * NCLASS)(*(u if u is not None else DEFAULT_U))
    return emu_mp_opts(eps, prec_mask, int(diag_fp64), uu, int(band), float(sp_frac))


def emu_potrf_mp(ctx: Context, A: Mat, eps: float = 0.0, prec_mask: int = 0b01011, diag_fp64: bool = False,
                 u=None, raise_on_error: bool = True, band: int = MAP_NORM, sp_frac: float = 0.0) -> FactorInfo:
    """band = MAP_NORM: eps <= 0 plain FP64, eps > 0 the norm rule; MAP_DP_SP / MAP_DP_SP_HP / MAP_DP_HP: the
    band maps (sp_frac 0 means 0.05)."""
    o = mp_opts(eps, prec_mask, diag_fp64, u, band, sp_frac)
    info = emu_factor_info()
    s = ctx.lib.emu_potrf_mp(ctx.h, A.h, ctypes.byref(o), ctypes.byref(info))
    fi = FactorInfo(s, info.n, info.nb, info.nt, info.pivot, list(info.tiles), list(info.update_flops),
                    info.frob, info.ms)
    if raise_on_error and s != EMU_OK:
        ctx._check(s, "emu_potrf_mp")
    return fi


def emu_sample(ctx: Context, L: Mat, nsamples: int, seed: int, stream_id: int = 0, out=None,
               return_z: bool = False):
    n = L.n
    if out is None:
        out = _colmajor_empty(n, nsamples, ctx.device)
    Z = _colmajor_empty(n, nsamples, ctx.device) if return_z else None
    ld = out.stride(1)
    if Z is not None and Z.stride(1) != ld:
        raise ValueError("Y and Z must share a leading dimension")
    ctx._check(ctx.lib.emu_sample(ctx.h, L.h, nsamples, seed, stream_id, ctypes.c_void_p(_ptr(out)), ld,
                                  ctypes.c_void_p(_ptr(Z))), "emu_sample")
    return (out, Z) if return_z else out


def emu_sample_host(ctx: Context, L: Mat, nsamples: int, seed: int, stream_id: int = 0, out=None):
    """Samples into a host buffer: out is a float64 (n x s) column-major numpy array
    or CPU tensor (pinned memory gives full copy bandwidth)."""
    n = L.n
    if out is None:
        out = np.empty((n, nsamples), dtype=np.float64, order="F")
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    ctx._check(ctx.lib.emu_sample_host(ctx.h, L.h, nsamples, seed, stream_id, ctypes.c_void_p(ptr), n),
               "emu_sample_host")
    return out


def emu_potrs(ctx: Context, L: Mat, B, out=None):
    n, r = B.shape
    if B.stride() != (1, n):
        B = B.t().contiguous().t()
    if out is None:
        out = _colmajor_empty(n, r, ctx.device)
    ctx._check(ctx.lib.emu_potrs(ctx.h, L.h, ctypes.c_void_p(_ptr(B)), n, ctypes.c_void_p(_ptr(out)),
                                 out.stride(1), r), "emu_potrs")
    return out


@dataclass
class RefineInfo:
    status: int
    iters: int
    rel_resid: float
    ms: float


def emu_solve_refine(ctx: Context, L: Mat, S: Mat, B, tol: float = 1e-14, maxit: int = 50, out=None,
                     raise_on_error: bool = True):
    n, r = B.shape
    if B.stride() != (1, n):
        B = B.t().contiguous().t()
    if out is None:
        out = _colmajor_empty(n, r, ctx.device)
    info = emu_refine_info()
    s = ctx.lib.emu_solve_refine(ctx.h, L.h, S.h, ctypes.c_void_p(_ptr(B)), n, ctypes.c_void_p(_ptr(out)),
                                 out.stride(1), r, tol, maxit, ctypes.byref(info))
    ri = RefineInfo(s, info.iters, info.rel_resid, info.ms)
    if raise_on_error and s != EMU_OK:
        ctx._check(s, "emu_solve_refine")
    return out, ri


def emu_batch_potrf_sample(ctx: Context, params, nb: int = 256, eps: float = 0.0, prec_mask: int = 0b01011,
                           diag_fp64: bool = False, u=None, nsamples: int = 0, seed: int = 0, want_L: bool = False,
                           raise_on_error: bool = True, out_Y=None, band: int = MAP_NORM, sp_frac: float = 0.0):
    """params: sequence of (L, beta) or (L, beta, sigma_exp, nugget_rel).
    Returns (Ys, Ls, infos, status): lists of column-major CUDA tensors
    (n_b x nsamples and n_b x n_b; None where not asked) and FactorInfo.
    out_Y: optional list of preallocated Y_b (column-major, ld n_b)."""
    count = len(params)
    P = (emu_cov_params * count)()
    for b, q in enumerate(params):
        sexp = float(q[2]) if len(q) > 2 else 1.5
        nug = float(q[3]) if len(q) > 3 else 1e-8
        P[b] = emu_cov_params(int(q[0]), float(q[1]), sexp, nug)
    Ys = None
    if nsamples > 0:
        Ys = out_Y if out_Y is not None else [_colmajor_empty(int(q[0]) ** 2, nsamples, ctx.device) for q in params]
    Ls = [_colmajor_empty(int(q[0]) ** 2, int(q[0]) ** 2, ctx.device) for q in params] if want_L else None
    yp = (ctypes.c_void_p * count)(*[_ptr(t) for t in Ys]) if Ys else None
    lp = (ctypes.c_void_p * count)(*[_ptr(t) for t in Ls]) if Ls else None
    o = mp_opts(eps, prec_mask, diag_fp64, u, band, sp_frac)
    infos = (emu_factor_info * count)()
    s = ctx.lib.emu_batch_potrf_sample(ctx.h, count, P, nb, ctypes.byref(o), nsamples, seed,
                                       ctypes.cast(yp, ctypes.c_void_p) if yp else None,
                                       ctypes.cast(lp, ctypes.c_void_p) if lp else None, infos)
    fis = [FactorInfo(s, f.n, f.nb, f.nt, f.pivot, list(f.tiles), list(f.update_flops), f.frob, f.ms)
           for f in infos]
    if raise_on_error and s != EMU_OK:
        ctx._check(s, "emu_batch_potrf_sample")
    return Ys, Ls, fis, s


def emu_batch_release(ctx: Context):
    ctx._check(ctx.lib.emu_batch_release(ctx.h), "emu_batch_release")
