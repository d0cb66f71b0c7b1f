"""Plain CPU FP64 oracle for the covariance factor / sampling path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  The arithmetic lives in ``emu_oracle.c`` (plain loops, FP64); this module
compiles it with gcc on first use and exposes numpy-friendly wrappers.

Every matrix is a Fortran-ordered (column-major) float64 numpy array.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emu_oracle.c")
_HDR = os.path.join(_HERE, "emu_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Unit roundoff of each precision class, most precise first:
# FP64, FP32 (computed on tensor cores as split TF32), TF32, BF16, FP8-E4M3.
CLASS_NAMES = ("fp64", "fp32", "tf32", "bf16", "e4m3")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i, lg, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
    L.orc_lm_of_index.argtypes = [lg, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.orc_cov_build.argtypes = [i, d, d, d, dp, lg]
    L.orc_cov_rows.argtypes = [i, d, d, d, ctypes.POINTER(lg), i, dp]
    L.orc_tile_norms.argtypes = [i, dp, lg, i, dp]
    L.orc_frob_from_tiles.argtypes = [i, dp]
    L.orc_frob_from_tiles.restype = d
    L.orc_precision_map.argtypes = [i, dp, d, dp, i, ctypes.c_uint, i, u8p]
    L.orc_precision_map_band.argtypes = [i, i, d, u8p]
    L.orc_cov_from_residuals.argtypes = [i, lg, dp, lg, d, dp]
    L.orc_var_recursion.argtypes = [i, i, dp, lg, dp, i, dp, lg]
    L.orc_mean_trend.argtypes = [lg, d, d, d, d, d, i, dp, dp, dp]
    L.orc_mean_trend.restype = d
    L.orc_emulate_grid.argtypes = [lg, i, dp, lg, dp, lg, i, d, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, lg]
    L.orc_real_sh.argtypes = [i, i, d, d]
    L.orc_real_sh.restype = d
    L.orc_isht.argtypes = [i, i, dp, lg, i, i, dp, lg]
    L.orc_sht.argtypes = [i, i, dp, lg, i, i, dp, lg]
    L.orc_I_pub.argtypes = [i, dp, dp]
    L.orc_precision_map_band.restype = i
    L.orc_potrf_unblocked.argtypes = [i, dp, lg]
    L.orc_potrf_unblocked.restype = i
    L.orc_potrf_blocked.argtypes = [i, i, dp, lg, i]
    L.orc_potrf_blocked.restype = i
    L.orc_potrf_blocked_steps.argtypes = [i, i, dp, lg, i, i]
    L.orc_potrf_blocked_steps.restype = i
    L.orc_trmm_lower.argtypes = [i, i, dp, lg, dp, lg, dp, lg]
    L.orc_potrs.argtypes = [i, i, dp, lg, dp, lg, dp, lg]
    L.orc_logdet_chol.argtypes = [i, dp, lg]
    L.orc_logdet_chol.restype = d
    L.orc_backward_error.argtypes = [i, dp, lg, dp, lg]
    L.orc_backward_error.restype = d
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_normal_matrix.argtypes = [ctypes.c_uint64, ctypes.c_uint32, i, i, dp, lg]
    L.orc_uniform_pair.argtypes = [ctypes.c_uint64, ctypes.c_uint32, lg, i, dp, dp]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    a = np.asarray(a, dtype=np.float64)
    return np.asfortranarray(a)


def lm_of_index(k: int):
    l, m = ctypes.c_int(), ctypes.c_int()
    lib().orc_lm_of_index(k, ctypes.byref(l), ctypes.byref(m))
    return l.value, m.value


def cov_build(L: int, beta: float, sigma_exp: float = 1.5, nugget_rel: float = 1e-8):
    n = L * L
    S = np.zeros((n, n), dtype=np.float64, order="F")
    lib().orc_cov_build(L, beta, sigma_exp, nugget_rel, _dp(S), n)
    return S


def cov_rows(L: int, beta: float, rows, sigma_exp: float = 1.5, nugget_rel: float = 1e-8):
    """Rows `rows` of the covariance (len(rows) x L^2), without the full matrix."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), L * L), dtype=np.float64, order="F")
    lib().orc_cov_rows(L, beta, sigma_exp, nugget_rel, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                       len(rows), _dp(out))
    return out


def tile_norms(S, nb: int):
    S = _f64(S)
    n = S.shape[0]
    NT = (n + nb - 1) // nb
    t = np.zeros((NT, NT), dtype=np.float64, order="F")
    lib().orc_tile_norms(n, _dp(S), S.shape[0], nb, _dp(t))
    return t


def frob_from_tiles(t):
    t = _f64(t)
    return lib().orc_frob_from_tiles(t.shape[0], _dp(t))


def precision_map(t, eps: float, u, mask: int, diag_fp64: bool = False):
    t = _f64(t)
    NT = t.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    cls = np.zeros((NT, NT), dtype=np.uint8, order="F")
    lib().orc_precision_map(NT, _dp(t), eps, _dp(u), len(u), mask, int(diag_fp64),
                            cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return cls


def precision_map_band(NT: int, band: int, sp_frac: float = 0.05):
    """Band map of the paper's variants (1 DP/SP, 2 DP/SP/HP, 3 DP/HP): (classes NT x NT, number of SP bands)."""
    cls = np.zeros((NT, NT), dtype=np.uint8, order="F")
    nsp = lib().orc_precision_map_band(NT, band, sp_frac, cls.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return cls, nsp


def cov_from_residuals(Xi, nugget_rel: float = 0.0):
    """U = Xi Xi^T / m with nugget_rel * max diag added to the diagonal (full symmetric n x n)."""
    Xi = np.asfortranarray(Xi, dtype=np.float64)
    n, m = Xi.shape
    U = np.zeros((n, n), dtype=np.float64, order="F")
    lib().orc_cov_from_residuals(n, m, _dp(Xi), n, nugget_rel, _dp(U))
    return U


def var_recursion(Xi, Phi):
    """f_t = sum_p Phi[:, p-1] f_{t-p} + Xi[:, t], f before t = 0 zero (n x T)."""
    Xi = np.asfortranarray(Xi, dtype=np.float64)
    n, T = Xi.shape
    P = 0 if Phi is None else Phi.shape[1]
    Ph = np.asfortranarray(Phi if P else np.zeros((n, 1)), dtype=np.float64)
    F = np.zeros((n, T), dtype=np.float64, order="F")
    lib().orc_var_recursion(n, T, _dp(Xi), n, _dp(Ph), P, _dp(F), n)
    return F


def mean_trend(t: int, tau: float, b0: float, b1: float, b2: float, rho: float, a, b, x) -> float:
    """m_t at one grid point (Eq. decouple's trend): a, b the K harmonic amplitudes, x the forcing x[0..Y]."""
    K = len(a)
    a = np.ascontiguousarray(list(a) + [0.0], dtype=np.float64)  # never empty
    b = np.ascontiguousarray(list(b) + [0.0], dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_mean_trend(t, tau, b0, b1, b2, rho, K, _dp(a), _dp(b), _dp(x))


def emulate_grid(Zs, E, tau: float, b0, b1, b2, rho, A, B, x, sigma, v):
    """y_t(g) = m_t(g) + sigma(g) (Zs_t(g) + v(g) E_t(g)) for t = 1..T (columns); Zs, E are G x T; A, B are K x G."""
    Zs = np.asfortranarray(Zs, dtype=np.float64)
    E = np.asfortranarray(E, dtype=np.float64)
    G, T = Zs.shape
    A = np.asfortranarray(A, dtype=np.float64).reshape(-1, G, order="F")
    B = np.asfortranarray(B, dtype=np.float64).reshape(-1, G, order="F")
    K = A.shape[0]
    if K == 0:
        A = B = np.zeros((1, G), order="F")
    vec = [np.ascontiguousarray(q, dtype=np.float64) for q in (b0, b1, b2, rho, x, sigma, v)]
    Y = np.zeros((G, T), dtype=np.float64, order="F")
    lib().orc_emulate_grid(G, T, _dp(Zs), G, _dp(E), G, K, tau, _dp(vec[0]), _dp(vec[1]), _dp(vec[2]),
                           _dp(vec[3]), _dp(A), _dp(B), _dp(vec[4]), _dp(vec[5]), _dp(vec[6]), _dp(Y), G)
    return Y


def real_sh(l: int, m: int, theta: float, phi: float) -> float:
    return lib().orc_real_sh(l, m, theta, phi)


def isht(F, L: int, ntheta: int, nphi: int):
    """Synthesis of each column of F (L^2 x T) on the grid: (ntheta*nphi x T), point (i, j) at row i + j*ntheta."""
    F = np.asfortranarray(F, dtype=np.float64)
    n, T = F.shape
    Z = np.zeros((ntheta * nphi, T), dtype=np.float64, order="F")
    lib().orc_isht(L, T, _dp(F), n, ntheta, nphi, _dp(Z), ntheta * nphi)
    return Z


def sht(Z, L: int, ntheta: int, nphi: int):
    """Forward SHT (the paper's method: DFT in longitude, circle extension in colatitude, I(q) contraction) of
    each column of Z ((ntheta*nphi) x T, point (i, j) at row i + j*ntheta): real-form coefficients (L^2 x T)."""
    Z = np.asfortranarray(Z, dtype=np.float64)
    T = Z.shape[1]
    F = np.zeros((L * L, T), dtype=np.float64, order="F")
    lib().orc_sht(L, T, _dp(Z), ntheta * nphi, ntheta, nphi, _dp(F), L * L)
    return F


def I_of(k: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_I_pub(k, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def potrf_unblocked(A):
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    info = lib().orc_potrf_unblocked(A.shape[0], _dp(A), A.shape[0])
    return np.tril(A), info


def potrf_blocked(A, nb: int, kmax: int = -1, inplace: bool = False):
    if inplace:
        assert A.dtype == np.float64 and A.flags.f_contiguous
    else:
        A = np.array(A, dtype=np.float64, order="F", copy=True)
    info = lib().orc_potrf_blocked(A.shape[0], nb, _dp(A), A.shape[0], kmax)
    if inplace:
        return A, info
    return np.tril(A), info


def trmm_lower(Lf, Z):
    Lf = _f64(Lf)
    Z = _f64(Z)
    n, s = Z.shape
    Y = np.zeros((n, s), dtype=np.float64, order="F")
    lib().orc_trmm_lower(n, s, _dp(Lf), Lf.shape[0], _dp(Z), n, _dp(Y), n)
    return Y


def potrs(Lf, B):
    Lf = _f64(Lf)
    B = _f64(B)
    n, r = B.shape
    X = np.zeros((n, r), dtype=np.float64, order="F")
    lib().orc_potrs(n, r, _dp(Lf), Lf.shape[0], _dp(B), n, _dp(X), n)
    return X


def logdet_chol(Lf):
    Lf = _f64(Lf)
    return lib().orc_logdet_chol(Lf.shape[0], _dp(Lf), Lf.shape[0])


def backward_error(A, Lf):
    A = _f64(A)
    Lf = _f64(Lf)
    return lib().orc_backward_error(A.shape[0], _dp(A), A.shape[0], _dp(Lf), Lf.shape[0])


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def uniform_pair(seed: int, stream: int, p: int, c: int):
    u1, u2 = ctypes.c_double(), ctypes.c_double()
    lib().orc_uniform_pair(seed, stream, p, c, ctypes.byref(u1), ctypes.byref(u2))
    return u1.value, u2.value


def normal_matrix(seed: int, stream: int, n: int, s: int):
    Z = np.zeros((n, s), dtype=np.float64, order="F")
    lib().orc_normal_matrix(seed, stream, n, s, _dp(Z), n)
    return Z
