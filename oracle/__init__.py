"""CPU FP64 oracle for the Chebyshev-Hutchinson log-determinant estimator.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously-correct
reference the GPU library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it;
the library in ``paper_1503_06394_gb300`` never does, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over rows); this
module compiles it on first use, wraps it with ctypes, and adds the closed-form
exact references that are easiest to state in numpy:

* ``kms_logdet`` -- log det of the Kac-Murdock-Szego matrix rho^|i-k|,
  (d - 1) log(1 - rho^2).
* ``grid_laplacian_logdet`` -- log det(kappa^2 I + L) for the 5-point Dirichlet
  Laplacian on an N x N grid, from its separable eigenvalues
  kappa^2 + 4 sin^2(pi i / (2(N+1))) + 4 sin^2(pi j / (2(N+1))).
* ``thm1_degree`` -- the sufficient degree of Theorem 1, and
  ``chebyshev_error_bound`` -- the per-eigenvalue bound
  20 log(2(1/delta - 1)) / ((K-1) K^n) of Sec. 4.1.

Every arithmetic function here is pinned by a CPU test against something other
than itself (closed forms, numpy's eigensolver and slogdet, exhaustive sign
enumeration, finite differences, cuRAND's host Philox); none is parity
unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
               "-fPIC", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_rademacher.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_rademacher.restype = ctypes.c_double
            lib.oracle_rademacher_fill.argtypes = [ctypes.c_uint64, ctypes.c_int64, _i64p,
                                                   ctypes.c_int64, _f64p]
            lib.oracle_rademacher_fill.restype = None
            lib.oracle_cheb_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _f64p]
            lib.oracle_cheb_coeffs.restype = None
            lib.oracle_cheb_coeffs_alg1.argtypes = [ctypes.c_int, ctypes.c_double, _f64p]
            lib.oracle_cheb_coeffs_alg1.restype = None
            lib.oracle_moments.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int64, _f64p, _f64p]
            lib.oracle_moments.restype = ctypes.c_int
            lib.oracle_finalize.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p]
            lib.oracle_finalize.restype = None
            lib.oracle_alg1_literal.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int64, _f64p, _f64p]
            lib.oracle_alg1_literal.restype = ctypes.c_int
            lib.oracle_alg2_literal.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int64, _f64p,
                                                _f64p]
            lib.oracle_alg2_literal.restype = ctypes.c_int
            lib.oracle_gershgorin.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p]
            lib.oracle_gershgorin.restype = None
            lib.oracle_sigma_max_bound.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p]
            lib.oracle_sigma_max_bound.restype = ctypes.c_double
            lib.oracle_dominance_margins.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p]
            lib.oracle_dominance_margins.restype = None
            lib.oracle_logdet_cholesky.argtypes = [ctypes.c_int64, _f64p, _f64p]
            lib.oracle_logdet_cholesky.restype = ctypes.c_int
            lib.oracle_grad.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int64, _f64p, _f64p]
            lib.oracle_grad.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(arr, ptype):
    return arr.ctypes.data_as(ptype)


def _csr(rowptr, col, val):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    d = rowptr.shape[0] - 1
    if d < 0 or rowptr[-1] != col.shape[0] or col.shape[0] != val.shape[0]:
        raise ValueError("inconsistent CSR arrays")
    return d, rowptr, col, val


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# ----------------------------------------------------------------------------- probes
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: counter (4 x uint32), key (2 x uint32) -> 4 x uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def rademacher(seed: int, d: int, probes) -> np.ndarray:
    """d x len(probes) matrix of Rademacher signs v[i, probes[q]] (FP64)."""
    pr = np.ascontiguousarray(np.atleast_1d(probes), dtype=np.int64)
    V = np.empty((d, pr.shape[0]), dtype=np.float64)
    _load().oracle_rademacher_fill(ctypes.c_uint64(seed), d, _p(pr, _i64p), pr.shape[0], _p(V, _f64p))
    return V


# ----------------------------------------------------------------------------- estimator
def cheb_coeffs(n: int, a: float, b: float) -> np.ndarray:
    """c_0..c_n of the degree-n Chebyshev interpolant of log on [a, b] (Sec. 2.1)."""
    c = np.empty(n + 1, dtype=np.float64)
    _load().oracle_cheb_coeffs(n, a, b, _p(c, _f64p))
    return c


def cheb_coeffs_alg1(n: int, delta: float) -> np.ndarray:
    """Coefficients of log(1 - ((1-2 delta) x + 1)/2), as Algorithm 1 states them."""
    c = np.empty(n + 1, dtype=np.float64)
    _load().oracle_cheb_coeffs_alg1(n, delta, _p(c, _f64p))
    return c


def moments(rowptr, col, val, a: float, b: float, n: int, V, kind: int = 0) -> np.ndarray:
    """t[j, p] = v_p^T T_j(At) v_p for j = 0..n, At = (2X - (a+b)I)/(b-a).

    X is the CSR matrix (kind 0) or C^T C for the CSR matrix C (kind 1).
    V is d x M (any real probes).  Returns an (n+1) x M FP64 array."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim != 2 or V.shape[0] != d:
        raise ValueError("V must be d x M")
    M = V.shape[1]
    t = np.zeros((n + 1, M), dtype=np.float64)
    rc = _load().oracle_moments(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p), kind,
                                a, b, n, M, _p(V, _f64p), _p(t, _f64p))
    if rc != 0:
        raise ValueError("oracle_moments failed with %d" % rc)
    return t


def finalize(c, t):
    """(Gamma_p per probe, Gamma) from coefficients and moments (Algorithm 1)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    n = c.shape[0] - 1
    M = t.shape[1]
    gp = np.empty(M, dtype=np.float64)
    g = ctypes.c_double()
    _load().oracle_finalize(n, M, _p(c, _f64p), _p(t, _f64p), _p(gp, _f64p), ctypes.byref(g))
    return gp, g.value


def estimate(rowptr, col, val, a, b, n, M, seed=0, probes=None, kind=0):
    """Chebyshev-Hutchinson estimate with the Philox Rademacher stream.

    Returns dict(gamma, gamma_p, stderr, t, c).  For kind 1 (general C) gamma
    estimates logdet(C^T C) = 2 log|det C|."""
    d = len(rowptr) - 1
    pr = np.arange(M, dtype=np.int64) if probes is None else np.asarray(probes, dtype=np.int64)
    V = rademacher(seed, d, pr)
    t = moments(rowptr, col, val, a, b, n, V, kind=kind)
    c = cheb_coeffs(n, a, b)
    gp, g = finalize(c, t)
    m = gp.shape[0]
    se = float(np.std(gp, ddof=1) / np.sqrt(m)) if m > 1 else float("nan")
    return {"gamma": g, "gamma_p": gp, "stderr": se, "t": t, "c": c}


def alg1_literal(rowptr, col, val, delta, n, V) -> float:
    """Algorithm 1 as printed (with the documented readings), probes V (d x m)."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    V = np.ascontiguousarray(V, dtype=np.float64)
    g = ctypes.c_double()
    rc = _load().oracle_alg1_literal(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p), delta,
                                     n, V.shape[1], _p(V, _f64p), ctypes.byref(g))
    if rc != 0:
        raise ValueError("oracle_alg1_literal failed with %d" % rc)
    return g.value


def alg2_literal(rowptr, col, val, sigma_min, sigma_max, n, V) -> float:
    """Algorithm 2 as printed: estimate of log|det C| for CSR matrix C."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    V = np.ascontiguousarray(V, dtype=np.float64)
    g = ctypes.c_double()
    rc = _load().oracle_alg2_literal(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p),
                                     sigma_min, sigma_max, n, V.shape[1], _p(V, _f64p),
                                     ctypes.byref(g))
    if rc != 0:
        raise ValueError("oracle_alg2_literal failed with %d" % rc)
    return g.value


def grad(rowptr, col, val, a, b, n, V) -> np.ndarray:
    """dGamma / d(stored value), Gamma averaged over the probes in V, [a,b] fixed."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    V = np.ascontiguousarray(V, dtype=np.float64)
    G = np.zeros(val.shape[0], dtype=np.float64)
    rc = _load().oracle_grad(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p), a, b, n,
                             V.shape[1], _p(V, _f64p), _p(G, _f64p))
    if rc != 0:
        raise ValueError("oracle_grad failed with %d" % rc)
    return G


# ----------------------------------------------------------------------------- bounds
def gershgorin(rowptr, col, val):
    """(lo, hi) Gershgorin enclosure of the spectrum of a symmetric CSR matrix."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().oracle_gershgorin(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p),
                              ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def sigma_max_bound(rowptr, col, val) -> float:
    """sqrt(||C||_1 ||C||_inf) >= sigma_max(C) (Sec. 3.2)."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    return float(_load().oracle_sigma_max_bound(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p)))


def dominance_margins(rowptr, col, val):
    """(alpha, beta): row and column diagonal-dominance margins of a general C."""
    d, rowptr, col, val = _csr(rowptr, col, val)
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().oracle_dominance_margins(d, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p),
                                     ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


# ----------------------------------------------------------------------------- exact
def logdet_cholesky(A) -> float:
    """2 sum log L_ii from a dense FP64 Cholesky factorisation (Sec. 1)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix required")
    out = ctypes.c_double()
    rc = _load().oracle_logdet_cholesky(A.shape[0], _p(A, _f64p), ctypes.byref(out))
    if rc != 0:
        raise ValueError("matrix is not positive definite")
    return out.value


def grid_laplacian_logdet(N: int, kappa2: float) -> float:
    """log det(kappa^2 I + L), L the 5-point Dirichlet Laplacian on an N x N grid.

    The eigenvalues are kappa^2 + 4 sin^2(pi i/(2(N+1))) + 4 sin^2(pi j/(2(N+1))),
    i, j = 1..N; the sum of their logs is accumulated with math.fsum."""
    import math
    s = 4.0 * np.sin(np.pi * np.arange(1, N + 1) / (2.0 * (N + 1))) ** 2
    lam = kappa2 + s[:, None] + s[None, :]
    return math.fsum(np.log(lam).ravel().tolist())


def kms_logdet(d: int, rho: float) -> float:
    """log det of the d x d Kac-Murdock-Szego matrix A_ik = rho^|i-k|, |rho| < 1.

    With white noise e, x_0 = e_0 and x_i = rho x_{i-1} + sqrt(1 - rho^2) e_i
    has covariance rho^|i-k|; x = L e for a lower triangular L whose diagonal
    is 1, sqrt(1 - rho^2), ..., sqrt(1 - rho^2), so A = L L^T and
    det A = (1 - rho^2)^(d-1)."""
    import math
    if d <= 0:
        return 0.0
    return (d - 1) * math.log1p(-rho * rho)


def chebyshev_error_bound(delta: float, n: int) -> float:
    """20 log(2(1/delta - 1)) / ((K-1) K^n), K = (sqrt(2-delta)+sqrt(delta))/(sqrt(2-delta)-sqrt(delta))
    (Sec. 4.1: the per-eigenvalue bound for log(1-x) on [delta, 1-delta])."""
    K = (np.sqrt(2 - delta) + np.sqrt(delta)) / (np.sqrt(2 - delta) - np.sqrt(delta))
    return 20.0 * np.log(2.0 * (1.0 / delta - 1.0)) / ((K - 1.0) * K ** n)


def thm1_degree(delta: float, eps: float) -> float:
    """Right-hand side of Theorem 1's condition on n (real-valued)."""
    K = (np.sqrt(2 - delta) + np.sqrt(delta)) / (np.sqrt(2 - delta) - np.sqrt(delta))
    num = np.log(20.0 / eps * (np.sqrt(2.0 / delta - 1.0) - 1.0)
                 * np.log(2.0 * (1.0 / delta - 1.0)) / np.log(1.0 / (1.0 - delta)))
    return float(num / np.log(K))

