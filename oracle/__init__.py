"""FP64 CPU oracle for the layered-media Laplace potential (arXiv 1908.10863).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1908_10863_gb300``; the C source
``lfmm_oracle.c`` is compiled here with gcc and loaded through ctypes.

Functions follow the paper's definitions:

* :func:`sigma` -- reaction densities sigma^{ab}_{l l'}(k) from a direct solve
  of the spectral interface problem (Appendix A, eqs. A.1-A.3).
* :func:`sigma3_closed` -- the explicit three-layer densities of Appendix A
  (densitythreelayer1-3), with the kappa and sigma^{22}_{22} corrections.
* :func:`sommerfeld_K` / :func:`sommerfeld_K_images` -- the Sommerfeld-type
  integral of eq. uniformintegral (unnormalised: K = sqrt((N+mu)!(N-mu)!) I)
  by adaptive Gauss-Kronrod, or by the exact three-layer image series.
* :func:`direct` -- Phi and E = -grad Phi at target charges by direct
  summation (eqs. potential1, totalinteraction), 1/(4 pi) included, free-space
  self term excluded, reaction self term included.  In quadrature mode the
  density's k -> infinity limit is integrated in closed form (Lipschitz
  integral) and only the decaying rest by adaptive quadrature, so charges
  next to an interface converge.  A quadrature that runs out of panels raises
  :class:`OracleNotConverged` instead of returning a partial sum.
* :func:`err2`, :func:`errmax` -- the error norms of Section 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class OracleNotConverged(RuntimeError):
    """An adaptive quadrature ran out of panels before meeting its tolerance;
    the oracle refuses to return the partial sum."""


def build(force: bool = False) -> str:
    """Compile ``lfmm_oracle.c`` into ``liboracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Werror=implicit-function-declaration", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_sigma.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp]
        lib.oracle_sigma.restype = ctypes.c_int
        lib.oracle_sigma3_closed.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _dp]
        lib.oracle_sigma3_closed.restype = ctypes.c_int
        lib.oracle_sommerfeld_K.argtypes = [ctypes.c_int, _dp, _dp] + [ctypes.c_int] * 6 + [
            ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double]
        lib.oracle_sommerfeld_K.restype = ctypes.c_double
        lib.oracle_sommerfeld_K_images.argtypes = [_dp, _dp] + [ctypes.c_int] * 6 + [ctypes.c_double,
                                                                                       ctypes.c_double]
        lib.oracle_sommerfeld_K_images.restype = ctypes.c_double
        lib.oracle_legendre_nocs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.oracle_legendre_nocs.restype = ctypes.c_double
        lib.oracle_direct.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int64, _dp, _i32p, _dp, ctypes.c_int64,
                                      _i64p, ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int]
        lib.oracle_direct.restype = ctypes.c_int
        lib.oracle_reaction_pair.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                             ctypes.c_int, ctypes.c_double, _dp]
        lib.oracle_reaction_pair.restype = ctypes.c_int
        lib.oracle_forward_recurrence.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_forward_recurrence.restype = None
        _lib = lib
    return _lib


def _arr(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def sigma(d, eps, k: float, lp: int) -> np.ndarray:
    """All sigma^{ab}_{l,lp}(k) as an array [L+1, 2, 2] indexed (l, a-1, b-1)."""
    d = _arr(d); eps = _arr(eps)
    L = len(d)
    out = np.zeros(4 * (L + 1))
    if _load().oracle_sigma(L, _ptr(d), _ptr(eps), float(k), int(lp), _ptr(out)):
        raise ValueError("oracle_sigma failed")
    return out.reshape(L + 1, 2, 2)


def sigma3_closed(d, eps, k: float, l: int, lp: int, a: int, b: int) -> float:
    d = _arr(d); eps = _arr(eps)
    out = np.zeros(1)
    if _load().oracle_sigma3_closed(_ptr(d), _ptr(eps), float(k), l, lp, a, b, _ptr(out)):
        raise ValueError("component (%d,%d,%d,%d) does not exist" % (l, lp, a, b))
    return float(out[0])


def sommerfeld_K(d, eps, l, lp, a, b, N, mu, rho, z, sigma_one=False, tol=1e-13) -> float:
    """int_0^inf J_mu(k rho) k^N e^{-kz} sigma^{ab}_{l lp}(k) dk by adaptive quadrature."""
    d = _arr(d); eps = _arr(eps)
    v = _load().oracle_sommerfeld_K(len(d), _ptr(d), _ptr(eps), l, lp, a, b, N, mu, float(rho), float(z),
                                    1 if sigma_one else 0, float(tol))
    if not np.isfinite(v):
        raise OracleNotConverged("sommerfeld_K: invalid component or the adaptive quadrature did not converge")
    return v


def sommerfeld_K_images(d, eps, l, lp, a, b, N, mu, rho, z) -> float:
    """Same integral by the exact three-layer image series."""
    d = _arr(d); eps = _arr(eps)
    return _load().oracle_sommerfeld_K_images(_ptr(d), _ptr(eps), l, lp, a, b, N, mu, float(rho), float(z))


def legendre_nocs(n, m, x) -> float:
    return _load().oracle_legendre_nocs(n, m, float(x))


MODE_QUAD, MODE_IMAGES, MODE_SIGMA_ONE, MODE_FREE_ONLY = 0, 1, 2, 3


def direct(d, eps, xyz, layer, q, targets=None, mode=MODE_QUAD, tol=1e-12, threads=0):
    """Phi[nt] and E[nt,3] at ``targets`` (indices into the charge arrays)."""
    d = _arr(d); eps = _arr(eps)
    xyz = _arr(xyz).reshape(-1, 3)
    n = xyz.shape[0]
    layer = _arr(layer, np.int32)
    q = _arr(q)
    if targets is None:
        targets = np.arange(n, dtype=np.int64)
    targets = _arr(targets, np.int64)
    nt = targets.shape[0]
    phi = np.zeros(nt)
    field = np.zeros((nt, 3))
    rc = _load().oracle_direct(len(d), _ptr(d), _ptr(eps), n, _ptr(xyz), _ptr(layer, _i32p), _ptr(q), nt,
                               _ptr(targets, _i64p), int(mode), float(tol), _ptr(phi), _ptr(field), int(threads))
    if rc == -2:
        raise OracleNotConverged("oracle_direct: an adaptive quadrature ran out of panels before its tolerance")
    if rc:
        raise ValueError("oracle_direct rejected the input")
    return phi, field


def reaction_pair(d, eps, l, lp, r, rp, mode=MODE_QUAD, tol=1e-13):
    """(4 pi u^r_{l lp}(r, r'), 4 pi grad_r u^r) for one pair."""
    d = _arr(d); eps = _arr(eps)
    r = _arr(r); rp = _arr(rp)
    g = np.zeros(4)
    rc = _load().oracle_reaction_pair(len(d), _ptr(d), _ptr(eps), l, lp, _ptr(r), _ptr(rp), int(mode), float(tol),
                                      _ptr(g))
    if rc == -2:
        raise OracleNotConverged("oracle_reaction_pair: the adaptive quadrature did not converge")
    if rc:
        raise ValueError("oracle_reaction_pair failed")
    return g[0], g[1:].copy()


def forward_recurrence(P, S, rho, In0, In1):
    """The paper's forward recurrence (eq. recurrence) on S^n I_{n,m}."""
    In0 = _arr(In0); In1 = _arr(In1)
    out = np.zeros((2 * P + 1) * (2 * P + 1))
    _load().oracle_forward_recurrence(P, float(S), float(rho), _ptr(In0), _ptr(In1), _ptr(out))
    return out.reshape(2 * P + 1, 2 * P + 1)


def err2(ref, approx) -> float:
    """Relative l2 error Err_2 of Section 4."""
    ref = np.asarray(ref); approx = np.asarray(approx)
    return float(np.sqrt(np.sum(np.abs(ref - approx) ** 2) / np.sum(np.abs(ref) ** 2)))


def errmax(ref, approx) -> float:
    """Maximum pointwise relative error Err_max of Section 4."""
    ref = np.asarray(ref); approx = np.asarray(approx)
    return float(np.max(np.abs(ref - approx) / np.abs(ref)))
