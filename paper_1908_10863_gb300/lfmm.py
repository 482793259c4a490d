"""Python binding of the C ABI in ``include/lfmm.h`` (argument marshalling only).

Every computation runs in the CUDA library ``liblfmm.so``; this module only
converts numpy arrays / torch CUDA tensors to pointers and status codes to
exceptions.  Importing it fails loudly when the library cannot be built or
loaded: there is no host fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENUMERIC = range(7)
OPT_PRECISION, OPT_LEAF_CAP, OPT_PROFILE, OPT_QUAD_NODES, OPT_SURROGATE, OPT_SURROGATE_TOL = 1, 2, 3, 4, 5, 6
OPT_TENSOR_CORES, OPT_P2P_SPLIT, OPT_TC_GROUPS, OPT_NEAR_TABLES, OPT_TC_PERSISTENT = 7, 8, 9, 10, 11
OPT_P2P_STAGED, OPT_SERIAL_NEAR = 12, 13
TUNE_COLS = ["leaf_cap", "tensor_cores", "split", "depth", "ms", "chosen"]
BATCH_TUNE_COLS = ["tc_min_charges", "split", "tables", "ms", "chosen"]
STAT_NAMES = ["n", "depth", "boxes", "leaves", "m2l_free", "m2l_reaction", "p2p_free", "p2p_reaction",
              "components", "m2m_edges", "launches", "reaction_keys", "surr_net_pairs", "surr_quad_pairs",
              "timeouts", "reaction_tables"]
SURR_NPARAM = 8835
SURR_INFO = ["trained", "max_err", "cells_ok", "loss", "n_train", "n_val", "samples_ok"]
TIME_NAMES = ["p2m", "m2m", "m2l_free", "m2l_reaction", "l2l", "l2p", "p2p", "total", "build"]
_STATUS = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ESTATE: "ESTATE", ETIMEOUT: "ETIMEOUT",
           ENUMERIC: "ENUMERIC"}


class LfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_ctxp = ctypes.c_void_p

EXPORTED = ["lfmm_create", "lfmm_set_option", "lfmm_build", "lfmm_build_device", "lfmm_evaluate",
            "lfmm_evaluate_device", "lfmm_last_error", "lfmm_destroy", "lfmm_get_stats", "lfmm_get_timings",
            "lfmm_sommerfeld_tables", "lfmm_reaction_kernel", "lfmm_reaction_kernel_noalloc", "lfmm_gauss_laguerre",
            "lfmm_surrogate_train", "lfmm_surrogate_info", "lfmm_surrogate_eval", "lfmm_surrogate_get_params",
            "lfmm_surrogate_set_params", "lfmm_surrogate_forward", "lfmm_surrogate_loss_grad",
            "lfmm_batch_create", "lfmm_batch_offsets", "lfmm_batch_evaluate_device", "lfmm_batch_evaluate",
            "lfmm_batch_info", "lfmm_batch_autotune", "lfmm_batch_last_error", "lfmm_batch_destroy", "lfmm_autotune",
            "lfmm_check_bounded_wait", "lfmm_near_tables", "lfmm_medium_components"]
BATCH_INFO = ["problems", "charges", "graph_nodes", "kernel_nodes", "captures", "graph_launches", "direct_runs",
              "timeouts"]
NOALLOC_MAX_POINTS = 65536


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("liblfmm.so is missing at %s (run build())" % path)
    lib = ctypes.CDLL(path)
    lib.lfmm_create.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.POINTER(_ctxp)]
    lib.lfmm_set_option.argtypes = [_ctxp, ctypes.c_int, ctypes.c_double]
    lib.lfmm_build.argtypes = [_ctxp, ctypes.c_int64, _dp, _ip]
    lib.lfmm_build_device.argtypes = [_ctxp, ctypes.c_int64, _vp, _vp, _vp]
    lib.lfmm_evaluate.argtypes = [_ctxp, ctypes.c_int, _dp, _dp, _dp]
    lib.lfmm_evaluate_device.argtypes = [_ctxp, ctypes.c_int, _vp, _vp, _vp, _vp]
    lib.lfmm_last_error.argtypes = [_ctxp]
    lib.lfmm_last_error.restype = ctypes.c_char_p
    lib.lfmm_destroy.argtypes = [_ctxp]
    lib.lfmm_destroy.restype = None
    lib.lfmm_get_stats.argtypes = [_ctxp, _lp, ctypes.c_int]
    lib.lfmm_get_timings.argtypes = [_ctxp, _dp, ctypes.c_int]
    lib.lfmm_sommerfeld_tables.argtypes = [_ctxp] + [ctypes.c_int] * 5 + [_dp, _dp, ctypes.c_double, ctypes.c_int,
                                                                          _dp]
    lib.lfmm_reaction_kernel.argtypes = [_ctxp] + [ctypes.c_int] * 5 + [_dp, _dp, _dp]
    lib.lfmm_reaction_kernel_noalloc.argtypes = [_ctxp] + [ctypes.c_int] * 5 + [_dp, _dp, _dp]
    lib.lfmm_gauss_laguerre.argtypes = [ctypes.c_int, _dp, _dp]
    lib.lfmm_medium_components.argtypes = [_dp, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    _fp = ctypes.POINTER(ctypes.c_float)
    comp = [ctypes.c_int] * 4
    lib.lfmm_surrogate_train.argtypes = [_ctxp, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
    lib.lfmm_surrogate_info.argtypes = [_ctxp] + comp + [_dp]
    lib.lfmm_surrogate_eval.argtypes = [_ctxp] + comp + [ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.lfmm_surrogate_get_params.argtypes = [_ctxp] + comp + [_fp]
    lib.lfmm_surrogate_set_params.argtypes = [_ctxp] + comp + [_fp]
    lib.lfmm_surrogate_forward.argtypes = [_ctxp] + comp + [ctypes.c_int, _fp, _fp]
    lib.lfmm_surrogate_loss_grad.argtypes = [_ctxp] + comp + [ctypes.c_int, _fp, _fp, _dp, _fp]
    lib.lfmm_check_bounded_wait.argtypes = [_ctxp, ctypes.c_double]
    lib.lfmm_near_tables.argtypes = [_ctxp, _dp]
    lib.lfmm_autotune.argtypes = [_ctxp, ctypes.c_int64, _dp, _ip, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int)]
    lib.lfmm_batch_create.argtypes = [ctypes.POINTER(_ctxp), ctypes.c_int, _ip, ctypes.c_int, ctypes.POINTER(_vp)]
    lib.lfmm_batch_offsets.argtypes = [_vp, _lp]
    lib.lfmm_batch_evaluate_device.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.lfmm_batch_evaluate.argtypes = [_vp, _dp, _dp, _dp]
    lib.lfmm_batch_info.argtypes = [_vp, _lp, ctypes.c_int]
    lib.lfmm_batch_autotune.argtypes = [_vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.lfmm_batch_last_error.argtypes = [_vp]
    lib.lfmm_batch_last_error.restype = ctypes.c_char_p
    lib.lfmm_batch_destroy.argtypes = [_vp]
    lib.lfmm_batch_destroy.restype = None
    for name in EXPORTED:
        if name not in ("lfmm_last_error", "lfmm_destroy", "lfmm_batch_last_error", "lfmm_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def gauss_laguerre(Q: int):
    """Nodes and weights of the Q-point Gauss-Laguerre rule (host-only call)."""
    t = np.zeros(Q)
    w = np.zeros(Q)
    st = load().lfmm_gauss_laguerre(int(Q), _ptr(t), _ptr(w))
    if st != OK:
        raise LfmmError(st, "lfmm_gauss_laguerre")
    return t, w


MEDIUM_COLS = ["l", "lp", "a", "b", "is_free", "s", "o", "iface", "C", "zeta", "zeta_r"]


def medium_components(d, eps):
    """The components a context for this medium evaluates, one dict each
    (host-only call; see ``lfmm_medium_components``)."""
    d = _f64(d)
    eps = _f64(eps)
    L = int(d.shape[0])
    lib = load()
    n = ctypes.c_int(0)
    st = lib.lfmm_medium_components(_ptr(d) if L else None, L, _ptr(eps), None, 0, ctypes.byref(n))
    if st != OK:
        raise LfmmError(st, "lfmm_medium_components")
    out = np.zeros((n.value, len(MEDIUM_COLS)))
    st = lib.lfmm_medium_components(_ptr(d) if L else None, L, _ptr(eps), _ptr(out), n.value, ctypes.byref(n))
    if st != OK:
        raise LfmmError(st, "lfmm_medium_components")
    ints = {"l", "lp", "a", "b", "is_free"}
    return [{k: (int(v) if k in ints else float(v)) for k, v in zip(MEDIUM_COLS, r)} for r in out[:n.value]]


class LayeredFMM:
    """One medium (interfaces d, permittivities eps) and expansion order p."""

    def __init__(self, d, eps, p: int, precision: int = 0, leaf_cap: int = 40, profile: bool = False):
        lib = load()
        self._lib = lib
        d = _f64(d)
        eps = _f64(eps)
        self.L = int(d.shape[0])
        self.p = int(p)
        ctx = _ctxp()
        st = lib.lfmm_create(_ptr(d) if self.L else None, self.L, _ptr(eps), self.p, ctypes.byref(ctx))
        if st != OK:
            raise LfmmError(st, "lfmm_create")
        self._ctx = ctx
        self.n = 0
        if precision:
            self.set_option(OPT_PRECISION, precision)
        if leaf_cap != 40:
            self.set_option(OPT_LEAF_CAP, leaf_cap)
        if profile:
            self.set_option(OPT_PROFILE, 1)

    def _check(self, st, what):
        if st != OK:
            msg = self._lib.lfmm_last_error(self._ctx)
            raise LfmmError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def set_option(self, opt: int, value: float):
        self._check(self._lib.lfmm_set_option(self._ctx, int(opt), float(value)), "lfmm_set_option")

    def build(self, xyz, layer):
        xyz = _f64(xyz).reshape(-1, 3)
        layer = np.ascontiguousarray(layer, dtype=np.int32)
        self._check(self._lib.lfmm_build(self._ctx, xyz.shape[0], _ptr(xyz), _ptr(layer, _ip)), "lfmm_build")
        self.n = xyz.shape[0]

    def build_device(self, xyz, layer, stream=None):
        """xyz: torch.float64 CUDA tensor [n,3]; layer: torch.int32 CUDA tensor [n]."""
        n = int(xyz.shape[0])
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(self._lib.lfmm_build_device(self._ctx, n, ctypes.c_void_p(xyz.data_ptr()),
                                                ctypes.c_void_p(layer.data_ptr()), s), "lfmm_build_device")
        self.n = n

    def evaluate(self, q, field: bool = True, out=None):
        """q: [n] or [nrhs, n] host charges -> (phi, E) host arrays.  `out`
        may give preallocated float64 C-contiguous arrays (phi shaped like q,
        E like q plus a trailing 3, or None) that are written and returned."""
        q = _f64(q)
        single = q.ndim == 1
        q2 = q.reshape(1, -1) if single else q
        nrhs = q2.shape[0]
        if out is not None:
            phi_o, fld_o = out
            for a, shp in ((phi_o, q.shape), (fld_o, q.shape + (3,))):
                if a is not None and (a.shape != shp or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]):
                    raise ValueError("out arrays must be C-contiguous float64 of shapes %s and %s"
                                     % (q.shape, q.shape + (3,)))
            field = fld_o is not None
            self._check(self._lib.lfmm_evaluate(self._ctx, nrhs, _ptr(q2), _ptr(phi_o),
                                                _ptr(fld_o) if field else None), "lfmm_evaluate")
            return phi_o, fld_o
        phi = np.zeros_like(q2)
        fld = np.zeros(q2.shape + (3,)) if field else None
        self._check(self._lib.lfmm_evaluate(self._ctx, nrhs, _ptr(q2), _ptr(phi), _ptr(fld) if field else None),
                    "lfmm_evaluate")
        if single:
            return phi[0], (fld[0] if field else None)
        return phi, fld

    def evaluate_device(self, q, phi, field=None, stream=None):
        """Device tensors (float64): q [n] or [nrhs, n], phi like q, field [.., n, 3] or None."""
        nrhs = 1 if q.dim() == 1 else int(q.shape[0])
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(self._lib.lfmm_evaluate_device(self._ctx, nrhs, ctypes.c_void_p(q.data_ptr()),
                                                   ctypes.c_void_p(phi.data_ptr()),
                                                   ctypes.c_void_p(field.data_ptr()) if field is not None else None,
                                                   s), "lfmm_evaluate_device")

    def autotune(self, xyz, layer, mode: int = 0, reps: int = 3):
        """Time candidate settings on this geometry and keep the fastest (the
        context is left built with it).  Returns one dict per timed setting."""
        xyz = _f64(xyz).reshape(-1, 3)
        layer = np.ascontiguousarray(layer, dtype=np.int32)
        rows = np.zeros((64, len(TUNE_COLS)))
        nrows = ctypes.c_int(0)
        self._check(self._lib.lfmm_autotune(self._ctx, xyz.shape[0], _ptr(xyz), _ptr(layer, _ip), int(mode),
                                            int(reps), _ptr(rows), 64, ctypes.byref(nrows)), "lfmm_autotune")
        self.n = xyz.shape[0]
        return [dict(zip(TUNE_COLS, r)) for r in rows[:nrows.value]]

    def near_tables(self) -> float:
        """Build (once) the near-field remainder tables; returns their largest
        relative deviation from the quadrature at the check points."""
        e = ctypes.c_double(0.0)
        self._check(self._lib.lfmm_near_tables(self._ctx, ctypes.byref(e)), "lfmm_near_tables")
        return e.value

    def check_bounded_wait(self, limit_ms: float = 10.0) -> int:
        """Run the device's bounded-wait self-check; returns its status code
        (ETIMEOUT is the expected outcome)."""
        st = self._lib.lfmm_check_bounded_wait(self._ctx, float(limit_ms))
        if st not in (OK, ETIMEOUT):
            self._check(st, "lfmm_check_bounded_wait")
        return st

    def stats(self) -> dict:
        out = np.zeros(16, dtype=np.int64)
        self._check(self._lib.lfmm_get_stats(self._ctx, _ptr(out, _lp), 16), "lfmm_get_stats")
        return {k: int(v) for k, v in zip(STAT_NAMES, out)}

    def timings(self) -> dict:
        out = np.zeros(12)
        self._check(self._lib.lfmm_get_timings(self._ctx, _ptr(out), 12), "lfmm_get_timings")
        return {k: float(v) for k, v in zip(TIME_NAMES, out)}

    def sommerfeld_tables(self, l, lp, a, b, rho, z, S, P):
        rho = _f64(rho).ravel()
        z = _f64(z).ravel()
        TS = 2 * P + 1
        out = np.zeros((rho.shape[0], TS, TS))
        self._check(self._lib.lfmm_sommerfeld_tables(self._ctx, l, lp, a, b, rho.shape[0], _ptr(rho), _ptr(z),
                                                     float(S), int(P), _ptr(out)), "lfmm_sommerfeld_tables")
        return out

    def reaction_kernel(self, l, lp, a, b, rho, h):
        rho = _f64(rho).ravel()
        h = _f64(h).ravel()
        out = np.zeros((rho.shape[0], 3))
        self._check(self._lib.lfmm_reaction_kernel(self._ctx, l, lp, a, b, rho.shape[0], _ptr(rho), _ptr(h),
                                                   _ptr(out)), "lfmm_reaction_kernel")
        return out

    def reaction_kernel_noalloc(self, l, lp, a, b, rho, h):
        """Same as reaction_kernel through the allocation-free entry point."""
        rho = _f64(rho).ravel()
        h = _f64(h).ravel()
        out = np.zeros((rho.shape[0], 3))
        self._check(self._lib.lfmm_reaction_kernel_noalloc(self._ctx, l, lp, a, b, rho.shape[0], _ptr(rho),
                                                           _ptr(h), _ptr(out)), "lfmm_reaction_kernel_noalloc")
        return out

    # ---- learned near-field reaction kernels ------------------------------
    def surrogate_train(self, nsamples: int = 1 << 20, epochs: int = 4, seed: int = 1):
        self._check(self._lib.lfmm_surrogate_train(self._ctx, int(nsamples), int(epochs), int(seed)),
                    "lfmm_surrogate_train")

    def surrogate_info(self, l, lp, a, b) -> dict:
        out = np.zeros(8)
        self._check(self._lib.lfmm_surrogate_info(self._ctx, l, lp, a, b, _ptr(out)), "lfmm_surrogate_info")
        return {k: float(v) for k, v in zip(SURR_INFO, out)}

    def surrogate_eval(self, l, lp, a, b, rho, ht, hs):
        """-> [n, 4]: network I_00, I_10, I_11 and the error-table acceptance flag."""
        rho, ht, hs = (_f64(v).ravel() for v in (rho, ht, hs))
        out = np.zeros((rho.shape[0], 4))
        self._check(self._lib.lfmm_surrogate_eval(self._ctx, l, lp, a, b, rho.shape[0], _ptr(rho), _ptr(ht),
                                                  _ptr(hs), _ptr(out)), "lfmm_surrogate_eval")
        return out

    def surrogate_params(self, l, lp, a, b):
        th = np.zeros(SURR_NPARAM, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self._lib.lfmm_surrogate_get_params(self._ctx, l, lp, a, b, _ptr(th, fp)),
                    "lfmm_surrogate_get_params")
        return th

    def surrogate_set_params(self, l, lp, a, b, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32).ravel()
        if th.shape[0] != SURR_NPARAM:
            raise ValueError("need %d parameters" % SURR_NPARAM)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self._lib.lfmm_surrogate_set_params(self._ctx, l, lp, a, b, _ptr(th, fp)),
                    "lfmm_surrogate_set_params")

    def surrogate_forward(self, l, lp, a, b, x):
        """Raw (standardised) network outputs [n, 3] for features x [n, 4] by the inference kernel."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        y = np.zeros((x.shape[0], 3), dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self._lib.lfmm_surrogate_forward(self._ctx, l, lp, a, b, x.shape[0], _ptr(x, fp), _ptr(y, fp)),
                    "lfmm_surrogate_forward")
        return y

    def surrogate_loss_grad(self, l, lp, a, b, x, y):
        """Loss and parameter gradient on the device for x [n,4], y [n,3] (n a multiple of 64)."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1, 3)
        fp = ctypes.POINTER(ctypes.c_float)
        loss = ctypes.c_double(0.0)
        g = np.zeros(SURR_NPARAM, dtype=np.float32)
        self._check(self._lib.lfmm_surrogate_loss_grad(self._ctx, l, lp, a, b, x.shape[0], _ptr(x, fp),
                                                       _ptr(y, fp), ctypes.byref(loss), _ptr(g, fp)),
                    "lfmm_surrogate_loss_grad")
        return loss.value, g

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.lfmm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class LayeredFMMBatch:
    """Many built problems (``LayeredFMM`` objects) evaluated together: one
    CUDA graph launch per evaluation when ``graph`` is true (see
    ``lfmm_batch_create`` in include/lfmm.h).  The members must stay open
    while the batch is used."""

    def __init__(self, members, nrhs=None, graph: bool = True):
        lib = load()
        self._lib = lib
        self.members = list(members)
        k = len(self.members)
        arr = (_ctxp * k)(*[m._ctx for m in self.members])
        nr = None if nrhs is None else np.ascontiguousarray(nrhs, dtype=np.int32)
        self.nrhs = [1] * k if nrhs is None else [int(v) for v in nr]
        h = _vp()
        st = lib.lfmm_batch_create(arr, k, _ptr(nr, _ip) if nr is not None else None, 1 if graph else 0,
                                   ctypes.byref(h))
        if st != OK:
            raise LfmmError(st, "lfmm_batch_create")
        self._b = h
        off = np.zeros(k + 1, dtype=np.int64)
        self._check(lib.lfmm_batch_offsets(self._b, _ptr(off, _lp)), "lfmm_batch_offsets")
        self.offsets = off
        self.total = int(off[-1])

    def _check(self, st, what):
        if st != OK:
            msg = self._lib.lfmm_batch_last_error(self._b)
            raise LfmmError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def concat(self, qs):
        """Per-problem charge arrays ([n_i] or [nrhs_i, n_i]) -> one concatenated host array."""
        return np.concatenate([_f64(q).ravel() for q in qs])

    def split(self, a, field=False):
        out = []
        for i, m in enumerate(self.members):
            o0, o1 = int(self.offsets[i]), int(self.offsets[i + 1])
            if field:
                v = a[3 * o0:3 * o1].reshape(self.nrhs[i], m.n, 3)
            else:
                v = a[o0:o1].reshape(self.nrhs[i], m.n)
            out.append(v[0] if self.nrhs[i] == 1 else v)
        return out

    def evaluate(self, qs, field: bool = True):
        """qs: list of per-problem host charges -> (list of phi, list of E or None)."""
        q = self.concat(qs)
        if q.shape[0] != self.total:
            raise ValueError("need %d charges in all, got %d" % (self.total, q.shape[0]))
        phi = np.zeros(self.total)
        fld = np.zeros(3 * self.total) if field else None
        self._check(self._lib.lfmm_batch_evaluate(self._b, _ptr(q), _ptr(phi), _ptr(fld) if field else None),
                    "lfmm_batch_evaluate")
        return self.split(phi), (self.split(fld, True) if field else None)

    def evaluate_host(self, q, phi, field=None):
        """Concatenated host arrays (float64, e.g. pinned torch tensors' numpy views) in and out."""
        self._check(self._lib.lfmm_batch_evaluate(self._b, _ptr(q), _ptr(phi),
                                                  _ptr(field) if field is not None else None),
                    "lfmm_batch_evaluate")

    def evaluate_device(self, q, phi, field=None, stream=None):
        """Concatenated float64 CUDA tensors: q, phi [total], field [3 total] or None."""
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(self._lib.lfmm_batch_evaluate_device(self._b, ctypes.c_void_p(q.data_ptr()),
                                                         ctypes.c_void_p(phi.data_ptr()),
                                                         ctypes.c_void_p(field.data_ptr())
                                                         if field is not None else None, s),
                    "lfmm_batch_evaluate_device")

    def info(self) -> dict:
        out = np.zeros(len(BATCH_INFO), dtype=np.int64)
        self._check(self._lib.lfmm_batch_info(self._b, _ptr(out, _lp), len(BATCH_INFO)), "lfmm_batch_info")
        return {k: int(v) for k, v in zip(BATCH_INFO, out)}

    def autotune(self, reps: int = 3):
        """Tune the batch as a whole (lfmm_batch_autotune); one dict per timed setting."""
        rows = np.zeros((32, len(BATCH_TUNE_COLS)))
        n = ctypes.c_int(0)
        self._check(self._lib.lfmm_batch_autotune(self._b, int(reps), _ptr(rows), 32, ctypes.byref(n)),
                    "lfmm_batch_autotune")
        return [dict(zip(BATCH_TUNE_COLS, r)) for r in rows[:n.value]]

    def close(self):
        if getattr(self, "_b", None):
            self._lib.lfmm_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
