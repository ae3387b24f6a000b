"""ctypes binding of include/h2eig.h: argument marshalling only.

Every entry point keeps its C name on the raw library object ``lib()``; the
``H2Matrix`` class wraps a handle.  Device-pointer entry points accept any
object with ``data_ptr()`` (a torch CUDA tensor) or a raw integer address.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

H2_K_LAPLACE_EPS, H2_K_YUKAWA_EPS, H2_K_GAUSS_PLUS_INV, H2_K_TRIDIAG_TEST, H2_K_MIN_TEST = 0, 1, 2, 3, 4
H2_ADM_BOX, H2_ADM_CENTER, H2_ADM_WEAK = 0, 1, 2
H2_PREC_FP64, H2_PREC_MIXED, H2_PREC_FP64_TC = 0, 1, 2

EXPORTED_SYMBOLS = ["h2_default_options", "h2_build", "h2_destroy", "h2_last_error", "h2_inertia",
                    "h2_inertia_device", "h2_kth_eig", "h2_info", "h2_tree_perm", "h2_level_ranks",
                    "h2_profile_batch", "h2_dense_inertia_noalloc", "h2_status", "h2_heartbeat",
                    "h2_group_create", "h2_group_inertia_device", "h2_group_launches", "h2_group_destroy",
                    "h2_autotune_choice", "h2_plan_summary", "h2_export", "h2_compression_error", "h2_kth_eig_in"]
KIND_NAMES = ["init", "recomp", "rotate", "ldl", "trsm", "schur", "merge", "other"]


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 4)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("admissibility", C.c_int), ("eps_h2", C.c_double),
                ("fill_cap", C.c_int), ("sketch_cols", C.c_int), ("seed", C.c_uint64),
                ("max_lanes", C.c_int), ("pivot_guard", C.c_double), ("stream", C.c_void_p),
                ("graphs", C.c_int), ("recomp_cluster_cols", C.c_int), ("autotune", C.c_int),
                ("hbm_budget", C.c_size_t), ("tc_schur", C.c_int), ("lookahead", C.c_int),
                ("shifts_per_interval", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int), ("leaves", C.c_int), ("max_rank", C.c_int),
                ("near_pairs", C.c_int64), ("fill_pairs", C.c_int64), ("norm_inf", C.c_double),
                ("gershgorin_lo", C.c_double), ("gershgorin_hi", C.c_double), ("trunc_tol", C.c_double),
                ("workspace_bytes", C.c_int64), ("lanes", C.c_int), ("kernels_per_batch", C.c_int),
                ("last_rounds", C.c_int), ("last_shifts", C.c_int64), ("last_mixed_rounds", C.c_int),
                ("guard_reruns", C.c_int64), ("bracket_resets", C.c_int64), ("cap_bound", C.c_int),
                ("max_residual", C.c_double), ("guard_checked", C.c_int64)]


class ExportBuf(C.Structure):
    _fields_ = [("level", C.c_int), ("nc", C.c_int), ("dq", C.c_int), ("nfar", C.c_int), ("rbmax", C.c_int),
                ("nnear", C.c_int), ("dm", C.c_int), ("offsets", C.c_void_p), ("ranks", C.c_void_p),
                ("residuals", C.c_void_p), ("colours", C.c_void_p), ("Q", C.c_void_p), ("far_pairs", C.c_void_p),
                ("C", C.c_void_p), ("near_pairs", C.c_void_p), ("B", C.c_void_p)]


class H2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("h2eig error %d: %s" % (code, msg))
        self.code = code


_LIB = None


def library_path() -> str:
    return os.path.join(HERE, "libh2eig.so")


def lib():
    """The loaded libh2eig.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError("libh2eig.so is not built: run `python -m paper_2311_08618_gb300.build`")
        L = C.CDLL(path)
        P = C.c_void_p
        L.h2_default_options.argtypes = [C.POINTER(Options)]
        L.h2_default_options.restype = None
        L.h2_build.argtypes = [P, C.c_int64, C.c_int, Kernel, C.c_int, C.c_int, C.c_double,
                               C.POINTER(Options), C.POINTER(P)]
        L.h2_destroy.argtypes = [P]
        L.h2_destroy.restype = None
        L.h2_last_error.restype = C.c_char_p
        L.h2_inertia.argtypes = [P, P, C.c_int64, P, P]
        L.h2_inertia_device.argtypes = [P, P, C.c_int64, P, P]
        L.h2_kth_eig.argtypes = [P, P, C.c_int64, C.c_double, P, P]
        L.h2_info.argtypes = [P, C.POINTER(Stats)]
        L.h2_tree_perm.argtypes = [P, P]
        L.h2_level_ranks.argtypes = [P, C.c_int, P]
        L.h2_profile_batch.argtypes = [P, P, C.c_int64, P, P, P, P, P]
        L.h2_dense_inertia_noalloc.argtypes = [P, C.c_int, C.c_int, P, C.c_int, P, P, P]
        L.h2_dense_inertia_noalloc.restype = C.c_int
        L.h2_heartbeat.argtypes = [P]
        L.h2_heartbeat.restype = None
        L.h2_status.argtypes = [P, P]
        L.h2_status.restype = C.c_int
        L.h2_group_create.argtypes = [P, C.c_int, C.POINTER(P)]
        L.h2_group_create.restype = C.c_int
        L.h2_group_inertia_device.argtypes = [P, P, P, P, P]
        L.h2_group_inertia_device.restype = C.c_int
        L.h2_group_launches.argtypes = [P]
        L.h2_group_launches.restype = C.c_int
        L.h2_group_destroy.argtypes = [P]
        L.h2_group_destroy.restype = None
        L.h2_autotune_choice.argtypes = [P, C.c_int, P]
        L.h2_autotune_choice.restype = C.c_int
        L.h2_plan_summary.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_int, P, P, P, P]
        L.h2_plan_summary.restype = C.c_int
        L.h2_kth_eig_in.argtypes = [P, P, C.c_int64, C.c_double, C.c_double, C.c_double, P, P]
        L.h2_kth_eig_in.restype = C.c_int
        L.h2_export.argtypes = [P, C.POINTER(ExportBuf)]
        L.h2_export.restype = C.c_int
        L.h2_compression_error.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.h2_compression_error.restype = C.c_int
        for f in ("h2_build", "h2_inertia", "h2_inertia_device", "h2_kth_eig", "h2_info",
                  "h2_tree_perm", "h2_level_ranks", "h2_profile_batch"):
            getattr(L, f).restype = C.c_int
        _LIB = L
    return _LIB


def _check(rc):
    if rc != 0:
        raise H2Error(rc, lib().h2_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(int(x))


def default_options() -> Options:
    o = Options()
    lib().h2_default_options(C.byref(o))
    return o


class H2Matrix:
    """A resident, factor-ready H^2 matrix (h2_build ... h2_destroy)."""

    def __init__(self, points, kernel: int, kparams=(1e-3, 0.0, 0.0, 0.0), leaf: int = 64,
                 rank: int = 16, eta: float = 1.0, **opts):
        pts = np.ascontiguousarray(points, dtype=np.float64)
        if pts.ndim == 1:
            pts = pts.reshape(-1, 1)
        o = default_options()
        for k, v in opts.items():
            if k == "stream" and v is not None and not isinstance(v, int):
                v = v.cuda_stream
            setattr(o, k, v)
        kr = Kernel(kernel, (C.c_double * 4)(*[float(v) for v in (list(kparams) + [0, 0, 0, 0])[:4]]))
        h = C.c_void_p()
        _check(lib().h2_build(pts.ctypes.data_as(C.c_void_p), pts.shape[0], pts.shape[1], kr, leaf, rank,
                              eta, C.byref(o), C.byref(h)))
        self._h = h
        self.n = pts.shape[0]

    def close(self):
        if getattr(self, "_h", None):
            lib().h2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def h2_inertia(self, shifts):
        s = np.ascontiguousarray(shifts, dtype=np.float64).ravel()
        counts = np.zeros(s.size, dtype=np.int64)
        mp = np.zeros(s.size, dtype=np.float64)
        _check(lib().h2_inertia(self._h, s.ctypes.data_as(C.c_void_p), s.size,
                                counts.ctypes.data_as(C.c_void_p), mp.ctypes.data_as(C.c_void_p)))
        return counts, mp

    def h2_inertia_device(self, d_shifts, ns, d_counts, d_minpiv=None):
        _check(lib().h2_inertia_device(self._h, _ptr(d_shifts), int(ns), _ptr(d_counts), _ptr(d_minpiv)))

    def h2_profile_batch(self, d_shifts, ns, d_counts):
        """Per kernel kind: (ms, launches, flops, bytes) of one profiled batch."""
        nk = len(KIND_NAMES)
        ms = np.zeros(nk)
        nl = np.zeros(nk, dtype=np.int64)
        fl = np.zeros(nk)
        by = np.zeros(nk)
        _check(lib().h2_profile_batch(self._h, _ptr(d_shifts), int(ns), _ptr(d_counts),
                                      ms.ctypes.data_as(C.c_void_p), nl.ctypes.data_as(C.c_void_p),
                                      fl.ctypes.data_as(C.c_void_p), by.ctypes.data_as(C.c_void_p)))
        return {k: {"ms": float(ms[i]), "launches": int(nl[i]), "flops": float(fl[i]), "bytes": float(by[i])}
                for i, k in enumerate(KIND_NAMES)}

    def h2_kth_eig(self, ks, tol):
        k = np.ascontiguousarray(ks, dtype=np.int64).ravel()
        out = np.zeros(k.size)
        eb = np.zeros(k.size)
        _check(lib().h2_kth_eig(self._h, k.ctypes.data_as(C.c_void_p), k.size, float(tol),
                                out.ctypes.data_as(C.c_void_p), eb.ctypes.data_as(C.c_void_p)))
        return out, eb

    def h2_kth_eig_in(self, ks, lo, hi, tol):
        """h2_kth_eig with every bracket starting from [lo, hi]."""
        k = np.ascontiguousarray(ks, dtype=np.int64).ravel()
        out = np.zeros(k.size)
        eb = np.zeros(k.size)
        _check(lib().h2_kth_eig_in(self._h, k.ctypes.data_as(C.c_void_p), k.size, float(lo), float(hi), float(tol),
                                   out.ctypes.data_as(C.c_void_p), eb.ctypes.data_as(C.c_void_p)))
        return out, eb

    def h2_info(self) -> dict:
        s = Stats()
        _check(lib().h2_info(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def h2_status(self):
        """(rc, info[8]) of the device error record (see include/h2eig.h)."""
        info = np.zeros(8, dtype=np.int64)
        rc = lib().h2_status(self._h, info.ctypes.data_as(C.c_void_p))
        return rc, info

    def h2_tree_perm(self):
        p = np.zeros(self.n, dtype=np.int64)
        _check(lib().h2_tree_perm(self._h, p.ctypes.data_as(C.c_void_p)))
        return p

    def h2_autotune_choice(self, level):
        """(threads per Bunch-Kaufman block: 32 for one warp, 128 or 256 for a
        CTA; 1 if the recompression is clustered) of a level."""
        out = np.zeros(2, dtype=np.int32)
        _check(lib().h2_autotune_choice(self._h, int(level), out.ctypes.data_as(C.c_void_p)))
        return int(out[0]), int(out[1])

    def h2_export(self, level):
        """One level of the resident representation (see h2_export in the
        header): dict with offsets, ranks, residuals, colours, Q [nc, dq, dq],
        far_pairs [nfar, 2], C [nfar, rbmax, rbmax], near_pairs, B."""
        b = ExportBuf()
        b.level = int(level)
        _check(lib().h2_export(self._h, C.byref(b)))
        out = {"offsets": np.zeros(b.nc + 1, dtype=np.int64), "ranks": np.zeros(b.nc, dtype=np.int32),
               "residuals": np.zeros(b.nc), "colours": np.zeros(b.nc, dtype=np.int32),
               "Q": np.zeros((b.nc, b.dq, b.dq)), "far_pairs": np.zeros((b.nfar, 2), dtype=np.int32),
               "C": np.zeros((b.nfar, b.rbmax, b.rbmax)), "near_pairs": np.zeros((b.nnear, 2), dtype=np.int32),
               "B": np.zeros((b.nnear, b.dm, b.dm))}
        for f in ("offsets", "ranks", "residuals", "colours", "Q", "far_pairs", "C", "near_pairs", "B"):
            setattr(b, f, out[f].ctypes.data_as(C.c_void_p) if out[f].size else None)
        _check(lib().h2_export(self._h, C.byref(b)))
        return out

    def h2_compression_error(self, iters=30):
        """(||A - A~||_2, ||A||_2) by power iteration on the device."""
        e = C.c_double()
        a = C.c_double()
        _check(lib().h2_compression_error(self._h, int(iters), C.byref(e), C.byref(a)))
        return e.value, a.value

    def h2_level_ranks(self, level):
        r = np.zeros(1 << level, dtype=np.int32)
        _check(lib().h2_level_ranks(self._h, int(level), r.ctypes.data_as(C.c_void_p)))
        return r


class H2Group:
    """One inertia batch over several resident H2Matrix handles (h2_group_create
    ... h2_group_destroy): one launch per tree level and colour for all of them.
    The handles must share max_lanes, precision and stream, and stay alive."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (C.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        g = C.c_void_p()
        _check(lib().h2_group_create(C.cast(arr, C.c_void_p), len(self.mats), C.byref(g)))
        self._g = g

    def close(self):
        if getattr(self, "_g", None):
            lib().h2_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launches(self) -> int:
        return int(lib().h2_group_launches(self._g))

    def h2_group_inertia_device(self, d_shifts, ns, d_counts, d_minpiv=None):
        """d_shifts, d_counts (, d_minpiv): device buffers of len(mats) * max_lanes;
        ns: shifts per handle (host sequence)."""
        n = np.ascontiguousarray(ns, dtype=np.int32).ravel()
        _check(lib().h2_group_inertia_device(self._g, _ptr(d_shifts), n.ctypes.data_as(C.c_void_p),
                                             _ptr(d_counts), _ptr(d_minpiv)))


def plan_summary(points, leaf: int, eta: float = 1.0, rule: int = 0):
    """h2_plan_summary: (perm, per-level [clusters, near, fill, far, colours],
    per-level colour arrays) of the structure h2_build would use (host only)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts.reshape(-1, 1)
    n, d = pts.shape
    perm = np.zeros(n, dtype=np.int64)
    lv = C.c_int(0)
    per = np.zeros(5 * 64, dtype=np.int64)
    _check(lib().h2_plan_summary(pts.ctypes.data_as(C.c_void_p), n, d, leaf, float(eta), rule,
                                 perm.ctypes.data_as(C.c_void_p), C.byref(lv), per.ctypes.data_as(C.c_void_p),
                                 None))
    L1 = lv.value
    per = per[:5 * L1].reshape(L1, 5)
    cols = np.zeros(int(per[:, 0].sum()), dtype=np.int32)
    _check(lib().h2_plan_summary(pts.ctypes.data_as(C.c_void_p), n, d, leaf, float(eta), rule,
                                 None, C.byref(lv), None, cols.ctypes.data_as(C.c_void_p)))
    out, pos = [], 0
    for l in range(L1):
        out.append(cols[pos:pos + per[l, 0]])
        pos += per[l, 0]
    return perm, per, out
