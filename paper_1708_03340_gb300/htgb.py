"""Thin ctypes binding of ``libhtgb.so`` (C-ABI in ``include/htgb.h``).

Only argument marshalling lives here; every step of the truncation runs in
the library's CUDA kernels.  The binding refuses to run without the built
library (no CPU fallback): ``load()`` raises if ``libhtgb.so`` is missing and
cannot be built.

Function names follow the C-ABI.  ``HTTensor`` is a small owner of an
``ht_tensor*`` handle with numpy conversions of the packed blob.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhtgb.so")

HT_OK, HT_EINVAL, HT_ENOMEM, HT_ECUDA, HT_ETIMEOUT, HT_ENUMERIC, HT_EUNSUPPORTED = range(7)
HT_F64, HT_F32 = 0, 1
HT_PREC_FP64, HT_PREC_FP32, HT_PREC_FP32_SQRT, HT_PREC_MIXED = 0, 1, 2, 3
HT_TRUNC_RANK, HT_TRUNC_EPS = 0, 1
HT_SCHED_LEVEL, HT_SCHED_NODE = 0, 1

# every symbol the header declares (checked by the ABI test)
EXPORTS = [
    "ht_tree_balanced", "ht_tree_free", "ht_tree_num_nodes", "ht_tree_node",
    "ht_tensor_create", "ht_tensor_free", "ht_tensor_ranks", "ht_tensor_blob_size",
    "ht_tensor_upload", "ht_tensor_download", "ht_tensor_node_ptr", "ht_scale",
    "ht_add", "ht_add_into", "ht_orthogonalize", "ht_gramians", "ht_truncate",
    "ht_truncate_batch", "ht_norm", "ht_eval_entries", "ht_last_error",
    "ht_profile_set", "ht_profile_read", "ht_launch_count", "ht_gramians_noalloc",
    "ht_graph_add_truncate", "ht_graph_launch", "ht_graph_kernels", "ht_graph_free", "ht_inner", "ht_apply",
    "ht_device_status", "ht_selftest_wait", "ht_set_gemm_tuning",
]
HT_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
HT_K_GEMM, HT_K_QR, HT_K_EIG, HT_K_COPY, HT_K_COMPACT, HT_K_RANKS, HT_K_ADD, HT_K_EVAL, HT_K_MISC, HT_K_SPLIT = range(10)
KERNEL_KINDS = ["gemm", "qr", "eig", "copy", "compact", "ranks", "add", "eval", "misc", "split"]


class HTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"htgb status {status}: {msg}")
        self.status = status


class TruncOpts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("eps_relative", ctypes.c_int),
        ("rank_cap", ctypes.c_int),
        ("ranks", ctypes.POINTER(ctypes.c_int)),
        ("prec", ctypes.c_int),
        ("schedule", ctypes.c_int),
        ("tensor_caps", ctypes.POINTER(ctypes.c_int)),
        ("qr_kernel", ctypes.c_int),
    ]


class TruncReport(ctypes.Structure):
    _fields_ = [
        ("norm", ctypes.c_double),
        ("discarded_sq", ctypes.c_double),
        ("bound", ctypes.c_double),
        ("ranks_out", ctypes.POINTER(ctypes.c_int)),
        ("korth_out", ctypes.POINTER(ctypes.c_int)),
        ("sigma_out", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libhtgb.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _b
            _b.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1708_03340_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64p, i32p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), \
            ctypes.POINTER(ctypes.c_double)
        sig = {
            "ht_tree_balanced": ([ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
            "ht_tree_free": ([vp], None),
            "ht_tree_num_nodes": ([vp], ctypes.c_int),
            "ht_tree_node": ([vp, ctypes.c_int] + [i32p] * 7, ctypes.c_int),
            "ht_tensor_create": ([vp, i64p, i32p, ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "ht_tensor_free": ([vp], ctypes.c_int),
            "ht_tensor_ranks": ([vp, i32p], ctypes.c_int),
            "ht_tensor_blob_size": ([vp, i64p], ctypes.c_int),
            "ht_tensor_upload": ([vp, vp], ctypes.c_int),
            "ht_tensor_download": ([vp, vp], ctypes.c_int),
            "ht_tensor_node_ptr": ([vp, ctypes.c_int, ctypes.POINTER(vp), i64p], ctypes.c_int),
            "ht_scale": ([vp, ctypes.c_double], ctypes.c_int),
            "ht_add": ([vp, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "ht_add_into": ([vp, vp, vp], ctypes.c_int),
            "ht_orthogonalize": ([vp, ctypes.c_int], ctypes.c_int),
            "ht_gramians": ([vp, vp, ctypes.c_int], ctypes.c_int),
            "ht_truncate": ([vp, ctypes.POINTER(TruncOpts), ctypes.POINTER(TruncReport)], ctypes.c_int),
            "ht_truncate_batch": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(TruncOpts),
                                   ctypes.POINTER(TruncReport)], ctypes.c_int),
            "ht_norm": ([vp, f64p], ctypes.c_int),
            "ht_eval_entries": ([vp, i64p, ctypes.c_int64, f64p], ctypes.c_int),
            "ht_last_error": ([], ctypes.c_char_p),
            "ht_profile_set": ([ctypes.c_uint], ctypes.c_int),
            "ht_profile_read": ([ctypes.c_int, i64p, f64p, f64p, ctypes.c_int], ctypes.c_int),
            "ht_launch_count": ([i64p], ctypes.c_int),
            "ht_device_status": ([], ctypes.c_int),
            "ht_gramians_noalloc": ([vp, vp, ctypes.c_int], ctypes.c_int),
            "ht_selftest_wait": ([ctypes.c_double, vp], ctypes.c_int),
            "ht_set_gemm_tuning": ([ctypes.c_int, ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "ht_graph_add_truncate": ([ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                       ctypes.POINTER(TruncOpts), ctypes.POINTER(vp)], ctypes.c_int),
            "ht_graph_launch": ([vp], ctypes.c_int),
            "ht_graph_kernels": ([vp, i32p], ctypes.c_int),
            "ht_graph_free": ([vp], ctypes.c_int),
            "ht_inner": ([vp, vp, f64p], ctypes.c_int),
            "ht_apply": ([vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _check(status):
    if status != HT_OK:
        msg = load().ht_last_error().decode(errors="replace")
        raise HTError(status, msg)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


# ---------------------------------------------------------------------------
# same names as the C-ABI
# ---------------------------------------------------------------------------

def ht_tree_balanced(d: int) -> int:
    h = ctypes.c_void_p()
    _check(load().ht_tree_balanced(int(d), ctypes.byref(h)))
    return h.value


def ht_tree_free(tree):
    load().ht_tree_free(tree)


def ht_tree_node(tree, t):
    vals = [ctypes.c_int() for _ in range(7)]
    _check(load().ht_tree_node(tree, int(t), *[ctypes.byref(v) for v in vals]))
    return dict(zip(["lo", "hi", "parent", "son1", "son2", "depth", "height"], [v.value for v in vals]))


def ht_tensor_create(tree, n, ranks, dtype=HT_F64, stream=None) -> int:
    n = np.ascontiguousarray(n, dtype=np.int64)
    r = np.ascontiguousarray(ranks, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().ht_tensor_create(tree, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(dtype),
                                   _stream_handle(stream), ctypes.byref(h)))
    return h.value


def ht_tensor_free(x):
    _check(load().ht_tensor_free(x))


def ht_tensor_ranks(x, nn):
    r = np.zeros(nn, np.int32)
    _check(load().ht_tensor_ranks(x, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return r


def ht_tensor_blob_size(x):
    c = ctypes.c_int64()
    _check(load().ht_tensor_blob_size(x, ctypes.byref(c)))
    return c.value


def ht_tensor_upload(x, host_array):
    _check(load().ht_tensor_upload(x, ctypes.c_void_p(host_array.ctypes.data)))


def ht_tensor_download(x, host_array):
    _check(load().ht_tensor_download(x, ctypes.c_void_p(host_array.ctypes.data)))


def ht_tensor_node_ptr(x, t):
    p, c = ctypes.c_void_p(), ctypes.c_int64()
    _check(load().ht_tensor_node_ptr(x, int(t), ctypes.byref(p), ctypes.byref(c)))
    return p.value, c.value


def ht_scale(x, alpha):
    _check(load().ht_scale(x, float(alpha)))


def ht_add(a, c) -> int:
    h = ctypes.c_void_p()
    _check(load().ht_add(a, c, ctypes.byref(h)))
    return h.value


def ht_add_into(a, c, out):
    _check(load().ht_add_into(a, c, out))


def ht_orthogonalize(x, prec=HT_PREC_FP64):
    _check(load().ht_orthogonalize(x, int(prec)))


def ht_gramians(x, dev_ptr, prec=HT_PREC_FP64):
    _check(load().ht_gramians(x, ctypes.c_void_p(dev_ptr), int(prec)))


def ht_gramians_noalloc(x, dev_ptr, prec=HT_PREC_FP64):
    """ht_gramians without any device allocation (fixed scratch inside the library)."""
    _check(load().ht_gramians_noalloc(x, ctypes.c_void_p(dev_ptr), int(prec)))


def make_opts(mode="rank", eps=0.0, eps_relative=True, rank_cap=0, ranks=None, prec=HT_PREC_FP64,
              schedule=HT_SCHED_LEVEL, tensor_caps=None, qr_kernel=0):
    o = TruncOpts()
    o.mode = HT_TRUNC_EPS if mode in ("eps", HT_TRUNC_EPS) else HT_TRUNC_RANK
    o.eps = float(eps)
    o.eps_relative = 1 if eps_relative else 0
    o.rank_cap = int(rank_cap)
    o.prec = int(prec)
    o.schedule = int(schedule)
    o.qr_kernel = int(qr_kernel)
    keep = None
    if ranks is not None:
        keep = np.ascontiguousarray(ranks, dtype=np.int32)
        o.ranks = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    keep_caps = None
    if tensor_caps is not None:
        keep_caps = np.ascontiguousarray(tensor_caps, dtype=np.int32)
        o.tensor_caps = keep_caps.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    o._keep = (keep, keep_caps)
    return o


def ht_truncate(x, opts: TruncOpts, report: bool = False, nn: int = 0, sigma_len: int = 0):
    if not report:
        _check(load().ht_truncate(x, ctypes.byref(opts), None))
        return None
    rk = np.zeros(nn, np.int32)
    ko = np.zeros(nn, np.int32)
    sg = np.zeros(max(sigma_len, 1), np.float64)
    rep = TruncReport()
    rep.ranks_out = rk.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rep.korth_out = ko.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rep.sigma_out = sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if sigma_len else None
    _check(load().ht_truncate(x, ctypes.byref(opts), ctypes.byref(rep)))
    return dict(norm=rep.norm, discarded_sq=rep.discarded_sq, bound=rep.bound, ranks=rk, korth=ko,
                sigma=sg[:sigma_len])


def ht_truncate_batch(xs, opts: TruncOpts, report: bool = False):
    arr = (ctypes.c_void_p * len(xs))(*xs)
    if not report:
        _check(load().ht_truncate_batch(arr, len(xs), ctypes.byref(opts), None))
        return None
    reps = (TruncReport * len(xs))()
    _check(load().ht_truncate_batch(arr, len(xs), ctypes.byref(opts), reps))
    return [dict(norm=r.norm, discarded_sq=r.discarded_sq, bound=r.bound) for r in reps]


def ht_graph_add_truncate(a, c, out, opts: TruncOpts):
    """Record out[i] = T(a[i] + c[i]) as one CUDA graph; returns its handle."""
    n = len(out)
    if len(a) != n or len(c) != n:
        raise ValueError("a, c and out must have the same length")
    arr = lambda hs: (ctypes.c_void_p * n)(*hs)
    g = ctypes.c_void_p()
    _check(load().ht_graph_add_truncate(arr(a), arr(c), arr(out), n, ctypes.byref(opts), ctypes.byref(g)))
    return g.value


def ht_graph_launch(g):
    _check(load().ht_graph_launch(g))


def ht_graph_kernels(g) -> int:
    k = ctypes.c_int()
    _check(load().ht_graph_kernels(g, ctypes.byref(k)))
    return k.value


def ht_graph_free(g):
    _check(load().ht_graph_free(g))


def ht_apply(op, x, out):
    _check(load().ht_apply(op, x, out))


def ht_inner(x, y) -> float:
    v = ctypes.c_double()
    _check(load().ht_inner(x, y, ctypes.byref(v)))
    return v.value


def ht_norm(x) -> float:
    v = ctypes.c_double()
    _check(load().ht_norm(x, ctypes.byref(v)))
    return v.value


def ht_eval_entries(x, idx) -> np.ndarray:
    idx = np.ascontiguousarray(np.atleast_2d(idx), dtype=np.int64)
    out = np.zeros(idx.shape[0], np.float64)
    _check(load().ht_eval_entries(x, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), idx.shape[0],
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def ht_profile_set(mask: int):
    _check(load().ht_profile_set(int(mask)))


def ht_profile_read(kind: int, reset: bool = True):
    """(launches, device ms, algorithmic flops) recorded for one kernel family."""
    n, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(load().ht_profile_read(int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl), 1 if reset else 0))
    return n.value, ms.value, fl.value


def ht_launch_count() -> int:
    n = ctypes.c_int64()
    _check(load().ht_launch_count(ctypes.byref(n)))
    return n.value


def ht_device_status() -> None:
    """Synchronises; raises HTError(HT_ETIMEOUT) if a kernel's bounded wait gave
    up, HTError(HT_ENUMERIC) if an eigensolver hit its iteration limit or a
    truncation met non-finite values, since the last call."""
    _check(load().ht_device_status())


def ht_selftest_wait(limit_ms: float, stream=None) -> None:
    """Enqueue the bounded-wait self-test kernel (its wait always runs out)."""
    _check(load().ht_selftest_wait(float(limit_ms), _stream_handle(stream)))


def ht_set_gemm_tuning(tall_m: int, tall_share: float, square_share: float) -> None:
    """Tile-shape rule of the SIMT contraction kernel (tall_m < 0: the committed table)."""
    _check(load().ht_set_gemm_tuning(int(tall_m), float(tall_share), float(square_share)))


# ---------------------------------------------------------------------------
# convenience owner
# ---------------------------------------------------------------------------

class HTTree:
    def __init__(self, d: int):
        self.d = int(d)
        self.nn = 2 * self.d - 1
        self.handle = ht_tree_balanced(self.d)

    def node(self, t):
        return ht_tree_node(self.handle, t)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            ht_tree_free(self.handle)
            self.handle = None


class HTTensor:
    """Owner of an ht_tensor handle.  ``from_blob`` uploads a packed float64 blob."""

    def __init__(self, tree: HTTree, handle: int, n, dtype: int):
        self.tree, self.handle, self.n, self.dtype = tree, handle, np.asarray(n, np.int64), dtype

    @classmethod
    def create(cls, tree: HTTree, n, ranks, dtype=HT_F64, stream=None):
        return cls(tree, ht_tensor_create(tree.handle, n, ranks, dtype, stream), n, dtype)

    @classmethod
    def from_blob(cls, tree: HTTree, n, ranks, blob, dtype=HT_F64, stream=None):
        x = cls.create(tree, n, ranks, dtype, stream)
        x.upload(blob)
        return x

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == HT_F64 else np.float32

    def upload(self, blob):
        a = np.ascontiguousarray(blob, dtype=self.np_dtype)
        ht_tensor_upload(self.handle, a)

    def ranks(self):
        return ht_tensor_ranks(self.handle, self.tree.nn)

    def download(self) -> np.ndarray:
        out = np.zeros(ht_tensor_blob_size(self.handle), self.np_dtype)
        ht_tensor_download(self.handle, out)
        return out

    def add(self, other: "HTTensor") -> "HTTensor":
        return HTTensor(self.tree, ht_add(self.handle, other.handle), self.n, self.dtype)

    def add_into(self, a: "HTTensor", c: "HTTensor"):
        """self = a + c (self created with capacities a.ranks + c.ranks)."""
        ht_add_into(a.handle, c.handle, self.handle)

    def orthogonalize(self, prec=None):
        ht_orthogonalize(self.handle, self.default_prec() if prec is None else prec)

    def default_prec(self):
        return HT_PREC_FP64 if self.dtype == HT_F64 else HT_PREC_FP32

    def truncate(self, report=True, **kw):
        kw.setdefault("prec", self.default_prec())
        o = make_opts(**kw)
        if not report:
            return ht_truncate(self.handle, o)
        nn = self.tree.nn
        # sigma length: korth is unknown before the call; the largest possible is sum of current ranks
        r = self.ranks()
        return ht_truncate(self.handle, o, True, nn, int(np.sum(r[1:])))

    def norm(self) -> float:
        return ht_norm(self.handle)

    def inner(self, other: "HTTensor") -> float:
        return ht_inner(self.handle, other.handle)

    def eval(self, idx) -> np.ndarray:
        return ht_eval_entries(self.handle, idx)

    def scale(self, alpha):
        ht_scale(self.handle, alpha)

    def free(self):
        if self.handle:
            ht_tensor_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                ht_tensor_free(self.handle)
                self.handle = None
        except Exception:
            pass
