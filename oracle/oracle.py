"""ctypes wrapper of the CPU FP64 oracle (``ht_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product library never imports, links or calls anything in this directory.

Each function restates one step of the paper (Grasedyck & Loebbert,
"Distributed Hierarchical SVD in the Hierarchical Tucker Format"); the C
source cites the section and equation of each.  Tensors are passed as
(ranks, blob): ``ranks`` has one entry per tree node in pre-order (root = 1)
and ``blob`` is the packed float64 array described in ``ht_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_LIB = os.path.join(_HERE, "libhtoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into ``oracle/libhtoracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int)
            f64p = ctypes.POINTER(ctypes.c_double)
            lib.ho_set_threads.argtypes = [ctypes.c_int]
            lib.ho_tree_info.argtypes = [ctypes.c_int] + [i32p] * 7
            lib.ho_size.argtypes = [ctypes.c_int, i64p, i32p]
            lib.ho_size.restype = ctypes.c_int64
            lib.ho_add.argtypes = [ctypes.c_int, i64p, i32p, f64p, i32p, f64p, i32p, f64p]
            lib.ho_orthogonalize.argtypes = [ctypes.c_int, i64p, i32p, f64p, f64p]
            lib.ho_gramians.argtypes = [ctypes.c_int, i64p, i32p, f64p, f64p]
            lib.ho_truncate.argtypes = [ctypes.c_int, i64p, i32p, f64p, ctypes.c_void_p, i32p, f64p, f64p, f64p]
            lib.ho_eval.argtypes = [ctypes.c_int, i64p, i32p, f64p, ctypes.c_int64, i64p, f64p]
            lib.ho_inner.argtypes = [ctypes.c_int, i64p, i32p, f64p, i32p, f64p]
            lib.ho_inner.restype = ctypes.c_double
            lib.ho_apply.argtypes = [ctypes.c_int, i64p, i64p, i32p, f64p, i32p, f64p, i32p, f64p]
            lib.ho_qr.argtypes = [ctypes.c_int64, ctypes.c_int, f64p, f64p, f64p]
            lib.ho_eig_sym.argtypes = [ctypes.c_int, f64p, f64p, f64p]
            _lib = lib
    return _lib


class _Opts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("eps_relative", ctypes.c_int),
        ("rank_cap", ctypes.c_int),
        ("ranks", ctypes.POINTER(ctypes.c_int)),
        ("noise", ctypes.c_double),
    ]


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (0 = runtime default); returns the count in use."""
    return int(_load().ho_set_threads(int(n)))


def tree_info(d: int) -> dict:
    """Balanced dimension tree (Sec. 2.1, eq. "balanced") in pre-order."""
    nn = 2 * d - 1
    arrs = [np.zeros(nn, np.int32) for _ in range(7)]
    rc = _load().ho_tree_info(d, *[_p(a, ctypes.c_int) for a in arrs])
    if rc != nn:
        raise ValueError(f"bad d={d}")
    keys = ["lo", "hi", "parent", "son1", "son2", "depth", "height"]
    return dict(zip(keys, arrs))


def size(d, n, k) -> int:
    n, k = _i64(n), _i32(k)
    return int(_load().ho_size(d, _p(n, ctypes.c_int64), _p(k, ctypes.c_int)))


def add(d, n, ka, xa, kc, xc):
    """Lemma "sum of two H-tensors": returns (k_out, blob_out)."""
    n, ka, kc, xa, xc = _i64(n), _i32(ka), _i32(kc), _f64(xa), _f64(xc)
    kout = np.zeros(2 * d - 1, np.int32)
    lib = _load()
    # output size needs kout; compute it the same way as the C code (sum of ranks, root 1)
    kk = ka + kc
    kk[0] = 1
    out = np.zeros(size(d, n, kk), np.float64)
    rc = lib.ho_add(d, _p(n, ctypes.c_int64), _p(ka, ctypes.c_int), _p(xa, ctypes.c_double),
                    _p(kc, ctypes.c_int), _p(xc, ctypes.c_double), _p(kout, ctypes.c_int),
                    _p(out, ctypes.c_double))
    if rc:
        raise RuntimeError("ho_add failed")
    return kout, out


def orthogonalize(d, n, k, x):
    """Sec. 3.4 orthogonalization: returns (k_orth, blob_orth)."""
    n, k, x = _i64(n), _i32(k).copy(), _f64(x)
    out = np.zeros(x.size, np.float64)
    rc = _load().ho_orthogonalize(d, _p(n, ctypes.c_int64), _p(k, ctypes.c_int), _p(x, ctypes.c_double),
                                  _p(out, ctypes.c_double))
    if rc:
        raise RuntimeError("ho_orthogonalize failed")
    return k, out[: size(d, n, k)].copy()


def gramians(d, n, k, x):
    """Reduced Gramians (Sec. 3.3) of an orthogonal tensor: list of k_t x k_t arrays (root: [[1]])."""
    n, k, x = _i64(n), _i32(k), _f64(x)
    kk = k.copy()
    kk[0] = 1
    g = np.zeros(int(np.sum(kk.astype(np.int64) ** 2)), np.float64)
    rc = _load().ho_gramians(d, _p(n, ctypes.c_int64), _p(k, ctypes.c_int), _p(x, ctypes.c_double),
                             _p(g, ctypes.c_double))
    if rc:
        raise RuntimeError("ho_gramians failed")
    out, o = [], 0
    for t in range(2 * d - 1):
        kt = int(kk[t])
        out.append(g[o:o + kt * kt].reshape(kt, kt).copy())
        o += kt * kt
    return out


def truncate(d, n, k, x, mode="rank", eps=0.0, eps_relative=True, rank_cap=0, ranks=None, noise=0.0):
    """HSVD truncation T(X) (Sec. 3.3 after Sec. 3.4).

    Returns a dict with ``k`` (truncated ranks), ``x`` (truncated blob),
    ``korth`` (ranks after orthogonalization), ``sigma`` (list per node of
    the singular values, root entry empty), ``norm`` (||X||),
    ``discarded_sq`` (sum of discarded sigma^2, root pair counted once) and
    ``tail2`` (per-node squared threshold in eps mode).  ``noise``: charge
    per dropped eigenvalue in eps mode, relative to the node's largest
    eigenvalue (0, the default, is the plain rule on the computed tail).
    """
    n, x = _i64(n), _f64(x)
    kk = _i32(k).copy()
    korth = np.zeros_like(kk)
    out = np.zeros(x.size, np.float64)
    sig = np.zeros(max(1, int(np.sum(kk[1:]))), np.float64)
    info = np.zeros(4, np.float64)
    opts = _Opts()
    opts.mode = 1 if mode == "eps" else 0
    opts.eps = float(eps)
    opts.eps_relative = 1 if eps_relative else 0
    opts.rank_cap = int(rank_cap)
    opts.noise = float(noise)
    rk = None
    if ranks is not None:
        rk = _i32(ranks)
        opts.ranks = _p(rk, ctypes.c_int)
    rc = _load().ho_truncate(d, _p(n, ctypes.c_int64), _p(kk, ctypes.c_int), _p(x, ctypes.c_double),
                             ctypes.byref(opts), _p(korth, ctypes.c_int), _p(out, ctypes.c_double),
                             _p(sig, ctypes.c_double), _p(info, ctypes.c_double))
    if rc:
        raise RuntimeError("ho_truncate failed")
    sigma, o = [np.zeros(0)], 0
    for t in range(1, 2 * d - 1):
        sigma.append(sig[o:o + korth[t]].copy())
        o += int(korth[t])
    return dict(k=kk, x=out[: size(d, n, kk)].copy(), korth=korth, sigma=sigma, norm=float(info[0]),
                discarded_sq=float(info[1]), tail2=float(info[2]))


def eval_entries(d, n, k, x, idx):
    """Entry evaluation (Sec. 3.1, eq. "transfermult"); idx is m x d."""
    n, k, x = _i64(n), _i32(k), _f64(x)
    idx = _i64(np.atleast_2d(idx))
    m = idx.shape[0]
    out = np.zeros(m, np.float64)
    rc = _load().ho_eval(d, _p(n, ctypes.c_int64), _p(k, ctypes.c_int), _p(x, ctypes.c_double), m,
                         _p(idx, ctypes.c_int64), _p(out, ctypes.c_double))
    if rc:
        raise RuntimeError("ho_eval failed")
    return out


def inner(d, n, ka, xa, kc, xc) -> float:
    """<A, C> by the Phi recursion (Definition/Lemma "phi", Sec. 3.2)."""
    n, ka, kc, xa, xc = _i64(n), _i32(ka), _i32(kc), _f64(xa), _f64(xc)
    return float(_load().ho_inner(d, _p(n, ctypes.c_int64), _p(ka, ctypes.c_int), _p(xa, ctypes.c_double),
                                  _p(kc, ctypes.c_int), _p(xc, ctypes.c_double)))


def apply(d, n, m, kop, xop, kx, xx):
    """C = L X (Lemma "operator", Sec. 3.6): L an HT tensor over the index pairs
    (j_mu, i_mu), mode sizes m_mu n_mu, pair (j, i) flattened as j + i m_mu.
    Returns (kout, xout) with kout_t = kop_t kx_t, pair (p, i) as p kx_t + i."""
    n, m = _i64(n), _i64(m)
    if n.size == 1:
        n = np.full(d, int(n[0]), np.int64)
    if m.size == 1:
        m = np.full(d, int(m[0]), np.int64)
    kop, kx, xop, xx = _i32(kop), _i32(kx), _f64(xop), _f64(xx)
    kout = np.array([1] + [int(kop[t]) * int(kx[t]) for t in range(1, 2 * d - 1)], np.int32)
    xout = np.zeros(size(d, m, kout), np.float64)
    rc = _load().ho_apply(d, _p(n, ctypes.c_int64), _p(m, ctypes.c_int64), _p(kop, ctypes.c_int), _p(xop, ctypes.c_double),
                          _p(kx, ctypes.c_int), _p(xx, ctypes.c_double), _p(kout, ctypes.c_int), _p(xout, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("ho_apply failed")
    return kout, xout


def qr(a):
    """Own Householder QR: a = Q R, Q (m x p) orthonormal, R (p x n) upper trapezoidal."""
    a = np.asfortranarray(a, dtype=np.float64)
    m, nc = a.shape
    p = min(m, nc)
    q = np.zeros((p, m), np.float64)  # column-major storage of m x p
    r = np.zeros((p, nc), np.float64)
    _load().ho_qr(m, nc, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _p(q, ctypes.c_double),
                  _p(r, ctypes.c_double))
    return q.T.copy(), r


def eig_sym(a):
    """Own cyclic Jacobi: returns (w descending, V with V[:, c] the eigenvector of w[c])."""
    a = _f64(a)
    nr = a.shape[0]
    w = np.zeros(nr, np.float64)
    v = np.zeros((nr, nr), np.float64)  # column-major storage
    _load().ho_eig_sym(nr, _p(a, ctypes.c_double), _p(w, ctypes.c_double), _p(v, ctypes.c_double))
    return w, v.T.copy()
