"""Seeded synthetic HT tensors: the input recipe of every workload.

This module only draws random numbers and lays them out.  It holds none of
the truncation arithmetic and is shared by the tests, the benchmark and the
CPU oracle's callers.  Random numbers come from a counter-based generator,
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) mapped to N(0,1) by the Box-Muller transform.

Layout of a tensor (the "packed blob", float64): nodes of the balanced
dimension tree in pre-order; a leaf {mu} stores U (n_mu x k) column-major, an
inner node t stores B_t (k_t x k_s1 x k_s2) with the last index fastest, the
root stores B_D (k_t1 x k_t2) row-major.  ``ranks`` has one entry per node,
the root's entry is 1.

Workload recipes (per node, "scaled along each mode j by sigma_j" means
B[a,b,c] = g_abc * sigma_a * sigma_b * sigma_c with 1-based a, b, c; every
inner transfer tensor is then scaled so that its first (largest) slice
B[1, :, :], weighted by the expected column norms of the sons' frames, has
unit norm, the root likewise as a whole, and every Gaussian leaf frame is
divided by sqrt(n) -- scalar factors of the whole tensor that keep ||X|| = O(1)
for deep trees without changing any singular value ratio, rank or relative
error):

* ``small``      d=8, n=32, k=8, Gaussian U, sigma_j = 2^-j  (two seeds added)
* ``brute``      d=4, n=8, k=4, as ``small``
* ``single``     d=64, n=1000, k=32, orthonormalised Gaussian U, sigma_j = 10^(-8j/32)
* ``batched``    4096 tensors, d~U{4..32}, n~U{16..512}, k~U{4..48}; each a sum of 4
                 ``small``-style tensors with sigma_j = 2^-j
* ``deep``       d=256, n=4096, k=64, Gaussian U, sigma_j = 10^(-10j/64)
* ``wide``       d=16, n=2048, k=128, orthonormalised Gaussian U, sigma_j = j^-2
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on uint64 arrays (wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _C1
    z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def _key(*parts: int) -> np.uint64:
    """Derive a stream key from integers (seed, node, purpose)."""
    with np.errstate(over="ignore"):
        k = np.uint64(0x243F6A8885A308D3)
        for p in parts:
            k = _mix(np.array([k + np.uint64(p & 0xFFFFFFFFFFFFFFFF) * _GAMMA], dtype=np.uint64))[0]
        return k


def uniform(key: np.uint64, count: int) -> np.ndarray:
    """count uniforms in (0, 1]: the i-th is a function of (key, i) only."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = _mix(key + i * _GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(key: np.uint64, count: int) -> np.ndarray:
    """count N(0,1) numbers by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(key, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, np.float64)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def randint(key: np.uint64, count: int, lo: int, hi: int) -> np.ndarray:
    """count integers uniform in {lo..hi}."""
    u = uniform(key, count)
    return np.minimum(lo + np.floor((1.0 - u) * (hi - lo + 1)).astype(np.int64), hi)


# ----------------------------------------------------------------------------
# dimension tree layout (pre-order), needed to lay nodes out
# ----------------------------------------------------------------------------

def tree(d: int) -> dict:
    """Balanced dimension tree in pre-order: lists lo, hi, son1, son2, parent.

    Node {mu..nu} (1-based) has sons {mu..floor((mu+nu-1)/2)} and the rest.
    """
    lo, hi, s1, s2, par = [], [], [], [], []

    def rec(a, b, p):
        i = len(lo)
        lo.append(a); hi.append(b); s1.append(-1); s2.append(-1); par.append(p)
        if a != b:
            last1 = (a + b + 1) // 2 - 1
            s1[i] = rec(a, last1, i)
            s2[i] = rec(last1 + 1, b, i)
        return i

    rec(0, d - 1, -1)
    return dict(lo=lo, hi=hi, son1=s1, son2=s2, parent=par, d=d)


def blob_size(d: int, n, ranks) -> int:
    tr = tree(d)
    n = np.broadcast_to(np.asarray(n, dtype=np.int64), (d,))
    s = 0
    for t in range(2 * d - 1):
        if tr["son1"][t] < 0:
            s += int(n[tr["lo"][t]]) * int(ranks[t])
        else:
            kt = 1 if t == 0 else int(ranks[t])
            s += kt * int(ranks[tr["son1"][t]]) * int(ranks[tr["son2"][t]])
    return s


def random_ht(d: int, n, k, seed: int, leaf: str = "gauss", sigma=None):
    """One random HT tensor.

    d: dimension; n: int or per-mode sizes; k: rank of every non-root node;
    leaf: "gauss" (i.i.d. N(0,1)) or "orth" (Q factor of a Gaussian, via
    numpy's Householder QR); sigma: function j -> weight (1-based j), or None.
    Returns (n_array[int64], ranks[int32], blob[float64]).
    """
    tr = tree(d)
    nn = 2 * d - 1
    n = np.broadcast_to(np.asarray(n, dtype=np.int64), (d,)).copy()
    ranks = np.full(nn, int(k), np.int32)
    ranks[0] = 1
    w = np.ones(int(k)) if sigma is None else np.array([sigma(j) for j in range(1, int(k) + 1)], np.float64)
    parts = []
    for t in range(nn):
        key = _key(seed, t, 1)
        if tr["son1"][t] < 0:
            nm = int(n[tr["lo"][t]])
            g = normal(key, nm * int(k)).reshape(int(k), nm).T  # column-major n x k
            if leaf == "orth":
                if nm < k:
                    raise ValueError("orthonormal leaf needs n >= k")
                g = np.linalg.qr(g)[0]
            else:
                # columns of unit expected norm: a scalar factor of the whole tensor that keeps
                # ||X|| finite for deep trees (256 leaves of norm sqrt(4096) would give ~64^256)
                g = g / np.sqrt(nm)
            parts.append(np.asfortranarray(g).ravel(order="F"))
        else:
            if t == 0:
                g = normal(key, int(k) * int(k)).reshape(int(k), int(k))
                b = g * w[:, None] * w[None, :]
            else:
                g = normal(key, int(k) ** 3).reshape(int(k), int(k), int(k))
                b = g * w[:, None, None] * w[None, :, None] * w[None, None, :]
            # scalar normalisation (a factor of the whole tensor that keeps ||X|| = O(1)
            # at any depth): column a of an inner node's frame has a norm close to
            # || b[a, :, :] weighted by the sons' column norms ||, the sons' columns
            # having norms 1 (leaves) or w_j / w_1 (inner nodes normalised this way);
            # the first (largest) column is scaled to norm 1, the root to unit norm
            def son_scale(s):
                return np.ones(int(k)) if tr["son1"][s] < 0 else w / w[0]
            s1, s2 = son_scale(tr["son1"][t]), son_scale(tr["son2"][t])
            if t == 0:
                parts.append((b / np.linalg.norm(b * s1[:, None] * s2[None, :])).ravel())
            else:
                parts.append((b / np.linalg.norm(b[0] * s1[:, None] * s2[None, :])).ravel())
    return n, ranks, np.concatenate(parts)


def blob_nodes(d: int, n, ranks, blob) -> list:
    """Split a blob into per-node arrays: leaves (n x k), inner (kt, k1, k2), root (k1, k2)."""
    tr = tree(d)
    n = np.broadcast_to(np.asarray(n, dtype=np.int64), (d,))
    out, o = [], 0
    for t in range(2 * d - 1):
        if tr["son1"][t] < 0:
            nm, kt = int(n[tr["lo"][t]]), int(ranks[t])
            out.append(blob[o:o + nm * kt].reshape(kt, nm).T)
            o += nm * kt
        else:
            k1, k2 = int(ranks[tr["son1"][t]]), int(ranks[tr["son2"][t]])
            kt = 1 if t == 0 else int(ranks[t])
            a = blob[o:o + kt * k1 * k2]
            out.append(a.reshape(k1, k2) if t == 0 else a.reshape(kt, k1, k2))
            o += kt * k1 * k2
    return out


def nodes_blob(d: int, nodes: list) -> np.ndarray:
    """Inverse of blob_nodes."""
    tr = tree(d)
    parts = []
    for t, a in enumerate(nodes):
        if tr["son1"][t] < 0:
            parts.append(np.asarray(a, np.float64).ravel(order="F"))
        else:
            parts.append(np.asarray(a, np.float64).ravel())
    return np.concatenate(parts)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def small_pair(seed: int = 1, d: int = 8, n: int = 32, k: int = 8):
    """``small``: two d=8, n=32, k=8 tensors (seeds s, s+1), Gaussian leaves, sigma_j = 2^-j.
    Truncated back to rank k after the addition."""
    sig = lambda j: 2.0 ** (-j)
    a = random_ht(d, n, k, seed, "gauss", sig)
    c = random_ht(d, n, k, seed + 1, "gauss", sig)
    return a, c


def brute_pair(seed: int = 1):
    """``brute``: the d=4, n=8, k=4 variant of ``small`` for full-tensor checks."""
    return small_pair(seed, d=4, n=8, k=4)


def single_pair(seed: int = 11, d: int = 64, n: int = 1000, k: int = 32):
    """``single``: d=64, n=1000, k=32, orthonormalised Gaussian leaves,
    sigma_j = 10^(-8j/32); the sum (rank 64) is truncated to relative eps=1e-8
    with rank cap 32."""
    sig = lambda j: 10.0 ** (-8.0 * j / 32.0)
    return random_ht(d, n, k, seed, "orth", sig), random_ht(d, n, k, seed + 1, "orth", sig)


SINGLE_OPTS = dict(mode="eps", eps=1e-8, eps_relative=True, rank_cap=32)


def deep_pair(seed: int = 21, d: int = 256, n: int = 4096, k: int = 64):
    """``deep``: d=256, n=4096, k=64, Gaussian leaves, sigma_j = 10^(-10j/64); eps=1e-6 relative."""
    sig = lambda j: 10.0 ** (-10.0 * j / 64.0)
    return random_ht(d, n, k, seed, "gauss", sig), random_ht(d, n, k, seed + 1, "gauss", sig)


DEEP_OPTS = dict(mode="eps", eps=1e-6, eps_relative=True, rank_cap=0)


def wide_pair(seed: int = 31, d: int = 16, n: int = 2048, k: int = 128):
    """``wide``: d=16, n=2048, k=128, orthonormalised Gaussian leaves, sigma_j = j^-2; rank 128."""
    sig = lambda j: float(j) ** -2.0
    return random_ht(d, n, k, seed, "orth", sig), random_ht(d, n, k, seed + 1, "orth", sig)


WIDE_OPTS = dict(mode="rank", rank_cap=128)


def batched_specs(count: int = 4096, seed: int = 41, d_range=(4, 32), n_range=(16, 512), k_range=(4, 48)):
    """``batched``: per tensor (d, n, k, seed) with d, n, k uniform in the ranges."""
    key = _key(seed, 0, 7)
    ds = randint(_key(seed, 1, 7), count, *d_range)
    ns = randint(_key(seed, 2, 7), count, *n_range)
    ks = randint(_key(seed, 3, 7), count, *k_range)
    del key
    return [(int(ds[i]), int(ns[i]), int(ks[i]), int(seed * 1000003 + i * 17)) for i in range(count)]


def batched_terms(spec, terms: int = 4):
    """The 4 addends of one ``batched`` tensor: ``small``-style with sigma_j = 2^-j."""
    d, n, k, s = spec
    sig = lambda j: 2.0 ** (-j)
    return [random_ht(d, n, k, s + 101 * i, "gauss", sig) for i in range(terms)]
