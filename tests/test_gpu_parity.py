"""GPU path vs the CPU FP64 oracle, through the C-ABI, on the same seeded inputs.

Tolerances: FP64 path 1e-12 (normwise on sigma^2 per node, i.e.
|sigma_i^2 - sigma_oracle_i^2| <= 1e-12 sigma_max^2, and relative to ||X|| on
tensor entries); FP32 path 1e-6 on the same measures for sigma >= 1e-5 sigma_max.
Ranks (integers) must agree exactly; byte-moving steps (addition) bit-exactly.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, check_ranks, check_sigma, gpu_sum, noise_floor, sample_idx, split_sigma

pytestmark = pytest.mark.gpu

F64, F32 = htgb.HT_F64, htgb.HT_F32
TOL = {F64: 1e-12, F32: 1e-6}


def test_add_bit_exact():
    (n, ka, xa), (_, kc, xc) = I.small_pair(3)
    tree, A, C, X = gpu_sum(8, n, (n, ka, xa), (n, kc, xc), F64)
    k, x = O.add(8, n, ka, xa, kc, xc)
    assert list(X.ranks()) == list(k)
    assert np.array_equal(X.download(), x)
    # uneven tree, unequal ranks
    a = I.random_ht(5, [3, 9, 2, 5, 4], 2, 7)
    c = I.random_ht(5, [3, 9, 2, 5, 4], 3, 8)
    tree, A, C, X = gpu_sum(5, a[0], a, c, F64)
    k, x = O.add(5, a[0], a[1], a[2], c[1], c[2])
    assert np.array_equal(X.download(), x)


def test_eval_entries():
    (n, ka, xa), _ = I.small_pair(5)
    tree = htgb.HTTree(8)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, F64)
    idx = sample_idx(n, 257)
    got = A.eval(idx)
    ref = O.eval_entries(8, n, ka, xa, idx)
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("case", ["small", "uneven", "tall", "wide_leaf", "d2", "big_rank", "rank128", "rank200"])
def test_orthogonalize(dtype, case):
    d, n, a, c = _case(case)
    tree, A, C, X = gpu_sum(d, n, a, c, dtype)
    k, x = O.add(d, n, a[1], as_stored(a[2], dtype), c[1], as_stored(c[2], dtype))
    ko_ref, xo_ref = O.orthogonalize(d, n, k, x)
    X.orthogonalize()
    ko = X.ranks()
    assert list(ko) == list(ko_ref)
    xo = X.download().astype(np.float64)
    nodes = I.blob_nodes(d, n, ko, xo)
    tr = I.tree(d)
    orth_tol = 1e-13 if dtype == F64 else 2e-6
    for t in range(1, 2 * d - 1):
        M = nodes[t] if tr["son1"][t] < 0 else nodes[t].reshape(nodes[t].shape[0], -1).T
        assert np.abs(M.T @ M - np.eye(M.shape[1])).max() <= orth_tol, t
    idx = sample_idx(n, 200)
    ref = O.eval_entries(d, n, k, x, idx)
    got = O.eval_entries(d, n, ko, xo, idx)
    scale = np.linalg.norm(nodes[0])
    assert np.abs(got - ref).max() <= TOL[dtype] * 10 * scale
    # ||X|| = ||B_D||_F
    ref_norm = np.linalg.norm(I.blob_nodes(d, n, ko_ref, xo_ref)[0])
    assert abs(scale - ref_norm) <= TOL[dtype] * ref_norm


def _case(case):
    if case == "small":
        (n, ka, xa), (_, kc, xc) = I.small_pair(2)
        return 8, n, (n, ka, xa), (n, kc, xc)
    if case == "uneven":
        nn = [7, 30, 12, 5, 40]
        return 5, np.array(nn), I.random_ht(5, nn, 4, 31), I.random_ht(5, nn, 3, 32)
    if case == "tall":  # leaf frames taller than one shared-memory block (multi-level TSQR)
        nn = [3000, 2500, 2100, 4000]
        return 4, np.array(nn), I.random_ht(4, nn, 9, 41), I.random_ht(4, nn, 7, 42)
    if case == "wide_leaf":  # n < k at the leaves: Q = I, R = U
        nn = [5, 3, 20, 6]
        return 4, np.array(nn), I.random_ht(4, nn, 4, 51), I.random_ht(4, nn, 3, 52)
    if case == "d2":
        nn = [40, 33]
        return 2, np.array(nn), I.random_ht(2, nn, 6, 61), I.random_ht(2, nn, 5, 62)
    if case == "big_rank":  # rank 81 > 64 after the addition: two QR panels
        nn = [700, 200, 450, 180]
        return 4, np.array(nn), I.random_ht(4, nn, 40, 71), I.random_ht(4, nn, 41, 72)
    if case == "rank128":  # rank 128: two full panels, leaves taller than one block
        nn = [600, 300, 520, 400]
        return 4, np.array(nn), I.random_ht(4, nn, 64, 81), I.random_ht(4, nn, 64, 82)
    if case == "rank200":  # rank 200: four panels (64, 64, 64, 8), n < k at one leaf
        nn = [700, 150, 420, 640]
        return 4, np.array(nn), I.random_ht(4, nn, 100, 91), I.random_ht(4, nn, 100, 92)
    raise ValueError(case)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_gramians(dtype):
    (n, ka, xa), (_, kc, xc) = I.small_pair(4)
    d = 8
    tree, A, C, X = gpu_sum(d, n, (n, ka, xa), (n, kc, xc), dtype)
    X.orthogonalize()
    ko = X.ranks()
    import torch
    sizes = [1] + [int(v) ** 2 for v in ko[1:]]
    buf = torch.zeros(sum(sizes), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    htgb.ht_gramians(X.handle, buf.data_ptr(), X.default_prec())
    torch.cuda.synchronize()
    g = buf.cpu().numpy()
    # oracle Gramians of the oracle's orthogonal tensor: compare spectra (frames differ by rotations)
    k, x = O.add(d, n, ka, as_stored(xa, dtype), kc, as_stored(xc, dtype))
    ko_ref, xo_ref = O.orthogonalize(d, n, k, x)
    G_ref = O.gramians(d, n, ko_ref, xo_ref)
    o = 1
    for t in range(1, 2 * d - 1):
        G = g[o:o + sizes[t]].reshape(int(ko[t]), int(ko[t]))
        o += sizes[t]
        lam = np.sort(np.linalg.eigvalsh(0.5 * (G + G.T)))[::-1]
        lam_ref = np.sort(np.linalg.eigvalsh(G_ref[t]))[::-1]
        assert np.abs(lam - lam_ref).max() <= TOL[dtype] * lam_ref[0], t


def _trunc_compare(d, n, a, c, dtype, opts, entries_tol_scale=10.0, floor=0.0, prec=None, tol=None, **kernel_opts):
    tree, A, C, X = gpu_sum(d, n, a, c, dtype)
    k, x = O.add(d, n, a[1], as_stored(a[2], dtype), c[1], as_stored(c[2], dtype))
    if prec is None:
        prec = htgb.HT_PREC_FP64 if dtype == F64 else htgb.HT_PREC_FP32
    tol = TOL[dtype] if tol is None else tol
    ref = O.truncate(d, n, k, x, noise=noise_floor(d, dtype, prec), **opts)
    rep = X.truncate(prec=prec, **opts, **kernel_opts)
    assert list(rep["korth"]) == list(ref["korth"])
    assert list(X.ranks()) == list(rep["ranks"])
    differ, energy = check_ranks(rep["ranks"], ref, tol, opts.get("mode") == "eps", d, dtype, prec)
    sg = split_sigma(rep["korth"], rep["sigma"])
    check_sigma(sg, ref["sigma"], tol, floor)
    assert abs(rep["norm"] - ref["norm"]) <= tol * ref["norm"]
    assert abs(rep["discarded_sq"] - ref["discarded_sq"]) <= tol * ref["norm"] ** 2 + 2 * energy ** 2
    idx = sample_idx(n, 300, 7)
    xt = X.download().astype(np.float64)
    got = O.eval_entries(d, n, X.ranks(), xt, idx)
    want = O.eval_entries(d, n, ref["k"], ref["x"], idx)
    # entries of T(X) relative to ||X|| (plus the effect of near-threshold rank decisions)
    assert np.abs(got - want).max() <= entries_tol_scale * tol * ref["norm"] + 2 * energy
    # the device-side evaluation agrees with the oracle's on the same data
    dev = X.eval(idx)
    assert np.abs(dev - got).max() <= 1e-12 * ref["norm"] + (1e-6 * ref["norm"] if dtype == F32 else 0.0)
    return rep, ref


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("case", ["small", "uneven", "tall", "wide_leaf", "d2", "big_rank", "rank128", "rank200"])
def test_truncate_rank(dtype, case):
    d, n, a, c = _case(case)
    r = {"small": 8, "uneven": 3, "tall": 5, "wide_leaf": 3, "d2": 4, "big_rank": 30, "rank128": 64,
         "rank200": 100}[case]
    _trunc_compare(d, n, a, c, dtype, dict(mode="rank", rank_cap=r))


@pytest.mark.parametrize("dtype", [F64, F32])
def test_truncate_eps(dtype):
    d, n, a, c = _case("small")
    _trunc_compare(d, n, a, c, dtype, dict(mode="eps", eps=1e-3, eps_relative=True))


@pytest.mark.parametrize("dtype", [F64, F32])
def test_truncate_to_ranks_per_node(dtype):
    """Target ranks given per node: 0 keeps every rank left after
    orthogonalization, the root's two sons keep the smaller of their targets."""
    d, n, a, c = _case("uneven")
    ranks = np.array([1, 4, 2, 3, 5, 0, 3, 2, 4])
    rep, ref = _trunc_compare(d, n, a, c, dtype, dict(mode="rank", ranks=ranks))
    assert list(ref["k"]) == [1, 4, 2, 3, 4, 7, 3, 2, 4]


def test_truncate_x_plus_x():
    (n, ka, xa), _ = I.small_pair(9)
    d = 8
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, F64)
    X = A.add(A)
    X.truncate(mode="rank", rank_cap=8)
    assert list(X.ranks()) == [1] + [8] * (2 * d - 2)
    idx = sample_idx(n, 300, 3)
    got = X.eval(idx)
    want = 2.0 * O.eval_entries(d, n, ka, xa, idx)
    scale = 2.0 * A.norm()  # ||2X||
    assert np.abs(got - want).max() <= 1e-12 * scale


def test_truncate_eps_zero_keeps_tensor():
    d, n, a, c = _case("small")
    tree, A, C, X = gpu_sum(d, n, a, c, F64)
    idx = sample_idx(n, 200, 5)
    before = X.eval(idx)
    scale = X.norm()
    X.truncate(mode="eps", eps=0.0, eps_relative=False)
    after = X.eval(idx)
    assert np.abs(after - before).max() <= 1e-12 * scale


def test_norm_and_scale():
    d, n, a, c = _case("uneven")
    tree, A, C, X = gpu_sum(d, n, a, c, F64)
    k, x = O.add(d, n, a[1], a[2], c[1], c[2])
    ref = O.truncate(d, n, k, x, mode="eps", eps=0.0)["norm"]
    assert abs(X.norm() - ref) <= 1e-13 * ref
    X.scale(-2.0)
    assert abs(X.norm() - 2 * ref) <= 1e-13 * ref


def test_node_schedule_matches_level_schedule():
    d, n, a, c = _case("uneven")
    out = []
    for sched in [htgb.HT_SCHED_LEVEL, htgb.HT_SCHED_NODE]:
        tree, A, C, X = gpu_sum(d, n, a, c, F64)
        rep = X.truncate(mode="rank", rank_cap=3, schedule=sched)
        out.append((rep, X.eval(sample_idx(n, 100, 1))))
    assert list(out[0][0]["ranks"]) == list(out[1][0]["ranks"])
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-13 * np.abs(out[0][1]).max()


def test_golden_diagonal_tensor():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "diag_d4.json")))
    d, n = g["d"], np.array(g["n"])
    tree = htgb.HTTree(d)
    X = htgb.HTTensor.from_blob(tree, n, g["ranks"], np.array(g["blob"]), F64)
    rep = X.truncate(mode="rank", rank_cap=g["rank"])
    sg = split_sigma(rep["korth"], rep["sigma"])
    for t in range(1, 2 * d - 1):
        assert np.abs(sg[t] - np.array(g["sigma"])).max() <= 1e-14
    assert abs(rep["norm"] - g["norm"]) <= 1e-14
    assert abs(np.sqrt(rep["discarded_sq"] / (2 * d - 3)) - g["trunc_err"]) <= 1e-13


@pytest.mark.parametrize("case", ["big_rank", "rank128", "rank200"])
def test_two_column_qr_kernel(case):
    """The two-column TSQR block kernel (two blocks per SM, chosen for FP32
    launches of 64-column blocks with more blocks than SMs) forced onto every
    such launch (qr_kernel = 2), then the one-column kernel forced everywhere
    (qr_kernel = 1): both truncations against the oracle."""
    d, n, a, c = _case(case)
    r = {"big_rank": 30, "rank128": 64, "rank200": 100}[case]
    for qk in (2, 1):
        _trunc_compare(d, n, a, c, F32, dict(mode="rank", rank_cap=r), qr_kernel=qk)