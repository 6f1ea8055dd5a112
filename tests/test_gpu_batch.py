"""ht_truncate_batch: many HT tensors of uneven d, n and rank, each level of
all tensors in one batched launch, against the oracle tensor by tensor.

The tensors follow the batched recipe at reduced size (d in 4..9, n in
12..90, k in 3..16; each the sum of 4 tensors with sigma_j = 2^-j, truncated
back to its k), so that the oracle finishes in seconds."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, check_sigma, sample_idx, split_sigma

pytestmark = pytest.mark.gpu


def _sum4(spec, dtype):
    d, n, k, s = spec
    terms = I.batched_terms(spec)
    tree = htgb.HTTree(d)
    X = None
    ko, xo = None, None
    for (nv, kv, xv) in terms:
        T = htgb.HTTensor.from_blob(tree, nv, kv, xv, dtype)
        X = T if X is None else X.add(T)
        xs = as_stored(xv, dtype)
        if ko is None:
            ko, xo = kv, xs
        else:
            ko, xo = O.add(d, nv, ko, xo, kv, xs)
    return tree, terms[0][0], X, ko, xo


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
def test_truncate_batch_uneven(dtype):
    specs = I.batched_specs(count=7, seed=5, d_range=(4, 9), n_range=(12, 90), k_range=(3, 16))
    built = [_sum4(sp, dtype) for sp in specs]
    xs = [b[2] for b in built]
    # every tensor goes back to its own k (per-tensor rank caps), all in one call
    caps = [sp[2] for sp in specs]
    prec = htgb.HT_PREC_FP64 if dtype == htgb.HT_F64 else htgb.HT_PREC_FP32
    tol = 1e-12 if dtype == htgb.HT_F64 else 1e-6
    opts = htgb.make_opts(mode="rank", rank_cap=1, prec=prec, tensor_caps=caps)
    reps = htgb.ht_truncate_batch([x.handle for x in xs], opts, report=True)
    for i, rep in enumerate(reps):
        d, n, k, s = specs[i]
        tree, nvec, X, kin, xin = built[i]
        ref = O.truncate(d, nvec, kin, xin, mode="rank", rank_cap=k)
        assert list(X.ranks()) == list(ref["k"])
        assert max(X.ranks()[1:]) <= k
        assert abs(rep["norm"] - ref["norm"]) <= tol * ref["norm"]
        idx = sample_idx(nvec, 150, i)
        got = X.eval(idx)
        want = O.eval_entries(d, nvec, ref["k"], ref["x"], idx)
        assert np.abs(got - want).max() <= 10 * tol * ref["norm"], (i, specs[i])


def test_batch_equals_single_calls():
    """One batched call gives the same tensors as one call per tensor."""
    specs = I.batched_specs(count=5, seed=9, d_range=(4, 7), n_range=(10, 40), k_range=(4, 8))
    out = []
    for mode in ("batch", "single"):
        built = [_sum4(sp, htgb.HT_F64) for sp in specs]
        opts = htgb.make_opts(mode="rank", rank_cap=4, prec=htgb.HT_PREC_FP64)
        if mode == "batch":
            htgb.ht_truncate_batch([b[2].handle for b in built], opts)
        else:
            for b in built:
                htgb.ht_truncate(b[2].handle, opts)
        out.append([b[2].eval(sample_idx(b[1], 60, 2)) for b in built])
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-13 * max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
def test_batch_mixed_gramian_sizes(dtype):
    """One batch whose eigen launch holds Gramians of 4..140 rows: the launch's
    shared-memory layout is decided by its largest Gramian (above 128 rows the
    eigenvectors live in global scratch for every item, above 64 the FP64
    refinement does), and every item must follow it."""
    big_n = [300, 200, 250, 180]
    sig = lambda j: 0.9 ** j  # 10% gaps between neighbouring singular values: a well-posed cut
    ht = lambda d, nn, k, s: I.random_ht(d, nn, k, s, "gauss", sig)
    small_n, mid_n = [20, 9, 14, 11, 30], [40, 50, 60]
    cases = [(4, big_n, ht(4, big_n, 70, 51), ht(4, big_n, 70, 52), 60),
             (5, small_n, ht(5, small_n, 4, 53), ht(5, small_n, 4, 54), 3),
             (3, mid_n, ht(3, mid_n, 30, 55), ht(3, mid_n, 30, 56), 20)]
    xs, refs = [], []
    for d, nn, a, c, cap in cases:
        tree = htgb.HTTree(d)
        A = htgb.HTTensor.from_blob(tree, a[0], a[1], a[2], dtype)
        C = htgb.HTTensor.from_blob(tree, c[0], c[1], c[2], dtype)
        xs.append(A.add(C))
        k, x = O.add(d, a[0], a[1], as_stored(a[2], dtype), c[1], as_stored(c[2], dtype))
        refs.append((d, a[0], O.truncate(d, a[0], k, x, mode="rank", rank_cap=cap)))
    prec = htgb.HT_PREC_FP64 if dtype == htgb.HT_F64 else htgb.HT_PREC_FP32
    opts = htgb.make_opts(mode="rank", rank_cap=1, prec=prec, tensor_caps=[cs[-1] for cs in cases])
    htgb.ht_truncate_batch([x.handle for x in xs], opts)
    tol = 1e-12 if dtype == htgb.HT_F64 else 1e-5
    for i, (X, (d, nvec, ref)) in enumerate(zip(xs, refs)):
        assert list(X.ranks()) == list(ref["k"])
        idx = sample_idx(nvec, 200, i)
        got = X.eval(idx)
        want = O.eval_entries(d, nvec, ref["k"], ref["x"], idx)
        assert np.abs(got - want).max() <= tol * ref["norm"], i


def test_batched_wave_in_benchmark_configuration():
    """The batched workload as the benchmark runs it: a CUDA graph over a wave
    of uneven tensors (sums of 4, ranks 4k up to 192, per-tensor caps), FP32
    path.  The three cheapest tensors of the wave are recomputed by the oracle
    (on the FP32-rounded addends) and compared entrywise; every tensor's ranks
    obey its cap."""
    specs = I.batched_specs(count=4096, seed=41)[:16]
    dtype = htgb.HT_F32
    A, C, X, trees = [], [], [], []
    for (d, n, k, s) in specs:
        tr = htgb.HTTree(d)
        trees.append(tr)
        T = [htgb.HTTensor.from_blob(tr, nv, kv, xv, dtype) for (nv, kv, xv) in I.batched_terms((d, n, k, s))]
        a, c = T[0].add(T[1]), T[2].add(T[3])
        kk = a.ranks() + c.ranks()
        kk[0] = 1
        A.append(a), C.append(c), X.append(htgb.HTTensor.create(tr, a.n, kk, dtype))
    opts = htgb.make_opts(mode="rank", prec=htgb.HT_PREC_FP32, tensor_caps=[sp[2] for sp in specs])
    g = htgb.ht_graph_add_truncate([a.handle for a in A], [c.handle for c in C], [x.handle for x in X], opts)
    try:
        htgb.ht_graph_launch(g)
        for x, sp in zip(X, specs):
            assert max(x.ranks()[1:]) <= sp[2]
        cost = [(sp[0] - 2) * (4 * sp[2]) ** 4 + sp[0] * sp[1] * (4 * sp[2]) ** 2 for sp in specs]
        for i in np.argsort(cost)[:3]:
            d, n, k, s = specs[i]
            terms = I.batched_terms((d, n, k, s))
            nv = terms[0][0]
            kk, xx = terms[0][1], as_stored(terms[0][2], dtype)
            for (_, kv, xv) in terms[1:]:
                kk, xx = O.add(d, nv, kk, xx, kv, as_stored(xv, dtype))
            ref = O.truncate(d, nv, kk, xx, mode="rank", rank_cap=k)
            assert list(X[i].ranks()) == list(ref["k"])
            idx = sample_idx(nv, 200, int(i))
            got = X[i].eval(idx)
            want = O.eval_entries(d, nv, ref["k"], ref["x"], idx)
            assert np.abs(got - want).max() <= 1e-5 * ref["norm"], (i, specs[i])
    finally:
        htgb.ht_graph_free(g)
