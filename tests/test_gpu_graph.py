"""CUDA-graph form of the hot path (ht_graph_add_truncate / ht_graph_launch):
one replay gives bit for bit what ht_add_into + ht_truncate_batch give on the
same inputs, replays are repeatable, and the result matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, sample_idx

pytestmark = pytest.mark.gpu


def _pairs(dtype):
    """Three small pairs (d=8, n=32, k=8, sigma_j = 2^-j) and one uneven pair."""
    out = []
    for s in (1, 3, 5):
        a, c = I.small_pair(s)
        out.append((8, a, c))
    nn = [40, 17, 33, 25, 9]
    out.append((5, I.random_ht(5, nn, 6, 7), I.random_ht(5, nn, 4, 8)))
    return out


def _build(dtype):
    trees, A, C, X = [], [], [], []
    for d, a, c in _pairs(dtype):
        tr = htgb.HTTree(d)
        ta = htgb.HTTensor.from_blob(tr, a[0], a[1], a[2], dtype)
        tc = htgb.HTTensor.from_blob(tr, c[0], c[1], c[2], dtype)
        cap = np.asarray(a[1]) + np.asarray(c[1])
        cap[0] = 1
        tx = htgb.HTTensor.create(tr, a[0], cap, dtype)
        trees.append(tr), A.append(ta), C.append(tc), X.append(tx)
    return trees, A, C, X


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
def test_graph_replay_equals_direct_calls(dtype):
    prec = htgb.HT_PREC_FP64 if dtype == htgb.HT_F64 else htgb.HT_PREC_FP32
    opts = htgb.make_opts(mode="rank", rank_cap=4, prec=prec)
    trees, A, C, X = _build(dtype)
    g = htgb.ht_graph_add_truncate([a.handle for a in A], [c.handle for c in C], [x.handle for x in X], opts)
    try:
        assert htgb.ht_graph_kernels(g) > 0
        htgb.ht_graph_launch(g)
        first = [(x.ranks().copy(), x.download().copy()) for x in X]
        htgb.ht_graph_launch(g)
        htgb.ht_graph_launch(g)
        again = [(x.ranks().copy(), x.download().copy()) for x in X]
    finally:
        htgb.ht_graph_free(g)
    # direct calls on fresh outputs
    _, A2, C2, X2 = _build(dtype)
    for x, a, c in zip(X2, A2, C2):
        x.add_into(a, c)
    htgb.ht_truncate_batch([x.handle for x in X2], opts)
    for (r1, b1), (r2, b2), x in zip(first, again, X2):
        assert list(r1) == list(r2) == list(x.ranks())
        assert np.array_equal(b1, b2)
        assert np.array_equal(b1, x.download())


def test_graph_matches_oracle():
    dtype = htgb.HT_F64
    opts = htgb.make_opts(mode="rank", rank_cap=8, prec=htgb.HT_PREC_FP64)
    trees, A, C, X = _build(dtype)
    g = htgb.ht_graph_add_truncate([a.handle for a in A], [c.handle for c in C], [x.handle for x in X], opts)
    try:
        htgb.ht_graph_launch(g)
        for i, ((d, a, c), x) in enumerate(zip(_pairs(dtype), X)):
            k, xs = O.add(d, a[0], a[1], a[2], c[1], c[2])
            ref = O.truncate(d, a[0], k, xs, mode="rank", rank_cap=8)
            assert list(x.ranks()) == list(ref["k"])
            idx = sample_idx(a[0], 200, i)
            got = x.eval(idx)
            want = O.eval_entries(d, a[0], ref["k"], ref["x"], idx)
            assert np.abs(got - want).max() <= 1e-12 * ref["norm"]
    finally:
        htgb.ht_graph_free(g)


def test_graph_rejects_bad_capacity():
    trees, A, C, X = _build(htgb.HT_F64)
    bad = htgb.HTTensor.create(trees[0], A[0].n, np.full(trees[0].nn, 3), htgb.HT_F64)
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_graph_add_truncate([A[0].handle], [C[0].handle], [bad.handle], htgb.make_opts(mode="rank", rank_cap=4))
    assert e.value.status == htgb.HT_EINVAL
