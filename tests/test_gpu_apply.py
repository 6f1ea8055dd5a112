"""ht_apply (Lemma "operator", Sec. 3.6): C = L X on the GPU against the
oracle's operator application (pinned against the full operator-times-tensor
product), then the truncation of C against the oracle's."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, sample_idx

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "d4":
        d, m, n = 4, [3, 5, 2, 4], [4, 6, 3, 5]
        op = I.random_ht(d, np.multiply(m, n), 2, 41)
        x = I.random_ht(d, n, 3, 42)
    else:  # deeper, taller leaves, larger ranks (leaf products of 40 x 60 matrices)
        d, m, n = 6, [40, 30, 20, 40, 30, 20], [60, 50, 40, 60, 50, 40]
        op = I.random_ht(d, np.multiply(m, n), 3, 43, "gauss", lambda j: 2.0 ** -j)
        x = I.random_ht(d, n, 6, 44, "gauss", lambda j: 2.0 ** -j)
    return d, np.asarray(m, np.int64), np.asarray(n, np.int64), op, x


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
@pytest.mark.parametrize("name", ["d4", "d6"])
def test_apply_matches_oracle(name, dtype):
    d, m, n, op, x = _case(name)
    tree = htgb.HTTree(d)
    L = htgb.HTTensor.from_blob(tree, op[0], op[1], op[2], dtype)
    X = htgb.HTTensor.from_blob(tree, x[0], x[1], x[2], dtype)
    kc = np.asarray(op[1]) * np.asarray(x[1])
    kc[0] = 1
    C = htgb.HTTensor.create(tree, m, kc, dtype)
    htgb.ht_apply(L.handle, X.handle, C.handle)
    kref, xref = O.apply(d, n, m, op[1], as_stored(op[2], dtype), x[1], as_stored(x[2], dtype))
    assert list(C.ranks()) == list(kref)
    got = C.download().astype(np.float64)
    tol = 1e-13 if dtype == htgb.HT_F64 else 4e-6
    # leaves are sums of n products; transfer tensors are single products
    assert np.abs(got - xref).max() <= tol * np.abs(xref).max() * np.sqrt(float(max(n)))
    # and the truncation of L X
    rep = C.truncate(mode="rank", rank_cap=4)
    ref = O.truncate(d, m, kref, xref, mode="rank", rank_cap=4)
    assert list(C.ranks()) == list(ref["k"])
    idx = sample_idx(m, 200, 5)
    e_tol = 1e-12 if dtype == htgb.HT_F64 else 1e-5
    assert np.abs(C.eval(idx) - O.eval_entries(d, m, ref["k"], ref["x"], idx)).max() <= e_tol * ref["norm"]


def test_apply_rejects_bad_shapes():
    d, m, n, op, x = _case("d4")
    tree = htgb.HTTree(d)
    L = htgb.HTTensor.from_blob(tree, op[0], op[1], op[2], htgb.HT_F64)
    X = htgb.HTTensor.from_blob(tree, x[0], x[1], x[2], htgb.HT_F64)
    kc = np.asarray(op[1]) * np.asarray(x[1])
    kc[0] = 1
    bad = htgb.HTTensor.create(tree, m + 1, kc, htgb.HT_F64)
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_apply(L.handle, X.handle, bad.handle)
    assert e.value.status == htgb.HT_EINVAL
