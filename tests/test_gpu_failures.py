"""Failure reporting of the library on the GPU, with no fault, trap or hang.

- A bounded device-side wait that runs out: the self-test kernel waits on a
  flag that no code sets, its time bound ends the wait, the kernel returns
  and the host reads HT_ETIMEOUT; the context stays usable.
- Non-finite input: a NaN in a leaf frame reaches ||X|| and the Gramian
  eigenvalues; the truncation with a report returns HT_ENUMERIC, and the
  device status words are cleared afterwards.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _drain_status():
    """Read and clear the status words; return the status raised (or HT_OK)."""
    try:
        htgb.ht_device_status()
        return htgb.HT_OK
    except htgb.HTError as e:
        return e.status


def _small_truncation_ok():
    (n, ka, xa), (_, kc, xc) = I.small_pair(1)
    tree = htgb.HTTree(8)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, htgb.HT_F64)
    C = htgb.HTTensor.from_blob(tree, n, kc, xc, htgb.HT_F64)
    X = A.add(C)
    rep = X.truncate(mode="rank", rank_cap=8)
    k, x = O.add(8, n, ka, xa, kc, xc)
    ref = O.truncate(8, n, k, x, mode="rank", rank_cap=8)
    assert list(rep["ranks"]) == list(ref["k"])
    assert abs(rep["norm"] - ref["norm"]) <= 1e-12 * ref["norm"]


@pytest.mark.parametrize("limit_ms", [0.0, 2.0])
def test_bounded_wait_times_out_and_context_survives(limit_ms):
    assert _drain_status() == htgb.HT_OK
    htgb.ht_selftest_wait(limit_ms)
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_device_status()
    assert e.value.status == htgb.HT_ETIMEOUT
    # the word was cleared by the read, and the device still computes
    assert _drain_status() == htgb.HT_OK
    _small_truncation_ok()


def test_selftest_rejects_bad_limit():
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_selftest_wait(-1.0)
    assert e.value.status == htgb.HT_EINVAL


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
def test_nan_input_reports_enumeric(dtype):
    assert _drain_status() == htgb.HT_OK
    (n, ka, xa), (_, kc, xc) = I.small_pair(2)
    xa = np.array(xa, dtype=np.float64, copy=True)
    tr = I.tree(8)
    # a NaN inside the first leaf's frame (the leaf slot follows the root and inner nodes in pre-order)
    leaf = next(t for t in range(15) if tr["son1"][t] < 0)
    off = sum(b.size for b in I.blob_nodes(8, n, ka, xa)[:leaf])
    xa[off + 3] = np.nan
    tree = htgb.HTTree(8)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, dtype)
    C = htgb.HTTensor.from_blob(tree, n, kc, xc, dtype)
    X = A.add(C)
    with pytest.raises(htgb.HTError) as e:
        X.truncate(mode="eps", eps=1e-3)
    assert e.value.status == htgb.HT_ENUMERIC
    assert "not finite" in str(e.value)
    # whatever else the NaN left in the status words is reported once, then cleared
    assert _drain_status() in (htgb.HT_OK, htgb.HT_ENUMERIC)
    assert _drain_status() == htgb.HT_OK
    _small_truncation_ok()
