"""C-ABI library: loads, exports every symbol include/htgb.h declares, and its
host-side tree agrees with the paper's balanced tree.  No GPU needed."""
import os
import re

import numpy as np
import pytest

from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "htgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ht_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = htgb.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"libhtgb.so does not export {n}"
    assert sorted(htgb.EXPORTS) == names


def test_symbols_are_c_linkage():
    out = os.popen(f"nm -D --defined-only {htgb.LIB_PATH}").read()
    for n in declared_symbols():
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


@pytest.mark.parametrize("d", [2, 3, 5, 8, 17, 64])
def test_tree_matches_generator(d):
    tr = htgb.HTTree(d)
    g = I.tree(d)
    for t in range(2 * d - 1):
        info = tr.node(t)
        assert info["lo"] == g["lo"][t] and info["hi"] == g["hi"][t]
        assert info["son1"] == g["son1"][t] and info["son2"] == g["son2"][t]
        assert info["parent"] == g["parent"][t]


def test_errors_are_status_codes():
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_tree_balanced(1)
    assert e.value.status == htgb.HT_EINVAL
    assert "d must be" in str(e.value)
    tr = htgb.HTTree(4)
    with pytest.raises(htgb.HTError):
        htgb.ht_tree_node(tr.handle, 99)


def _einval(fn, *args, match=None):
    with pytest.raises(htgb.HTError) as e:
        fn(*args)
    assert e.value.status == htgb.HT_EINVAL
    if match:
        assert match in str(e.value)


def test_argument_errors_are_reported_before_any_device_work():
    """Bad arguments come back as HT_EINVAL with a message, checked on the host
    before the library touches a device (so this runs without a GPU)."""
    tr = htgb.HTTree(4)
    ok_n, ok_r = [5, 6, 7, 8], [1] + [2] * 6
    _einval(htgb.ht_tensor_create, tr.handle, [5, 0, 7, 8], ok_r, match="mode sizes")
    _einval(htgb.ht_tensor_create, tr.handle, ok_n, [1, 2, 2, 0, 2, 2, 2], match="ranks")
    _einval(htgb.ht_tensor_create, tr.handle, ok_n, ok_r, 7, match="dtype")
    opts = htgb.make_opts(mode="rank", rank_cap=2)
    _einval(htgb.ht_truncate, None, opts, match="null tensor")
    _einval(htgb.ht_truncate_batch, [None, None], opts, match="null tensor")
    _einval(htgb.ht_truncate, None, htgb.make_opts(mode="eps", eps=-1.0), match="eps")
    _einval(htgb.ht_truncate, None, htgb.make_opts(qr_kernel=7), match="qr_kernel")
    bad_mode = htgb.make_opts()
    bad_mode.mode = 9
    _einval(htgb.ht_truncate, None, bad_mode, match="mode")
    _einval(htgb.ht_orthogonalize, None)
    _einval(htgb.ht_gramians, None, 0)
    _einval(htgb.ht_gramians_noalloc, None, 0)
    _einval(htgb.ht_add, None, None)
    _einval(htgb.ht_add_into, None, None, None)
    _einval(htgb.ht_inner, None, None)
    _einval(htgb.ht_norm, None)
    _einval(htgb.ht_scale, None, 2.0)
    _einval(htgb.ht_apply, None, None, None)
    _einval(htgb.ht_eval_entries, None, np.zeros((1, 4), np.int64))
    _einval(htgb.ht_tensor_node_ptr, None, 0)
    _einval(htgb.ht_graph_launch, None)
    _einval(htgb.ht_selftest_wait, -1.0)
    _einval(htgb.ht_profile_read, 99)
