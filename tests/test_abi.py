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
