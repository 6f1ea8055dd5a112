"""ht_inner (Sec. 3.2, Lemma "phi"): <X, Y> by the Phi recursion on the GPU
against the oracle's Phi recursion (itself pinned against full tensors), on
tensors of different ranks, uneven trees, and against ||X||^2 from the
orthogonalization path."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import U32, as_stored

pytestmark = pytest.mark.gpu


def _cases():
    yield "small", 8, 32, I.random_ht(8, 32, 8, 1), I.random_ht(8, 32, 5, 2)
    nn = [40, 17, 33, 25, 9]
    yield "uneven", 5, nn, I.random_ht(5, nn, 6, 3), I.random_ht(5, nn, 9, 4)
    yield "d2", 2, [50, 70], I.random_ht(2, [50, 70], 12, 5), I.random_ht(2, [50, 70], 7, 6)
    nn = [700, 300, 450, 600]
    yield "long_leaves_big_rank", 4, nn, I.random_ht(4, nn, 70, 7), I.random_ht(4, nn, 90, 8)


@pytest.mark.parametrize("dtype", [htgb.HT_F64, htgb.HT_F32])
@pytest.mark.parametrize("case", ["small", "uneven", "d2", "long_leaves_big_rank"])
def test_inner_matches_oracle(dtype, case):
    name, d, n, a, c = next(cs for cs in _cases() if cs[0] == case)
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, a[0], a[1], a[2], dtype)
    C = htgb.HTTensor.from_blob(tree, c[0], c[1], c[2], dtype)
    xa, xc = as_stored(a[2], dtype), as_stored(c[2], dtype)
    want = O.inner(d, a[0], a[1], xa, c[1], xc)
    scale = np.sqrt(O.inner(d, a[0], a[1], xa, a[1], xa) * O.inner(d, c[0], c[1], xc, c[1], xc))
    got = A.inner(C)
    # FP32: one rounding per contraction and level, reductions up to n long (split, FP64 partial sums)
    tol = 1e-12 if dtype == htgb.HT_F64 else 64 * np.sqrt(2 * d - 1) * U32
    assert abs(got - want) <= tol * scale, (got, want, scale)


def test_inner_with_itself_is_norm_squared():
    (n, ka, xa), (_, kc, xc) = I.single_pair(11)
    tree = htgb.HTTree(64)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, htgb.HT_F64)
    C = htgb.HTTensor.from_blob(tree, n, kc, xc, htgb.HT_F64)
    X = A.add(C)
    nrm = X.norm()
    assert abs(X.inner(X) - nrm ** 2) <= 1e-12 * nrm ** 2
    # bilinearity through the addition lemma: <A + C, A> = <A, A> + <C, A>
    lhs = X.inner(A)
    rhs = A.inner(A) + C.inner(A)
    assert abs(lhs - rhs) <= 1e-12 * nrm * A.norm()
