"""HT_PREC_FP32_SQRT: FP32 storage and contractions with square-root Gramian
factors (double-float Gram products, FP64 Cholesky), against the oracle on the
FP32-rounded inputs.  The singular values must be accurate to the FP32
tolerance ABSOLUTELY (|sigma - sigma_ref| <= tol sigma_max), i.e. small
singular values to O(u_32) sigma_max, where the squared-Gramian FP32 path
only gets O(sqrt(u_32)) sigma_max."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, fp32_tol, gpu_sum, sample_idx, split_sigma
from tests.test_gpu_parity import _case

pytestmark = pytest.mark.gpu
F32 = htgb.HT_F32
SQRT = htgb.HT_PREC_FP32_SQRT


def _sigma_abs_worst(sg, ref):
    worst = 0.0
    for t in range(1, len(ref)):
        b = np.asarray(ref[t], np.float64)
        if len(b) == 0 or b[0] == 0:
            continue
        a = np.asarray(sg[t], np.float64)[:len(b)]
        worst = max(worst, float(np.max(np.abs(a - b)) / b[0]))
    return worst


@pytest.mark.parametrize("case", ["small", "uneven", "tall", "d2", "big_rank", "rank128"])
def test_sqrt_gramians_truncate_rank(case):
    d, n, a, c = _case(case)
    r = {"small": 8, "uneven": 3, "tall": 5, "d2": 4, "big_rank": 30, "rank128": 64}[case]
    tree, A, C, X = gpu_sum(d, n, a, c, F32)
    rep = X.truncate(mode="rank", rank_cap=r, prec=SQRT)
    k, x = O.add(d, n, a[1], as_stored(a[2], F32), c[1], as_stored(c[2], F32))
    ref = O.truncate(d, n, k, x, mode="rank", rank_cap=r)
    assert list(X.ranks()) == list(ref["k"])
    K = int(max(k[1:]))
    tol = fp32_tol(d, K)
    worst = _sigma_abs_worst(split_sigma(rep["korth"], rep["sigma"]), ref["sigma"])
    print(f"{case}: sigma abs worst / sigma_max = {worst:.2e} (tol {tol:.2e})")
    assert worst <= tol
    assert abs(rep["norm"] - ref["norm"]) <= tol * ref["norm"]
    idx = sample_idx(n, 300, 3)
    got = X.eval(idx)
    want = O.eval_entries(d, n, ref["k"], ref["x"], idx)
    assert np.abs(got - want).max() <= 10 * tol * ref["norm"]


def test_sqrt_gramians_single_workload():
    """d=64, n=1000, k=32: the FP32 path with square-root Gramians against the
    FP64 oracle on the same FP32-representable inputs."""
    D = 64
    (n, ka, xa), (_, kc, xc) = I.single_pair(11)
    tree, A, C, X = gpu_sum(D, n, (n, ka, xa), (n, kc, xc), F32)
    rep = X.truncate(prec=SQRT, **I.SINGLE_OPTS)
    k, x = O.add(D, n, ka, as_stored(xa, F32), kc, as_stored(xc, F32))
    ref = O.truncate(D, n, k, x, **I.SINGLE_OPTS)
    tol = fp32_tol(D, 64)
    worst = _sigma_abs_worst(split_sigma(rep["korth"], rep["sigma"]), ref["sigma"])
    kt, xt = X.ranks(), X.download().astype(np.float64)
    Y = htgb.HTTensor.from_blob(tree, n, kt, xt, htgb.HT_F64)
    Z = htgb.HTTensor.from_blob(tree, n, ref["k"], ref["x"], htgb.HT_F64)
    Z.scale(-1.0)
    dist = Y.add(Z).norm() / ref["norm"]
    print(f"single sqrt: sigma abs worst / sigma_max = {worst:.2e} (tol {tol:.2e}), "
          f"||T(X) - T_ref(X)|| / ||X|| = {dist:.2e}, ranks[1:6] = {list(kt[1:6])}")
    assert worst <= tol
    assert abs(rep["norm"] - ref["norm"]) <= tol * ref["norm"]
    # the truncated tensors agree to the FP32 tolerance (the squared-Gramian FP32
    # path is a factor ~15 further away here: cuts below sqrt(u_32) sigma_max)
    assert dist <= tol
