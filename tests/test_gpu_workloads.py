"""Full-size parity on the benchmark workload, in the launch configuration the
benchmark times (level schedule, the F32 tensor with FP64 eigensolves and the
F64 plain path):  d=64, n=1000, k=32 (rank 64 after the addition),
orthonormal Gaussian leaves, sigma_j = 10^(-8j/32), eps = 1e-8 relative,
rank cap 32.

Differences of HT tensors are measured as ||Y - Z|| = ||Y + (-Z)|| with the
norm of the orthogonalized sum (backward stable), never through
<Y,Y> - 2<Y,Z> + <Z,Z>.

Rank decisions near the eps threshold are discontinuous: a node whose rank
differs from the oracle's is accepted only if the oracle's discarded tail at
the GPU's cut lies within the arithmetic's error of the per-node threshold.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import as_stored, check_ranks, check_sigma, fp32_tol, fp32_tol_sigma, gpu_sum, split_sigma

pytestmark = pytest.mark.gpu

D = 64


@pytest.fixture(scope="module", params=[htgb.HT_F64, htgb.HT_F32])
def single(request):
    dtype = request.param
    (n, ka, xa), (_, kc, xc) = I.single_pair(11)
    k, x = O.add(D, n, ka, as_stored(xa, dtype), kc, as_stored(xc, dtype))
    ref = O.truncate(D, n, k, x, **I.SINGLE_OPTS)
    return dtype, n, (n, ka, xa), (n, kc, xc), k, x, ref


def negated(k, x):
    """-Z as a blob: the root block (first in pre-order) changes sign."""
    y = np.array(x, dtype=np.float64, copy=True)
    tr = I.tree(D)
    y[: int(k[tr["son1"][0]]) * int(k[tr["son2"][0]])] *= -1.0
    return y


def diff_norm(n, k1, x1, k2, x2):
    """||Y - Z|| as ||B_D|| of the orthogonalized sum Y + (-Z) (oracle, FP64)."""
    ks, xs = O.add(D, n, k1, x1, k2, negated(k2, x2))
    ko, xo = O.orthogonalize(D, n, ks, xs)
    root = int(ko[I.tree(D)["son1"][0]]) * int(ko[I.tree(D)["son2"][0]])
    return float(np.linalg.norm(xo[:root]))


def test_single_workload(single):
    dtype, n, a, c, k, x, ref = single
    tree, A, C, X = gpu_sum(D, n, a, c, dtype)
    prec = htgb.HT_PREC_FP64 if dtype == htgb.HT_F64 else htgb.HT_PREC_FP32
    rep = X.truncate(prec=prec, **I.SINGLE_OPTS)
    nrm = ref["norm"]
    tol = 1e-12 if dtype == htgb.HT_F64 else fp32_tol(D)
    assert list(rep["korth"]) == list(ref["korth"])
    norm_err = abs(rep["norm"] - nrm) / nrm
    print(f"dtype={dtype} tol={tol:.2e} norm rel err={norm_err:.2e}")
    assert norm_err <= tol
    sg = split_sigma(rep["korth"], rep["sigma"])
    tol_sig = 1e-12 if dtype == htgb.HT_F64 else fp32_tol_sigma(D)
    worst = check_sigma(sg, ref["sigma"], tol_sig, floor=1e-5)
    kt = X.ranks()
    xt = X.download().astype(np.float64)
    differ, energy = check_ranks(kt, ref, tol_sig, True, D, dtype)
    dist = diff_norm(n, kt, xt, ref["k"], ref["x"]) / nrm
    err_gpu = diff_norm(n, k, x, kt, xt) / nrm
    err_ref = diff_norm(n, k, x, ref["k"], ref["x"]) / nrm
    print(f"dtype={dtype} sigma worst={worst:.2e} (tol {tol_sig:.2e}) rank_diffs={len(differ)} energy={energy / nrm:.2e} "
          f"dist={dist:.2e} err_gpu={err_gpu:.3e} err_ref={err_ref:.3e}")
    # the HSVD error bound: ||X - T(X)|| <= sqrt(sum of the discarded sigma^2)
    assert err_ref <= np.sqrt(ref["discarded_sq"]) / nrm * (1 + 1e-9)
    if dtype == htgb.HT_F64:  # keeping more rank than the oracle never increases the error beyond these parts
        assert err_gpu <= err_ref + energy / nrm + tol
    # Directions whose Gramian eigenvalue lies below the path's resolution
    # (tol_sig * lambda_max of the node) cannot be told apart: the truncated
    # tensors may differ by X's energy in them (oracle spectra, summed over nodes).
    unresolved = 0.0
    for t in range(1, 2 * D - 1):
        lam = np.asarray(ref["sigma"][t], dtype=np.float64) ** 2
        if len(lam) and lam[0] > 0:
            unresolved += float(np.sqrt(np.sum(lam[lam <= 2 * tol_sig * lam[0]])))
    print(f"dtype={dtype} unresolved energy bound={unresolved / nrm:.2e}")
    # relative Frobenius distance to the oracle's T(X), and of the truncation errors
    assert dist <= tol + 2 * energy / nrm + unresolved / nrm
    assert abs(err_gpu - err_ref) <= tol + 2 * energy / nrm + unresolved / nrm
    if dtype == htgb.HT_F64:
        assert dist <= 1e-12 + 2 * energy / nrm  # FP64 resolves everything the oracle does
