"""Full-size workloads against the CPU FP64 oracle, through the C-ABI, in the
launch configuration the benchmark times (one batched launch per tree level).

  deep   d=256, n=4096, k=64 -> rank 128, sigma_j = 10^(-10j/64), eps = 1e-6 relative
  wide   d=16, n=2048, k=128 -> rank 256, sigma_j = j^-2, truncated to rank 128
  C3     a sample of the batched workload at its full ranges (K = 4k up to 192,
         n up to 512), all tensors in one batched call

Tolerances (per result): the mixed path 1e-6 on sigma normwise per node
(|sigma_i - sigma_ref_i| <= 1e-6 sigma_max for sigma_ref_i >= 1e-5 sigma_max);
the FP64 path 1e-12 on sigma^2 normwise per node (|sigma_i^2 - sigma_ref_i^2|
<= 1e-12 sigma_max^2, times depth / 4 beyond depth 4 since the top-down
Gramian recursion adds one contraction's rounding per level: two FP64
Gramian computations differ by about u lambda_max per eigenvalue, i.e. by
about u sigma_max^2 / (2 sigma) on sigma, which is 2e-11 sigma_max at
sigma = 1e-5 sigma_max); both on ||X|| relative
and on ||T(X) - T_ref(X)|| / ||X||; in eps mode the truncation error
||X - T(X)|| stays within eps ||X|| (5% for decisions at rounding level).  Ranks are discontinuous in the eigenvalues: in
eps mode a node may differ only where the oracle's tail at the library's cut
lies within the tolerance of the per-node budget, and the truncated tensors
may then differ by the oracle's energy between the two cuts (added to the
bound and printed).  Tensor differences are norms of the orthogonalized sum
Y + (-Z) (FP64 path on the GPU, pinned against the oracle's norm), never
inner products.  The oracle's wall time is printed with each reference.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import check_ranks, gap_allowance, gpu_sum, split_sigma

pytestmark = pytest.mark.gpu

TOLS = {htgb.HT_PREC_MIXED: 1e-6, htgb.HT_PREC_FP64: 1e-12}
# Gramian error (normwise, per node) of each path, as measured on the deep and
# wide workloads (sigma^2 normwise against the oracle, with margin)
GRAM_EPS = {htgb.HT_PREC_MIXED: 3e-10, htgb.HT_PREC_FP64: 2e-12}


def _oracle(d, n, ka, xa, kc, xc, opts):
    O.set_threads(0)
    t0 = time.perf_counter()
    k, x = O.add(d, n, ka, xa, kc, xc)
    ref = O.truncate(d, n, k, x, **opts)
    print(f"oracle d={d}: {time.perf_counter() - t0:.1f} s on {O.set_threads(0)} threads")
    return k, x, ref


def _sigma_errors(rep, ref, d):
    """Worst per-node sigma errors against the oracle: (sigma normwise and
    relative for sigma_ref >= 1e-5 sigma_max, sigma^2 normwise over all)."""
    sg = split_sigma(rep["korth"], rep["sigma"])
    nw = rl = nw2 = 0.0
    for t in range(1, 2 * d - 1):
        a, b = np.asarray(sg[t], np.float64), np.asarray(ref["sigma"][t], np.float64)
        assert a.shape == b.shape, t
        if len(b) == 0 or b[0] <= 0:
            continue
        sel = b >= 1e-5 * b[0]
        nw = max(nw, float(np.max(np.abs(a[sel] - b[sel])) / b[0]))
        rl = max(rl, float(np.max(np.abs(a[sel] - b[sel]) / b[sel])))
        nw2 = max(nw2, float(np.max(np.abs(a ** 2 - b ** 2)) / b[0] ** 2))
    return nw, rl, nw2


def _diff_norm(tree, n, k1, x1, k2, x2):
    P = htgb.HTTensor.from_blob(tree, n, k1, x1, htgb.HT_F64)
    Q = htgb.HTTensor.from_blob(tree, n, k2, x2, htgb.HT_F64)
    Q.scale(-1.0)
    return P.add(Q).norm()


def _compare(d, n, pair, ref, k, x, opts, prec, label):
    tol = TOLS[prec]
    (ka, xa), (kc, xc) = pair
    tree, A, C, X = gpu_sum(d, n, (n, ka, xa), (n, kc, xc), htgb.HT_F64)
    t0 = time.perf_counter()
    rep = X.truncate(prec=prec, **opts)
    secs = time.perf_counter() - t0
    nrm = ref["norm"]
    assert list(rep["korth"]) == list(ref["korth"])
    nw, rl, nw2 = _sigma_errors(rep, ref, d)
    kt, xt = X.ranks(), X.download()
    eps_mode = opts.get("mode") == "eps"
    differ, energy = check_ranks(kt, ref, tol, eps_mode, d, htgb.HT_F64, prec)
    dist = _diff_norm(tree, n, kt, xt, ref["k"], ref["x"]) / nrm
    err = _diff_norm(tree, n, k, x, kt, xt) / nrm
    err_ref = _diff_norm(tree, n, k, x, ref["k"], ref["x"]) / nrm
    # closely spaced singular values at a cut make T(X) itself ill-conditioned:
    # the allowance of a Gramian error of the measured size at every node
    gap = gap_allowance(ref["sigma"], ref["k"], max(nw2, 1e-16)) / nrm
    print(f"{label} prec={prec}: {secs:.2f} s, sigma normwise {nw:.2e} relative {rl:.2e} sigma^2 normwise {nw2:.2e}, "
          f"||X|| {abs(rep['norm'] - nrm) / nrm:.2e}, ||T - T_ref|| {dist:.2e}, err {err:.3e} (oracle {err_ref:.3e}), "
          f"rank diffs {len(differ)} (energy {energy / nrm:.2e}), gap allowance {gap:.2e}, ranks {list(kt[1:8])}")
    if prec == htgb.HT_PREC_FP64:
        # one FP64 contraction's rounding per level of the top-down Gramian
        # recursion: 1e-12 up to depth 4, proportionally deeper
        depth = int(np.ceil(np.log2(d)))
        assert nw2 <= tol * max(1.0, depth / 4.0)
    else:
        assert nw <= tol
    assert abs(rep["norm"] - nrm) <= tol * nrm
    if eps_mode:
        assert err <= opts["eps"] * 1.05
    assert dist <= tol + 2 * energy / nrm + gap
    assert abs(err - err_ref) <= tol + 2 * energy / nrm + gap
    # the HSVD error bound of the oracle's own truncation
    assert err_ref <= np.sqrt(ref["discarded_sq"]) / nrm * (1 + 1e-9) + 1e-12
    return rep


@pytest.fixture(scope="module")
def deep_ref():
    d = 256
    (n, ka, xa), (_, kc, xc) = I.deep_pair(21)
    k, x, ref = _oracle(d, n, ka, xa, kc, xc, I.DEEP_OPTS)
    return d, n, ((ka, xa), (kc, xc)), ref, k, x


@pytest.mark.parametrize("prec", [htgb.HT_PREC_MIXED, htgb.HT_PREC_FP64])
def test_deep_against_oracle(deep_ref, prec):
    d, n, pair, ref, k, x = deep_ref
    rep = _compare(d, n, pair, ref, k, x, I.DEEP_OPTS, prec, "deep")
    # eps = 1e-6 truncates: the ranks fall below the post-addition 128 at the root's sons
    assert min(int(v) for v in rep["ranks"][1:]) < 128


@pytest.fixture(scope="module")
def wide_ref():
    d = 16
    (n, ka, xa), (_, kc, xc) = I.wide_pair(31)
    k, x, ref = _oracle(d, n, ka, xa, kc, xc, I.WIDE_OPTS)
    return d, n, ((ka, xa), (kc, xc)), ref, k, x


@pytest.mark.parametrize("prec", [htgb.HT_PREC_MIXED, htgb.HT_PREC_FP64])
def test_wide_against_oracle(wide_ref, prec):
    d, n, pair, ref, k, x = wide_ref
    _compare(d, n, pair, ref, k, x, I.WIDE_OPTS, prec, "wide")


def _c3_full_range_sample():
    """Tensors of the batched workload's 4096 specs whose post-addition rank
    4k spans the full range (up to 192, i.e. three QR panels) and whose n
    reaches 512, plus small ones, so that one batched call mixes shapes."""
    specs = I.batched_specs(count=4096, seed=41)
    big = sorted([s for s in specs if s[1] >= 400], key=lambda s: -s[2])[:3]
    small = [s for s in specs if s[2] <= 8 and s[1] <= 64][:2]
    tall = [s for s in specs if s[1] >= 500 and 24 <= s[2] <= 32][:1]
    return big + small + tall


@pytest.mark.parametrize("prec,dtype", [(htgb.HT_PREC_MIXED, htgb.HT_F64), (htgb.HT_PREC_FP64, htgb.HT_F64)])
def test_batched_full_range_against_oracle(prec, dtype):
    sample = _c3_full_range_sample()
    assert max(4 * s[2] for s in sample) >= 180 and max(s[1] for s in sample) >= 500
    O.set_threads(0)
    Xs, refs = [], []
    t0 = time.perf_counter()
    for (d, nn, kk, seed) in sample:
        terms = I.batched_terms((d, nn, kk, seed))
        tree = htgb.HTTree(d)
        T = [htgb.HTTensor.from_blob(tree, nv, kv, xv, dtype) for (nv, kv, xv) in terms]
        Xs.append(T[0].add(T[1]).add(T[2].add(T[3])))
        nv = terms[0][0]
        ka, xa = O.add(d, nv, terms[0][1], terms[0][2], terms[1][1], terms[1][2])
        kc, xc = O.add(d, nv, terms[2][1], terms[2][2], terms[3][1], terms[3][2])
        k, x = O.add(d, nv, ka, xa, kc, xc)
        refs.append((d, nv, k, x, O.truncate(d, nv, k, x, mode="rank", rank_cap=kk)))
    print(f"oracle, {len(sample)} tensors {[(s[0], s[1], 4 * s[2]) for s in sample]}: {time.perf_counter() - t0:.1f} s")
    caps = [s[2] for s in sample]
    htgb.ht_truncate_batch([X.handle for X in Xs], htgb.make_opts(mode="rank", prec=prec, tensor_caps=caps))
    tol = TOLS[prec]
    for X, (d, nv, k, x, ref) in zip(Xs, refs):
        assert list(X.ranks()) == list(ref["k"])
        tree = X.tree
        xt = X.download()
        dist = _diff_norm(tree, nv, X.ranks(), xt, ref["k"], ref["x"]) / ref["norm"]
        # ill-conditioning of T(X) at closely spaced cuts, for a Gramian error of the path's tolerance
        gap = gap_allowance(ref["sigma"], ref["k"], GRAM_EPS[prec]) / ref["norm"]
        print(f"  d={d} n={nv[0]} K={int(max(k))}: ||T - T_ref|| / ||X|| = {dist:.2e} (gap allowance {gap:.2e})")
        assert dist <= tol + gap
