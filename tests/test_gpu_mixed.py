"""The mixed-precision path (HT_PREC_MIXED: F64 storage, QR blocks in
double-float arithmetic on the FP32 pipe (FP64 Householder blocks with
qr_kernel 3), FP64 eigensolves, every contraction on the tcgen05 tensor cores
by exact BF16 slicing) against the CPU FP64 oracle, through the C-ABI.

Tolerance: 1e-9, normwise on sigma^2 per node and relative to ||X|| on
entries and norms.  The slicing carries about 2^-40 of |a| |b| per product
(5 slices), far below this; 1e-9 leaves room for the random walk over a
tree's contractions and is still three orders below the 1e-6 the path is
built for.  Ranks: equal in rank mode; in eps mode the rule is the FP64 one
(no noise charge) and a differing node must sit at the threshold within the
tolerance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I
from tests.gpu_util import check_sigma, gpu_sum, sample_idx, split_sigma
from tests.test_gpu_parity import _case, _trunc_compare

pytestmark = pytest.mark.gpu

F64, MIXED = htgb.HT_F64, htgb.HT_PREC_MIXED
TOL = 1e-9


@pytest.mark.parametrize("case", ["small", "uneven", "tall", "wide_leaf", "d2", "big_rank", "rank128", "rank200"])
def test_mixed_orthogonalize(case):
    d, n, a, c = _case(case)
    tree, A, C, X = gpu_sum(d, n, a, c, F64)
    k, x = O.add(d, n, a[1], a[2], c[1], c[2])
    ko_ref, xo_ref = O.orthogonalize(d, n, k, x)
    X.orthogonalize(MIXED)
    ko = X.ranks()
    assert list(ko) == list(ko_ref)
    xo = X.download()
    nodes = I.blob_nodes(d, n, ko, xo)
    tr = I.tree(d)
    for t in range(1, 2 * d - 1):
        M = nodes[t] if tr["son1"][t] < 0 else nodes[t].reshape(nodes[t].shape[0], -1).T
        # block Gram-Schmidt between 32-column panels: every Q column passes
        # through up to two tensor-core projections per earlier panel (about
        # 2^-40 each, 5 slices), so orthogonality holds to about 1e-11
        assert np.abs(M.T @ M - np.eye(M.shape[1])).max() <= 1e-10, t
    idx = sample_idx(n, 200)
    ref = O.eval_entries(d, n, k, x, idx)
    got = O.eval_entries(d, n, ko, xo, idx)
    scale = np.linalg.norm(nodes[0])
    assert np.abs(got - ref).max() <= TOL * scale
    ref_norm = np.linalg.norm(I.blob_nodes(d, n, ko_ref, xo_ref)[0])
    assert abs(scale - ref_norm) <= TOL * ref_norm


@pytest.mark.parametrize("case", ["small", "uneven", "tall", "wide_leaf", "d2", "big_rank", "rank128", "rank200"])
def test_mixed_truncate_rank(case):
    d, n, a, c = _case(case)
    r = {"small": 8, "uneven": 3, "tall": 5, "wide_leaf": 3, "d2": 4, "big_rank": 30, "rank128": 64,
         "rank200": 100}[case]
    _trunc_compare(d, n, a, c, F64, dict(mode="rank", rank_cap=r), prec=MIXED, tol=TOL)


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_mixed_truncate_eps(eps):
    d, n, a, c = _case("small")
    _trunc_compare(d, n, a, c, F64, dict(mode="eps", eps=eps, eps_relative=True), prec=MIXED, tol=TOL)


def test_mixed_node_schedule():
    d, n, a, c = _case("uneven")
    _trunc_compare(d, n, a, c, F64, dict(mode="rank", rank_cap=3), prec=MIXED, tol=TOL,
                   schedule=htgb.HT_SCHED_NODE)


def test_mixed_x_plus_x_is_2x():
    (n, ka, xa), _ = I.small_pair(9)
    d = 8
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, F64)
    X = A.add(A)
    X.truncate(mode="rank", rank_cap=8, prec=MIXED)
    assert list(X.ranks()) == [1] + [8] * (2 * d - 2)
    idx = sample_idx(n, 300, 3)
    got = X.eval(idx)
    want = 2.0 * O.eval_entries(d, n, ka, xa, idx)
    scale = 2.0 * A.norm()
    assert np.abs(got - want).max() <= TOL * scale


def test_mixed_gramians():
    import torch
    (n, ka, xa), (_, kc, xc) = I.small_pair(4)
    d = 8
    tree, A, C, X = gpu_sum(d, n, (n, ka, xa), (n, kc, xc), F64)
    X.orthogonalize(MIXED)
    ko = X.ranks()
    sizes = [1] + [int(v) ** 2 for v in ko[1:]]
    buf = torch.zeros(sum(sizes), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    htgb.ht_gramians(X.handle, buf.data_ptr(), MIXED)
    torch.cuda.synchronize()
    g = buf.cpu().numpy()
    k, x = O.add(d, n, ka, xa, kc, xc)
    ko_ref, xo_ref = O.orthogonalize(d, n, k, x)
    G_ref = O.gramians(d, n, ko_ref, xo_ref)
    o = 1
    for t in range(1, 2 * d - 1):
        G = g[o:o + sizes[t]].reshape(int(ko[t]), int(ko[t]))
        o += sizes[t]
        lam = np.sort(np.linalg.eigvalsh(0.5 * (G + G.T)))[::-1]
        lam_ref = np.sort(np.linalg.eigvalsh(G_ref[t]))[::-1]
        assert np.abs(lam - lam_ref).max() <= TOL * lam_ref[0], t


def test_mixed_rejects_f32_tensor():
    (n, ka, xa), _ = I.small_pair(1)
    tree = htgb.HTTree(8)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, htgb.HT_F32)
    with pytest.raises(htgb.HTError) as e:
        A.truncate(mode="rank", rank_cap=4, prec=MIXED)
    assert e.value.status == htgb.HT_EUNSUPPORTED


@pytest.mark.parametrize("case", ["small", "big_rank", "rank128"])
def test_mixed_fp64_qr_blocks(case):
    """qr_kernel 3: the mixed path with FP64 Householder blocks in place of the
    double-float ones, against the oracle at the same tolerance."""
    d, n, a, c = _case(case)
    r = {"small": 8, "big_rank": 30, "rank128": 64}[case]
    _trunc_compare(d, n, a, c, F64, dict(mode="rank", rank_cap=r), prec=MIXED, tol=TOL, qr_kernel=3)


@pytest.mark.parametrize("case", ["uneven", "rank200"])
def test_double_float_qr_blocks_match_fp64_blocks(case):
    """The same mixed truncation with double-float QR blocks (default) and with
    FP64 blocks: both carry the contractions' 2^-40 per product, the blocks
    themselves 2^-47 and 2^-53, so every node's singular values agree to
    1e-10 of the largest and the truncated tensors to 1e-9 of ||X||."""
    d, n, a, c = _case(case)
    r = {"uneven": 3, "rank200": 100}[case]
    out = []
    for qk in (0, 3):
        _, _, _, X = gpu_sum(d, n, a, c, F64)
        rep = X.truncate(prec=MIXED, mode="rank", rank_cap=r, qr_kernel=qk)
        out.append((rep, X))
    (r0, X0), (r3, X3) = out
    assert list(r0["korth"]) == list(r3["korth"]) and list(r0["ranks"]) == list(r3["ranks"])
    s0 = np.concatenate([np.ravel(v) for v in split_sigma(r0["korth"], r0["sigma"])])
    s3 = np.concatenate([np.ravel(v) for v in split_sigma(r3["korth"], r3["sigma"])])
    assert np.abs(s0 - s3).max() <= 1e-10 * np.abs(s0).max()
    assert abs(r0["norm"] - r3["norm"]) <= 1e-12 * r3["norm"]
    idx = sample_idx(n, 300, 11)
    assert np.abs(X0.eval(idx) - X3.eval(idx)).max() <= 1e-9 * r3["norm"]
