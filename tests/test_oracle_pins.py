"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check goes through an
independent route (numpy SVD / eigh / QR of full matricizations, full
tensors built from the definition, closed forms, brute force).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1708_03340_gb300 import inputs as I
from tests import fulltensor as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# --- dimension tree (Sec. 2.1, eq. "balanced") ------------------------------

@pytest.mark.parametrize("d", [2, 3, 4, 5, 7, 8, 13, 32, 64])
def test_tree_balanced(d):
    tr = O.tree_info(d)
    nn = 2 * d - 1
    for t in range(nn):
        lo, hi = tr["lo"][t], tr["hi"][t]
        if tr["son1"][t] >= 0:
            s1, s2 = tr["son1"][t], tr["son2"][t]
            size = hi - lo + 1
            # left son gets floor(size/2) leaves, sons partition t
            assert tr["hi"][s1] - tr["lo"][s1] + 1 == size // 2
            assert tr["lo"][s1] == lo and tr["hi"][s2] == hi and tr["hi"][s1] + 1 == tr["lo"][s2]
            assert tr["parent"][s1] == t and tr["parent"][s2] == t
        else:
            assert lo == hi
    assert int(tr["depth"].max()) == int(np.ceil(np.log2(d)))
    # the generator's own tree layout agrees (same pre-order)
    g = I.tree(d)
    assert list(tr["lo"]) == g["lo"] and list(tr["son1"]) == g["son1"]


# --- dense building blocks ---------------------------------------------------

@pytest.mark.parametrize("m,n", [(40, 7), (7, 7), (5, 9), (200, 16)])
def test_householder_qr(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n))
    Q, R = O.qr(A)
    p = min(m, n)
    assert Q.shape == (m, p) and R.shape == (p, n)
    assert np.abs(Q.T @ Q - np.eye(p)).max() < 1e-14
    assert rel(Q @ R, A) < 1e-14
    assert np.abs(np.tril(R, -1)).max() == 0.0
    # R is unique up to the signs of its rows: compare with numpy's Householder QR
    Rn = np.linalg.qr(A, mode="r")
    assert np.allclose(np.abs(R), np.abs(Rn[:p]), atol=1e-12 * np.abs(Rn).max())


def test_householder_qr_rank_deficient():
    rng = np.random.default_rng(3)
    U = rng.standard_normal((30, 4))
    A = np.hstack([U, U])  # exactly rank 4 in 8 columns, as in X + X
    Q, R = O.qr(A)
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-14
    assert rel(Q @ R, A) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_jacobi_eig(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    A = X @ X.T
    w, V = O.eig_sym(A)
    wn = np.linalg.eigvalsh(A)[::-1]
    assert np.all(np.diff(w) <= 0)
    assert np.abs(w - wn).max() < 1e-13 * max(1.0, wn.max())
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    assert np.abs(A @ V - V * w).max() < 1e-12 * max(1.0, wn.max())


def test_jacobi_eig_degenerate():
    rng = np.random.default_rng(5)
    Qr, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([3.0, 3.0, 1.0, 1.0, 1.0, 0.0])
    A = (Qr * lam) @ Qr.T
    w, V = O.eig_sym(A)
    assert np.abs(w - lam).max() < 1e-14 * 3
    assert np.abs(V.T @ V - np.eye(6)).max() < 1e-13


# --- evaluation, addition, inner product (Sec. 3.1, 3.5, 3.2) --------------

def _full(d, n, k, x):
    return F.frames(d, n, k, x)[1]


@pytest.mark.parametrize("case", ["brute", "uneven"])
def test_eval_matches_full_tensor(case):
    """Sec. 3.1 (eq. "transfermult") against the full tensor built from the
    definition of the transfer tensors (tests/fulltensor.py, numpy only).  The
    uneven case has distinct mode sizes and unequal ranks of the two sons of
    every node, so a swap of the sons' indices (j, l) of B_t, of two modes, or
    of the parent index with a son's index changes the values."""
    if case == "brute":
        (n, k, x), _ = I.brute_pair(3)
        d = 4
    else:
        d, n = 5, np.array([3, 4, 2, 5, 6])
        tr = I.tree(d)
        k = np.array([1] + [2 + (t % 3) for t in range(1, 2 * d - 1)], np.int32)
        rng = np.random.default_rng(11)
        nodes = []
        for t in range(2 * d - 1):
            if tr["son1"][t] < 0:
                nodes.append(rng.standard_normal((int(n[tr["lo"][t]]), int(k[t]))))
            else:
                kt = 1 if t == 0 else int(k[t])
                B = rng.standard_normal((kt, int(k[tr["son1"][t]]), int(k[tr["son2"][t]])))
                nodes.append(B[0] if t == 0 else B)
        x = I.nodes_blob(d, nodes)
        assert any(k[tr["son1"][t]] != k[tr["son2"][t]] for t in range(2 * d - 1) if tr["son1"][t] >= 0)
    full = F.frames(d, n, k, x)[1]
    rng = np.random.default_rng(0)
    idx = np.stack([rng.integers(0, int(v), 80) for v in n], axis=1)
    vals = O.eval_entries(d, n, k, x, idx)
    ref = full[tuple(idx.T)]
    assert np.abs(vals - ref).max() < 1e-15 * np.abs(full).max() * 10


def test_add_lemma_entries():
    (n, ka, xa), (_, kc, xc) = I.brute_pair(4)
    k, x = O.add(4, n, ka, xa, kc, xc)
    assert list(k) == [1] + [8] * 6
    assert rel(_full(4, n, k, x), _full(4, n, ka, xa) + _full(4, n, kc, xc)) < 1e-15
    # uneven tree and unequal ranks
    a = I.random_ht(5, [3, 4, 2, 5, 3], 2, 7)
    c = I.random_ht(5, [3, 4, 2, 5, 3], 3, 8)
    k, x = O.add(5, a[0], a[1], a[2], c[1], c[2])
    assert rel(_full(5, a[0], k, x), _full(5, a[0], a[1], a[2]) + _full(5, c[0], c[1], c[2])) < 1e-15


def test_inner_product_phi():
    (n, ka, xa), (_, kc, xc) = I.brute_pair(6)
    v = O.inner(4, n, ka, xa, kc, xc)
    ref = float(np.sum(_full(4, n, ka, xa) * _full(4, n, kc, xc)))
    assert abs(v - ref) < 1e-13 * abs(ref) + 1e-15


# --- orthogonalization (Sec. 3.4) -------------------------------------------

@pytest.mark.parametrize("d,n", [(4, 8), (5, [3, 4, 2, 5, 3]), (2, 6)])
def test_orthogonalize(d, n):
    a = I.random_ht(d, n, 3, 12)
    c = I.random_ht(d, n, 2, 13)
    k, x = O.add(d, a[0], a[1], a[2], c[1], c[2])
    ko, xo = O.orthogonalize(d, a[0], k, x)
    tr = I.tree(d)
    nodes = I.blob_nodes(d, a[0], ko, xo)
    for t in range(1, 2 * d - 1):
        if tr["son1"][t] < 0:
            U = nodes[t]
            assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-13
        else:
            M = nodes[t].reshape(nodes[t].shape[0], -1).T  # M_{2,3}(B)
            assert np.abs(M.T @ M - np.eye(M.shape[1])).max() < 1e-13
    f0, f1 = _full(d, a[0], k, x), _full(d, a[0], ko, xo)
    assert rel(f1, f0) < 1e-13
    # ||A|| = ||B_D||_F of the orthogonal representation
    assert abs(np.linalg.norm(nodes[0]) - np.linalg.norm(f0)) < 1e-13 * np.linalg.norm(f0)


# --- Gramians vs SVDs of the full matricizations (Sec. 3.3) ----------------

@pytest.mark.parametrize("seed", [1, 2])
def test_gramian_eigs_are_squared_singular_values(seed):
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    ko, xo = O.orthogonalize(d, n, k, x)
    G = O.gramians(d, n, ko, xo)
    full = _full(d, n, k, x)
    tr = I.tree(d)
    for t in range(1, 2 * d - 1):
        s = np.linalg.svd(F.matricization(full, tr["lo"][t], tr["hi"][t]), compute_uv=False)
        lam = np.sort(np.linalg.eigvalsh(G[t]))[::-1]
        kk = min(len(s), len(lam))
        smax = s[0]
        # |sigma_i^2 - lambda_i| <= 1e-12 sigma_max^2 (normwise on eigenvalues)
        assert np.abs(s[:kk] ** 2 - lam[:kk]).max() <= 1e-12 * smax ** 2
        assert np.all(np.abs(lam[kk:]) <= 1e-12 * smax ** 2)
        # plain relative 1e-12 on the O(1) singular values of this case
        big = s[:kk] > 1e-3 * smax
        assert np.abs(np.sqrt(np.maximum(lam[:kk][big], 0)) - s[:kk][big]).max() <= 1e-12 * smax


def test_gramian_eigs_uneven_tree():
    d, n = 5, [3, 4, 2, 5, 3]
    a = I.random_ht(d, n, 3, 21)
    ko, xo = O.orthogonalize(d, a[0], a[1], a[2])
    G = O.gramians(d, a[0], ko, xo)
    full = _full(d, a[0], a[1], a[2])
    tr = I.tree(d)
    for t in range(1, 2 * d - 1):
        s = np.linalg.svd(F.matricization(full, tr["lo"][t], tr["hi"][t]), compute_uv=False)
        lam = np.sort(np.linalg.eigvalsh(G[t]))[::-1]
        kk = min(len(s), len(lam))
        assert np.abs(s[:kk] ** 2 - lam[:kk]).max() <= 1e-12 * s[0] ** 2


# --- truncation (Sec. 3.3) ---------------------------------------------------

@pytest.mark.parametrize("seed,r", [(1, 2), (2, 3), (5, 1)])
def test_truncation_equals_full_svd_truncation(seed, r):
    """HSVD of the HT tensor = truncation by SVDs of all matricizations of the full tensor."""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    res = O.truncate(d, n, k, x, mode="rank", rank_cap=r)
    full = _full(d, n, k, x)
    ref = F.brute_truncate(d, full, [1] + [r] * 6)
    assert rel(_full(d, n, res["k"], res["x"]), ref) < 1e-11


@pytest.mark.parametrize("seed,ranks,effective", [
    (3, [1, 5, 3, 2, 3, 0, 4], [1, 3, 3, 2, 3, 8, 4]),
    (4, [1, 2, 4, 1, 6, 2, 5], [1, 2, 4, 1, 2, 2, 5]),
])
def test_truncation_to_prescribed_ranks_per_node(seed, ranks, effective):
    """Target ranks given per node (Sec. 3.5, truncation to prescribed ranks):
    node t keeps ranks[t] (0: every rank left after orthogonalization), and the
    root's two sons, whose matricizations are transposes of each other, keep
    the smaller of their two targets.  The result is the projection of the full
    tensor onto the leading singular vectors of each matricization with those
    ranks; a rank read from the wrong node (a father's, a brother's) or a root
    pair left unequal gives a different tensor."""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    res = O.truncate(d, n, k, x, mode="rank", ranks=np.array(ranks))
    assert list(res["k"]) == effective
    full = _full(d, n, k, x)
    ref = F.brute_truncate(d, full, effective)
    assert rel(_full(d, n, res["k"], res["x"]), ref) < 1e-11


@pytest.mark.parametrize("seed", [1, 3, 8])
def test_truncation_error_bounds(seed):
    """||A - T(A)|| <= sqrt(sum discarded sigma^2) <= sqrt(2d-3) max_t tail_t <= sqrt(2d-3) best."""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    res = O.truncate(d, n, k, x, mode="rank", rank_cap=2)
    full = _full(d, n, k, x)
    err = np.linalg.norm(full - _full(d, n, res["k"], res["x"]))
    tr = I.tree(d)
    tails = []
    for t in range(1, 2 * d - 1):
        s = np.linalg.svd(F.matricization(full, tr["lo"][t], tr["hi"][t]), compute_uv=False)
        tails.append(np.sum(s[2:] ** 2))
    best_lower = np.sqrt(max(tails))  # Eckart-Young at the node with the largest tail
    disc = np.sqrt(res["discarded_sq"])
    assert err <= disc * (1 + 1e-12)
    assert disc <= np.sqrt(2 * d - 3) * best_lower * (1 + 1e-12)
    # the discarded energy the oracle reports equals the SVD tails (root pair once)
    t1, t2 = tr["son1"][0], tr["son2"][0]
    ref = sum(tl for t, tl in zip(range(1, 2 * d - 1), tails) if t != t2)
    assert abs(res["discarded_sq"] - ref) <= 1e-12 * np.sum(full ** 2)


def test_truncate_x_plus_x_is_2x():
    (n, ka, xa), _ = I.small_pair(9)
    d = 8
    k, x = O.add(d, n, ka, xa, ka, xa)
    res = O.truncate(d, n, k, x, mode="rank", rank_cap=8)
    assert list(res["k"]) == [1] + [8] * (2 * d - 2)
    idx = np.stack([np.random.default_rng(1).integers(0, 32, 300) for _ in range(d)], axis=1)
    got = O.eval_entries(d, n, res["k"], res["x"], idx)
    ref = 2.0 * O.eval_entries(d, n, ka, xa, idx)
    scale = res["norm"]  # ||X + X|| = ||2X||
    assert abs(scale - 2.0 * O.truncate(d, n, ka, xa, mode="eps", eps=0.0)["norm"]) <= 1e-13 * scale
    assert np.abs(got - ref).max() <= 1e-12 * scale


def test_d2_is_matrix_svd():
    """d = 2: A = U1 B_D U2^T; the truncation is the best rank-r approximation."""
    rng = np.random.default_rng(4)
    n = [9, 7]
    U1, U2, BD = rng.standard_normal((9, 5)), rng.standard_normal((7, 5)), rng.standard_normal((5, 5))
    x = I.nodes_blob(2, [BD, U1, U2])
    k = np.array([1, 5, 5])
    res = O.truncate(2, n, k, x, mode="rank", rank_cap=3)
    A = U1 @ BD @ U2.T
    u, s, vt = np.linalg.svd(A)
    best = (u[:, :3] * s[:3]) @ vt[:3]
    got = _full(2, n, res["k"], res["x"])
    assert rel(got, best) < 1e-12
    assert np.abs(res["sigma"][1] - s[:5]).max() < 1e-12 * s[0]


def test_eps_zero_returns_input():
    (n, ka, xa), (_, kc, xc) = I.brute_pair(2)
    k, x = O.add(4, n, ka, xa, kc, xc)
    res = O.truncate(4, n, k, x, mode="eps", eps=0.0, eps_relative=False)
    assert rel(_full(4, n, res["k"], res["x"]), _full(4, n, k, x)) < 1e-12


def test_eps_truncation_meets_eps():
    (n, ka, xa), (_, kc, xc) = I.brute_pair(7)
    k, x = O.add(4, n, ka, xa, kc, xc)
    full = _full(4, n, k, x)
    for eps in [1e-1, 1e-2, 1e-4]:
        res = O.truncate(4, n, k, x, mode="eps", eps=eps, eps_relative=True)
        err = np.linalg.norm(full - _full(4, n, res["k"], res["x"]))
        assert err <= eps * np.linalg.norm(full) * (1 + 1e-10)
        assert abs(res["norm"] - np.linalg.norm(full)) < 1e-13 * np.linalg.norm(full)



def _eps_ranks_from_svds(d, full, korth, eps, noise):
    """Ranks of the eps rule written out on the singular values of the full
    tensor's matricizations: r_t = smallest r >= 1 with
    sum_{i>r} (sigma_{t,i}^2 + nu_t) <= (eps ||A||)^2 / (2d-3), nu_t = noise sigma_{t,1}^2,
    the root's second son taking the first son's rank."""
    budget = (eps * np.linalg.norm(full)) ** 2 / (2 * d - 3)
    tr = I.tree(d)
    want = [1] * (2 * d - 1)
    for t in range(1, 2 * d - 1):
        s = np.linalg.svd(F.matricization(full, tr["lo"][t], tr["hi"][t]), compute_uv=False)[: int(korth[t])]
        lam = s ** 2 + noise * s[0] ** 2
        tails = [float(np.sum(lam[r:])) for r in range(len(lam) + 1)]
        # no tail within 1e-9 of the budget: the cut is decided by the reading, not by rounding
        assert all(abs(tl - budget) > 1e-9 * budget for tl in tails)
        want[t] = next(r for r in range(1, len(lam) + 1) if tails[r] <= budget)
    want[tr["son2"][0]] = want[tr["son1"][0]]
    return want


@pytest.mark.parametrize("seed,eps", [(5, 3e-1), (5, 1e-1), (7, 3e-2), (7, 1e-2), (2, 1e-3)])
def test_eps_rank_rule_against_full_svds(seed, eps):
    """The eps rank rule (the paper cites [Gr10] without stating it; reading:
    r_t is the smallest r >= 1 whose tail sum_{i>r} sigma_{t,i}^2 fits
    (eps ||A||)^2 / (2d-3), the root's two sons share the rank of the first)
    against singular values of the full tensor's matricizations: a divisor of
    2d-2 or 2d-1, or a cut one place late, changes some rank in these cases.
    (That the root pair's tail is counted once is pinned by the discarded
    energy in the bounds test.)"""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    full = F.frames(d, n, k, x)[1]
    res = O.truncate(d, n, k, x, mode="eps", eps=eps, eps_relative=True)
    want = _eps_ranks_from_svds(d, full, res["korth"], eps, 0.0)
    assert list(res["k"]) == want
    assert len(set(want[1:])) > 1  # the cases cut at different ranks per node


@pytest.mark.parametrize("seed,eps,cap", [(7, 1e-2, 5), (2, 1e-1, 4), (5, 3e-2, 5)])
def test_eps_rank_rule_with_rank_cap(seed, eps, cap):
    """Accuracy with a rank cap (Sec. 5 truncates to an accuracy with a bound
    on the ranks): each node takes the eps rule's rank, then the cap; the
    root's second son follows the first.  The cap cuts below the eps rank at
    some nodes and not at others in these cases."""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    full = F.frames(d, n, k, x)[1]
    res = O.truncate(d, n, k, x, mode="eps", eps=eps, eps_relative=True, rank_cap=cap)
    plain = _eps_ranks_from_svds(d, full, res["korth"], eps, 0.0)
    want = [1] + [min(r, cap) for r in plain[1:]]
    assert list(res["k"]) == want
    assert any(r > cap for r in plain[1:]) and any(r < cap for r in plain[1:])
    # the discarded energy is what the capped ranks leave out, root pair once
    tr = I.tree(d)
    disc = 0.0
    for t in range(1, 2 * d - 1):
        if t == tr["son2"][0]:
            continue
        s = np.linalg.svd(F.matricization(full, tr["lo"][t], tr["hi"][t]), compute_uv=False)
        disc += float(np.sum(s[want[t]:] ** 2))
    assert abs(res["discarded_sq"] - disc) <= 1e-12 * float(np.sum(full ** 2))


@pytest.mark.parametrize("seed,eps,noise", [(7, 1e-2, 3e-6), (7, 3e-2, 1e-5), (5, 1e-1, 3e-4), (5, 3e-1, 3e-3)])
def test_eps_rank_rule_noise_floor(seed, eps, noise):
    """The rule with a charge nu_t = noise * sigma_{t,1}^2 per dropped
    eigenvalue (the charge the FP32 paths apply: an eps below what their
    arithmetic resolves keeps rank) against the full-tensor singular values.
    In these cases the charge decides: the plain rule cuts lower at some node,
    so an oracle that ignored the charge would fail."""
    (n, ka, xa), (_, kc, xc) = I.brute_pair(seed)
    d = 4
    k, x = O.add(d, n, ka, xa, kc, xc)
    full = F.frames(d, n, k, x)[1]
    res = O.truncate(d, n, k, x, mode="eps", eps=eps, eps_relative=True, noise=noise)
    want = _eps_ranks_from_svds(d, full, res["korth"], eps, noise)
    plain = _eps_ranks_from_svds(d, full, res["korth"], eps, 0.0)
    assert list(res["k"]) == want
    assert want != plain and all(w >= p for w, p in zip(want, plain))


def test_golden_diagonal_tensor():
    g = json.load(open(os.path.join(GOLDEN, "diag_d4.json")))
    d, n, k, x = g["d"], np.array(g["n"]), np.array(g["ranks"]), np.array(g["blob"])
    res = O.truncate(d, n, k, x, mode="rank", rank_cap=g["rank"])
    for t in range(1, 2 * d - 1):
        assert np.abs(res["sigma"][t] - np.array(g["sigma"])).max() < 1e-14
    assert abs(res["norm"] - g["norm"]) < 1e-14
    full = _full(d, n, k, x)
    err = np.linalg.norm(full - _full(d, n, res["k"], res["x"]))
    assert abs(err - g["trunc_err"]) < 1e-13
    res = O.truncate(d, n, k, x, mode="eps", eps=g["eps_abs"], eps_relative=False)
    assert list(res["k"][1:]) == [g["eps_rank"]] * 6


def _full_by_eval(d, n, k, x):
    """All entries of an HT tensor by the oracle's evaluation (pinned above
    against the definition), C order.  Used only by the operator-application
    pins below, whose operators live on index pairs."""
    n = np.broadcast_to(np.asarray(n, np.int64), (d,))
    idx = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), axis=-1).reshape(-1, d)
    return O.eval_entries(d, n, k, x, idx).reshape(tuple(int(v) for v in n))


def test_operator_application_equals_full_matrix_vector():
    """Lemma "operator" (Sec. 3.6): the HT representation of C = L X equals the
    product of the full operator (built entry by entry from its own HT
    representation over the index pairs (j, i) = j + i m) with the full tensor."""
    d, m, n = 4, 3, 4
    op = I.random_ht(d, m * n, 2, 31)
    x = I.random_ht(d, n, 3, 32)
    kc, xc = O.apply(d, n, m, op[1], op[2], x[1], x[2])
    assert list(kc[1:]) == [2 * 3] * (2 * d - 2)
    L = _full_by_eval(d, m * n, op[1], op[2])          # L[(j1,i1), ..., (j4,i4)]
    L = L.reshape(n, m, n, m, n, m, n, m)        # axis pair (i, j) from e = j + i m
    X = _full_by_eval(d, n, x[1], x[2])
    C = np.einsum("aebfcgdh,abcd->efgh", L, X)   # axes (i1, j1, ..., i4, j4); C[j] = sum_i L[(j,i)] X[i]
    got = _full_by_eval(d, m, kc, xc)
    assert np.abs(got - C).max() <= 1e-12 * np.abs(C).max()


def test_identity_operator_returns_the_tensor():
    d, n = 5, [4, 6, 3, 5, 2]
    x = I.random_ht(d, n, 3, 33)
    tr = I.tree(d)
    nodes = []
    for t in range(2 * d - 1):
        if tr["son1"][t] < 0:
            nm = n[tr["lo"][t]]
            nodes.append(np.eye(nm).reshape(-1, 1, order="F"))
        else:
            nodes.append(np.ones((1, 1)) if t == 0 else np.ones((1, 1, 1)))
    kop = np.ones(2 * d - 1, np.int32)
    xop = I.nodes_blob(d, nodes)
    kc, xc = O.apply(d, n, n, kop, xop, x[1], x[2])
    assert list(kc) == list(x[1])
    assert np.array_equal(xc, np.asarray(x[2], np.float64))
