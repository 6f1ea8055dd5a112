"""Writes tests/golden/diag_d4.json: a closed-form HT tensor and its exact HSVD data.

The tensor is A = sum_i c_i e_i (x) e_i (x) e_i (x) e_i (d = 4, n = 6, k = 4)
written in the HT format of Sec. 2.2 with NON-orthonormal leaf frames:
leaf mu has U_mu = [e_1 .. e_k] diag(w_mu), the inner nodes t = {1,2}, {3,4}
have B_t[i,j,l] = delta_{ijl} / (w_s1[j] w_s2[l]) so that U_t = [e_i (x) e_i]
(Lemma "transfer tensor transformation" with Y = diag(w)), and the root is
B_D = diag(c).  Every matricization M_t(A) is sum_i c_i (e_i..)(e_i..)^T, so
its singular values are |c_i| sorted (Definition "matricization"); the
truncation to rank r keeps the r largest |c_i| and its error is
sqrt(sum of the discarded c_i^2) (Sec. 3.3).  All numbers below follow from
these closed forms; no library or oracle routine is called.
"""
import json
import os

d, n, k = 4, 6, 4
c = [3.0, -5.0, 0.5, 2.0]
w = [[1.0, 2.0, 4.0, 8.0], [1.0, 1.0, 1.0, 1.0], [0.5, 0.5, 2.0, 2.0], [3.0, 1.0, 1.0, 1.0]]
# pre-order nodes for d = 4: 0 root, 1 {0,1}, 2 leaf 0, 3 leaf 1, 4 {2,3}, 5 leaf 2, 6 leaf 3
leaf_of = {2: 0, 3: 1, 5: 2, 6: 3}
inner_sons = {1: (2, 3), 4: (5, 6)}
blob = []
for t in range(7):
    if t == 0:
        blob += [c[j] if j == l else 0.0 for j in range(k) for l in range(k)]
    elif t in leaf_of:
        mu = leaf_of[t]
        for col in range(k):  # column-major n x k
            blob += [w[mu][col] if row == col else 0.0 for row in range(n)]
    else:
        s1, s2 = inner_sons[t]
        w1, w2 = w[leaf_of[s1]], w[leaf_of[s2]]
        blob += [(1.0 / (w1[j] * w2[l]) if (i == j == l) else 0.0) for i in range(k) for j in range(k) for l in range(k)]
sig = sorted([abs(v) for v in c], reverse=True)
r = 2
err2 = sum(s * s for s in sig[r:])
# eps rank: the smallest r with sum_{i>r} sig_i^2 <= eps^2/(2d-3).  Tails: r=2 -> 4.25,
# r=3 -> 0.25.  With absolute eps = 1.2 the per-node budget is 1.44/5 = 0.288, so r = 3.
eps_abs = 1.2
out = dict(
    d=d, n=[n] * d, ranks=[1] + [k] * 6, blob=blob,
    sigma=sig, norm=sum(v * v for v in c) ** 0.5,
    rank=r, trunc_err=err2 ** 0.5,
    trunc_kept=[v for v in c if abs(v) in sig[:r]],
    eps_abs=eps_abs, eps_rank=3,
    cite="closed form; Definition 'matricization', Sec. 2.2 eq. 'transfer', Sec. 3.3",
)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "diag_d4.json"), "w") as f:
    json.dump(out, f, indent=1)
