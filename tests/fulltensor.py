"""Independent dense helpers for the brute-force pins (numpy only).

Builds the full tensor of an HT representation straight from the definition
of the transfer tensors (Sec. 2.2, eq. "transfer"), forms matricizations
(Definition "matricization") and runs the full-tensor truncation by SVDs of
all matricizations (Sec. 3.3, the three-step procedure before the HSVD).
None of this calls the oracle.
"""
import numpy as np

from paper_1708_03340_gb300 import inputs as I


def frames(d, n, ranks, blob):
    """Frames U_t (N_t x k_t) of every node, bottom-up; returns (frames, full tensor as d-dim array)."""
    tr = I.tree(d)
    nodes = I.blob_nodes(d, n, ranks, blob)
    nn = 2 * d - 1
    U = [None] * nn

    def rec(t):
        if tr["son1"][t] < 0:
            U[t] = np.asarray(nodes[t])
            return
        s1, s2 = tr["son1"][t], tr["son2"][t]
        rec(s1)
        rec(s2)
        B = nodes[t] if t != 0 else nodes[t][None, :, :]
        # (U_t)_{-,i} = sum_{j,l} B[i,j,l] U_s1[:,j] (x) U_s2[:,l]; the row index of
        # U_t is (row of s1, row of s2) with the s2 row fastest (numpy kron order)
        Ut = np.einsum("ijl,aj,bl->abi", B, U[s1], U[s2])
        U[t] = Ut.reshape(U[s1].shape[0] * U[s2].shape[0], B.shape[0])

    rec(0)
    nvec = np.broadcast_to(np.asarray(n), (d,))
    full = U[0][:, 0].reshape(tuple(int(v) for v in nvec))
    return U, full


def matricization(full, lo, hi):
    """M_t(A) for t = {lo..hi}: rows the modes of t, columns the rest."""
    d = full.ndim
    rows = list(range(lo, hi + 1))
    cols = [m for m in range(d) if m < lo or m > hi]
    A = np.transpose(full, rows + cols)
    nr = int(np.prod([full.shape[m] for m in rows]))
    return A.reshape(nr, -1)


def brute_truncate(d, full, ranks):
    """Truncation of a full tensor by SVDs of all matricizations (Sec. 3.3):
    U_t = leading r_t left singular vectors of M_t(A); B_t[i,j,l] = <U_t[:,i],
    U_s1[:,j] (x) U_s2[:,l]>; B_D[j,l] = <M_D(A), U_t1[:,j] (x) U_t2[:,l]>.
    Returns the full tensor of the result."""
    tr = I.tree(d)
    nn = 2 * d - 1
    U = [None] * nn
    for t in range(1, nn):
        M = matricization(full, tr["lo"][t], tr["hi"][t])
        u, s, vt = np.linalg.svd(M, full_matrices=False)
        U[t] = u[:, : ranks[t]]
    B = [None] * nn
    for t in range(nn):
        if tr["son1"][t] < 0:
            continue
        s1, s2 = tr["son1"][t], tr["son2"][t]
        K = np.einsum("aj,bl->abjl", U[s1], U[s2]).reshape(U[s1].shape[0] * U[s2].shape[0], U[s1].shape[1] * U[s2].shape[1])
        Ut = full.reshape(-1, 1) if t == 0 else U[t]
        B[t] = (Ut.T @ K).reshape(Ut.shape[1], U[s1].shape[1], U[s2].shape[1])
    # rebuild the full tensor top-down from leaves
    def rec(t):
        if tr["son1"][t] < 0:
            return U[t]
        s1, s2 = tr["son1"][t], tr["son2"][t]
        a, b = rec(s1), rec(s2)
        return np.einsum("ijl,aj,bl->abi", B[t], a, b).reshape(a.shape[0] * b.shape[0], B[t].shape[0])
    return rec(0)[:, 0].reshape(full.shape)
