"""Helpers of the GPU parity tests: run a workload through the C-ABI and
through the oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I


U32 = 2.0 ** -24


def fp32_tol(d, K=64):
    """Tolerance of the FP32-storage path on ||X|| and on the truncated tensor.
    Householder QR applies up to K reflectors to every column of a node's K
    columns, each a rounding in FP32, so a node's orthogonalization perturbs X
    by about sqrt(K) u_32 (a random walk over the K roundings); the 2d-1 nodes
    round independently and add like a random walk over the nodes, and a
    factor 4 covers the tail: 4 sqrt(K (2d-1)) u_32, at least 1e-6."""
    return max(1e-6, 4.0 * np.sqrt(K * (2 * d - 1)) * U32)


def fp32_tol_sigma(d, K=64):
    """Tolerance of the FP32-storage path on sigma^2 (normwise per node): every
    Gramian carries twice the relative error of ||X||^2's scale, plus one FP32
    contraction error per level of the top-down recursion (depth = ceil(log2 d))."""
    depth = int(np.ceil(np.log2(d)))
    return max(1e-6, 2.0 * fp32_tol(d, K) + 4.0 * depth * U32)


def as_stored(blob, dtype):
    """The tensor the GPU path actually holds: F32 tensors store FP32-rounded
    inputs, so the oracle is run on the same rounded values (input rounding is
    not an error of the path)."""
    b = np.asarray(blob, dtype=np.float64)
    return b.astype(np.float32).astype(np.float64) if dtype == htgb.HT_F32 else b


def gpu_sum(d, n, a, c, dtype):
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, n, a[1], a[2], dtype)
    C = htgb.HTTensor.from_blob(tree, n, c[1], c[2], dtype)
    X = A.add(C)
    return tree, A, C, X


def split_sigma(korth, sig):
    out, o = [np.zeros(0)], 0
    for t in range(1, len(korth)):
        out.append(sig[o:o + korth[t]])
        o += int(korth[t])
    return out


def sample_idx(n, m, seed=0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, int(v), m) for v in n], axis=1)


def check_sigma(sg_gpu, sg_ref, tol, floor=0.0):
    """|sigma_i^2 - sigma_ref_i^2| <= tol * sigma_max^2 for sigma_ref_i >= floor * sigma_max (per node).
    Returns the worst normwise error seen."""
    worst = 0.0
    for t in range(1, len(sg_ref)):
        a, b = np.asarray(sg_gpu[t]), np.asarray(sg_ref[t])
        assert a.shape == b.shape, (t, a.shape, b.shape)
        smax = max(b.max(), 1e-300)
        sel = b >= floor * smax
        err = np.abs(a[sel] ** 2 - b[sel] ** 2).max() / smax ** 2 if sel.any() else 0.0
        worst = max(worst, err)
        assert err <= tol, (t, err)
    return worst


def noise_floor(d, dtype, prec=None):
    """Charge per dropped eigenvalue (relative to the node's largest
    eigenvalue) that the library's eps rule applies on a path: none on the
    FP64 and mixed paths (the plain rule on the computed tail, as the oracle
    runs by default); 4 sqrt(2d-1) u_32 on the FP32 path, whose Gramians do
    not resolve eigenvalues below that; its square on the square-root path.
    The oracle is run with the same charge, so both sides apply one rule."""
    if prec is None:
        prec = htgb.HT_PREC_FP64 if dtype == htgb.HT_F64 else htgb.HT_PREC_FP32
    if prec in (htgb.HT_PREC_FP64, getattr(htgb, "HT_PREC_MIXED", -1)):
        return 0.0
    nu = 4.0 * np.sqrt(2 * d - 1) * 2.0 ** -24
    return nu * nu if prec == htgb.HT_PREC_FP32_SQRT else nu


def rank_diff_energy(sig_ref, r_gpu, r_ref):
    """sqrt of the oracle's sigma^2 between two cuts of one node."""
    lo, hi = min(r_gpu, r_ref), max(r_gpu, r_ref)
    return float(np.sqrt(np.sum(np.asarray(sig_ref[lo:hi], dtype=np.float64) ** 2)))


def check_ranks(ranks_gpu, ref, tol_rel, eps_mode, d=None, dtype=None, prec=None):
    """Compare ranks with the oracle's (run with the path's own noise charge).

    Rank mode: equal.  Eps mode: ranks are discontinuous in the eigenvalues,
    so a node may differ where the oracle's tail at the library's cut lies
    within the path's eigenvalue error (tol_rel * lambda_max per eigenvalue)
    of the per-node budget: one more kept direction than the oracle only if
    dropping it fails the budget within that error, one fewer only if dropping
    it fits the budget within that error.
    Returns (differing nodes, bound on the effect on the truncated tensor:
    the sum over those nodes of the oracle's energy between the two cuts)."""
    differ = [t for t in range(1, len(ranks_gpu)) if int(ranks_gpu[t]) != int(ref["k"][t])]
    if not eps_mode:
        assert not differ, (list(ranks_gpu), list(ref["k"]))
        return differ, 0.0
    nu = noise_floor(d, dtype, prec)
    energy = 0.0
    for t in differ:
        s = np.asarray(ref["sigma"][t], dtype=np.float64)
        rg, rr = int(ranks_gpu[t]), int(ref["k"][t])
        lam = np.maximum(s, 0.0) ** 2
        lam_max = lam[0] if len(lam) else 0.0
        charged = lam + nu * lam_max
        slack = len(lam) * tol_rel * lam_max
        if rg > rr:  # the library could not drop eigenvalue rg-1 (0-based)
            assert float(np.sum(charged[rg - 1:])) + slack >= ref["tail2"], (t, rg, rr)
        else:        # the library dropped down to rg where the oracle stopped at rr
            assert float(np.sum(charged[rg:])) - slack <= ref["tail2"], (t, rg, rr)
        energy += rank_diff_energy(s, rg, rr)
    return differ, float(energy)


def gap_allowance(sig_ref, ranks, eps_g):
    """Bound on how far two truncations of the same tensor may lie apart when
    their Gramians differ by eps_g * lambda_max per node: at node t the kept
    r_t-dimensional eigenspace turns by at most eps_g lambda_1 / (lambda_r -
    lambda_{r+1}) (Davis-Kahan), which moves the projection by that angle
    times the energy of the two directions at the cut.  Summed over the
    nodes; the truncated tensor is unique only where lambda_r > lambda_{r+1}."""
    total = 0.0
    for t in range(1, len(ranks)):
        lam = np.asarray(sig_ref[t], dtype=np.float64) ** 2
        r = int(ranks[t])
        if r >= len(lam) or len(lam) == 0:
            continue
        gap = lam[r - 1] - lam[r]
        near = np.sqrt(lam[r - 1] + lam[r])
        angle = 1.0 if gap <= 0 else min(1.0, eps_g * lam[0] / gap)
        total += angle * near
    return float(total)
