"""Helpers of the GPU parity tests: run a workload through the C-ABI and
through the oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I


U32 = 2.0 ** -24


def fp32_tol(d):
    """Tolerance of the FP32-storage path on ||X|| and on the truncated tensor:
    1e-6, widened for deep trees to 4 sqrt(2d-1) u_32 because every one of the
    2d-1 nodes rounds its orthogonalized factors to FP32 independently (the
    errors add like a random walk over the nodes)."""
    return max(1e-6, 4.0 * np.sqrt(2 * d - 1) * U32)


def fp32_tol_sigma(d):
    """Tolerance of the FP32-storage path on sigma^2 (normwise per node): every
    Gramian carries twice the relative error of ||X||^2's scale, plus one FP32
    contraction error per level of the top-down recursion (depth = ceil(log2 d))."""
    depth = int(np.ceil(np.log2(d)))
    return max(1e-6, 2.0 * fp32_tol(d) + 4.0 * depth * U32)


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


def rank_noise_ok(sig_ref, r_gpu, r_ref, tail2, tol):
    """A rank decision differing from the oracle's is acceptable only if the
    oracle's discarded tails at every cut between the two lie within tol of
    the per-node threshold tail2 (the decision is then below the arithmetic's
    resolution)."""
    lam = np.maximum(np.asarray(sig_ref, dtype=np.float64) ** 2, 0.0)
    tails = [float(np.sum(lam[r:])) for r in range(len(lam) + 1)]
    lo, hi = min(r_gpu, r_ref), max(r_gpu, r_ref)
    # keeping lo must (nearly) violate, keeping hi must (nearly) satisfy the threshold
    return tails[hi] <= tail2 + tol and tails[lo] >= tail2 - tol


def rank_diff_energy(sig_ref, r_gpu, r_ref):
    """sqrt of the oracle's sigma^2 between two cuts of one node."""
    lo, hi = min(r_gpu, r_ref), max(r_gpu, r_ref)
    return float(np.sqrt(np.sum(np.asarray(sig_ref[lo:hi], dtype=np.float64) ** 2)))


def check_ranks(ranks_gpu, ref, tol_rel, eps_mode):
    """Compare ranks; returns (differing nodes, energy bound of their effect)."""
    differ = [t for t in range(1, len(ranks_gpu)) if int(ranks_gpu[t]) != int(ref["k"][t])]
    if not eps_mode:
        assert not differ, (list(ranks_gpu), list(ref["k"]))
    e2 = 0.0
    for t in differ:
        s = ref["sigma"][t]
        lam_max = float(s[0]) ** 2 if len(s) else 0.0
        assert rank_noise_ok(s, int(ranks_gpu[t]), int(ref["k"][t]), ref["tail2"], len(s) * tol_rel * lam_max), \
            (t, int(ranks_gpu[t]), int(ref["k"][t]))
        e2 += rank_diff_energy(s, int(ranks_gpu[t]), int(ref["k"][t]))
    # projections that differ at several nodes: the truncated tensors differ by at
    # most the sum (telescoping over the nodes) of the energies between the cuts
    return differ, float(e2)
