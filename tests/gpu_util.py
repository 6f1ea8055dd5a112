"""Helpers of the GPU parity tests: run a workload through the C-ABI and
through the oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I


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
