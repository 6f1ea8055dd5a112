"""The arithmetic of the mixed path's eigenvector accumulation, checked on
the CPU with numpy: the QL sweeps' Givens rotations, computed in FP64 by the
recurrence, applied to the eigenvector matrix in double-float arithmetic
(pairs of FP32 numbers; each rotation's c and s converted to pairs, products
exact by FMA, sums by two-sum and renormalised).  This emulates the number
format and the update, not the kernel's layout.

Claim checked: after as many rotations as a 128 x 128 solve takes (about k
per eigenvalue), the eigenvectors stay orthonormal to 1e-12 and within 1e-12
of the same rotations applied in FP64; plain FP32 rotations do not."""
import numpy as np

from tests.test_double_float_qr import fast_two_sum, to_df, two_prod, two_sum

f32 = np.float32


def df_prod(ah, al, bh, bl):
    """Unnormalised product (p, e): p + e = (ah + al)(bh + bl) to 2^-47."""
    p, e = two_prod(ah, bh)
    return p, e + (ah * bl + al * bh)


def test_double_float_rotations_keep_eigenvectors_orthonormal():
    k, n_rot = 128, 128 * 128
    rng = np.random.default_rng(0)
    theta = rng.uniform(0.0, 2.0 * np.pi, n_rot)
    cols = rng.integers(0, k - 1, n_rot)
    c64, s64 = np.cos(theta), np.sin(theta)
    zh, zl = np.eye(k, dtype=f32), np.zeros((k, k), f32)
    z64, z32 = np.eye(k), np.eye(k, dtype=f32)
    for q in range(n_rot):
        i = cols[q]
        ch, cl = to_df(np.array(c64[q]))
        sh, sl = to_df(np.array(s64[q]))
        bh0, bl0, h1, l1 = zh[:, i].copy(), zl[:, i].copy(), zh[:, i + 1].copy(), zl[:, i + 1].copy()
        # a = s z_i + c z_{i+1}, b = c z_i - s z_{i+1}, each renormalised
        p1, e1 = df_prod(sh, sl, bh0, bl0)
        p2, e2 = df_prod(ch, cl, h1, l1)
        ah, t = two_sum(p1, p2)
        ah, al = fast_two_sum(ah, t + (e1 + e2))
        p1, e1 = df_prod(ch, cl, bh0, bl0)
        p2, e2 = df_prod(sh, sl, h1, l1)
        bh, t = two_sum(p1, -p2)
        bh, bl = fast_two_sum(bh, t + (e1 - e2))
        zh[:, i + 1], zl[:, i + 1], zh[:, i], zl[:, i] = ah, al, bh, bl
        a64 = s64[q] * z64[:, i] + c64[q] * z64[:, i + 1]
        z64[:, i] = c64[q] * z64[:, i] - s64[q] * z64[:, i + 1]
        z64[:, i + 1] = a64
        c, s = f32(c64[q]), f32(s64[q])
        a32 = s * z32[:, i] + c * z32[:, i + 1]
        z32[:, i] = c * z32[:, i] - s * z32[:, i + 1]
        z32[:, i + 1] = a32
    eye = np.eye(k)
    z = zh.astype(np.float64) + zl.astype(np.float64)
    assert np.abs(z.T @ z - eye).max() <= 1e-12
    assert np.abs(z - z64).max() <= 1e-12
    z32 = z32.astype(np.float64)
    assert np.abs(z32.T @ z32 - eye).max() > 1e-8
