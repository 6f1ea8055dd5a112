"""The arithmetic of the mixed path's TSQR row blocks, checked on the CPU
with numpy: Householder QR of FP64 blocks carried out in double-float
arithmetic (every value an unevaluated sum h + l of two FP32 numbers; exact
products by FMA, Knuth's two-sum, Dekker's fast two-sum; square root and
reciprocal from the FP32 operation plus one correction), with every column
scaled by a power of two on conversion.  This emulates the number format and
the steps of the factorisation, not the kernel's layout.

Claims checked: ||a_c - Q r_c|| / ||a_c|| for every column c and
||Q^T Q - I|| stay at a small multiple of 2^-47 (far below the 2^-40 per product of the path's contractions), also for
exactly dependent columns and for columns outside FP32's exponent range; the
same steps in plain FP32 do not get near that (so the checks can tell the
two apart)."""
import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fast_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def two_prod(a, b):
    p = a * b
    # the error of an FP32 product is an FP32 number: exact through FP64
    return p, (a.astype(np.float64) * b.astype(np.float64) - p.astype(np.float64)).astype(f32)


def df_mul(ah, al, bh, bl):
    p, e = two_prod(ah, bh)
    return fast_two_sum(p, e + (ah * bl + al * bh))


def df_add(ah, al, bh, bl):
    s, e = two_sum(ah, bh)
    return fast_two_sum(s, e + (al + bl))


def df_sum(h, l):
    """Sum over axis 0 by a pairwise tree of double-float additions."""
    while h.shape[0] > 1:
        if h.shape[0] % 2:
            z = np.zeros((1,) + h.shape[1:], f32)
            h, l = np.concatenate([h, z]), np.concatenate([l, z])
        h, l = df_add(h[0::2], l[0::2], h[1::2], l[1::2])
    return h[0], l[0]


def df_sqrt(xh, xl):
    r = np.sqrt(xh)
    p, e = two_prod(r, r)
    d = ((xh - p) - e) + xl  # x - r^2
    return fast_two_sum(r, d / (f32(2) * r))


def df_recip(bh, bl):
    q = f32(1) / bh
    ph, pl = df_mul(bh, bl, q, f32(0))
    rh, rl = df_add(f32(1), f32(0), -ph, -pl)  # 1 - b q
    return fast_two_sum(q, q * rh)


def to_df(x):
    h = x.astype(f32)
    return h, (x - h.astype(np.float64)).astype(f32)


def householder_df(A):
    """Q (m x n) and R (n x n) of A (m >= n) in double-float arithmetic."""
    m, n = A.shape
    E = np.zeros(n, np.int64)
    nz = np.abs(A).max(axis=0) > 0
    E[nz] = np.frexp(np.abs(A).max(axis=0)[nz])[1]
    h, l = to_df(np.ldexp(A, -E[None, :]))  # column c scaled by 2^-E_c: exact
    Y = []
    for j in range(n):
        xh, xl = h[j:, j].copy(), l[j:, j].copy()
        ah, al = xh[0], xl[0]
        s2h, s2l = df_sum(*df_mul(xh[1:, None], xl[1:, None], xh[1:, None], xl[1:, None])) if m - j > 1 \
            else (np.array([f32(0)]), np.array([f32(0)]))
        s2h, s2l = s2h[0], s2l[0]
        kh = kl = f32(0)
        bh, bl = ah, al
        yh, yl = xh.copy(), xl.copy()
        if s2h != 0:
            x2h, x2l = df_add(*df_mul(ah, al, ah, al), s2h, s2l)
            nh, nl = df_sqrt(x2h, x2l)
            bh, bl = (nh, nl) if ah <= 0 else (-nh, -nl)
            uh, ul = df_add(ah, al, -bh, -bl)
            ph, pl = df_mul(bh, bl, uh, ul)
            kh, kl = df_recip(-ph, -pl)  # kappa = -1 / (beta u)
            yh[0], yl[0] = uh, ul
        Y.append((yh, yl, kh, kl))
        # trailing columns: a <- a - kappa (y^T a) y
        if j + 1 < n:
            th, tl = df_sum(*df_mul(yh[:, None], yl[:, None], h[j:, j + 1:], l[j:, j + 1:]))
            ch, cl = df_mul(th, tl, kh, kl)
            dh, dl = df_mul(ch[None, :], cl[None, :], yh[:, None], yl[:, None])
            h[j:, j + 1:], l[j:, j + 1:] = df_add(h[j:, j + 1:], l[j:, j + 1:], -dh, -dl)
        h[j, j], l[j, j] = bh, bl
    R = np.triu(h[:n].astype(np.float64) + l[:n].astype(np.float64))
    R = np.ldexp(R, E[None, :])  # column c scaled back by 2^E_c
    # Q = H_0 ... H_{n-1} [I; 0], accumulated backwards
    qh, ql = np.eye(m, n, dtype=f32), np.zeros((m, n), f32)
    for j in reversed(range(n)):
        yh, yl, kh, kl = Y[j]
        th, tl = df_sum(*df_mul(yh[:, None], yl[:, None], qh[j:], ql[j:]))
        ch, cl = df_mul(th, tl, kh, kl)
        dh, dl = df_mul(ch[None, :], cl[None, :], yh[:, None], yl[:, None])
        qh[j:], ql[j:] = df_add(qh[j:], ql[j:], -dh, -dl)
    return qh.astype(np.float64) + ql.astype(np.float64), R


def householder_f32(A):
    """The same steps in plain FP32 (for contrast)."""
    a = A.astype(f32)
    m, n = a.shape
    Y = []
    for j in range(n):
        x = a[j:, j].copy()
        alpha, s2 = x[0], np.dot(x[1:], x[1:])
        kappa, beta, y = f32(0), alpha, x.copy()
        if s2 != 0:
            nrm = np.sqrt(alpha * alpha + s2)
            beta = nrm if alpha <= 0 else -nrm
            y[0] = alpha - beta
            kappa = f32(-1) / (beta * y[0])
        Y.append((y, kappa))
        a[j:, j + 1:] -= kappa * np.outer(y, y @ a[j:, j + 1:])
        a[j, j] = beta
    q = np.eye(m, n, dtype=f32)
    for j in reversed(range(n)):
        y, kappa = Y[j]
        q[j:] -= kappa * np.outer(y, y @ q[j:])
    return q.astype(np.float64), np.triu(a[:n]).astype(np.float64)


def _errors(A, Q, R):
    """Largest columnwise backward error ||a_c - Q r_c|| / ||a_c|| (Householder
    QR is backward stable column by column, so columns 2^600 apart are each
    held to it) and largest entry of Q^T Q - I."""
    back = (np.linalg.norm(A - Q @ R, axis=0) / np.linalg.norm(A, axis=0)).max()
    orth = np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()
    return back, orth


def _block(kind, m=256, n=32, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    if kind == "dependent":  # exactly dependent columns, as in the QR of X + X
        A[:, n // 2:] = A[:, : n - n // 2]
    elif kind == "range":  # columns far outside FP32's exponent range, and graded within
        A *= np.exp2(rng.integers(-300, 300, n))[None, :]
    elif kind == "graded":  # singular values over 12 decades
        U, _ = np.linalg.qr(rng.standard_normal((m, n)))
        V, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = (U * np.logspace(0, -12, n)) @ V.T
    return A


@pytest.mark.parametrize("kind", ["gauss", "dependent", "range", "graded"])
def test_double_float_householder_at_2_to_minus_47(kind):
    A = _block(kind)
    Q, R = householder_df(A)
    back, orth = _errors(A, Q, R)
    u = 2.0 ** -47
    assert back <= 16 * u and orth <= 16 * u, (back / u, orth / u)
    assert np.abs(np.tril(R, -1)).max() == 0.0


def test_plain_fp32_is_far_from_it():
    A = _block("gauss")
    Q, R = householder_f32(A)
    back, orth = _errors(A, Q, R)
    assert back > 2.0 ** -30 and orth > 2.0 ** -30
