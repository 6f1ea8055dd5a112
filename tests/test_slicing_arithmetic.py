"""The arithmetic the mixed path's tensor-core contractions rest on, checked
on the CPU with numpy (an emulation of the number formats, not of the
kernels): FP64 operands cut into S balanced base-256 digits on a per-row grid
(the splitting idea of Ozaki et al., "Error-free transformations of matrix
multiplication", for BF16 operands).

Claims checked:
  * the digits rebuild the rounded row exactly, and every slice is a BF16
    value (its FP32 bits have a zero low half);
  * over <= 256 products the slice products of the diagonals i + j = 0 and
    i + j = 1 sum exactly in FP32, in any order, even for digits at their
    extremes;
  * with the remaining products accumulated in FP32 (one accumulator for
    i + j >= 2 with S = 5; i + j = 2 and i + j >= 3 apart with S = 6), a
    256-long dot product stays within a few steps of the operands' row grids,
    2^(E_a - 8S) sum |b| + 2^(E_b - 8S) sum |a|: about 2^-40 (S = 5) and 2^-48
    (S = 6) of the row scale per product; for Gaussian rows about 5e-12 and
    3e-14 of |a| |b|."""
import math

import numpy as np
import pytest

CHUNK = 256


def grid_exponents(x):
    """Per row: the smallest E with |x| < 2^E over the row (0 for a zero row)."""
    m = np.abs(x).max(axis=1)
    e = np.zeros(len(m), np.int64)
    nz = m > 0
    e[nz] = np.frexp(m[nz])[1]  # m = f 2^e with f in [0.5, 1): m < 2^e
    return e


def digits(x, S):
    """Balanced base-256 digits of round(|x| 2^(8S - E)) per entry: d_0 in
    [0, 256], d_i in [-128, 127]; returns (d (S, rows, K) int64, sign, E)."""
    E = grid_exponents(x)
    X = np.ldexp(np.abs(x), (8 * S - E)[:, None])  # exact: a power-of-two scaling
    F = np.rint(X).astype(np.int64)
    assert F.max() <= 2 ** (8 * S)
    bias = sum(128 << (8 * j) for j in range(S - 1))
    G = F + bias
    d = np.zeros((S,) + x.shape, np.int64)
    for i in range(1, S):
        d[i] = ((G >> (8 * (S - 1 - i))) & 255) - 128
    d[0] = G >> (8 * (S - 1))
    return d, np.sign(x).astype(np.int64), E


def slices(d, sign, S):
    """Slice i = sign d_i 2^(-8(i+1)) as FP32 values."""
    return np.stack([np.ldexp((sign * d[i]).astype(np.float64), -8 * (i + 1)) for i in range(S)]).astype(np.float32)


def _rows(rng, rows, K, kind):
    if kind == "gauss":
        return rng.standard_normal((rows, K)) * np.exp2(rng.integers(-30, 30, (rows, 1)))
    if kind == "spread":  # entries across 40 binades within a row
        return rng.standard_normal((rows, K)) * np.exp2(rng.integers(-40, 0, (rows, K)))
    raise ValueError(kind)


@pytest.mark.parametrize("S", [2, 5, 6])
@pytest.mark.parametrize("kind", ["gauss", "spread"])
def test_digits_rebuild_the_row_and_slices_are_bf16(S, kind):
    rng = np.random.default_rng(S)
    x = _rows(rng, 32, CHUNK, kind)
    x[0, :] = 0.0
    x[1, :5] = [1.0, -1.0, 0.5, 2.0 ** -60, -(1 - 2.0 ** -53)]  # exact powers of two, a value rounding up
    d, sign, E = digits(x, S)
    assert d[0].min() >= 0 and d[0].max() <= 256
    if S > 1:
        assert d[1:].min() >= -128 and d[1:].max() <= 127
    # the digits rebuild F = round(|x| 2^(8S - E)) exactly
    F = sum(d[i] << (8 * (S - 1 - i)) for i in range(S))
    assert np.array_equal(F, np.rint(np.ldexp(np.abs(x), (8 * S - E)[:, None])).astype(np.int64))
    # ... so the slices sum to x within half a grid step, 2^(E - 8S - 1)
    s = slices(d, sign, S).astype(np.float64)
    back = np.ldexp(s.sum(axis=0), E[:, None])
    assert np.all(np.abs(back - x) <= np.ldexp(1.0, E - 8 * S - 1)[:, None])
    # every slice is a BF16 value: the low 16 bits of its FP32 pattern are zero
    assert np.all((s.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def _fp32_sums_any_order(terms, rng, orders=4):
    """FP32 sums of the last axis in several random orders (sequential)."""
    out = []
    for _ in range(orders):
        p = rng.permutation(terms.shape[-1])
        out.append(np.cumsum(terms[..., p], axis=-1, dtype=np.float32)[..., -1])
    return out


@pytest.mark.parametrize("S", [5, 6])
def test_leading_diagonals_sum_exactly_in_fp32(S):
    rng = np.random.default_rng(10 + S)
    a = _rows(rng, 8, CHUNK, "gauss")
    b = _rows(rng, 8, CHUNK, "gauss")
    # extremes: rows whose digits sit at the ends of their ranges
    a[0] = 1.0 - 2.0 ** -(8 * S + 1)        # rounds up to d_0 = 256, other digits 0
    b[0] = -(1.0 - 2.0 ** -(8 * S + 1))
    a[1] = 0.5 + 127 / 256 * 2.0 ** -8      # d_0 = 128, d_1 = 127
    b[1] = -(0.75 + 128 / 256 * 2.0 ** -8)  # d_0 = 193, d_1 = -128 (the balancing carry)
    da, sa, _ = digits(a, S)
    db, sb, _ = digits(b, S)
    assert (da[0, 0, 0], db[0, 0, 0]) == (256, 256)
    assert (da[0, 1, 0], da[1, 1, 0], db[0, 1, 0], db[1, 1, 0]) == (128, 127, 193, -128)
    A = slices(da, sa, S)  # (S, rows, K)
    B = slices(db, sb, S)
    for diag in (0, 1):
        pairs = [(i, diag - i) for i in range(diag + 1)]
        # products of BF16 values are exact in FP32; the terms of one output
        terms = np.concatenate([A[i][:, None, :] * B[j][None, :, :] for i, j in pairs], axis=-1)
        # the exact sum, in integers of the diagonal's grid 2^(-8(diag + 2))
        ia = np.stack([sa * da[i] for i in range(S)])
        ib = np.stack([sb * db[j] for j in range(S)])
        exact = sum(ia[i][:, None, :] * ib[j][None, :, :] for i, j in pairs).sum(axis=-1)
        assert np.abs(exact).max() <= 2 ** 24
        for got in _fp32_sums_any_order(terms.astype(np.float32), rng):
            assert np.array_equal(np.ldexp(got.astype(np.float64), 8 * (diag + 2)), exact.astype(np.float64))


@pytest.mark.parametrize("S,gauss_bound", [(5, 1e-11), (6, 5e-14)])
@pytest.mark.parametrize("ka,kb", [("gauss", "gauss"), ("spread", "gauss"), ("spread", "spread")])
def test_sliced_dot_products_within_the_stated_error(S, gauss_bound, ka, kb):
    rng = np.random.default_rng(20 + S)
    a = _rows(rng, 8, CHUNK, ka)
    b = _rows(rng, 8, CHUNK, kb)
    da, sa, Ea = digits(a, S)
    db, sb, Eb = digits(b, S)
    A, B = slices(da, sa, S), slices(db, sb, S)
    groups = [[0], [1], list(range(2, S))] if S == 5 else [[0], [1], [2], list(range(3, S))]
    acc = []
    for g in groups:
        terms = np.concatenate([A[i][:, None, :] * B[s - i][None, :, :] for s in g for i in range(s + 1)], axis=-1)
        acc.append(_fp32_sums_any_order(terms.astype(np.float32), rng, orders=1)[0].astype(np.float64))
    got = np.ldexp(sum(acc), Ea[:, None] + Eb[None, :])
    for r in range(a.shape[0]):
        for c in range(b.shape[0]):
            exact = math.fsum(float(u) * float(v) for u, v in zip(a[r], b[c]))
            err = abs(got[r, c] - exact)
            grid = np.ldexp(np.abs(b[c]).sum(), int(Ea[r]) - 8 * S) + np.ldexp(np.abs(a[r]).sum(), int(Eb[c]) - 8 * S)
            assert err <= 4 * grid, (r, c, err / grid)
            if ka == kb == "gauss":
                assert err <= gauss_bound * np.linalg.norm(a[r]) * np.linalg.norm(b[c])
