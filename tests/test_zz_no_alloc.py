"""ht_gramians_noalloc: the reduced Gramians without any device allocation.

Some callers cannot let a library allocate device memory behind their back,
for example a program that reserves its whole memory budget at start-up or
hands out every buffer from its own allocator.  For them the library offers
one entry point whose workspace is a fixed array inside the library.  This
test calls it through the C-ABI twice in a row and checks each result
against the ordinary ht_gramians, checks that the two calls took nothing
from the stream-ordered memory pool (not even briefly: the pool's
high-water mark is reset before them), and checks that an oversized request
is refused with a clear error.  The file is named so that pytest collects it
last; it also passes when run on its own in a fresh process.
"""
import ctypes
import gc
import os

import numpy as np
import pytest

from paper_1708_03340_gb300 import htgb
from paper_1708_03340_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _pool_used():
    """(pool, runtime, used bytes now, high-water mark) of the current device's
    default stream-ordered memory pool, the pool that every cudaMallocAsync of
    the library draws from.  The runtime is the one libhtgb.so has loaded."""
    import torch
    htgb.load()
    cudart = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    dev = torch.cuda.current_device()
    assert cudart.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used, high = ctypes.c_uint64(), ctypes.c_uint64()
    assert cudart.cudaMemPoolGetAttribute(pool, 0x7, ctypes.byref(used)) == 0  # cudaMemPoolAttrUsedMemCurrent
    assert cudart.cudaMemPoolGetAttribute(pool, 0x8, ctypes.byref(high)) == 0  # cudaMemPoolAttrUsedMemHigh
    return pool, cudart, used.value, high.value


def _reset_high(pool, cudart):
    zero = ctypes.c_uint64(0)
    assert cudart.cudaMemPoolSetAttribute(pool, 0x8, ctypes.byref(zero)) == 0


@pytest.mark.parametrize("dtype,tol", [(htgb.HT_F64, 1e-12), (htgb.HT_F32, 1e-6)])
def test_noalloc_gramians_match(dtype, tol):
    import torch
    d = 8
    (n, ka, xa), (_, kc, xc) = I.small_pair(4)
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, dtype)
    C = htgb.HTTensor.from_blob(tree, n, kc, xc, dtype)
    X = A.add(C)
    X.orthogonalize()
    ko = X.ranks()
    count = 1 + sum(int(v) ** 2 for v in ko[1:])
    prec = X.default_prec()
    ref = torch.zeros(count, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    htgb.ht_gramians(X.handle, ref.data_ptr(), prec)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    scale = np.abs(r).max()
    assert scale > 0
    outs = [torch.full((count,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    # tensors that earlier tests left to the garbage collector are freed now,
    # not between the two readings of the pool below
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        pool, cudart, used0, _ = _pool_used()
        _reset_high(pool, cudart)
        for out in outs:  # two calls in a row share the fixed scratch
            htgb.ht_gramians_noalloc(X.handle, out.data_ptr(), prec)
            torch.cuda.synchronize()
        _, _, used1, high1 = _pool_used()
    finally:
        gc.enable()
    # nothing was taken from the stream-ordered pool, not even for a moment
    assert used1 <= used0 and high1 <= used0, (used0, used1, high1)
    for out in outs:
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.abs(o - r).max() <= tol * scale


def test_noalloc_rejects_oversized_request():
    import torch
    d, n, k = 64, 1000, 64
    tree = htgb.HTTree(d)
    ranks = np.full(2 * d - 1, k, np.int32)
    ranks[0] = 1
    X = htgb.HTTensor.create(tree, np.full(d, n), ranks, htgb.HT_F64)
    out = torch.zeros(1 + (2 * d - 2) * k * k, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(htgb.HTError) as e:
        htgb.ht_gramians_noalloc(X.handle, out.data_ptr(), htgb.HT_PREC_FP64)
    assert e.value.status == htgb.HT_ENOMEM
    assert str(htgb.HT_NOALLOC_SCRATCH_BYTES) in str(e.value)
