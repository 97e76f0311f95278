"""lt_product_noalloc: the *_L-product for callers that cannot allocate device memory.

Such callers (an application whose own pool owns all GPU memory, or code that must not
call cudaMalloc because it may synchronise the device) cannot hand lt_product a
workspace; lt_product_noalloc uses a fixed array inside the library instead.  These
tests call it through the C ABI and check it against lt_product on the same inputs,
for two calls in a row with different operands (the array keeps the previous call's
contents, which must not leak into the next result).  This file is collected last so
that a run stopping at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_02870_gb300 import lt
from tests.gpu_util import empty_dev, make_ctx, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


def call_noalloc(ctx, A, B, Cout, I1, l, I2):
    st = torch.cuda.current_stream().cuda_stream
    return lt.lib().lt_product_noalloc(ctx.handle, I1, l, I2, ctypes.c_void_p(A.data_ptr()),
                                       ctypes.c_void_p(B.data_ptr()),
                                       ctypes.c_void_p(Cout.data_ptr()), ctypes.c_void_p(st))


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
def test_noalloc_matches_lt_product_on_two_calls(prec):
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    transforms = [("dct", 3), ("dct", 8)]
    ctx = make_ctx(transforms, prec)
    rng = np.random.default_rng(2024)
    for I1, l, I2 in ((32, 24, 16), (65, 9, 40)):  # two calls, different operands
        A = rng.uniform(-1, 1, (I1, l, 3, 8))
        B = rng.uniform(-1, 1, (l, I2, 3, 8))
        Ad, Bd = to_dev(A, dt), to_dev(B, dt)
        ref = empty_dev((I1, I2, 3, 8), dt)
        lt.lt_product(ctx, Ad, Bd, ref)
        out = empty_dev((I1, I2, 3, 8), dt).fill_(float("nan"))
        assert call_noalloc(ctx, Ad, Bd, out, I1, l, I2) == lt.LT_OK
        torch.cuda.synchronize()
        assert rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL[prec]


def test_noalloc_rejects_sizes_beyond_its_array():
    ctx = make_ctx([("dct", 4)])
    # L(A) alone would need 4 * 1024 * 1024 * 8 bytes = 32 MiB: over the limit with L(B)
    I1, l, I2 = 1024, 1024, 1
    A = torch.zeros((4, l, I1), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, I2, l), dtype=torch.float64, device="cuda")
    Cout = torch.zeros((4, I2, I1), dtype=torch.float64, device="cuda")
    assert call_noalloc(ctx, A, B, Cout, I1, l, I2) == -2  # LT_ERR_SHAPE, nothing enqueued
