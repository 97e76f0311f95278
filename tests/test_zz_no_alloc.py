"""lt_product_noalloc: the *_L-product for callers that cannot allocate device memory.

Such callers (an application whose own pool owns all GPU memory, or code that must not
call cudaMalloc because it may synchronise the device) cannot hand lt_product a
workspace; lt_product_noalloc uses a fixed array inside the library instead.  These
tests call it through the C ABI and check it against lt_product and against the FP64
oracle on the same inputs, for two calls in a row with different operands (the array
keeps the previous call's contents, which must not leak into the next result), in FP64,
FP32 and LT_MIXED (whose face-wise GEMM then runs on the tensor cores with its TMA
descriptors over the fixed array), and check that a warm call leaves the device's free
memory unchanged.  This file is collected last so
that a run stopping at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt
from tests.gpu_util import empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}


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


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32, lt.LT_MIXED])
def test_noalloc_matches_lt_product_on_two_calls(prec):
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    transforms = [("dct", 3), ("dct", 8)]
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, prec)
    rng = np.random.default_rng(2024)
    # two calls, different operands; for LT_MIXED both keep I1 and l multiples of 4 so
    # that the face-wise GEMM takes the tensor-core kernel
    shapes = ((32, 24, 16), (132, 36, 40)) if prec == lt.LT_MIXED else ((32, 24, 16), (65, 9, 40))
    for I1, l, I2 in shapes:
        A = rng.uniform(-1, 1, (I1, l, 3, 8))
        B = rng.uniform(-1, 1, (l, I2, 3, 8))
        Ad, Bd = to_dev(A, dt), to_dev(B, dt)
        ref = empty_dev((I1, I2, 3, 8), dt)
        lt.lt_product(ctx, Ad, Bd, ref)
        lt.lt_ctx_get_stats(ctx, reset=True)
        out = empty_dev((I1, I2, 3, 8), dt).fill_(float("nan"))
        assert call_noalloc(ctx, Ad, Bd, out, I1, l, I2) == lt.LT_OK
        torch.cuda.synchronize()
        assert rel(out.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL[prec]
        assert rel(from_dev(out, (I1, I2, 3, 8)), O.product(A, B, Ms)) <= TOL[prec]
        # tc_launches counts every tensor-core launch, this call's included
        tc = lt.lt_ctx_get_stats(ctx, reset=True)["tc_launches"]
        assert tc == (1 if prec == lt.LT_MIXED else 0)
        assert lt.lt_last_device_status(ctx) == 0


def test_noalloc_warm_call_leaves_free_memory_unchanged():
    ctx = make_ctx([("dct", 3), ("dct", 8)], lt.LT_MIXED)
    rng = np.random.default_rng(7)
    A = to_dev(rng.uniform(-1, 1, (64, 32, 3, 8)), torch.float32)
    B = to_dev(rng.uniform(-1, 1, (32, 48, 3, 8)), torch.float32)
    out = empty_dev((64, 48, 3, 8), torch.float32)
    assert call_noalloc(ctx, A, B, out, 64, 32, 48) == lt.LT_OK  # loads the kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call_noalloc(ctx, A, B, out, 64, 32, 48) == lt.LT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_wrapping_sizes():
    """Sizes whose byte count overflows 64 bits are refused on the host, not wrapped
    below the array's limit: with P = 64^4 = 2^24 slices, I1 = l = 2^20 gives
    I1 * l * P * 8 = 2^67 bytes for L(A), which wraps to 0 in 64-bit arithmetic.  The
    check runs before anything is enqueued, so the small buffers are never touched."""
    ctx = make_ctx([("dct", 64)] * 4)
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    A, B, Cout = buf[:16], buf[16:32], buf[32:48]
    for I1, l, I2 in ((1 << 20, 1 << 20, 1), (1, 1 << 20, 1 << 20), (1 << 20, 1 << 20, 1 << 20)):
        assert call_noalloc(ctx, A, B, Cout, I1, l, I2) == -2  # LT_ERR_SHAPE
    torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_array():
    ctx = make_ctx([("dct", 4)])
    # L(A) alone would need 4 * 1024 * 1024 * 8 bytes = 32 MiB: over the limit with L(B)
    I1, l, I2 = 1024, 1024, 1
    A = torch.zeros((4, l, I1), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, I2, l), dtype=torch.float64, device="cuda")
    Cout = torch.zeros((4, I2, I1), dtype=torch.float64, device="cuda")
    assert call_noalloc(ctx, A, B, Cout, I1, l, I2) == -2  # LT_ERR_SHAPE, nothing enqueued
