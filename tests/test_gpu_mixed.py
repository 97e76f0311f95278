"""Parity of the LT_MIXED path: face-wise products (Algorithm 2) and the mode products of
large modes (Sec. 3.2) on the tcgen05 tensor cores in split TF32 x 3, against the FP64
oracle on the same seeded inputs.

Tolerance: 1e-5 relative Frobenius error (the mixed-path bound).  Split TF32 keeps about
21 significant bits per product (hi = tf32(x), lo = tf32(x - hi); the dropped lo*lo term
and the rounding of lo are below 2^-21 |a b|) and accumulates in FP32, so products of
length K carry a relative error of a few 2^-22 sqrt(K); with cond(L) = 10 transforms the
inverse amplifies that, as on the FP32 path, hence 10x the bound there.

Each case also checks that the tensor-core kernel ran (lt_ctx_get_stats' tc_launches)
where its alignment rules hold, and that it did not run where they fail (the FP32 SIMT
kernels take those operands).
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-5
MIXED = lt.LT_MIXED


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


def random_transforms(rng, sizes, cond=10.0):
    return [("matrix", synth.conditioned_matrix(rng, n, cond, two_sided=True)) for n in sizes]


def tc_launches(ctx):
    return lt.lt_ctx_get_stats(ctx, reset=True)["tc_launches"]


def test_mixed_product_config1():
    """*_L-product of the 32x24x8 and 24x16x8 operands (DCT-II 8), face-wise GEMM on the
    tensor cores."""
    c = synth.config1()
    Ms = oracle_mats(c["transforms"])
    ctx = make_ctx(c["transforms"], MIXED)
    A, B = to_dev(c["A"], torch.float32), to_dev(c["B"], torch.float32)
    Cd = empty_dev((32, 16, 8), torch.float32)
    lt.lt_product(ctx, A, B, Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, (32, 16, 8)), O.product(c["A"], c["B"], Ms)) <= TOL
    assert tc_launches(ctx) == 1
    assert lt.lt_last_device_status(ctx) == 0


# (I1, l, I2, trailing modes): several 128-row tiles with a ragged tail, K chunks of 32
# with a ragged tail, N tiles of every width with a ragged tail, one and two outer modes.
TC_SHAPES = [(4, 4, 1, (2,)), (128, 32, 64, (3,)), (132, 36, 72, (2, 3)),
             (260, 100, 130, (3,)), (64, 256, 300, (2,)), (8, 12, 256, (4,))]


@pytest.mark.parametrize("tile_n", [0, 32, 64, 128, 256])
@pytest.mark.parametrize("I1,l,I2,trailing", TC_SHAPES)
def test_mixed_product_tiles(I1, l, I2, trailing, tile_n):
    rng = np.random.default_rng(I1 * 7 + l * 3 + I2)
    A = rng.uniform(-1, 1, (I1, l) + trailing)
    B = rng.uniform(-1, 1, (l, I2) + trailing)
    tr = random_transforms(rng, trailing)
    ctx = make_ctx(tr, MIXED)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TILE_N, tile_n)
    Cd = empty_dev((I1, I2) + trailing, torch.float32)
    lt.lt_product(ctx, to_dev(A, torch.float32), to_dev(B, torch.float32), Cd)
    torch.cuda.synchronize()
    err = rel(from_dev(Cd, (I1, I2) + trailing), O.product(A, B, oracle_mats(tr)))
    assert err <= TOL * 10, err
    assert tc_launches(ctx) == 1
    assert lt.lt_last_device_status(ctx) == 0


@pytest.mark.parametrize("I1,l,I2", [(5, 4, 8), (8, 6, 8), (130, 64, 129)])
def test_mixed_product_unaligned_takes_simt(I1, l, I2):
    """I1 or l not a multiple of 4: the TMA descriptors cannot address the slices, the
    FP32 SIMT kernel computes the product, and the result is the same to the bound."""
    rng = np.random.default_rng(I1 + l + I2)
    A = rng.uniform(-1, 1, (I1, l, 3))
    B = rng.uniform(-1, 1, (l, I2, 3))
    tr = [("dct", 3)]
    ctx = make_ctx(tr, MIXED)
    Cd = empty_dev((I1, I2, 3), torch.float32)
    lt.lt_product(ctx, to_dev(A, torch.float32), to_dev(B, torch.float32), Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, (I1, I2, 3)), O.product(A, B, oracle_mats(tr))) <= TOL * 10
    assert tc_launches(ctx) == 0


def test_mixed_product_differs_from_fp32_but_agrees():
    """The mixed and FP32 paths are different arithmetic (the products are not bitwise
    equal) with the same result to the bound: the tensor cores really computed it."""
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (64, 32, 4))
    B = rng.uniform(-1, 1, (32, 48, 4))
    tr = [("dct", 4)]
    out = {}
    for prec in (lt.LT_FP32, MIXED):
        ctx = make_ctx(tr, prec)
        Cd = empty_dev((64, 48, 4), torch.float32)
        lt.lt_product(ctx, to_dev(A, torch.float32), to_dev(B, torch.float32), Cd)
        torch.cuda.synchronize()
        out[prec] = Cd.clone()
    assert not torch.equal(out[lt.LT_FP32], out[MIXED])
    ref = O.product(A, B, oracle_mats(tr))
    for prec in out:
        assert rel(from_dev(out[prec], (64, 48, 4)), ref) <= TOL


# (I1, I2, transforms, tensor-core passes per transform)
TC_TRANSFORMS = [
    ((8, 6), [("dct", 3), ("dct", 32)], 1),           # the benchmark's transform pair
    ((4, 5), [("dct", 3), ("dct", 120)], 1),          # the large completion's pair
    ((16, 2), [("dct", 2), ("dct", 64), ("dct", 3)], 1),
    ((4, 4), [("dct", 4), "random40", ("dct", 36)], 2),
    ((5, 7), [("dct", 3), ("dct", 32)], 0),           # S = 105: SIMT passes only
]


@pytest.mark.parametrize("shape,transforms,ntc", TC_TRANSFORMS)
def test_mixed_transform_and_inverse(shape, transforms, ntc):
    rng = np.random.default_rng(17 + shape[0])
    transforms = [random_transforms(rng, (40,))[0] if t == "random40" else t for t in transforms]
    sizes = tuple(t[1] if t[0] == "dct" else np.asarray(t[1]).shape[0] for t in transforms)
    full = tuple(shape) + sizes
    X = rng.uniform(-1, 1, size=full)
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, MIXED)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_MODE_MIN, 32)
    Xd = to_dev(X, torch.float32)
    Xh = empty_dev(full, torch.float32)
    lt.lt_transform(ctx, Xd, Xh)
    Xb = empty_dev(full, torch.float32)
    lt.lt_inverse(ctx, Xh, Xb)
    torch.cuda.synchronize()
    assert rel(from_dev(Xh, full), O.transform(X, Ms)) <= TOL
    assert rel(from_dev(Xb, full), X) <= TOL * 10
    assert tc_launches(ctx) == 2 * ntc
    # in place (every tensor-core pass then covers all columns of its mode in one tile)
    lt.lt_transform(ctx, Xd, Xd)
    lt.lt_inverse(ctx, Xd, Xd)
    torch.cuda.synchronize()
    assert rel(from_dev(Xd, full), X) <= TOL * 10
    assert tc_launches(ctx) == 2 * ntc
    assert lt.lt_last_device_status(ctx) == 0


def test_mixed_tc_mode_min_option_routes_passes():
    """LT_OPT_TC_MODE_MIN routes the mode-32 products (0: never on the tensor cores; 32:
    on them; 33 and the default 64: not); the results agree to the bound."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (8, 6, 3, 32))
    tr = [("dct", 3), ("dct", 32)]
    Ms = oracle_mats(tr)
    ref = O.transform(X, Ms)
    for mode_min, ntc in ((0, 0), (32, 1), (33, 0), (None, 0)):
        ctx = make_ctx(tr, MIXED)
        if mode_min is not None:  # None: the default (64) keeps mode 32 in the SIMT pass
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_MODE_MIN, mode_min)
        Xh = empty_dev(X.shape, torch.float32)
        lt.lt_transform(ctx, to_dev(X, torch.float32), Xh)
        torch.cuda.synchronize()
        assert rel(from_dev(Xh, X.shape), ref) <= TOL
        assert tc_launches(ctx) == ntc


def test_mixed_pga_small():
    """PGA (Algorithm 5) on a 24 x 20 x 3 x 32 completion problem in LT_MIXED with the
    mode-4 products routed to the tensor cores (LT_OPT_TC_MODE_MIN = 32) inside every
    iteration."""
    c = synth.completion_case(11, 24, 20, (3, 32), rank=3, rho=0.4)
    tr = [("dct", 3), ("dct", 32)]
    Ms = oracle_mats(tr)
    X0 = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    obs = c["mask"] * (X0 + c["noise"])
    ref, _ = O.pga(c["mask"], obs, 0.3, 1.0, 20, Ms)
    ctx = make_ctx(tr, MIXED)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_MODE_MIN, 32)
    X = torch.zeros((32, 3, 20, 24), dtype=torch.float32, device="cuda")
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs, torch.float32), 0.3, 1.0, 20, X,
                       report=rep)
    torch.cuda.synchronize()
    assert rep.iters_done == 20 and rep.device_status == 0
    assert rel(from_dev(X, obs.shape), ref) <= TOL
    assert tc_launches(ctx) == 2 * 20


def test_mixed_options_reject_bad_values():
    ctx = make_ctx([("dct", 3)], MIXED)
    for opt, bad in ((lt.LT_OPT_TC_TILE_N, 48), (lt.LT_OPT_TC_TILE_N, 512),
                     (lt.LT_OPT_TC_MODE_MIN, -1), (lt.LT_OPT_TC_MODE_MIN, 2.5)):
        with pytest.raises(lt.LtError):
            lt.lt_ctx_set_option(ctx, opt, bad)
    for opt, bad in ((lt.LT_OPT_TC_WAIT_US, -1.0), (lt.LT_OPT_TC_WAIT_US, 1e9),
                     (lt.LT_OPT_TC_TEST_NO_LOADS, 2)):
        with pytest.raises(lt.LtError):
            lt.lt_ctx_set_option(ctx, opt, bad)


def test_tc_bounded_wait_expires_then_context_recovers():
    """Failure detection of the tensor-core kernel without a GPU fault: with the test
    switch LT_OPT_TC_TEST_NO_LOADS the producer issues no copies, so the converters' and
    the issuer's first waits (limit 5 ms) expire and every role returns (no copy or MMA
    in flight, TMEM freed).  The call reports LT_DEV_TIMEOUT through the device status
    word; with the switch off the same context then computes the product correctly."""
    rng = np.random.default_rng(515)
    A = rng.uniform(-1, 1, (128, 32, 3))
    B = rng.uniform(-1, 1, (32, 64, 3))
    tr = [("dct", 3)]
    ctx = make_ctx(tr, MIXED)
    Ad, Bd = to_dev(A, torch.float32), to_dev(B, torch.float32)
    Cd = empty_dev((128, 64, 3), torch.float32)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_WAIT_US, 5000)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TEST_NO_LOADS, 1)
    lt.lt_product(ctx, Ad, Bd, Cd)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) & lt.LT_DEV_TIMEOUT
    assert tc_launches(ctx) == 1
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TEST_NO_LOADS, 0)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_WAIT_US, 0)
    lt.lt_product(ctx, Ad, Bd, Cd)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0
    assert tc_launches(ctx) == 1
    assert rel(from_dev(Cd, (128, 64, 3)), O.product(A, B, oracle_mats(tr))) <= TOL


def test_tma_transform_bounded_wait_expires_then_context_recovers():
    """Failure detection of the TMA transform passes without a GPU fault: with the test
    switch LT_OPT_TC_TEST_NO_LOADS the copy warp issues no loads, so the compute warps'
    first waits (limit 5 ms) expire, they agree on it on their named barrier and stop, and
    the copy thread's wait for their first tile expires in turn (nothing in flight).  The
    call reports LT_DEV_TIMEOUT through the device status word; with the switch off the
    same context then transforms correctly (both passes, {16, 16} and {8})."""
    rng = np.random.default_rng(516)
    full = (24, 20, 16, 16, 8)
    X = rng.uniform(-1, 1, full)
    tr = [("dct", 16), ("matrix", synth.conditioned_matrix(rng, 16, 10.0, True)), ("dct", 8)]
    ctx = make_ctx(tr, lt.LT_FP32)
    Xd = to_dev(X, torch.float32)
    Y = empty_dev(full, torch.float32)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_WAIT_US, 5000)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TEST_NO_LOADS, 1)
    lt.lt_transform(ctx, Xd, Y)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) & lt.LT_DEV_TIMEOUT
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TEST_NO_LOADS, 0)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_WAIT_US, 0)
    lt.lt_transform(ctx, Xd, Y)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0
    assert rel(from_dev(Y, full), O.transform(X, oracle_mats(tr))) <= 1e-6


# (I1, I2, trailing): a 256-slice pass of two modes plus a single-mode pass with wide tiles
# (16, 16, 8), ragged tiles (Sg = 468), a single mode of 8, a view that is not a multiple
# of 4 (SIMT fallback), and mode sizes 3 and 32 (one pass of 96 slices)
TMA_SHAPES = [(24, 20, (16, 16, 8)), (36, 13, (16, 16)), (20, 10, (8,)), (33, 7, (5, 3)),
              (64, 64, (3, 32))]


@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("I1,I2,trailing", TMA_SHAPES)
def test_transform_tma_equals_simt(I1, I2, trailing, inplace):
    """FP32 transform and inverse passes through the tensor memory accelerator
    (LT_OPT_TRANSFORM_TMA = 1, the default) give the same bits as the SIMT loads and
    stores (0): the mode products are the same code; and both match the oracle."""
    rng = np.random.default_rng(I1 * 5 + I2)
    full = (I1, I2) + trailing
    X = rng.uniform(-1, 1, full)
    tr = [("dct", n) if k % 2 == 0 else ("matrix", synth.conditioned_matrix(rng, n, 10.0, True))
          for k, n in enumerate(trailing)]
    Ms = oracle_mats(tr)
    outs = {}
    for tma in (1, 0):
        ctx = make_ctx(tr, lt.LT_FP32)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_TRANSFORM_TMA, tma)
        Xd = to_dev(X, torch.float32)
        Y = Xd if inplace else empty_dev(full, torch.float32)
        lt.lt_transform(ctx, Xd, Y)
        Z = Y if inplace else empty_dev(full, torch.float32)
        Yc = Y.clone()
        lt.lt_inverse(ctx, Y, Z)
        torch.cuda.synchronize()
        assert lt.lt_last_device_status(ctx) == 0
        outs[tma] = (Yc, Z.clone())
    assert torch.equal(outs[1][0], outs[0][0]) and torch.equal(outs[1][1], outs[0][1])
    assert rel(from_dev(outs[1][0], full), O.transform(X, Ms)) <= 1e-6
    assert rel(from_dev(outs[1][1], full), X) <= 1e-5
