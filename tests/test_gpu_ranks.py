"""Parity of lt_truncate (the Eckart-Young rank-k approximation of Sec. 3.2) and
lt_norms (nuclear and spectral norms, multirank, average and tubal rank of Sec. 3.2)
with the FP64 oracle, through the C ABI.

Tolerances: relative Frobenius error 1e-12 (FP64) / 1e-5 (FP32) for A_k on tensors with
distinct singular values; the ranks are integers and must match exactly on tensors built
with prescribed transform-domain slice ranks; the norms are compared at 1e-12 / 1e-5
relative.
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt
from tests.gpu_util import dtype_of, empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}
U = {lt.LT_FP64: 2.0 ** -53, lt.LT_FP32: 2.0 ** -24, lt.LT_MIXED: 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
@pytest.mark.parametrize("shape,transforms", [((12, 9), [("dct", 3), ("dct", 2)]),
                                              ((9, 14), [("dct", 4)]),
                                              ((40, 33), [("dct", 3)])])
@pytest.mark.parametrize("k", [0, 1, 3, 100])
def test_truncate(prec, shape, transforms, k):
    rng = np.random.default_rng(shape[0] * 10 + k)
    sizes = tuple(t[1] for t in transforms)
    full = tuple(shape) + sizes
    A = rng.standard_normal(full)
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    Ak = empty_dev(full, dt)
    lt.lt_truncate(ctx, to_dev(A, dt), k, Ak)
    torch.cuda.synchronize()
    ref = O.truncate(A, k, Ms)
    got = from_dev(Ak, full)
    if k == 0:
        assert np.abs(got).max() == 0.0
    else:
        assert rel(got, ref) <= TOL[prec], rel(got, ref)
    assert lt.lt_last_device_status(ctx) == 0
    # in place
    Ad = to_dev(A, dt)
    lt.lt_truncate(ctx, Ad, k, Ad)
    torch.cuda.synchronize()
    if k:
        assert rel(from_dev(Ad, full), ref) <= TOL[prec]


def prescribed_rank_tensor(rng, I1, I2, transforms, ranks):
    Ms = oracle_mats(transforms)
    trailing = tuple(t[1] for t in transforms)
    P = int(np.prod(trailing))
    Ah = np.zeros((I1, I2, P))
    for p in range(P):
        r = ranks[p % len(ranks)]
        Ah[:, :, p] = rng.standard_normal((I1, r)) @ rng.standard_normal((r, I2))
    return O.inverse_transform(O.from_slices(Ah, trailing), Ms), Ms


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
@pytest.mark.parametrize("I1,I2,transforms,ranks", [
    (20, 16, [("dct", 3), ("dct", 4)], [3, 0, 7, 1, 16, 5]),
    (11, 30, [("dct", 5)], [2, 11, 0, 4, 9]),
    (144, 176, [("dct", 3), ("dct", 2)], [10, 0, 144, 57, 1, 99])])
def test_norms_and_ranks(prec, I1, I2, transforms, ranks):
    rng = np.random.default_rng(I1 + I2)
    A, Ms = prescribed_rank_tensor(rng, I1, I2, transforms, ranks)
    ref = O.ranks_and_norms(A, Ms, U[prec])
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    P = int(np.prod([t[1] for t in transforms]))
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    mr = torch.full((P,), -1, dtype=torch.int32, device="cuda")
    lt.lt_norms(ctx, to_dev(A, dt), out, mr)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert list(mr.cpu().numpy()) == list(ref["multirank"])
    assert o[2] == ref["tubal"] and o[3] == ref["average"]
    assert abs(o[1] - ref["spectral"]) <= TOL[prec] * ref["spectral"]
    assert abs(o[0] - ref["nuclear"]) <= TOL[prec] * ref["nuclear"]
    assert lt.lt_last_device_status(ctx) == 0


def test_norms_without_multirank_and_zero_tensor():
    ctx = make_ctx([("dct", 3)], lt.LT_FP64)
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    lt.lt_norms(ctx, torch.zeros((3, 5, 6), dtype=torch.float64, device="cuda"), out)
    torch.cuda.synchronize()
    assert list(out.cpu().numpy()) == [0.0, 0.0, 0.0, 0.0]


def test_truncate_rejects_negative_rank():
    ctx = make_ctx([("dct", 3)], lt.LT_FP64)
    A = torch.zeros((3, 5, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(lt.LtError):
        lt.lt_truncate(ctx, A, -1, A)


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
def test_autotune_svt_picks_a_form_and_keeps_parity(prec):
    """lt_autotune_svt times the SVT kernel forms on the caller's slices, sets the fastest
    on the context (never slower than the planner's default by its own measurement), and
    the SVT computed with it still matches the oracle."""
    rng = np.random.default_rng(31)
    full = (48, 56, 3, 2)
    A = rng.standard_normal(full)
    tr = [("dct", 3), ("dct", 2)]
    ctx = make_ctx(tr, prec)
    dt = dtype_of(prec)
    Ad, D = to_dev(A, dt), empty_dev(full, dt)
    rep = lt.lt_autotune_svt(ctx, Ad, 0.5, D)
    assert rep.candidates >= 4 and rep.best_ms <= rep.default_ms
    D2 = empty_dev(full, dt)
    lt.lt_svt(ctx, Ad, 0.5, D2)
    torch.cuda.synchronize()
    ref = O.svt(A, 0.5, oracle_mats(tr))
    assert rel(from_dev(D2, full), ref) <= TOL[prec]
    assert lt.lt_last_device_status(ctx) == 0
    with pytest.raises(lt.LtError):  # D must not alias A
        lt.lt_autotune_svt(ctx, Ad, 0.5, Ad)


def test_autotune_product_picks_a_tile_width():
    rng = np.random.default_rng(32)
    A = rng.uniform(-1, 1, (128, 64, 4))
    B = rng.uniform(-1, 1, (64, 96, 4))
    tr = [("dct", 4)]
    ctx = make_ctx(tr, lt.LT_MIXED)
    Cd = empty_dev((128, 96, 4), torch.float32)
    Ad, Bd = to_dev(A, torch.float32), to_dev(B, torch.float32)
    rep = lt.lt_autotune_product(ctx, Ad, Bd, Cd)
    assert rep.candidates == 4 and rep.tc_tile_n in (0, 32, 64, 128)
    assert rep.best_ms <= rep.default_ms
    lt.lt_product(ctx, Ad, Bd, Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, (128, 96, 4)), O.product(A, B, oracle_mats(tr))) <= 1e-5
