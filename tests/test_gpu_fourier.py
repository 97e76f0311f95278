"""Parity of the Fourier operator (M_3 = F_{I3}: the t-product of Sec. 2 and the TNN-PGA-F
completion of Sec. 5) with the FP64 oracle's complex arithmetic, on the same seeded
inputs.

The library works on real slots (the coefficients of F_n x in the orthonormal real DFT
basis, lt_ctx_create_fourier); `slots_of` maps the oracle's complex transform to that
layout for the transform test.  Products, SVTs and completions are compared in the
tensor domain, where both sides are real.

Tolerances: 1e-12 (FP64) and 1e-5 (FP32 and LT_MIXED) relative Frobenius error, as for
the real transforms; products and transforms through a random mode-4 matrix of
condition 10 get 10x (the inverse amplifies rounding by cond).
"""
import math

import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import dtype_of, empty_dev, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}
PRECS = [lt.LT_FP64, lt.LT_FP32]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


def fourier_ctx(trailing, rest, prec):
    return lt.lt_ctx_create_fourier(list(trailing), rest, prec)


def slots_of(Xh):
    """Complex L(X) (mode 3 = F_n, axis 2) -> the library's real slots along axis 2."""
    n = Xh.shape[2]
    out = np.empty(Xh.shape, dtype=np.float64)
    out[:, :, 0] = Xh[:, :, 0].real / math.sqrt(n)
    for k in range(1, (n + 1) // 2):
        out[:, :, 2 * k - 1] = math.sqrt(2.0 / n) * Xh[:, :, k].real
        out[:, :, 2 * k] = math.sqrt(2.0 / n) * Xh[:, :, k].imag
    if n % 2 == 0:
        out[:, :, n - 1] = Xh[:, :, n // 2].real / math.sqrt(n)
    return out


def rest_mats(rng, sizes, kind):
    if kind == "dct":
        return [O.dct_matrix(n) for n in sizes]
    return [synth.conditioned_matrix(rng, n, 10.0, two_sided=True) for n in sizes]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("trailing,kind", [((1,), "dct"), ((2,), "dct"), ((3,), "dct"),
                                           ((4,), "dct"), ((7,), "dct"), ((8, 3), "dct"),
                                           ((5, 4), "random"), ((3, 2, 3), "dct")])
def test_fourier_transform_slots_and_inverse(prec, trailing, kind):
    rng = np.random.default_rng(sum(trailing) * 11 + len(trailing))
    rest = rest_mats(rng, trailing[1:], kind)
    full = (6, 5) + trailing
    X = rng.uniform(-1, 1, full)
    ctx = fourier_ctx(trailing, rest, prec)
    dt = dtype_of(prec)
    Xh = empty_dev(full, dt)
    lt.lt_transform(ctx, to_dev(X, dt), Xh)
    Xb = empty_dev(full, dt)
    lt.lt_inverse(ctx, Xh, Xb)
    torch.cuda.synchronize()
    f = 10 if kind == "random" else 1
    assert rel(from_dev(Xh, full), slots_of(O.fourier_transform(X, rest))) <= TOL[prec] * f
    assert rel(from_dev(Xb, full), X) <= TOL[prec] * f


# (I1, l, I2, trailing, kind): several 64-wide tiles with ragged tails, odd and even n
PRODUCTS = [(4, 3, 5, (1,), "dct"), (8, 6, 7, (2,), "dct"), (70, 20, 66, (3,), "dct"),
            (33, 65, 17, (4,), "dct"), (16, 12, 20, (5, 3), "random"),
            (9, 7, 11, (6, 2, 2), "dct")]


@pytest.mark.parametrize("prec", PRECS + [lt.LT_MIXED])
@pytest.mark.parametrize("I1,l,I2,trailing,kind", PRODUCTS)
def test_fourier_product_is_the_tproduct(prec, I1, l, I2, trailing, kind):
    rng = np.random.default_rng(I1 + 3 * l + 7 * I2)
    rest = rest_mats(rng, trailing[1:], kind)
    A = rng.uniform(-1, 1, (I1, l) + trailing)
    B = rng.uniform(-1, 1, (l, I2) + trailing)
    ctx = fourier_ctx(trailing, rest, prec)
    dt = dtype_of(prec)
    Cd = empty_dev((I1, I2) + trailing, dt)
    lt.lt_product(ctx, to_dev(A, dt), to_dev(B, dt), Cd)
    torch.cuda.synchronize()
    f = 10 if kind == "random" else 1
    assert rel(from_dev(Cd, (I1, I2) + trailing), O.tproduct(A, B, rest)) <= TOL[prec] * f
    assert lt.lt_ctx_get_stats(ctx)["tc_launches"] == 0
    assert lt.lt_last_device_status(ctx) == 0


def test_fourier_product_third_order_circulant_case():
    """A tube-constant A (every frontal slice A_0) times B: the t-product is
    C_k = A_0 sum_j B_j for every k (bcirc of a constant tube)."""
    rng = np.random.default_rng(9)
    A0 = rng.standard_normal((5, 4))
    A = np.repeat(A0[:, :, None], 6, axis=2)
    B = rng.standard_normal((4, 3, 6))
    ctx = fourier_ctx((6,), [], lt.LT_FP64)
    Cd = empty_dev((5, 3, 6))
    lt.lt_product(ctx, to_dev(A), to_dev(B), Cd)
    torch.cuda.synchronize()
    C = from_dev(Cd, (5, 3, 6))
    for k in range(6):
        assert rel(C[:, :, k], A0 @ B.sum(axis=2)) <= 1e-13


SVTS = [((8, 6), (3,), 0.8), ((6, 9), (4,), 0.5), ((24, 20), (3, 4), 1.5),
        ((33, 17), (5, 2), 1.0), ((16, 40), (2, 3), 0.7), ((12, 12), (1, 3), 0.9),
        ((70, 50), (3, 2), 2.0)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,trailing,tau", SVTS)
def test_fourier_svt(prec, shape, trailing, tau):
    rng = np.random.default_rng(shape[0] * 5 + shape[1] + sum(trailing))
    rest = [O.dct_matrix(n) for n in trailing[1:]]
    full = tuple(shape) + trailing
    A = rng.standard_normal(full)
    ctx = fourier_ctx(trailing, rest, prec)
    dt = dtype_of(prec)
    D = empty_dev(full, dt)
    lt.lt_svt(ctx, to_dev(A, dt), tau, D)
    torch.cuda.synchronize()
    ref = O.tsvt(A, tau, rest)
    assert rel(from_dev(D, full), ref) <= TOL[prec]
    assert lt.lt_last_device_status(ctx) == 0
    # in place, and tau = 0 gives A back
    Ad = to_dev(A, dt)
    lt.lt_svt(ctx, Ad, 0.0, Ad)
    torch.cuda.synchronize()
    assert rel(from_dev(Ad, full), A) <= TOL[prec]


def fourier_completion(seed, I1, I2, trailing, rank, rho, rest):
    c = synth.completion_case(seed, I1, I2, trailing, rank=rank, rho=rho)
    X = O.tproduct(c["U"], np.swapaxes(c["V"], 0, 1), rest)
    obs = c["mask"] * (X + c["noise"])
    return X, c["mask"], obs


@pytest.mark.parametrize("prec", PRECS + [lt.LT_MIXED])
def test_fourier_pga_small(prec):
    rest = [O.dct_matrix(4)]
    X, mask, obs = fourier_completion(31, 24, 20, (3, 4), 3, 0.4, rest)
    ref, info = O.pga(mask, obs, 0.3, 1.0, 25, rest, fourier=True)
    ctx = fourier_ctx((3, 4), rest, prec)
    dt = dtype_of(prec)
    Xd = torch.zeros(tuple(reversed(obs.shape)), dtype=dt, device="cuda")
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(mask), to_dev(obs, dt), 0.3, 1.0, 25, Xd, report=rep)
    torch.cuda.synchronize()
    assert rep.iters_done == 25 and rep.device_status == 0
    assert rel(from_dev(Xd, obs.shape), ref) <= TOL[prec]
    assert abs(rep.rel_residual - info["residual"][-1]) <= 1e-8 + TOL[prec] * 10


@pytest.mark.parametrize("n", [2, 4, 5])
def test_fourier_pga_even_and_odd_tubes(n):
    """Nyquist slots (even n) and two conjugate pairs (n = 5), FP64, with continuation
    (mu_0 = nu ||M||_F, nu = 0.9)."""
    rest = [O.dct_matrix(3)]
    X, mask, obs = fourier_completion(32 + n, 18, 22, (n, 3), 2, 0.5, rest)
    mu0 = 0.9 * float(np.linalg.norm(obs))
    ref, _ = O.pga(mask, obs, 0.2, 1.0, 30, rest, fourier=True, mu0=mu0, nu=0.9)
    ctx = fourier_ctx((n, 3), rest, lt.LT_FP64)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_MU0, mu0)
    Xd = torch.zeros(tuple(reversed(obs.shape)), dtype=torch.float64, device="cuda")
    lt.lt_pga_complete(ctx, to_dev(mask), to_dev(obs), 0.2, 1.0, 30, Xd)
    torch.cuda.synchronize()
    assert rel(from_dev(Xd, obs.shape), ref) <= 1e-12


def test_fourier_pga_batched_with_real_contexts():
    """A batch mixing Fourier and DCT contexts: every problem equals its single run bit
    for bit and the Fourier one matches TNN-PGA-F of the oracle."""
    rest = [O.dct_matrix(4)]
    X, mask, obs = fourier_completion(33, 20, 16, (3, 4), 2, 0.5, rest)
    c2 = synth.completion_case(34, 16, 12, (3, 2), rank=2, rho=0.5)
    Ms2 = [O.dct_matrix(3), O.dct_matrix(2)]
    X2 = O.product(c2["U"], O.transpose(c2["V"], Ms2), Ms2)
    obs2 = c2["mask"] * X2
    ctxs = [fourier_ctx((3, 4), rest, lt.LT_FP64),
            lt.Context([3, 2], [lt.lt_make_dct(3), lt.lt_make_dct(2)], lt.LT_FP64)]
    masks = [to_dev(mask), to_dev(c2["mask"])]
    obss = [to_dev(obs), to_dev(obs2)]
    Xs = [torch.zeros(tuple(reversed(o.shape)), dtype=torch.float64, device="cuda")
          for o in (obs, obs2)]
    reps = []
    lt.lt_pga_complete_batched(ctxs, masks, obss, [0.3, 0.2], [1.0, 1.0], 7, Xs, reports=reps)
    torch.cuda.synchronize()
    for i in range(2):
        X1 = torch.zeros_like(Xs[i])
        lt.lt_pga_complete(ctxs[i], masks[i], obss[i], [0.3, 0.2][i], 1.0, 7, X1)
        torch.cuda.synchronize()
        assert torch.equal(Xs[i], X1)
    ref, _ = O.pga(mask, obs, 0.3, 1.0, 7, rest, fourier=True)
    assert rel(from_dev(Xs[0], obs.shape), ref) <= 1e-12


@pytest.fixture(scope="module")
def full_size_case():
    rest = [O.dct_matrix(32)]
    X, mask, obs = fourier_completion(2, 144, 176, (3, 32), 10, 0.3, rest)
    ref, _ = O.pga(mask, obs, 0.5, 1.0, 10, rest, fourier=True)
    return rest, mask, obs, ref


@pytest.mark.parametrize("prec", PRECS)
def test_fourier_pga_full_size(prec, full_size_case):
    """The benchmarked completion size with the Fourier operator (TNN-PGA-F):
    144x176x3x32, F_3 on mode 3, DCT 32 on mode 4, t-rank 10, 30% observed, tau 0.5,
    10 iterations."""
    rest, mask, obs, ref = full_size_case
    ctx = fourier_ctx((3, 32), rest, prec)
    dt = dtype_of(prec)
    Xd = torch.zeros(tuple(reversed(obs.shape)), dtype=dt, device="cuda")
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(mask), to_dev(obs, dt), 0.5, 1.0, 10, Xd, report=rep)
    torch.cuda.synchronize()
    assert rep.iters_done == 10 and rep.device_status == 0
    assert rel(from_dev(Xd, obs.shape), ref) <= (1e-12 if prec == lt.LT_FP64 else 1e-5)


def test_fourier_unsupported_calls_enqueue_nothing():
    ctx = fourier_ctx((3,), [], lt.LT_FP64)
    A = torch.zeros((3, 4, 5), dtype=torch.float64, device="cuda")
    U = torch.zeros((3, 5, 5), dtype=torch.float64, device="cuda")
    V = torch.zeros((3, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for call in (lambda: lt.lt_svd(ctx, A, U, torch.zeros_like(A), V),
                 lambda: lt.lt_truncate(ctx, A, 1, torch.zeros_like(A)),
                 lambda: lt.lt_norms(ctx, A, out)):
        with pytest.raises(lt.LtError) as e:
            call()
        assert e.value.status == lt.STATUS_CODE["LT_ERR_UNSUPPORTED"]
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_OBJECTIVE, 1)
    mask = torch.ones((3, 4, 5), dtype=torch.uint8, device="cuda")
    with pytest.raises(lt.LtError) as e:
        lt.lt_pga_complete(ctx, mask, A, 0.1, 1.0, 2, torch.zeros_like(A))
    assert e.value.status == lt.STATUS_CODE["LT_ERR_UNSUPPORTED"]
    with pytest.raises(lt.LtError):
        lt.lt_ctx_create_fourier([0], [])
