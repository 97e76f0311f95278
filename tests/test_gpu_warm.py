"""Warm start of the SVT across PGA iterations (LT_OPT_WARM_START): Algorithm 5 with the
previous iteration's singular vectors applied to each transform-domain slice before the
Jacobi SVT (and the result mapped back) gives the same iterates as the cold path, since
the SVT is unitarily invariant.  Checked against the FP64 oracle (1e-12 FP64, 1e-5 FP32 /
LT_MIXED) on the benchmark completion at full size and on small problems of both slice
orientations (I1 < I2: left vectors; I1 >= I2: right vectors), with rank-deficient
slices (the kernel's basis falls back to the identity), the tolerance stop and the
objective; the warm-started run must spend fewer Jacobi flops than the cold one.
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import dtype_of, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


def inputs(c):
    Ms = oracle_mats(c["transforms"])
    X = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    return c["mask"] * (X + c["noise"]), Ms


def run(c, obs, prec, iters, warm, tol=0.0, objective=False):
    ctx = make_ctx(c["transforms"], prec)
    if warm:
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, warm)
    if objective:
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_OBJECTIVE, 1)
    dt = dtype_of(prec)
    X = to_dev(np.zeros(obs.shape), dt)
    rep = lt.lt_pga_report()
    lt.lt_ctx_get_stats(ctx, reset=True)
    lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs, dt), c["tau"], c["step"], iters, X,
                       tol=tol, report=rep)
    torch.cuda.synchronize()
    st = lt.lt_ctx_get_stats(ctx, reset=True)
    return from_dev(X, obs.shape), rep, st


@pytest.fixture(scope="module")
def config2():
    c = synth.config2()
    obs, Ms = inputs(c)
    ref, info = O.pga(c["mask"], obs, c["tau"], c["step"], c["iters"], Ms)
    return c, obs, ref


# warm-start periods: FP64 keeps the accumulated basis orthogonal to ~1e-14 per
# iteration; in FP32 the basis loses ~1e-6 of orthogonality per warm iteration (the
# Jacobi tolerance and the rounding of its update), and the 100-iteration error against
# the oracle measured 6.7e-6 at period 4, 1.26e-5 at 8, 2.1e-5 at 16
PERIOD = {lt.LT_FP64: 8, lt.LT_FP32: 4}


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
def test_warm_config2_full(config2, prec):
    """The benchmark completion 144x176x3x32 (slices I1 < I2: left singular vectors),
    100 iterations with a cold iteration every 8 (FP64) or 4 (FP32): against the oracle,
    and fewer Jacobi flops than the cold run of the same problem."""
    c, obs, ref = config2
    got, rep, st = run(c, obs, prec, c["iters"], PERIOD[prec])
    err = rel(got, ref)
    _, rep0, st0 = run(c, obs, prec, c["iters"], 0)
    print(f"warm config2 prec {prec}: rel err {err:.2e}, jacobi GFLOP warm "
          f"{st['jacobi']['flops'] / 1e9:.2f} vs cold {st0['jacobi']['flops'] / 1e9:.2f}, "
          f"max sweeps {rep.max_sweeps_used} vs {rep0.max_sweeps_used}")
    assert rep.iters_done == 100 and rep.device_status == 0
    assert err <= TOL[prec]
    assert st["jacobi"]["flops"] < 0.9 * st0["jacobi"]["flops"]
    assert st["gemm"]["launches"] > 0


# (I1, I2, trailing, rank, rho, tau, period, iters)
SMALL = [(24, 20, (3, 4), 3, 0.4, 0.3, 2, 25),   # I1 > I2: right vectors
         (20, 24, (3, 4), 3, 0.4, 0.3, 3, 25),   # I1 < I2: left vectors
         (18, 18, (2, 3), 2, 0.5, 0.2, 5, 30),   # square
         (40, 33, (3, 2), 4, 0.3, 0.4, 4, 12)]


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32, lt.LT_MIXED])
@pytest.mark.parametrize("I1,I2,trailing,rank,rho,tau,period,iters", SMALL)
def test_warm_small(prec, I1, I2, trailing, rank, rho, tau, period, iters):
    c = synth.completion_case(31, I1, I2, trailing, rank=rank, rho=rho)
    c.update(tau=tau, step=1.0)
    obs, Ms = inputs(c)
    ref, _ = O.pga(c["mask"], obs, tau, 1.0, iters, Ms)
    got, rep, _ = run(c, obs, prec, iters, period)
    assert rep.iters_done == iters and rep.device_status == 0
    assert rel(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
def test_warm_rank_deficient_slices(prec):
    """With M_4 = I (so L keeps mode-4 indices apart) and nothing observed at mode-4 index
    1, the two transform-domain slices of that index are exactly zero in every iteration:
    their Jacobi columns have zero norm and the kernel returns the identity basis for
    them.  The slices of mode-4 index 2 are observed on 5 of 22 columns only (rank <= 5
    in the first iteration).  The iterates must still match the oracle."""
    c = synth.completion_case(32, 16, 22, (2, 3), rank=2, rho=0.5)
    c["transforms"] = [("dct", 2), ("matrix", np.eye(3))]
    c.update(tau=0.2, step=1.0)
    obs, Ms = inputs(c)
    c["mask"][:, :, :, 1] = 0
    c["mask"][:, 5:, :, 2] = 0
    obs = c["mask"] * obs
    ref, _ = O.pga(c["mask"], obs, 0.2, 1.0, 15, Ms)
    got, rep, _ = run(c, obs, prec, 15, 3)
    assert rep.iters_done == 15 and rep.device_status == 0
    assert np.all(got[:, :, :, 1] == 0.0)
    assert rel(got, ref) <= TOL[prec]


def test_warm_tolerance_stop_and_objective():
    c = synth.completion_case(21, 18, 26, (2, 3), rank=2, rho=0.6)
    c.update(tau=0.05, step=0.7)
    obs, Ms = inputs(c)
    ref, info = O.pga(c["mask"], obs, 0.05, 0.7, 300, Ms, tol=1e-5, objective=True)
    got, rep, _ = run(c, obs, lt.LT_FP64, 300, 6, tol=1e-5, objective=True)
    assert rep.iters_done == info["iters"] < 300
    assert rel(got, ref) <= 1e-12
    assert abs(rep.objective - info["objective"][-1]) <= 1e-12 * abs(info["objective"][-1])


def test_warm_option_values_and_workspace():
    ctx = make_ctx([("dct", 3), ("dct", 4)])
    cold = lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 20, 24)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, 4)
    warm = lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 20, 24)
    n, P, N = 20, 12, 20 * 24 * 12
    assert warm >= cold + (3 * n * n * P + N) * 8 + n * P * 4
    for bad in (1, -1, 2.5):
        with pytest.raises(lt.LtError):
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, bad)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, 0)
    assert lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 20, 24) == cold


def test_warm_ignored_by_the_batched_call():
    """One captured graph for all problems: the batched call runs the cold path even when
    the contexts ask for a warm start, bit for bit what cold single runs give."""
    probs = []
    for i, (I1, I2) in enumerate(((24, 20), (20, 24))):
        c = synth.completion_case(33, I1, I2, (3, 4), rank=3, rho=0.4, problem=i)
        c.update(tau=0.3, step=1.0)
        obs, _ = inputs(c)
        ctx = make_ctx(c["transforms"], lt.LT_FP64)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, 2)
        probs.append((c, obs, ctx))
    Xs = [to_dev(np.zeros(o.shape)) for _, o, _ in probs]
    lt.lt_pga_complete_batched([p[2] for p in probs], [to_dev(p[0]["mask"]) for p in probs],
                               [to_dev(p[1]) for p in probs], [0.3, 0.3], [1.0, 1.0], 6, Xs)
    torch.cuda.synchronize()
    for (c, obs, _), Xb in zip(probs, Xs):
        cold, _, _ = run(c, obs, lt.LT_FP64, 6, 0)
        assert np.array_equal(from_dev(Xb, obs.shape), cold)


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
def test_autotune_option_single_and_batched(prec):
    """LT_OPT_AUTOTUNE: the first PGA call on a new slice shape times the SVT kernel forms
    on the problem's first-iterate input and keeps the fastest; the iterates stay within
    the bound of the oracle (single call, a second call on the tuned context, and a batch
    of three problems of two shapes, one tuning per shape)."""
    probs = []
    for i, (I1, I2) in enumerate(((24, 20), (20, 24), (24, 20))):
        c = synth.completion_case(34, I1, I2, (3, 4), rank=3, rho=0.4, problem=i)
        c.update(tau=0.3, step=1.0)
        obs, Ms = inputs(c)
        ref, _ = O.pga(c["mask"], obs, 0.3, 1.0, 8, Ms)
        probs.append((c, obs, ref))
    dt = dtype_of(prec)
    c, obs, ref = probs[0]
    ctx = make_ctx(c["transforms"], prec)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_AUTOTUNE, 1)
    for _ in range(2):
        X = to_dev(np.zeros(obs.shape), dt)
        lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs, dt), 0.3, 1.0, 8, X)
        torch.cuda.synchronize()
        assert rel(from_dev(X, obs.shape), ref) <= TOL[prec]
    ctxs = [make_ctx(p[0]["transforms"], prec) for p in probs]
    for cx in ctxs:
        lt.lt_ctx_set_option(cx, lt.LT_OPT_AUTOTUNE, 1)
    Xs = [to_dev(np.zeros(p[1].shape), dt) for p in probs]
    lt.lt_pga_complete_batched(ctxs, [to_dev(p[0]["mask"]) for p in probs],
                               [to_dev(p[1], dt) for p in probs], [0.3] * 3, [1.0] * 3, 8, Xs)
    torch.cuda.synchronize()
    for (c, obs, ref), Xb in zip(probs, Xs):
        assert rel(from_dev(Xb, obs.shape), ref) <= TOL[prec]
    with pytest.raises(lt.LtError):
        lt.lt_ctx_set_option(ctxs[0], lt.LT_OPT_AUTOTUNE, 2)
