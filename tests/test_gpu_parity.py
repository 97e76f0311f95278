"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element
on the same seeded inputs.

Tolerances (relative Frobenius error against the oracle):
  FP64 path: 1e-12 (orthonormal or moderately conditioned L).
  FP32 path: 1e-5 -- single precision with unit roundoff u = 6e-8; transforms of
             size I accumulate ~sqrt(I) u of relative error per mode and the Jacobi SVT
             stops at sqrt(m) u pair orthogonality (a few 1e-7 for these sizes), which
             the momentum of Algorithm 5 amplifies about tenfold over 100 iterations.
"""
import math

import numpy as np
import pytest
import torch

from oracle import definitions as Def
from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import (dtype_of, empty_dev, from_dev, make_ctx, oracle_mats, rel,
                            to_dev)

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5}
PRECS = [lt.LT_FP64, lt.LT_FP32]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


def random_transforms(rng, sizes, cond=10.0):
    return [("matrix", synth.conditioned_matrix(rng, n, cond, two_sided=True)) for n in sizes]


# ------------------------------------------------------------------ transforms
TRANSFORM_CASES = [
    ((32, 24), [("dct", 8)]),
    ((5, 7), [("dct", 3), ("dct", 4)]),
    ((1, 1), [("dct", 2), ("dct", 3), ("dct", 2)]),
    ((13, 9), [("dct", 1)]),
    ((33, 3), "random3"),
    ((3, 5), [("dct", 16), ("dct", 16), ("dct", 8)]),     # P = 2048: grouped passes
    ((7, 6), [("dct", 120)]),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,transforms", TRANSFORM_CASES)
def test_transform_and_inverse(prec, shape, transforms):
    rng = np.random.default_rng(100 + shape[0])
    if transforms == "random3":
        transforms = random_transforms(rng, (4, 3, 5))
    full = tuple(shape) + tuple(
        t[1] if t[0] == "dct" else np.asarray(t[1]).shape[0] for t in transforms)
    X = rng.uniform(-1, 1, size=full)
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    Xd = to_dev(X, dt)
    Xh = empty_dev(full, dt)
    lt.lt_transform(ctx, Xd, Xh)
    Xb = empty_dev(full, dt)
    lt.lt_inverse(ctx, Xh, Xb)
    torch.cuda.synchronize()
    assert rel(from_dev(Xh, full), O.transform(X, Ms)) <= TOL[prec]
    assert rel(from_dev(Xb, full), X) <= TOL[prec] * 10
    # in place
    lt.lt_transform(ctx, Xd, Xd)
    torch.cuda.synchronize()
    assert rel(from_dev(Xd, full), O.transform(X, Ms)) <= TOL[prec]


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("prec", PRECS)
def test_product_config1(prec):
    """*_L-product of the 32x24x8 and 24x16x8 operands (DCT-II 8)."""
    c = synth.config1()
    Ms = oracle_mats(c["transforms"])
    ctx = make_ctx(c["transforms"], prec)
    dt = dtype_of(prec)
    A, B = to_dev(c["A"], dt), to_dev(c["B"], dt)
    Cd = empty_dev((32, 16, 8), dt)
    lt.lt_product(ctx, A, B, Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, (32, 16, 8)), O.product(c["A"], c["B"], Ms)) <= TOL[prec]


@pytest.mark.parametrize("shapes", [((3, 2, 4), (2, 3, 4)), ((2, 3, 3, 2), (3, 2, 3, 2)),
                                    ((4, 2, 2, 3, 2), (2, 5, 2, 3, 2))])
def test_product_equals_cproduct_definition(shapes):
    """With M = W^{-1} C (I+Z) from lt_make_cproduct on every mode the GPU product is
    the generalized c-product ten(btph(A) btph(B)) of Def. 9."""
    rng = np.random.default_rng(7)
    A, B = rng.standard_normal(shapes[0]), rng.standard_normal(shapes[1])
    tr = [("cprod", n) for n in shapes[0][2:]]
    ctx = make_ctx(tr)
    Cshape = (shapes[0][0], shapes[1][1]) + tuple(shapes[0][2:])
    Cd = empty_dev(Cshape)
    lt.lt_product(ctx, to_dev(A), to_dev(B), Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, Cshape), Def.cproduct_def(A, B)) <= 1e-12


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("I1,l,I2,trailing", [(65, 17, 70, (3,)), (1, 1, 1, (2, 2)),
                                              (130, 64, 129, (2, 3))])
def test_product_ragged_tiles(prec, I1, l, I2, trailing):
    rng = np.random.default_rng(I1 + l + I2)
    A = rng.uniform(-1, 1, (I1, l) + trailing)
    B = rng.uniform(-1, 1, (l, I2) + trailing)
    tr = random_transforms(rng, trailing)
    ctx = make_ctx(tr, prec)
    dt = dtype_of(prec)
    Cd = empty_dev((I1, I2) + trailing, dt)
    lt.lt_product(ctx, to_dev(A, dt), to_dev(B, dt), Cd)
    torch.cuda.synchronize()
    assert rel(from_dev(Cd, (I1, I2) + trailing), O.product(A, B, oracle_mats(tr))) <= TOL[prec] * 10


# ------------------------------------------------------------------ SVD
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,transforms", [((32, 24), [("dct", 8)]), ((24, 32), [("dct", 8)]),
                                              ((7, 7), [("dct", 3), ("dct", 2)]),
                                              ((9, 4), "random2")])
def test_svd_invariants(prec, shape, transforms):
    """Theorem of Eq. tsvd1: A = U * S * V^T, L(U)^p and L(V)^p orthogonal, L(S)^p
    diagonal with the oracle's singular values (descending).  Vectors are not unique,
    so they are checked through these invariants."""
    rng = np.random.default_rng(shape[0] * 31 + shape[1])
    if transforms == "random2":
        transforms = random_transforms(rng, (3, 2))
    if shape == (32, 24):
        A = synth.config1()["A"]
    else:
        trailing = tuple(t[1] if t[0] == "dct" else np.asarray(t[1]).shape[0] for t in transforms)
        A = rng.uniform(-1, 1, tuple(shape) + trailing)
    trailing = A.shape[2:]
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    I1, I2 = shape
    P = int(np.prod(trailing))
    U, S, V = empty_dev((I1, I1) + trailing, dt), empty_dev((I1, I2) + trailing, dt), \
        empty_dev((I2, I2) + trailing, dt)
    sig = torch.empty((P, min(I1, I2)), dtype=dt, device="cuda")
    lt.lt_svd(ctx, to_dev(A, dt), U, S, V, sigma=sig)
    torch.cuda.synchronize()
    Uh, Sh, Vh = (from_dev(t, s) for t, s in ((U, (I1, I1) + trailing), (S, (I1, I2) + trailing),
                                                (V, (I2, I2) + trailing)))
    tol = TOL[prec]
    rec = O.product(O.product(Uh, Sh, Ms), O.transpose(Vh, Ms), Ms)
    e_rec = rel(rec, A)
    _, _, _, sig_ref = O.svd(A, Ms)
    e_sig = rel(sig.double().cpu().numpy().T, sig_ref)
    Lu, Ls, Lv = (O.slices(O.transform(T, Ms)) for T in (Uh, Sh, Vh))
    e_u = max(np.abs(Lu[:, :, p].T @ Lu[:, :, p] - np.eye(I1)).max() for p in range(P))
    e_v = max(np.abs(Lv[:, :, p].T @ Lv[:, :, p] - np.eye(I2)).max() for p in range(P))
    e_off = 0.0
    for p in range(P):
        off = Ls[:, :, p].copy()
        np.fill_diagonal(off, 0)
        e_off = max(e_off, np.abs(off).max() / np.abs(Ls).max())
    print(f"svd invariants prec {prec} {shape}: reconstruction {e_rec:.2e}, sigma {e_sig:.2e}, "
          f"L(U) orth {e_u:.2e}, L(V) orth {e_v:.2e}, L(S) off-diagonal {e_off:.2e}")
    assert e_rec <= tol and e_sig <= tol
    assert e_u <= tol and e_v <= tol
    assert e_off <= tol


# ------------------------------------------------------------------ SVT
SVT_CASES = [((32, 24), [("dct", 8)], 0.5), ((24, 32), [("dct", 8)], 0.5),
             ((17, 17), [("dct", 3), ("dct", 4)], 0.3), ((144, 176), [("dct", 3)], 2.0),
             ((176, 144), [("dct", 2)], 2.0), ((5, 31), "random2", 0.1),
             ((40, 9), [("dct", 2)], 0.0), ((8, 6), [("dct", 2)], 1e6)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,transforms,tau", SVT_CASES)
def test_svt(prec, shape, transforms, tau):
    rng = np.random.default_rng(shape[0] + 1000 * shape[1])
    if transforms == "random2":
        transforms = random_transforms(rng, (2, 3))
    trailing = tuple(t[1] if t[0] == "dct" else np.asarray(t[1]).shape[0] for t in transforms)
    full = tuple(shape) + trailing
    A = synth.config1()["A"] if full == (32, 24, 8) else rng.standard_normal(full)
    Ms = oracle_mats(transforms)
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    Ad = to_dev(A, dt)
    D = empty_dev(full, dt)
    lt.lt_svt(ctx, Ad, tau, D)
    torch.cuda.synchronize()
    ref = O.svt(A, tau, Ms)
    if np.linalg.norm(ref) == 0:
        assert np.abs(from_dev(D, full)).max() <= TOL[prec] * np.abs(A).max()
    else:
        assert rel(from_dev(D, full), ref) <= TOL[prec]
    # in place (D aliases A)
    lt.lt_svt(ctx, Ad, tau, Ad)
    torch.cuda.synchronize()
    if np.linalg.norm(ref) > 0:
        assert rel(from_dev(Ad, full), ref) <= TOL[prec]
    assert lt.lt_last_device_status(ctx) == 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("group,pairwise", [(0, 0), (0, 1), (8, 0), (16, 0), (32, 0)])
@pytest.mark.parametrize("shape", [(37, 23), (144, 176), (300, 290)])
def test_svt_kernel_variants(prec, group, pairwise, shape):
    """Every instantiated form of the SVT kernel (lanes per pair, register-blocked or
    pairwise sweeps) against the oracle, on an odd shape, the benchmark's slice shape
    and a slice that needs the large-column forms."""
    rng = np.random.default_rng(shape[0])
    transforms = [("dct", 2)]
    full = tuple(shape) + (2,)
    A = rng.standard_normal(full)
    ctx = make_ctx(transforms, prec)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_GROUP, group)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_BLOCK, pairwise)
    dt = dtype_of(prec)
    D = empty_dev(full, dt)
    max_rows = {lt.LT_FP64: {8: 144, 16: 224, 32: 512}, lt.LT_FP32: {8: 192, 16: 384, 32: 1024}}
    if group and min(shape) > max_rows[prec][group]:
        # a forced group width too narrow for the slice is refused, nothing enqueued
        with pytest.raises(lt.LtError) as err:
            lt.lt_svt(ctx, to_dev(A, dt), 1.0, D)
        assert err.value.status == -2
        return
    lt.lt_svt(ctx, to_dev(A, dt), 1.0, D)
    torch.cuda.synchronize()
    assert rel(from_dev(D, full), O.svt(A, 1.0, oracle_mats(transforms))) <= TOL[prec]
    assert lt.lt_last_device_status(ctx) == 0


@pytest.mark.parametrize("group", [8, 16, 32])
@pytest.mark.parametrize("shape", [(37, 23), (144, 176)])
def test_svt_forced_register_blocks(group, shape):
    """FP32 register-blocked sweeps with a forced group width (LT_OPT_JACOBI_BLOCK = 2:
    8-lane groups with blocks of 2 columns, 16 with blocks of 4, 32 with blocks of 2)
    against the oracle."""
    rng = np.random.default_rng(shape[0] + group)
    transforms = [("dct", 2)]
    full = tuple(shape) + (2,)
    A = rng.standard_normal(full)
    ctx = make_ctx(transforms, lt.LT_FP32)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_GROUP, group)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_BLOCK, 2)
    D = empty_dev(full, torch.float32)
    lt.lt_svt(ctx, to_dev(A, torch.float32), 1.0, D)
    torch.cuda.synchronize()
    assert rel(from_dev(D, full), O.svt(A, 1.0, oracle_mats(transforms))) <= TOL[lt.LT_FP32]
    assert lt.lt_last_device_status(ctx) == 0


@pytest.mark.parametrize("shape", [(37, 23), (100, 130), (144, 176), (176, 144), (17, 3)])
def test_svt_wide_register_blocks(shape):
    """FP32 wide form (LT_OPT_JACOBI_BLOCK = 3: 16-lane groups with blocks of 2, one group
    per block pair of a round, up to 576 threads) against the oracle, on shapes with
    npad padded (37, 23 and 17, 3), 7 and 9 rows per lane, both orientations."""
    rng = np.random.default_rng(shape[0] * 3 + shape[1])
    transforms = [("dct", 3)]
    full = tuple(shape) + (3,)
    A = rng.standard_normal(full)
    ctx = make_ctx(transforms, lt.LT_FP32)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_BLOCK, 3)
    D = empty_dev(full, torch.float32)
    lt.lt_svt(ctx, to_dev(A, torch.float32), 1.0, D)
    torch.cuda.synchronize()
    assert rel(from_dev(D, full), O.svt(A, 1.0, oracle_mats(transforms))) <= TOL[lt.LT_FP32]
    assert lt.lt_last_device_status(ctx) == 0


@pytest.mark.parametrize("prec,scale", [(lt.LT_FP64, 1e-150), (lt.LT_FP64, 1e-30),
                                        (lt.LT_FP64, 1e30), (lt.LT_FP64, 1e150),
                                        (lt.LT_FP32, 1e-25), (lt.LT_FP32, 1e25)])
def test_svt_is_scale_equivariant(prec, scale):
    """D_{c tau}(c A) = c D_tau(A) (the SVT is positively homogeneous), for data far from
    unit scale: squared norms of such slices leave the FP32 range (and, at 1e+-150, the
    FP64 range), so this checks that the kernel keeps its arithmetic in range."""
    rng = np.random.default_rng(77)
    transforms = [("dct", 3)]
    full = (40, 31, 3)
    A = rng.standard_normal(full)
    ref = O.svt(A, 1.5, oracle_mats(transforms)) * scale
    ctx = make_ctx(transforms, prec)
    dt = dtype_of(prec)
    D = empty_dev(full, dt)
    lt.lt_svt(ctx, to_dev(A * scale, dt), 1.5 * scale, D)
    torch.cuda.synchronize()
    assert rel(from_dev(D, full), ref) <= TOL[prec]
    assert lt.lt_last_device_status(ctx) == 0


# ------------------------------------------------------------------ PGA
def completion_inputs(c):
    Ms = oracle_mats(c["transforms"])
    X = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    obs = c["mask"] * (X + c["noise"])
    return X, obs, Ms


def run_pga(c, obs, prec, iters, tol=0.0, X0=None, state=None):
    ctx = make_ctx(c["transforms"], prec)
    dt = dtype_of(prec)
    shape = obs.shape
    X = to_dev(np.zeros(shape) if X0 is None else X0, dt)
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs, dt), c["tau"], c["step"], iters, X,
                       tol=tol, report=rep, state=state)
    torch.cuda.synchronize()
    return X, rep, ctx


@pytest.mark.parametrize("prec", PRECS)
def test_pga_small(prec):
    c = synth.completion_case(20, 24, 20, (3, 4), rank=3, rho=0.4)
    c.update(tau=0.3, step=1.0)
    Xt, obs, Ms = completion_inputs(c)
    X, rep, _ = run_pga(c, obs, prec, 25)
    ref, info = O.pga(c["mask"], obs, 0.3, 1.0, 25, Ms)
    assert rep.iters_done == 25
    assert rel(from_dev(X, obs.shape), ref) <= TOL[prec]
    # r = ||Y - X^{k+1}|| / ||X^{k+1}|| with Y = X^k + beta (X^k - X^{k-1}), beta < 1:
    # relative errors e of the iterates (e <= TOL) move r by at most (3 + 1 + r) e
    dr = abs(rep.rel_residual - info["residual"][-1])
    print(f"pga small prec {prec}: residual {info['residual'][-1]:.6e}, |dr| {dr:.2e}")
    assert dr <= (4.0 + info["residual"][-1]) * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_pga_objective(prec):
    """The objective of the last iterate, F = tau sum_p ||L(X^{k+1})^p||_* +
    1/2 ||P_Omega(X^{k+1} - M)||^2 (Theorem 21 / Eq. 24 with orthonormal L, the g + f of
    Sec. 4), accumulated on the device from the shrunk singular values and the fused
    inverse transform (LT_OPT_OBJECTIVE), against the oracle's objective, which takes a
    fresh SVD of every L(X^{k+1})^p.  Checked after 1, 7 and 25 iterations."""
    c = synth.completion_case(23, 24, 20, (3, 4), rank=3, rho=0.4)
    c.update(tau=0.3, step=1.0)
    Xt, obs, Ms = completion_inputs(c)
    dt = dtype_of(prec)
    for iters in (1, 7, 25):
        ctx = make_ctx(c["transforms"], prec)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_OBJECTIVE, 1)
        X = to_dev(np.zeros(obs.shape), dt)
        rep = lt.lt_pga_report()
        lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs, dt), c["tau"], c["step"], iters,
                           X, report=rep)
        torch.cuda.synchronize()
        _, info = O.pga(c["mask"], obs, c["tau"], c["step"], iters, Ms, objective=True)
        ref = info["objective"][-1]
        err = abs(rep.objective - ref) / abs(ref)
        print(f"pga objective prec {prec} iters {iters}: {rep.objective:.15e} vs "
              f"{ref:.15e}, rel {err:.2e}")
        assert rep.iters_done == iters and rep.device_status == 0
        assert err <= TOL[prec], (iters, err)


def test_pga_step_and_tolerance_stop():
    c = synth.completion_case(21, 18, 26, (2, 3), rank=2, rho=0.6)
    c.update(tau=0.05, step=0.7)
    Xt, obs, Ms = completion_inputs(c)
    X, rep, _ = run_pga(c, obs, lt.LT_FP64, 300, tol=1e-5)
    ref, info = O.pga(c["mask"], obs, 0.05, 0.7, 300, Ms, tol=1e-5)
    assert rep.iters_done == info["iters"] < 300
    assert rel(from_dev(X, obs.shape), ref) <= 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_pga_continuation(prec):
    """Algorithm 5 with continuation (LT_OPT_MU0 = nu ||M||_F, the paper's choice, and
    nu = 0.9; mu_bar = tau): 40 iterations against the oracle, and a 20 + 20 resume
    through the checkpoint equal to the single run bit for bit (the schedule counts
    iterations from the start of the run)."""
    c = synth.completion_case(12, 24, 20, (3, 4), rank=3, rho=0.4)
    tr = [("dct", 3), ("dct", 4)]
    Ms = oracle_mats(tr)
    X0 = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    obs = c["mask"] * (X0 + c["noise"])
    mu0 = 0.9 * float(np.linalg.norm(obs))
    ref, _ = O.pga(c["mask"], obs, 0.3, 1.0, 40, Ms, mu0=mu0, nu=0.9)
    dt = dtype_of(prec)
    ctx = make_ctx(tr, prec)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_MU0, mu0)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_NU, 0.9)
    mask_d, obs_d = to_dev(c["mask"]), to_dev(obs, dt)
    X = torch.zeros((4, 3, 20, 24), dtype=dt, device="cuda")
    lt.lt_pga_complete(ctx, mask_d, obs_d, 0.3, 1.0, 40, X)
    torch.cuda.synchronize()
    assert rel(from_dev(X, obs.shape), ref) <= TOL[prec]
    Xr = torch.zeros_like(X)
    Xp = torch.empty_like(X)
    state = lt.lt_pga_state(Xp.data_ptr(), 0.0, 0.0, 0)
    lt.lt_pga_complete(ctx, mask_d, obs_d, 0.3, 1.0, 20, Xr, state=state)
    torch.cuda.synchronize()
    lt.lt_pga_complete(ctx, mask_d, obs_d, 0.3, 1.0, 20, Xr, state=state)
    torch.cuda.synchronize()
    assert torch.equal(Xr, X)
    # one graph per batch: continuation is refused there, nothing enqueued
    with pytest.raises(lt.LtError):
        lt.lt_pga_complete_batched([ctx], [mask_d], [obs_d], [0.3], [1.0], 2, [Xr])
    for bad in (-1.0, float("nan")):
        with pytest.raises(lt.LtError):
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_MU0, bad)
    for bad in (0.0, 1.5):
        with pytest.raises(lt.LtError):
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_NU, bad)


def test_pga_resume_is_bitwise():
    """50 + 50 iterations through the checkpoint state equal 100 in one call, bit for bit
    (fixed-order reductions)."""
    c = synth.completion_case(22, 16, 12, (3, 2), rank=2, rho=0.5)
    c.update(tau=0.2, step=1.0)
    _, obs, _ = completion_inputs(c)
    Xa, _, _ = run_pga(c, obs, lt.LT_FP64, 100)
    ctx = make_ctx(c["transforms"])
    Xb = to_dev(np.zeros(obs.shape))
    prev = torch.zeros_like(Xb)
    st = lt.lt_pga_state(X_prev=prev.data_ptr(), t_prev=1.0, t=1.0, k=0)
    m, o = to_dev(c["mask"]), to_dev(obs)
    lt.lt_pga_complete(ctx, m, o, 0.2, 1.0, 50, Xb, state=st)
    torch.cuda.synchronize()
    assert st.k == 50
    lt.lt_pga_complete(ctx, m, o, 0.2, 1.0, 50, Xb, state=st)
    torch.cuda.synchronize()
    assert st.k == 100
    assert torch.equal(Xa, Xb)


@pytest.mark.parametrize("prec", PRECS)
def test_pga_config2_full(prec):
    """The benchmarked workload at full size: 144x176x3x32, L-rank 10, 30% observed,
    DCT 3 / DCT 32, tau 0.5, step 1, 100 iterations."""
    c = synth.config2()
    Xt, obs, Ms = completion_inputs(c)
    X, rep, _ = run_pga(c, obs, prec, c["iters"])
    ref, info = O.pga(c["mask"], obs, c["tau"], c["step"], c["iters"], Ms)
    got = from_dev(X, obs.shape)
    assert rep.iters_done == 100
    assert rep.device_status == 0
    assert rel(got, ref) <= (1e-12 if prec == lt.LT_FP64 else 1e-5)
    # sanity of the completion itself (not parity): the low-rank truth is recovered
    assert O.rse(Xt, ref) < 0.05


# ------------------------------------------------------------------ boundary
def test_argument_errors_enqueue_nothing():
    ctx = make_ctx([("dct", 4)])
    x = torch.zeros((4, 3, 2), dtype=torch.float64, device="cuda")
    L = lt.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.lt_transform(None, 2, 3, x.data_ptr(), x.data_ptr(), None, 0, s) == -1
    assert L.lt_transform(ctx.handle, 0, 3, x.data_ptr(), x.data_ptr(), None, 0, s) == -1
    assert L.lt_svt(ctx.handle, 2, 3, x.data_ptr(), -1.0, x.data_ptr(), None, 0, s) == -1
    need = lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 2, 3)
    assert need > 0
    m = torch.zeros((4, 3, 2), dtype=torch.uint8, device="cuda")
    assert L.lt_pga_complete(ctx.handle, 2, 3, m.data_ptr(), x.data_ptr(), 0.1, 1.0, 5, 0.0,
                             x.data_ptr(), None, None, None, 0, s) == -8
    assert L.lt_pga_complete(ctx.handle, 2, 3, m.data_ptr(), x.data_ptr(), 0.1, 0.0, 5, 0.0,
                             x.data_ptr(), None, None, None, 0, s) == -1
    sing = np.zeros((3, 3))
    with pytest.raises(lt.LtError) as e:
        lt.Context([3], [sing])
    assert e.value.status == -3
    with pytest.raises(lt.LtError):
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_MAX_SWEEPS, 0)


def test_device_status_noconv_and_nonfinite():
    ctx = make_ctx([("dct", 2)])
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 12, 2))
    D = empty_dev(A.shape)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_MAX_SWEEPS, 1)
    lt.lt_svt(ctx, to_dev(A), 0.1, D)
    st = lt.lt_last_device_status(ctx)
    assert st & lt.LT_DEV_NOCONV
    assert np.all(np.isfinite(from_dev(D, A.shape)))
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_MAX_SWEEPS, 40)
    A[3, 4, 1] = np.nan
    lt.lt_svt(ctx, to_dev(A), 0.1, D)
    assert lt.lt_last_device_status(ctx) & lt.LT_DEV_NONFINITE
    assert lt.lt_last_device_status(ctx) == 0  # read-and-clear


def test_host_helpers_match_golden_and_oracle():
    from tests.conftest import load_golden_matrices
    g = load_golden_matrices()
    for n in (2, 3):
        assert np.allclose(lt.lt_make_dct(n), g[("dct", n)], atol=1e-15)
        assert np.allclose(lt.lt_make_cproduct(n), g[("cprod", n)], atol=1e-14)
    for n in (1, 5, 32, 120):
        assert np.abs(lt.lt_make_dct(n) - O.dct_matrix(n)).max() < 1e-14
        assert np.abs(lt.lt_make_cproduct(n) - O.cproduct_matrix(n)).max() < 1e-11


# ------------------------------------------------------------------ batched PGA
def batch_problems(specs, prec, rng_seed=40):
    """specs: list of (I1, I2, trailing, rank, rho, tau).  Returns contexts, device
    masks/obs, taus and the host obs/mask (oracle inputs)."""
    out = []
    for i, (I1, I2, trailing, rank, rho, tau) in enumerate(specs):
        c = synth.completion_case(rng_seed, I1, I2, trailing, rank=rank, rho=rho, problem=i)
        Ms = oracle_mats(c["transforms"])
        X = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
        obs = c["mask"] * (X + c["noise"])
        out.append({"ctx": make_ctx(c["transforms"], prec), "mask": c["mask"], "obs": obs,
                    "Ms": Ms, "tau": tau})
    return out


def run_batched(probs, prec, iters):
    dt = dtype_of(prec)
    Xs = [to_dev(np.zeros(p["obs"].shape), dt) for p in probs]
    reps = []
    lt.lt_pga_complete_batched([p["ctx"] for p in probs], [to_dev(p["mask"]) for p in probs],
                               [to_dev(p["obs"], dt) for p in probs], [p["tau"] for p in probs],
                               [1.0] * len(probs), iters, Xs, reports=reps)
    torch.cuda.synchronize()
    return Xs, reps[0]


SMALL_BATCH = [(24, 20, (3, 4), 3, 0.4, 0.3), (40, 18, (3, 8), 2, 0.3, 0.2),
               (17, 33, (3, 2), 4, 0.5, 0.5), (64, 48, (3, 8), 5, 0.25, 0.4),
               (9, 12, (3, 16), 2, 0.45, 0.1)]


@pytest.mark.parametrize("prec", PRECS)
def test_pga_batched_equals_single_runs(prec):
    """The batch (one CUDA graph with a branch per problem) gives exactly what separate
    lt_pga_complete calls give: same kernels, fixed-order reductions (7 iterations: three
    graph replays and one direct iteration)."""
    probs = batch_problems(SMALL_BATCH, prec)
    Xs, reps = run_batched(probs, prec, 7)
    dt = dtype_of(prec)
    for p, Xb, rep in zip(probs, Xs, reps):
        Xs1 = to_dev(np.zeros(p["obs"].shape), dt)
        lt.lt_pga_complete(p["ctx"], to_dev(p["mask"]), to_dev(p["obs"], dt), p["tau"], 1.0, 7, Xs1)
        torch.cuda.synchronize()
        assert torch.equal(Xb, Xs1)
        assert rep.iters_done == 7 and rep.device_status == 0


@pytest.mark.parametrize("prec", PRECS)
def test_pga_batched_vs_oracle(prec):
    probs = batch_problems(SMALL_BATCH[:3], prec)
    Xs, _ = run_batched(probs, prec, 10)
    for p, Xb in zip(probs, Xs):
        ref, _ = O.pga(p["mask"], p["obs"], p["tau"], 1.0, 10, p["Ms"])
        assert rel(from_dev(Xb, p["obs"].shape), ref) <= TOL[prec]


def test_pga_batched_with_tensor_core_passes_equals_single_runs():
    """LT_MIXED batch with the mode-4 products routed to the tensor cores
    (LT_OPT_TC_MODE_MIN = 8): the tcgen05 kernels captured in the batch graph give the
    same iterates as separate calls, bit for bit, and stay within the bound of the
    oracle."""
    probs = batch_problems(SMALL_BATCH, lt.LT_MIXED)
    for p in probs:
        lt.lt_ctx_set_option(p["ctx"], lt.LT_OPT_TC_MODE_MIN, 8)
    Xs, reps = run_batched(probs, lt.LT_MIXED, 7)
    assert sum(lt.lt_ctx_get_stats(p["ctx"])["tc_launches"] for p in probs) > 0
    for p, Xb, rep in zip(probs, Xs, reps):
        Xs1 = to_dev(np.zeros(p["obs"].shape), torch.float32)
        lt.lt_pga_complete(p["ctx"], to_dev(p["mask"]), to_dev(p["obs"], torch.float32), p["tau"],
                           1.0, 7, Xs1)
        torch.cuda.synchronize()
        assert torch.equal(Xb, Xs1)
        assert rep.iters_done == 7 and rep.device_status == 0
        ref, _ = O.pga(p["mask"], p["obs"], p["tau"], 1.0, 7, p["Ms"])
        assert rel(from_dev(Xb, p["obs"].shape), ref) <= 1e-5


@pytest.mark.parametrize("prec", [lt.LT_FP32, lt.LT_MIXED])
def test_pga_batched_config4_full(prec):
    """The 64-problem batch of uneven sizes (I1 x I2 from 64 x 48 to 512 x 384, I3 = 3,
    I4 in {8, 16, 32, 64}), FP32 and LT_MIXED (the benchmark's batched leg; its I4 = 64
    problems put the mode-4 products on the tensor cores): every problem completes its
    iterations without device errors, two of them (for LT_MIXED one with I4 = 64) equal
    their single-problem runs bit for bit, and the largest problem (512 x 384 x 3 x 16)
    and the first with I4 = 64 (320 x 240 x 3 x 64) match the FP64 oracle within 1e-5."""
    shapes = synth.config4_shapes()
    rng = np.random.default_rng(4)
    ctxs, masks, obss, Xs, host = [], [], [], [], []
    for i, sh in enumerate(shapes):
        full = (sh["I1"], sh["I2"]) + sh["trailing"]
        ctxs.append(make_ctx([("dct", n) for n in sh["trailing"]], prec))
        m = (rng.random(full) < sh["rho"]).astype(np.uint8)
        o = m * rng.standard_normal(full)
        host.append((m, o.astype(np.float32).astype(np.float64)))
        masks.append(to_dev(m))
        obss.append(to_dev(o, torch.float32))
        Xs.append(torch.zeros(tuple(reversed(full)), dtype=torch.float32, device="cuda"))
    reps = []
    lt.lt_pga_complete_batched(ctxs, masks, obss, [0.5] * 64, [1.0] * 64, 4, Xs, reports=reps)
    torch.cuda.synchronize()
    assert all(r.iters_done == 4 and r.device_status == 0 for r in reps[0])
    check = [0, 37]
    if prec == lt.LT_MIXED:
        check[1] = next(i for i, sh in enumerate(shapes) if sh["trailing"][1] == 64)
        assert lt.lt_ctx_get_stats(ctxs[check[1]])["tc_launches"] > 0
    for i in check:
        X1 = torch.zeros_like(Xs[i])
        lt.lt_pga_complete(ctxs[i], masks[i], obss[i], 0.5, 1.0, 4, X1)
        torch.cuda.synchronize()
        assert torch.equal(Xs[i], X1)
    largest = max(range(len(shapes)), key=lambda i: shapes[i]["I1"] * shapes[i]["I2"])
    first64 = next(i for i, sh in enumerate(shapes) if sh["trailing"][1] == 64)
    for i in (largest, first64):
        sh = shapes[i]
        full = (sh["I1"], sh["I2"]) + sh["trailing"]
        m, o = host[i]
        ref, _ = O.pga(m, o, 0.5, 1.0, 4, [O.dct_matrix(n) for n in sh["trailing"]])
        err = rel(from_dev(Xs[i], full), ref)
        print(f"batch problem {i} {full} prec {prec}: rel err vs oracle {err:.2e}")
        assert err <= 1e-5
