"""Full-size parity of the large workloads: the fifth-order product and L-SVT with
ill-conditioned transforms (256x256x16x16x8, cond(L_k) = 1e2 each, so cond(L) = 1e6) and
the large completion (540x960x3x120).  The oracle cannot redo these whole tensors in
seconds, so it checks sampled outputs it can compute one by one (full output tubes of
the product; transform-domain slices of the L-SVT) or one full PGA iteration.

Tolerances scale with the conditioning of L: a forward-stable evaluation of L^{-1}(.)
loses up to cond(L) u relative to the result, so the bound is 10 cond(L) u with u the
unit roundoff of the path (2^-53 FP64, 2^-24 FP32), floored at the orthonormal-L bounds
(1e-12 FP64, 1e-5 FP32).
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import dtype_of, empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

# unit roundoff of the arithmetic: LT_MIXED's face-wise GEMM carries about 21 bits
U = {lt.LT_FP64: 2.0 ** -53, lt.LT_FP32: 2.0 ** -24, lt.LT_MIXED: 2.0 ** -21}
FLOOR = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}


def tol_for(prec, Ms):
    kappa = float(np.prod([np.linalg.cond(M) for M in Ms]))
    return max(FLOOR[prec], 10.0 * kappa * U[prec]), kappa


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


@pytest.fixture(scope="module")
def config3():
    return synth.config3()


def kron_rows(Ms):
    """(M_5 kron M_4 kron M_3): maps the P slices of a tube to its transform."""
    K = np.eye(1)
    for M in Ms:
        K = np.kron(M, K)
    return K


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32, lt.LT_MIXED])
def test_config3_product_sampled_tubes(config3, prec):
    A, B = config3["A"], config3["B"]
    Ms = oracle_mats(config3["transforms"])
    ctx = make_ctx(config3["transforms"], prec)
    dt = dtype_of(prec)
    Ad, Bd = to_dev(A, dt), to_dev(B, dt)
    Cd = empty_dev((256, 128, 16, 16, 8), dt)
    lt.lt_product(ctx, Ad, Bd, Cd)
    torch.cuda.synchronize()
    del Ad, Bd
    tol, kappa = tol_for(prec, Ms)
    rng = np.random.default_rng(33)
    errs = []
    for _ in range(6):
        i, j = int(rng.integers(256)), int(rng.integers(128))
        Ah = O.transform(A[i:i + 1], Ms)           # row i of A, all slices
        Bh = O.transform(B[:, j:j + 1], Ms)        # column j of B, all slices
        Ch = np.einsum("alpqr,lbpqr->abpqr", Ah, Bh)
        ref = O.inverse_transform(Ch, Ms)[0, 0]    # the (i, j) tube of C
        got = Cd[:, :, :, j, i].double().cpu().numpy().transpose(2, 1, 0)
        errs.append(rel(got, ref))
    assert max(errs) <= tol, (max(errs), tol, kappa)
    if prec == lt.LT_MIXED:  # the face-wise GEMM ran on the tensor cores
        assert lt.lt_ctx_get_stats(ctx)["tc_launches"] == 1


def test_config3_svt_sampled_slices(config3):
    """FP32 L-SVT of the 256x256x16x16x8 tensor (working matrix in global memory):
    L(D)^p against the oracle's SVT of L(A)^p on sampled slices p; tau = 0.1 times the
    median largest singular value of the sampled transform-domain slices."""
    prec = lt.LT_FP32
    A = config3["A"]
    Ms = oracle_mats(config3["transforms"])
    K = kron_rows(Ms)                              # P x P
    P = K.shape[0]
    Aslices = O.slices(A).reshape(256 * 256, P, order="F")  # (i1 + 256 i2) x P
    samples = [0, 513, 1337, 2047]
    Ahat = {p: (Aslices @ K[p]).reshape(256, 256, order="F") for p in samples}
    tau = 0.1 * float(np.median([np.linalg.norm(Ahat[p], 2) for p in samples]))
    ctx = make_ctx(config3["transforms"], prec)
    Ad = to_dev(A, torch.float32)
    D = empty_dev(A.shape, torch.float32)
    lt.lt_svt(ctx, Ad, tau, D)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0
    del Ad
    # L(D) in FP64 on the GPU (an FP64 context over the same matrices)
    ctx64 = make_ctx(config3["transforms"], lt.LT_FP64)
    D64 = D.double()
    del D
    Dh = torch.empty_like(D64)
    lt.lt_transform(ctx64, D64, Dh)
    torch.cuda.synchronize()
    tol, kappa = tol_for(prec, Ms)
    for p in samples:
        k4, k3 = divmod(p, 16)
        k5, k4 = divmod(k4, 16)
        got = Dh[k5, k4, k3].cpu().numpy().T      # slice p, (I1, I2)
        u, s, vt = np.linalg.svd(Ahat[p], full_matrices=False)
        ref = (u * np.maximum(s - tau, 0)) @ vt
        assert rel(got, ref) <= tol, (p, rel(got, ref), tol)


@pytest.fixture(scope="module")
def config5():
    c = synth.config5()
    Ms = oracle_mats(c["transforms"])
    X = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    c["obs"] = c["mask"] * (X + c["noise"])
    c["Ms"] = Ms
    c["X1"] = O.svt(c["mask"] * c["obs"], c["tau"], Ms)   # the first PGA iterate
    return c


@pytest.mark.parametrize("prec", [lt.LT_FP32, lt.LT_FP64])
def test_config5_one_pga_iteration(config5, prec):
    """One PGA iteration of the 540x960x3x120 completion (X^1 = D_tau(P_Omega(M))) against
    the oracle, on every element."""
    c = config5
    ctx = make_ctx(c["transforms"], prec)
    dt = dtype_of(prec)
    X = to_dev(np.zeros(c["obs"].shape), dt)
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(c["obs"], dt), c["tau"], c["step"], 1, X,
                       report=rep)
    torch.cuda.synchronize()
    assert rep.iters_done == 1 and rep.device_status == 0
    ref = c["X1"]
    tol, _ = tol_for(prec, c["Ms"])
    assert rel(from_dev(X, c["obs"].shape), ref) <= tol


def test_config5_fp32_iterations_progress(config5):
    """A few FP32 iterations at full size through the checkpoint state: no device errors,
    the relative residual of the stopping test stays small (it need not decrease
    monotonically under momentum)."""
    c = config5
    ctx = make_ctx(c["transforms"], lt.LT_FP32)
    X = to_dev(np.zeros(c["obs"].shape), torch.float32)
    m, o = to_dev(c["mask"]), to_dev(c["obs"], torch.float32)
    prev = torch.zeros_like(X)  # checkpoint buffer: must outlive the calls
    st = lt.lt_pga_state(X_prev=prev.data_ptr(), t_prev=1.0, t=1.0, k=0)
    res = []
    for _ in range(3):
        rep = lt.lt_pga_report()
        lt.lt_pga_complete(ctx, m, o, c["tau"], c["step"], 2, X, state=st, report=rep)
        torch.cuda.synchronize()
        assert rep.device_status == 0
        res.append(rep.rel_residual)
    assert st.k == 6
    assert all(np.isfinite(r) and r < 1e-2 for r in res)
