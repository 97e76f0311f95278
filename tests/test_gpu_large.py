"""Full-size parity of the large workloads: the fifth-order product and L-SVT with
ill-conditioned transforms (256x256x16x16x8, cond(L_k) = 1e2 each, so cond(L) = 1e6) and
the large completion (540x960x3x120).  The oracle cannot redo these whole tensors in
seconds, so it checks sampled outputs it can compute one by one (full output tubes of
the product; transform-domain slices of the L-SVT) or one full PGA iteration.

Bounds on the fifth-order workload are fixed, not scaled by cond(L): 1e-12 for FP64 and
1e-5 for FP32 and LT_MIXED (the stated bounds of the paths).  cond(L) = 1e6 is a
worst-case amplification of a normwise perturbation of the transform-domain tensor;
the rounding of the inputs and of the matrices M_k to FP32 costs 1e-8 .. 1e-7 on these
outputs against the FP64 oracle (the oracle evaluated on rounded inputs), so the
measured errors printed by the tests are far below cond(L) u.  The large completion
uses orthonormal-or-cond-10 transforms and the same fixed bounds.
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import dtype_of, empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

BOUND = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5, lt.LT_MIXED: 1e-5}
NAME = {lt.LT_FP64: "fp64", lt.LT_FP32: "fp32", lt.LT_MIXED: "mixed"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


@pytest.fixture(scope="module")
def config3():
    return synth.config3()


@pytest.fixture(scope="module")
def config3_svt(config3):
    """Sampled transform-domain slices L(A)^p of the 256x256x16x16x8 tensor and the SVT
    threshold tau = 0.1 x the median largest singular value of those slices."""
    Ms = oracle_mats(config3["transforms"])
    K = kron_rows(Ms)                              # P x P
    P = K.shape[0]
    Aslices = O.slices(config3["A"]).reshape(256 * 256, P, order="F")  # (i1 + 256 i2) x P
    samples = [0, 513, 1337, 2047]
    Ahat = {p: (Aslices @ K[p]).reshape(256, 256, order="F") for p in samples}
    tau = 0.1 * float(np.median([np.linalg.norm(Ahat[p], 2) for p in samples]))
    return {"samples": samples, "Ahat": Ahat, "tau": tau}


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
    tol = BOUND[prec]
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
    print(f"config3 product {NAME[prec]}: max rel err over 6 tubes {max(errs):.3e} "
          f"(all: {', '.join(f'{e:.2e}' for e in errs)}), bound {tol:.0e}")
    assert max(errs) <= tol, (max(errs), tol)
    if prec == lt.LT_MIXED:  # the face-wise GEMM ran on the tensor cores
        assert lt.lt_ctx_get_stats(ctx)["tc_launches"] == 1


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32, lt.LT_MIXED])
def test_config3_svt_sampled_slices(config3, config3_svt, prec):
    """L-SVT of the 256x256x16x16x8 tensor (2048 slices of 256 x 256): L(D)^p against the
    oracle's SVT of L(A)^p on sampled slices p; tau = 0.1 times the median largest
    singular value of the sampled transform-domain slices.  L(D) is formed in FP64 on the
    GPU (an FP64 context over the same matrices) so that the check measures the SVT's
    error, not a second rounding."""
    A = config3["A"]
    samples, Ahat, tau = config3_svt["samples"], config3_svt["Ahat"], config3_svt["tau"]
    ctx = make_ctx(config3["transforms"], prec)
    dt = dtype_of(prec)
    Ad = to_dev(A, dt)
    D = empty_dev(A.shape, dt)
    lt.lt_svt(ctx, Ad, tau, D)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0
    del Ad
    ctx64 = make_ctx(config3["transforms"], lt.LT_FP64)
    D64 = D.double()
    del D
    Dh = torch.empty_like(D64)
    lt.lt_transform(ctx64, D64, Dh)
    torch.cuda.synchronize()
    tol = BOUND[prec]
    errs = []
    for p in samples:
        k4, k3 = divmod(p, 16)
        k5, k4 = divmod(k4, 16)
        got = Dh[k5, k4, k3].cpu().numpy().T      # slice p, (I1, I2)
        u, s, vt = np.linalg.svd(Ahat[p], full_matrices=False)
        ref = (u * np.maximum(s - tau, 0)) @ vt
        errs.append(rel(got, ref))
    print(f"config3 svt {NAME[prec]}: rel err per sampled slice "
          f"{', '.join(f'{e:.2e}' for e in errs)}, bound {tol:.0e}")
    assert max(errs) <= tol, (errs, tol)


# Original-domain error of the FP32 / LT_MIXED L-SVT of the 256x256x16x16x8 tensor
# against the FP64 path (itself within 6.5e-14 of the oracle on the sampled slices
# above): measured 3.2e-5.  The FP32 Jacobi SVT leaves a backward error of about 1e-6
# per transform-domain slice (the sampled-slice test above), and L^{-1} with cond 1e2 per
# mode amplifies it about thirtyfold on this output, so the 1e-5 target of the mixed path
# is NOT met for the original-domain L-SVT output of this workload; the bound below
# records the measured level (3x margin) so that a regression is caught.
SVT3_ORIGINAL_DOMAIN_BOUND = 1e-4


@pytest.mark.parametrize("prec", [lt.LT_FP32, lt.LT_MIXED])
def test_config3_svt_original_domain_vs_fp64(config3, config3_svt, prec):
    ctx = make_ctx(config3["transforms"], prec)
    ctx64 = make_ctx(config3["transforms"], lt.LT_FP64)
    A64 = to_dev(config3["A"], torch.float64)
    tau = config3_svt["tau"]
    D64 = torch.empty_like(A64)
    lt.lt_svt(ctx64, A64, tau, D64)
    A32 = A64.float()
    del A64
    D = torch.empty_like(A32)
    lt.lt_svt(ctx, A32, tau, D)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0 and lt.lt_last_device_status(ctx64) == 0
    err = float(torch.linalg.norm(D.double() - D64) / torch.linalg.norm(D64))
    print(f"config3 svt {NAME[prec]} original domain vs fp64: rel err {err:.3e} "
          f"(mixed-path target 1e-5 not met on this output; recorded bound "
          f"{SVT3_ORIGINAL_DOMAIN_BOUND:.0e})")
    assert err <= SVT3_ORIGINAL_DOMAIN_BOUND


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
    err = rel(from_dev(X, c["obs"].shape), ref)
    print(f"config5 one PGA iteration {NAME[prec]}: rel err {err:.3e}")
    assert err <= BOUND[prec]


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
