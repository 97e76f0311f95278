"""Parity of the cluster form of the SVT kernel (LT_OPT_JACOBI_CLUSTER: one slice on a
thread-block cluster of 3 or 4 CTAs, columns spread over their shared memory) with the
FP64 oracle, and its agreement with the one-CTA form.

Tolerances as for the one-CTA kernel: 1e-12 (FP64) and 1e-5 (FP32) relative Frobenius
error.  The cluster form orders the same rotations differently across CTAs, so it is
not bitwise equal to the one-CTA form; it is deterministic (fixed pairing and
reduction order), which the bitwise checks against itself test.
"""
import numpy as np
import pytest
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt, synth
from tests.gpu_util import dtype_of, empty_dev, from_dev, make_ctx, oracle_mats, rel, to_dev

pytestmark = pytest.mark.gpu

TOL = {lt.LT_FP64: 1e-12, lt.LT_FP32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2202_02870_gb300 import build
    build.build()
    torch.cuda.init()


# (I1, I2, transforms): ragged and padded column counts, both orientations, the
# benchmark's slices, and 288 columns (the largest the cluster form holds)
SHAPES = [(8, 6, [("dct", 3)]), (30, 50, [("dct", 2)]), (50, 30, [("dct", 3)]),
          (97, 61, [("dct", 2)]), (144, 176, [("dct", 3), ("dct", 4)]),
          (176, 144, [("dct", 3)]), (200, 190, [("dct", 2)])]


def run_svt(A, tau, transforms, prec, cluster, D=None):
    ctx = make_ctx(transforms, prec)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_CLUSTER, cluster)
    dt = dtype_of(prec)
    Dd = empty_dev(A.shape, dt)
    lt.lt_svt(ctx, to_dev(A, dt), tau, Dd)
    torch.cuda.synchronize()
    assert lt.lt_last_device_status(ctx) == 0
    return Dd


@pytest.mark.parametrize("prec", [lt.LT_FP64, lt.LT_FP32])
@pytest.mark.parametrize("cluster", [3, 4])
@pytest.mark.parametrize("I1,I2,transforms", SHAPES)
def test_cluster_svt_vs_oracle(prec, cluster, I1, I2, transforms):
    rng = np.random.default_rng(I1 * 3 + I2)
    sizes = tuple(t[1] for t in transforms)
    A = rng.standard_normal((I1, I2) + sizes)
    Ms = oracle_mats(transforms)
    s = np.linalg.svd(O.slices(O.transform(A, Ms))[:, :, 0], compute_uv=False)
    tau = float(s[len(s) // 3])  # shrinks about two thirds of the spectrum away
    D = run_svt(A, tau, transforms, prec, cluster)
    ref = O.svt(A, tau, Ms)
    assert rel(from_dev(D, A.shape), ref) <= TOL[prec]
    D1 = run_svt(A, tau, transforms, prec, 1)
    assert rel(from_dev(D, A.shape), from_dev(D1, A.shape)) <= TOL[prec]
    D2 = run_svt(A, tau, transforms, prec, cluster)
    assert torch.equal(D, D2)


def test_cluster_svt_288_columns_and_limits():
    """288 x 352 slices (FP64): four CTAs hold the working matrix; three cannot (their
    share exceeds a CTA's shared memory) and the forced form is refused."""
    rng = np.random.default_rng(288)
    A = rng.standard_normal((288, 352, 2))
    tr = [("dct", 2)]
    D = run_svt(A, 20.0, tr, lt.LT_FP64, 4)
    assert rel(from_dev(D, A.shape), O.svt(A, 20.0, oracle_mats(tr))) <= 1e-12
    ctx = make_ctx(tr, lt.LT_FP64)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_CLUSTER, 3)
    with pytest.raises(lt.LtError):
        lt.lt_svt(ctx, to_dev(A), 20.0, empty_dev(A.shape))
    with pytest.raises(lt.LtError):
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_CLUSTER, 2)


def test_cluster_svt_edge_cases():
    """tau = 0 returns A; tau above every singular value returns zeros; a zero slice and
    a rank-one slice."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 33, 3))
    A[:, :, 1] = 0.0
    A[:, :, 2] = np.outer(rng.standard_normal(40), rng.standard_normal(33))
    tr = [("matrix", np.eye(3))]
    D = run_svt(A, 0.0, tr, lt.LT_FP64, 3)
    assert rel(from_dev(D, A.shape), A) <= 1e-12
    D = run_svt(A, 1e6, tr, lt.LT_FP64, 4)
    assert np.abs(from_dev(D, A.shape)).max() == 0.0
    D = run_svt(A, 0.5, tr, lt.LT_FP64, 4)
    assert rel(from_dev(D, A.shape), O.svt(A, 0.5, [np.eye(3)])) <= 1e-12


@pytest.mark.parametrize("cluster", [3, 4])
def test_cluster_pga_vs_oracle(cluster):
    c = synth.completion_case(41, 40, 36, (3, 4), rank=3, rho=0.4)
    tr = [("dct", 3), ("dct", 4)]
    Ms = oracle_mats(tr)
    X0 = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    obs = c["mask"] * (X0 + c["noise"])
    ref, _ = O.pga(c["mask"], obs, 0.3, 1.0, 20, Ms)
    ctx = make_ctx(tr, lt.LT_FP64)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_CLUSTER, cluster)
    X = torch.zeros(tuple(reversed(obs.shape)), dtype=torch.float64, device="cuda")
    rep = lt.lt_pga_report()
    lt.lt_pga_complete(ctx, to_dev(c["mask"]), to_dev(obs), 0.3, 1.0, 20, X, report=rep)
    torch.cuda.synchronize()
    assert rep.iters_done == 20 and rep.device_status == 0
    assert rel(from_dev(X, obs.shape), ref) <= 1e-12


def test_cluster_auto_choice():
    """The planner's choice (LT_OPT_JACOBI_CLUSTER = 0) on FP64 144 x 176 slices, bit for
    bit: 12 slices go to clusters of 4 (48 CTAs instead of 12 on 152 SMs), the 96 of the
    benchmark to clusters of 3 (288 CTAs, two per SM)."""
    rng = np.random.default_rng(96)
    for I4, form in ((4, 4), (32, 3)):
        A = rng.standard_normal((144, 176, 3, I4))
        tr = [("dct", 3), ("dct", I4)]
        Da = run_svt(A, 5.0, tr, lt.LT_FP64, 0)
        Df = run_svt(A, 5.0, tr, lt.LT_FP64, form)
        assert torch.equal(Da, Df)
        assert rel(from_dev(Da, A.shape), O.svt(A, 5.0, oracle_mats(tr))) <= 1e-12
