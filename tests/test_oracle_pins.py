"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed forms derived
from the paper's definitions (tests/golden), a library routine that a special case
reduces to, brute force from a definition, or an identity/theorem the paper proves.
"""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import definitions as D
from oracle import lt_oracle as O
from tests.conftest import load_golden_matrices, rel


def rand(rng, *shape):
    return rng.standard_normal(size=shape)


def rand_invertible(rng, n, cond=10.0):
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.geomspace(1.0, cond, n)
    return (Q1 * d) @ Q2.T


# ---------------------------------------------------------------- transform matrices
def test_dct_matrix_closed_forms_and_scipy():
    g = load_golden_matrices()
    for n in (2, 3):
        assert np.allclose(O.dct_matrix(n), g[("dct", n)], atol=1e-15)
    # Special case that reduces to a library routine: C_n x == DCT-II (orthonormal).
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 5, 8, 32, 33):
        x = rng.standard_normal(n)
        assert np.allclose(O.dct_matrix(n) @ x, scipy.fft.dct(x, type=2, norm="ortho"),
                           atol=1e-14)
        C = O.dct_matrix(n)
        assert np.allclose(C @ C.T, np.eye(n), atol=1e-14)  # "C_n is orthogonal" (Sec. 2)


def test_cproduct_matrix_closed_forms():
    g = load_golden_matrices()
    for n in (2, 3):
        assert np.allclose(O.cproduct_matrix(n), g[("cprod", n)], atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_tph_diagonalisation_eq_d(n):
    """Eq. (d): C tph(a) C^T = diag(d), d = W^{-1} C (I+Z) vec(a)."""
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n)
    T = D.btph(a.reshape(1, 1, n))
    C = O.dct_matrix(n)
    Dm = C @ T @ C.T
    assert np.abs(Dm - np.diag(np.diag(Dm))).max() < 1e-13
    assert np.allclose(np.diag(Dm), O.cproduct_matrix(n) @ a, atol=1e-13)


# ---------------------------------------------------------------- mode products
@pytest.mark.parametrize("shape", [(3, 4, 2), (2, 3, 4, 2), (2, 2, 3, 2, 3)])
def test_mode_product_matricization(shape):
    """Y = X x_n U  <=>  Y_(n) = U X_(n) (Sec. 2), with X_(n) built element by element."""
    rng = np.random.default_rng(len(shape))
    X = rand(rng, *shape)
    for n in range(1, len(shape) + 1):
        U = rand(rng, 5, shape[n - 1])
        Y = O.mode_product(X, U, n)
        assert Y.shape[n - 1] == 5
        assert np.allclose(D.matricize(Y, n), U @ D.matricize(X, n), atol=1e-13)


def test_matricization_third_order_examples():
    """X_(1) = [X^(1), ..., X^(I3)] and X_(2) = [X^(1)T, ..., X^(I3)T] (Sec. 2)."""
    rng = np.random.default_rng(3)
    X = rand(rng, 3, 4, 2)
    assert np.allclose(D.matricize(X, 1), np.hstack([X[:, :, i] for i in range(2)]))
    assert np.allclose(D.matricize(X, 2), np.hstack([X[:, :, i].T for i in range(2)]))


def test_mode_products_commute():
    rng = np.random.default_rng(4)
    X = rand(rng, 2, 3, 4, 5)
    U, V = rand(rng, 4, 4), rand(rng, 5, 5)
    a = O.mode_product(O.mode_product(X, U, 3), V, 4)
    b = O.mode_product(O.mode_product(X, V, 4), U, 3)
    assert np.allclose(a, b, atol=1e-13)


@pytest.mark.parametrize("trailing", [(4,), (3, 2), (2, 3, 2)])
def test_transform_kronecker_brute_force(trailing):
    """vec(L(X)) = (M_K kron ... kron M_3 kron I) vec(X) and the round trip L^{-1}(L(X))."""
    rng = np.random.default_rng(sum(trailing))
    X = rand(rng, 3, 2, *trailing)
    Ms = [rand_invertible(rng, n) for n in trailing]
    Lx = O.transform(X, Ms)
    assert rel(Lx, D.kron_transform(X, Ms)) < 1e-13
    assert rel(O.inverse_transform(Lx, Ms), X) < 1e-12


# ---------------------------------------------------------------- products
@pytest.mark.parametrize("shapes", [((3, 2, 4), (2, 3, 4)), ((2, 3, 3, 2), (3, 2, 3, 2)),
                                    ((2, 2, 2, 3, 2), (2, 1, 2, 3, 2))])
def test_lemma_cproduct_equals_L_product(shapes):
    """Lemma of Sec. 3.1: A *_c B = ten(btph(A) btph(B)) equals L^{-1}(L(A) tri L(B))
    with M = W^{-1} C (I+Z) on every mode; plus btph(A *_c B) = btph(A) btph(B)."""
    rng = np.random.default_rng(7)
    A, B = rand(rng, *shapes[0]), rand(rng, *shapes[1])
    Ms = [O.cproduct_matrix(n) for n in shapes[0][2:]]
    C = O.product(A, B, Ms)
    assert rel(C, D.cproduct_def(A, B)) < 1e-12
    assert rel(D.btph(C), D.btph(A) @ D.btph(B)) < 1e-12
    assert rel(D.ten(D.btph(A), A.shape), A) < 1e-15


def test_dct_product_is_not_the_btph_cproduct():
    """With the orthonormal C instead of M_c the product differs (the reason the two
    transform kinds are kept apart)."""
    rng = np.random.default_rng(8)
    A, B = rand(rng, 3, 2, 4), rand(rng, 2, 3, 4)
    assert rel(O.product(A, B, [O.dct_matrix(4)]), D.cproduct_def(A, B)) > 1e-3


def test_slice_order_eq_3_5():
    """Representative matrices X^p with p = k3 + I3 k4 + I3 I4 k5 (Eq. 3.5, mode 3
    fastest), and the slices' round trip."""
    rng = np.random.default_rng(5)
    X = rand(rng, 2, 3, 3, 2, 2)
    S = O.slices(X)
    for k5 in range(2):
        for k4 in range(2):
            for k3 in range(3):
                assert np.array_equal(S[:, :, k3 + 3 * k4 + 6 * k5], X[:, :, k3, k4, k5])
    assert np.array_equal(O.from_slices(S, X.shape[2:]), X)


def test_facewise_product_brute_force():
    """(A tri B)^p = A^p B^p computed entry by entry from Eq. 3.5's slice order."""
    rng = np.random.default_rng(9)
    A, B = rand(rng, 3, 4, 2, 3), rand(rng, 4, 2, 2, 3)
    C = O.facewise(A, B)
    for k4 in range(3):
        for k3 in range(2):
            for i in range(3):
                for j in range(2):
                    s = sum(A[i, l, k3, k4] * B[l, j, k3, k4] for l in range(4))
                    assert abs(C[i, j, k3, k4] - s) < 1e-13


@pytest.mark.parametrize("kind", ["dct", "general"])
def test_ring_laws_identity_transpose(kind):
    rng = np.random.default_rng(10)
    trailing = (3, 4)
    Ms = ([O.dct_matrix(n) for n in trailing] if kind == "dct"
          else [rand_invertible(rng, n) for n in trailing])
    A, B, C = rand(rng, 3, 4, *trailing), rand(rng, 4, 2, *trailing), rand(rng, 2, 5, *trailing)
    # identity (Sec. 3.2): A * I = I * A = A
    assert rel(O.product(A, O.identity(4, trailing, Ms), Ms), A) < 1e-12
    assert rel(O.product(O.identity(3, trailing, Ms), A, Ms), A) < 1e-12
    # associativity and distributivity (ring theorem of Sec. 3.2)
    assert rel(O.product(O.product(A, B, Ms), C, Ms), O.product(A, O.product(B, C, Ms), Ms)) < 1e-12
    B2 = rand(rng, 4, 2, *trailing)
    assert rel(O.product(A, B + B2, Ms), O.product(A, B, Ms) + O.product(A, B2, Ms)) < 1e-12
    # commutativity of scalar-tensors
    a, b = rand(rng, 1, 1, *trailing), rand(rng, 1, 1, *trailing)
    assert rel(O.product(a, b, Ms), O.product(b, a, Ms)) < 1e-12
    # transpose reversal (A * B)^T = B^T * A^T
    lhs = O.transpose(O.product(A, B, Ms), Ms)
    rhs = O.product(O.transpose(B, Ms), O.transpose(A, Ms), Ms)
    assert rel(lhs, rhs) < 1e-12
    # for transforms on modes >= 3 the transpose is the swap of modes 1 and 2
    assert rel(O.transpose(A, Ms), np.swapaxes(A, 0, 1)) < 1e-12


def test_scalar_tensor_expansion_and_column_split():
    """Propositions of Sec. 3.2: (X * Y)_{ij} = sum_k X_{ik} * Y_{kj} (scalar-tensors),
    and A * B = [A * B_1, ..., A * B_{I2}]."""
    rng = np.random.default_rng(11)
    trailing = (3, 2)
    Ms = [rand_invertible(rng, n) for n in trailing]
    X, Y = rand(rng, 2, 3, *trailing), rand(rng, 3, 2, *trailing)
    XY = O.product(X, Y, Ms)
    for i in range(2):
        for j in range(2):
            acc = sum(O.product(X[i:i + 1, k:k + 1], Y[k:k + 1, j:j + 1], Ms) for k in range(3))
            assert rel(XY[i:i + 1, j:j + 1], acc) < 1e-12
    cols = np.concatenate([O.product(X, Y[:, j:j + 1], Ms) for j in range(2)], axis=1)
    assert rel(XY, cols) < 1e-12


# ---------------------------------------------------------------- SVD / SVT
@pytest.mark.parametrize("kind,shape", [("dct", (7, 5, 4)), ("dct", (4, 6, 3, 2)),
                                        ("general", (6, 6, 2, 3))])
def test_svd_invariants(kind, shape):
    """Theorem of Eq. tsvd1: A = U * S * V^T with U, V orthogonal (every L(U)^p, L(V)^p
    orthogonal), S f-diagonal; sigma >= 0 descending; for orthonormal L, ||A|| = ||S||
    and ||S_1|| >= ||S_2|| >= ... (Corollary of Sec. 3.2)."""
    rng = np.random.default_rng(12)
    A = rand(rng, *shape)
    trailing = shape[2:]
    Ms = ([O.dct_matrix(n) for n in trailing] if kind == "dct"
          else [rand_invertible(rng, n) for n in trailing])
    U, S, V, sig = O.svd(A, Ms)
    rec = O.product(O.product(U, S, Ms), O.transpose(V, Ms), Ms)
    assert rel(rec, A) < 1e-12
    Uh, Sh, Vh = (O.slices(O.transform(T, Ms)) for T in (U, S, V))
    for p in range(Uh.shape[2]):
        assert np.allclose(Uh[:, :, p].T @ Uh[:, :, p], np.eye(shape[0]), atol=1e-12)
        assert np.allclose(Vh[:, :, p].T @ Vh[:, :, p], np.eye(shape[1]), atol=1e-12)
        off = Sh[:, :, p].copy()
        np.fill_diagonal(off, 0.0)
        assert np.abs(off).max() < 1e-12
        s = np.diag(Sh[:, :, p])
        assert np.all(s >= -1e-13) and np.all(np.diff(s) <= 1e-13)
        # sigma equals the singular values of L(A)^p (brute: eigenvalues of the Gram)
        ev = np.sqrt(np.maximum(np.linalg.eigvalsh(
            O.slices(O.transform(A, Ms))[:, :, p].T @ O.slices(O.transform(A, Ms))[:, :, p]), 0))
        assert np.allclose(np.sort(ev)[::-1][: len(s)], s, atol=1e-10)
    # Q * Q^T = I (orthogonal tensor definition)
    I1 = shape[0]
    assert rel(O.product(U, O.transpose(U, Ms), Ms), O.identity(I1, trailing, Ms)) < 1e-12
    if kind == "dct":
        assert abs(np.linalg.norm(A) - np.linalg.norm(S)) < 1e-12 * np.linalg.norm(A)
        r = min(shape[:2])
        norms = [np.linalg.norm(S[i, i]) for i in range(r)]
        assert all(norms[i] >= norms[i + 1] - 1e-12 for i in range(r - 1))
        assert abs(sum(x * x for x in norms) - np.linalg.norm(A) ** 2) < 1e-10


def test_eckart_young_dct():
    """Eckart-Young theorem of Sec. 3.2: ||A - A_k||^2 = sum_{i>k} ||S_i||^2 (orthonormal
    L), and A_k beats other rank-k products."""
    rng = np.random.default_rng(13)
    trailing = (3, 2)
    Ms = [O.dct_matrix(n) for n in trailing]
    A = rand(rng, 6, 5, *trailing)
    U, S, V, _ = O.svd(A, Ms)
    for k in range(1, 5):
        Ak = O.product(O.product(U[:, :k], S[:k, :k], Ms), O.transpose(V[:, :k], Ms), Ms)
        err2 = np.linalg.norm(A - Ak) ** 2
        tail = sum(np.linalg.norm(S[i, i]) ** 2 for i in range(k, 5))
        assert abs(err2 - tail) < 1e-10 * np.linalg.norm(A) ** 2
        X, Y = rand(rng, 6, k, *trailing), rand(rng, k, 5, *trailing)
        assert np.linalg.norm(A - O.product(X, Y, Ms)) ** 2 >= err2 - 1e-10


def test_truncate_is_the_eckart_young_product():
    """O.truncate(A, k) equals the theorem's U(:,1:k) *_L S(1:k,1:k) *_L V(:,1:k)^T built
    with *_L-products from the full *_L-SVD (a different route: products and
    transposes of the SVD factors in the original domain), for DCT and a general
    invertible L; k = 0 gives zero, k >= min(I1, I2) gives A; and for I3 = 1 with the
    identity transform it is LAPACK's matrix rank-k truncation."""
    rng = np.random.default_rng(21)
    trailing = (3, 2)
    for Ms in ([O.dct_matrix(n) for n in trailing],
               [rng.standard_normal((n, n)) + 3 * np.eye(n) for n in trailing]):
        A = rand(rng, 6, 5, *trailing)
        U, S, V, _ = O.svd(A, Ms)
        for k in (1, 2, 4):
            Ak = O.product(O.product(U[:, :k], S[:k, :k], Ms), O.transpose(V[:, :k], Ms), Ms)
            assert np.linalg.norm(O.truncate(A, k, Ms) - Ak) <= 1e-11 * np.linalg.norm(A)
        assert np.linalg.norm(O.truncate(A, 0, Ms)) == 0.0
        assert np.linalg.norm(O.truncate(A, 7, Ms) - A) <= 1e-12 * np.linalg.norm(A)
    M = rng.standard_normal((7, 5))
    u, s, vt = np.linalg.svd(M, full_matrices=False)
    got = O.truncate(M[:, :, None], 2, [np.eye(1)])[:, :, 0]
    assert np.linalg.norm(got - (u[:, :2] * s[:2]) @ vt[:2]) <= 1e-13 * np.linalg.norm(M)


def test_ranks_and_norms_on_prescribed_ranks():
    """Tensors built in the transform domain with prescribed slice ranks r_p
    (L(A)^p = X_p Y_p, X_p I1 x r_p, Y_p r_p x I2): the multirank is r, the average
    rank mean(r), the tubal rank max(r) (Lemma of the tubal rank); with I3 = 1 and the
    identity transform the spectral and nuclear norms are LAPACK's matrix 2-norm and
    nuclear norm."""
    rng = np.random.default_rng(22)
    trailing = (3, 2)
    for Ms in ([O.dct_matrix(n) for n in trailing],
               [rng.standard_normal((n, n)) + 3 * np.eye(n) for n in trailing]):
        r = [2, 0, 5, 1, 3, 4]
        Ah = np.zeros((8, 6, 6))
        for p, rp in enumerate(r):
            Ah[:, :, p] = rng.standard_normal((8, rp)) @ rng.standard_normal((rp, 6))
        A = O.inverse_transform(O.from_slices(Ah, trailing), Ms)
        out = O.ranks_and_norms(A, Ms)
        assert list(out["multirank"]) == r
        assert out["tubal"] == 5 and out["average"] == sum(r) / 6
        sig = [np.linalg.svd(Ah[:, :, p], compute_uv=False) for p in range(6)]
        assert abs(out["spectral"] - max(x[0] for x in sig)) <= 1e-9 * out["spectral"]
    M = rng.standard_normal((7, 5))
    out = O.ranks_and_norms(M[:, :, None], [np.eye(1)])
    assert abs(out["spectral"] - np.linalg.norm(M, 2)) <= 1e-13 * np.linalg.norm(M, 2)
    assert abs(out["nuclear"] - np.linalg.norm(M, "nuc")) <= 1e-13 * np.linalg.norm(M, "nuc")
    assert out["tubal"] == 5 and list(out["multirank"]) == [5]


def test_svt_special_cases():
    rng = np.random.default_rng(14)
    trailing = (4,)
    Ms = [rand_invertible(rng, 4)]
    A = rand(rng, 5, 3, *trailing)
    assert rel(O.svt(A, 0.0, Ms), A) < 1e-12            # tau = 0 gives A back
    _, sig = O.svt(A, 0.0, Ms, return_sigma=True)
    assert np.abs(O.svt(A, float(sig.max()) * 1.0001, Ms)).max() < 1e-13  # tau >= sigma_max
    # I3 = 1 with M = [1]: the matrix SVT of Cai, Candes & Shen (via LAPACK)
    M = rand(rng, 6, 4)
    u, s, vt = np.linalg.svd(M, full_matrices=False)
    ref = (u * np.maximum(s - 0.7, 0)) @ vt
    assert rel(O.svt(M.reshape(6, 4, 1), 0.7, [np.eye(1)])[:, :, 0], ref) < 1e-13
    # scaled identity transform alpha * I leaves the product structure but scales sigma
    out = O.svt(M.reshape(6, 4, 1), 0.7, [np.array([[2.0]])])[:, :, 0]
    ref2 = (u * np.maximum(2 * s - 0.7, 0) / 2.0) @ vt
    assert rel(out, ref2) < 1e-13


def test_svt_is_the_prox_of_the_nuclear_norm():
    """Theorem 23 (orthonormal L): D_tau(A) minimises tau ||Y||_* + 1/2 ||Y - A||^2.
    Checked against random perturbations and by the subgradient condition in each
    transform-domain slice: A_hat - D_hat = tau (U1 V1^T + W) with ||W|| <= 1."""
    rng = np.random.default_rng(15)
    trailing = (3, 2)
    Ms = [O.dct_matrix(n) for n in trailing]
    A = rand(rng, 5, 4, *trailing)
    tau = 0.8
    Dt = O.svt(A, tau, Ms)

    def F(Y):
        return tau * O.nuclear_norm(Y, Ms) + 0.5 * np.linalg.norm(Y - A) ** 2

    f0 = F(Dt)
    for _ in range(200):
        P = rand(rng, *A.shape) * 10 ** rng.uniform(-4, 0)
        assert F(Dt + P) >= f0 - 1e-12
    Ah, Dh = O.slices(O.transform(A, Ms)), O.slices(O.transform(Dt, Ms))
    for p in range(Ah.shape[2]):
        Gp = (Ah[:, :, p] - Dh[:, :, p]) / tau
        assert np.linalg.norm(Gp, 2) <= 1 + 1e-10


# ---------------------------------------------------------------- PGA (Algorithm 5)
def small_completion(seed=16, I1=8, I2=7, trailing=(3, 4), rank=2, rho=0.5):
    rng = np.random.default_rng(seed)
    Ms = [O.dct_matrix(n) for n in trailing]
    U, V = rand(rng, I1, rank, *trailing), rand(rng, I2, rank, *trailing)
    X = O.product(U, O.transpose(V, Ms), Ms)
    mask = (rng.random(X.shape) < rho).astype(np.uint8)
    obs = mask * X
    return X, mask, obs, Ms


def test_pga_full_observation_reduces_to_one_svt():
    """Omega = everything and step = 1: G^k = M for every k (Eq. 51), so every iterate
    is D_tau(M) (Eq. 53) whatever the momentum."""
    X, mask, obs, Ms = small_completion()
    ones = np.ones_like(mask)
    Xk, info = O.pga(ones, X, 0.3, 1.0, 5, Ms)
    assert rel(Xk, O.svt(X, 0.3, Ms)) < 1e-13
    assert info["iters"] == 5


def test_pga_first_iterates_and_momentum_schedule():
    """With t_0 = t_1 = 1 the first two momentum weights vanish, so X^2 = D(P(M)) and
    X^3 = D(X^2 - P(X^2 - M)); the third weight is (t_2 - 1)/t_3 with t_2 the golden
    ratio (FISTA schedule t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2)."""
    X, mask, obs, Ms = small_completion()
    tau = 0.2
    m = mask.astype(float)
    x2 = O.svt(m * obs, tau, Ms)
    x3 = O.svt(x2 - m * (x2 - obs), tau, Ms)
    got2, _ = O.pga(mask, obs, tau, 1.0, 1, Ms)
    got3, info = O.pga(mask, obs, tau, 1.0, 2, Ms)
    assert rel(got2, x2) < 1e-14 and rel(got3, x3) < 1e-14
    phi = (1 + math.sqrt(5)) / 2
    assert abs(info["t"] - (1 + math.sqrt(1 + 4 * phi * phi)) / 2) < 1e-15
    y4 = x3 + (phi - 1) / info["t"] * (x3 - x2)
    got4, _ = O.pga(mask, obs, tau, 1.0, 3, Ms)
    assert rel(got4, O.svt(y4 - m * (y4 - obs), tau, Ms)) < 1e-13


def test_pga_ista_monotone_and_limit_is_optimal():
    """Without momentum the objective F = tau||X||_* + 1/2||P(X - M)||^2 never increases
    (proximal gradient with step 1 = 1/l_f, Sec. 4), FISTA converges to the same
    minimiser, and the limit beats random perturbations (convex optimality)."""
    X, mask, obs, Ms = small_completion(rho=0.6)
    tau = 0.05
    _, info = O.pga(mask, obs, tau, 1.0, 60, Ms, momentum=False, objective=True)
    f = info["objective"]
    assert all(f[i + 1] <= f[i] + 1e-12 for i in range(len(f) - 1))
    Xf, infof = O.pga(mask, obs, tau, 1.0, 400, Ms, objective=True)
    Fstar = infof["objective"][-1]
    rng = np.random.default_rng(0)
    for _ in range(100):
        P = rng.standard_normal(X.shape) * 10 ** rng.uniform(-4, -1)
        assert O.pga_objective(Xf + P, mask, obs, tau, Ms) >= Fstar - 1e-9
    # Beck-Teboulle rate for FISTA: F(X^k) - F* <= 2 ||X^0 - X*||^2 / (k+1)^2
    for k, fk in enumerate(infof["objective"][:100], start=1):
        assert fk - Fstar <= 2 * np.linalg.norm(Xf) ** 2 / (k + 1) ** 2 + 1e-9


def test_pga_continuation_schedule_and_limit():
    """Continuation of Algorithm 5 (mu_{k+1} = max(nu mu_k, mu_bar), mu_bar = tau):
    mu_0 <= tau is the fixed-tau run; nu = 1 is the fixed run at mu_0; the first iterate
    is D_{step mu_0}(step P_Omega(M)) (X^0 = 0); and the limit is a minimiser of the
    tau problem: its objective beats random perturbations and equals the fixed-tau
    limit's or lies below it (continuation reaches the optimum faster; convex
    optimality)."""
    X, mask, obs, Ms = small_completion(rho=0.6)
    tau = 0.05
    a, _ = O.pga(mask, obs, tau, 1.0, 12, Ms)
    b, _ = O.pga(mask, obs, tau, 1.0, 12, Ms, mu0=tau, nu=0.5)
    assert np.array_equal(a, b)
    c, _ = O.pga(mask, obs, 2.0, 1.0, 12, Ms)
    d, _ = O.pga(mask, obs, tau, 1.0, 12, Ms, mu0=2.0, nu=1.0)
    assert np.array_equal(c, d)
    x1, _ = O.pga(mask, obs, tau, 0.8, 1, Ms, mu0=3.0, nu=0.7)
    m = mask.astype(float)
    assert np.linalg.norm(x1 - O.svt(0.8 * m * obs, 0.8 * 3.0, Ms)) <= 1e-13 * np.linalg.norm(x1)
    mu0 = 0.9 * float(np.linalg.norm(m * obs))     # the paper's choice nu ||M||_F
    Xc, infoc = O.pga(mask, obs, tau, 1.0, 400, Ms, mu0=mu0, nu=0.9, objective=True)
    Xf, infof = O.pga(mask, obs, tau, 1.0, 400, Ms, objective=True)
    Fc = infoc["objective"][-1]
    assert Fc <= infof["objective"][-1] + 1e-9 * abs(Fc)
    assert infof["objective"][-1] - Fc <= 1e-5 * abs(Fc)
    assert infoc["objective"][0] > infof["objective"][0]   # early iterates over-shrink
    rng = np.random.default_rng(1)
    for _ in range(100):
        P = rng.standard_normal(X.shape) * 10 ** rng.uniform(-4, -1)
        assert O.pga_objective(Xc + P, mask, obs, tau, Ms) >= Fc - 1e-9


def test_pga_tolerance_stop_and_recovery():
    X, mask, obs, Ms = small_completion(I1=12, I2=10, rank=1, rho=0.7)
    Xk, info = O.pga(mask, obs, 0.01, 1.0, 500, Ms, tol=1e-6)
    assert info["iters"] < 500 and info["residual"][-1] <= 1e-6
    assert O.rse(X, Xk) < 0.05


# ---------------------------------------------------------------- Fourier (t-product)
def bcirc_product(A, B):
    """The t-product from its circulant definition (Kilmer and Martin), no transform:
    C = fold(bcirc(A) unfold(B)), i.e. C_k = sum_j A_{(k - j) mod n} B_j on the frontal
    slices."""
    n = A.shape[2]
    C = np.zeros((A.shape[0], B.shape[1], n))
    for k in range(n):
        for j in range(n):
            C[:, :, k] += A[:, :, (k - j) % n] @ B[:, :, j]
    return C


def tnn_fourier(Y, Ms_rest=()):
    """sum over the transform-domain slices of L(Y) = fft along mode 3 (numpy's FFT),
    then the real M_4, ..., of their nuclear norms (numpy's SVD)."""
    Yh = np.fft.fft(Y, axis=2)
    for k, M in enumerate(Ms_rest, start=3):
        Yh = np.moveaxis(np.tensordot(M, Yh, axes=(1, k)), 0, k)
    S = Yh.reshape(Y.shape[0], Y.shape[1], -1, order="F")
    return float(sum(np.linalg.svd(S[:, :, p], compute_uv=False).sum()
                     for p in range(S.shape[2])))


def test_fourier_matrix_is_numpy_fft_and_scaled_unitary():
    for n in (1, 2, 3, 4, 7):
        F = O.fourier_matrix(n)
        assert np.allclose(F, np.fft.fft(np.eye(n), axis=0), atol=1e-13)
        assert np.allclose(F @ F.conj().T, n * np.eye(n), atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_tproduct_is_the_block_circulant_product(n):
    """Third order: A *_L B with M_3 = F (Sec. 2) is the t-product fold(bcirc(A)
    unfold(B)); n = 1 is the matrix product."""
    rng = np.random.default_rng(40 + n)
    A, B = rand(rng, 4, 3, n), rand(rng, 3, 5, n)
    C = O.tproduct(A, B)
    assert rel(C, bcirc_product(A, B)) < 1e-13
    if n == 1:
        assert rel(C[:, :, 0], A[:, :, 0] @ B[:, :, 0]) < 1e-14


def test_tproduct_fourth_order_splits_along_mode_4():
    """With a real invertible M_4 the product is, for each mode-4 index of the
    M_4-transformed operands, the third-order t-product, then M_4^{-1} (the mode
    products on different modes commute)."""
    rng = np.random.default_rng(44)
    M4 = rand_invertible(rng, 3)
    A, B = rand(rng, 4, 3, 5, 3), rand(rng, 3, 2, 5, 3)
    At, Bt = O.mode_product(A, M4, 4), O.mode_product(B, M4, 4)
    Ct = np.stack([bcirc_product(At[..., j], Bt[..., j]) for j in range(3)], axis=3)
    assert rel(O.tproduct(A, B, [M4]), O.mode_product(Ct, np.linalg.inv(M4), 4)) < 1e-12


def test_tsvt_special_cases():
    """n = 1: the matrix SVT.  Equal frontal slices A_0: F(A) has the one nonzero slice
    n A_0, whose SVT at tau is n D_{tau/n}(A_0), so every frontal slice of the result is
    D_{tau/n}(A_0).  tau = 0 returns A; tau above every singular value returns 0."""
    rng = np.random.default_rng(45)
    A0 = rand(rng, 6, 4)

    def msvt(M, t):
        u, s, vt = np.linalg.svd(M, full_matrices=False)
        return (u * np.maximum(s - t, 0)) @ vt

    assert rel(O.tsvt(A0[:, :, None], 0.7)[:, :, 0], msvt(A0, 0.7)) < 1e-13
    n = 5
    A = np.repeat(A0[:, :, None], n, axis=2)
    D = O.tsvt(A, 2.0)
    for k in range(n):
        assert rel(D[:, :, k], msvt(A0, 2.0 / n)) < 1e-12
    X = rand(rng, 5, 4, 3, 2)
    Ms = [O.dct_matrix(2)]
    assert rel(O.tsvt(X, 0.0, Ms), X) < 1e-13
    assert np.abs(O.tsvt(X, 1e6, Ms)).max() == 0.0


@pytest.mark.parametrize("trailing", [(4,), (3, 2)])
def test_tsvt_is_the_prox_of_the_fourier_nuclear_norm(trailing):
    """With M_3 = F (M_3 M_3^* = n I) and orthonormal M_4, ||Y||_F^2 = ||L(Y)||_F^2 / n,
    so thresholding the slices of L(A) at tau minimises (tau / n) sum_p ||L(Y)^p||_* +
    1/2 ||Y - A||_F^2 over real Y (the unconstrained minimiser is conjugate-symmetric
    along mode 3, hence real).  Checked against random real perturbations, with the
    nuclear norm taken from numpy's FFT and SVD."""
    rng = np.random.default_rng(46)
    Ms = [O.dct_matrix(n) for n in trailing[1:]]
    A = rand(rng, 5, 4, *trailing)
    tau, n = 1.1, trailing[0]
    Dt = O.tsvt(A, tau, Ms)

    def F(Y):
        return tau / n * tnn_fourier(Y, Ms) + 0.5 * np.linalg.norm(Y - A) ** 2

    f0 = F(Dt)
    assert f0 < F(A) and f0 < F(np.zeros_like(A))
    for _ in range(150):
        P = rand(rng, *A.shape) * 10 ** rng.uniform(-4, 0)
        assert F(Dt + P) >= f0 - 1e-12


def test_pga_fourier_full_observation_and_limit():
    """TNN-PGA-F: Omega = everything with step 1 gives tsvt(M) at every iterate; on a
    partial mask the limit minimises 1/2 ||P(X - M)||^2 + (tau / n) sum_p ||F(X)^p||_*
    (the step's threshold step tau is the prox of step (tau / n) TNN_F, by the pin
    above)."""
    rng = np.random.default_rng(47)
    n = 3
    U, V = rand(rng, 8, 2, n, 4), rand(rng, 7, 2, n, 4)
    Ms = [O.dct_matrix(4)]
    X = O.tproduct(U, np.transpose(V, (1, 0, 2, 3)), Ms)
    Xk, _ = O.pga(np.ones(X.shape, np.uint8), X, 0.3, 1.0, 4, Ms, fourier=True)
    assert rel(Xk, O.tsvt(X, 0.3, Ms)) < 1e-13
    mask = (rng.random(X.shape) < 0.6).astype(np.uint8)
    obs = mask * X
    tau = 0.05
    Xf, _ = O.pga(mask, obs, tau, 1.0, 500, Ms, fourier=True)

    def F(Y):
        return 0.5 * float(np.sum((mask * (Y - obs)) ** 2)) + tau / n * tnn_fourier(Y, Ms)

    f0 = F(Xf)
    for _ in range(100):
        P = rand(rng, *X.shape) * 10 ** rng.uniform(-4, -1)
        assert F(Xf + P) >= f0 - 1e-9
    with pytest.raises(ValueError):
        O.pga(mask, obs, tau, 1.0, 2, Ms, fourier=True, objective=True)
