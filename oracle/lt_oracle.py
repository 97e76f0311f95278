"""Plain FP64 CPU oracle for the generalized *_L-product and *_L-SVT tensor completion.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the package entry
point and the CPU-baseline leg of the benchmark may import or run this module.  It
shares no code, table or helper with the CUDA library and imports nothing from it.

Every function states the passage of the paper (Bentbib, Elalj, El Hachimi, Jbilou,
Ratnani, "Generalized L-product for high order tensors with applications using GPU
computations", arXiv 2202.02870) that it writes out.  All arithmetic is float64.
Library primitives serve as single steps only: `np.tensordot` for the sum that defines
an n-mode product, `np.linalg.inv` for M^{-1}, `np.linalg.svd` (LAPACK) for the
per-slice SVD that the paper's algorithms call.

Conventions
-----------
* A K-th order tensor is a float64 array of shape (I1, I2, I3, ..., IK), indexed
  naturally; memory order is irrelevant here.
* Mode numbers are 1-based, as in the paper.
* `Ms` is the list [M_3, M_4, ..., M_K] of square transform matrices (Sec. 3.2).
* The p-th representative matrix (Eq. 3.5) of X is X[:, :, k3, k4, ..., kK] with
  p = k3 + I3*k4 + I3*I4*k5 + ... (0-based, mode 3 varying fastest).  The printed
  index formula of Eq. 3.5 is garbled; this is the column-major reading.

Readings of the paper taken here (the paper is ambiguous or garbled at these points):
* DCT matrix (Sec. 2, matrix C below Eq. (m)): the normalisation uses delta_{i,1}, which
  gives the orthonormal DCT-II; the printed delta_{i,j} is not orthogonal.
* Z in Eq. (m) is the plain superdiagonal of ones, exactly as its formula says.
* PGA (Algorithm 5): t_0 = t_1 = 1 (the printed 0 gives 0/0); the momentum weight is
  (t_{k-1} - 1)/t_k (Eq. 52); G = Y - step * P_Omega(Y - M) (Eq. 51, first form; the
  second printed form has a sign typo); X^{k+1} = D_{step*tau}(G) (Eq. 53 with the
  gradient step l_f^{-1} = step, l_f = 1 in the paper); the threshold is applied
  unscaled in the transform domain as Algorithm 4 does; the stopping quantity is
  ||Y^k - X^{k+1}||_F / ||X^{k+1}||_F (Sec. 5), taken as ||Y^k||_F when X^{k+1} = 0.
* Fourier operator (Sec. 2, t-product; Sec. 5, fft along mode 3): M_3 = F_{I3}
  unnormalised and complex, M_4, ..., M_K real; the SVT thresholds the complex slices
  of L(A) at tau as Algorithm 4 does, and L^{-1} keeps the real part.  The norm relation
  printed after the definition of L reads M_i M_i^* = alpha_i I (F: alpha = n).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "dct_matrix", "cproduct_matrix", "mode_product", "transform", "inverse_transform",
    "slices", "from_slices", "facewise", "product", "identity", "transpose",
    "svd", "svt", "truncate", "ranks_and_norms", "nuclear_norm", "fourier_matrix",
    "fourier_transform", "fourier_inverse", "tproduct", "tsvt", "pga", "pga_objective",
    "psnr", "rse",
]


# ----------------------------------------------------------------------------------
# Transform matrices
# ----------------------------------------------------------------------------------
def dct_matrix(n: int) -> np.ndarray:
    """DCT-II matrix C_n of Sec. 2 (the matrix used in Eq. (m) and, as "M_i = C_i",
    in the experiments of Sec. 5):

        (C_n)_{i,j} = sqrt((2 - delta_{i,1}) / n) * cos((i-1)(2j-1) pi / (2n)),
        1 <= i, j <= n.
    """
    C = np.empty((n, n), dtype=np.float64)
    for i in range(1, n + 1):
        scale = math.sqrt((2.0 - (1.0 if i == 1 else 0.0)) / n)
        for j in range(1, n + 1):
            C[i - 1, j - 1] = scale * math.cos((i - 1) * (2 * j - 1) * math.pi / (2 * n))
    return C


def cproduct_matrix(n: int) -> np.ndarray:
    """c-product transform M = W^{-1} C (I + Z) of Eq. (m), Sec. 2, with
    W = diag(C(:, 1)) and Z = diag(ones(n-1, 1), 1)."""
    C = dct_matrix(n)
    W = np.diag(C[:, 0])
    Z = np.diag(np.ones(n - 1), 1)
    return np.linalg.inv(W) @ C @ (np.eye(n) + Z)


# ----------------------------------------------------------------------------------
# n-mode product and the operator L (Def. 5, Sec. 3.1 definition of L, Sec. 3.2)
# ----------------------------------------------------------------------------------
def mode_product(X: np.ndarray, U: np.ndarray, n: int) -> np.ndarray:
    """n-mode product X x_n U of Eq. (3), Sec. 2:

        (X x_n U)_{i_1..i_{n-1}, j, i_{n+1}..i_K} = sum_{i_n} X_{i_1..i_K} U_{j, i_n}.
    """
    Y = np.tensordot(U, X, axes=([1], [n - 1]))  # axis 0 of Y is j
    return np.moveaxis(Y, 0, n - 1)


def transform(X: np.ndarray, Ms) -> np.ndarray:
    """L(X) = X x_3 M_3 x_4 M_4 ... x_K M_K (Sec. 3.2)."""
    for k, M in enumerate(Ms, start=3):
        X = mode_product(X, np.asarray(M, dtype=np.float64), k)
    return X


def inverse_transform(Xh: np.ndarray, Ms) -> np.ndarray:
    """L^{-1}(X) = X x_K M_K^{-1} ... x_3 M_3^{-1} (Sec. 3.1 definition of L; Sec. 3.2)."""
    K = len(Ms) + 2
    for k in range(K, 2, -1):
        Xh = mode_product(Xh, np.linalg.inv(np.asarray(Ms[k - 3], dtype=np.float64)), k)
    return Xh


# ----------------------------------------------------------------------------------
# Representative matrices and the face-wise product (Eq. 3.5, Sec. 3.1)
# ----------------------------------------------------------------------------------
def slices(X: np.ndarray) -> np.ndarray:
    """Stack of representative matrices X^p (Eq. 3.5) as an (I1, I2, P) array, p with
    mode 3 fastest."""
    I1, I2 = X.shape[:2]
    return X.reshape(I1, I2, -1, order="F")


def from_slices(S: np.ndarray, trailing) -> np.ndarray:
    """Inverse of `slices`: (I1, I2, P) back to (I1, I2, I3, ..., IK)."""
    return S.reshape(S.shape[0], S.shape[1], *trailing, order="F")


def facewise(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Generalized face-wise product (Sec. 3.1): C^p = A^p B^p for every p."""
    As, Bs = slices(A), slices(B)
    Cs = np.stack([As[:, :, p] @ Bs[:, :, p] for p in range(As.shape[2])], axis=2)
    return from_slices(Cs, A.shape[2:])


def product(A: np.ndarray, B: np.ndarray, Ms) -> np.ndarray:
    """*_L-product, Algorithm 2 (Sec. 3.2): A_hat = L(A), B_hat = L(B);
    C_hat^i = A_hat^i B_hat^i for i = 1..P; C = L^{-1}(C_hat)."""
    return inverse_transform(facewise(transform(A, Ms), transform(B, Ms)), Ms)


def identity(I1: int, trailing, Ms) -> np.ndarray:
    """Identity tensor of Sec. 3.2: L(I)^p = I for every p, i.e. I = L^{-1}(stack of I)."""
    P = int(np.prod(trailing)) if len(trailing) else 1
    Ih = from_slices(np.repeat(np.eye(I1)[:, :, None], P, axis=2), trailing)
    return inverse_transform(Ih, Ms)


def transpose(A: np.ndarray, Ms) -> np.ndarray:
    """Transpose of Sec. 3.2: L(A^T)^p = (L(A)^p)^T, applied literally in the
    transform domain."""
    Ah = slices(transform(A, Ms))
    return inverse_transform(from_slices(np.transpose(Ah, (1, 0, 2)), A.shape[2:]), Ms)


# ----------------------------------------------------------------------------------
# *_L-SVD and *_L-SVT (Theorem of Eq. tsvd1 / Algorithm 3; Definition of D_tau /
# Theorem 23 / Algorithm 4)
# ----------------------------------------------------------------------------------
def svd(A: np.ndarray, Ms):
    """*_L-SVD, Algorithm 3: A_hat = L(A); [U_hat^i, S_hat^i, V_hat^i] = svd(A_hat^i);
    U = L^{-1}(U_hat), S = L^{-1}(S_hat), V = L^{-1}(V_hat).  Full U (I1 x I1), S
    (I1 x I2), V (I2 x I2) as in the theorem's statement.  Returns (U, S, V, sigma)
    with sigma the (min(I1, I2), P) array of per-slice singular values, descending."""
    I1, I2 = A.shape[:2]
    trailing = A.shape[2:]
    Ah = slices(transform(A, Ms))
    P = Ah.shape[2]
    Uh = np.empty((I1, I1, P))
    Sh = np.zeros((I1, I2, P))
    Vh = np.empty((I2, I2, P))
    sig = np.empty((min(I1, I2), P))
    for p in range(P):
        u, s, vt = np.linalg.svd(Ah[:, :, p], full_matrices=True)
        Uh[:, :, p] = u
        Sh[: len(s), : len(s), p] = np.diag(s)
        Vh[:, :, p] = vt.T
        sig[:, p] = s
    U = inverse_transform(from_slices(Uh, trailing), Ms)
    S = inverse_transform(from_slices(Sh, trailing), Ms)
    V = inverse_transform(from_slices(Vh, trailing), Ms)
    return U, S, V, sig


def svt(A: np.ndarray, tau: float, Ms, return_sigma: bool = False):
    """*_L-SVT D_tau(A), Algorithm 4: A_hat = L(A); for every slice
    [U, S, V] = svd(A_hat^i), S = max(S - tau, 0), A_hat^i = U S V^T; A = L^{-1}(A_hat)."""
    trailing = A.shape[2:]
    Ah = slices(transform(A, Ms))
    Dh = np.empty_like(Ah)
    sig = []
    for p in range(Ah.shape[2]):
        u, s, vt = np.linalg.svd(Ah[:, :, p], full_matrices=False)
        s_shrunk = np.maximum(s - tau, 0.0)
        Dh[:, :, p] = (u * s_shrunk) @ vt
        sig.append(s)
    D = inverse_transform(from_slices(Dh, trailing), Ms)
    if return_sigma:
        return D, np.stack(sig, axis=1)
    return D


def truncate(A: np.ndarray, k: int, Ms) -> np.ndarray:
    """Rank-k approximation of the Eckart-Young theorem (Sec. 3.2):
    A_k = U(:, 1:k, ...) *_L S(1:k, 1:k, ...) *_L V(:, 1:k, ...)^T, i.e. per transform
    domain slice the first k singular triplets of A_hat^p (descending singular values),
    then L^{-1}.  k >= min(I1, I2) returns A (to rounding), k = 0 the zero tensor."""
    trailing = A.shape[2:]
    Ah = slices(transform(A, Ms))
    Dh = np.empty_like(Ah)
    for p in range(Ah.shape[2]):
        u, s, vt = np.linalg.svd(Ah[:, :, p], full_matrices=False)
        kk = min(int(k), len(s))
        Dh[:, :, p] = (u[:, :kk] * s[:kk]) @ vt[:kk, :]
    return inverse_transform(from_slices(Dh, trailing), Ms)


def ranks_and_norms(A: np.ndarray, Ms, unit_roundoff: float = 2.0 ** -53) -> dict:
    """The rank notions and norms of Sec. 3.2 from the per-slice singular values of
    L(A):
      multirank    rho_p = rank(L(A)^p)  (Definition "Multirank and average rank")
      average      mean_p rho_p
      tubal        card{i : sigma_i(L(A)^p) != 0 for some p}  (Definition and Lemma of
                   the tubal rank; with descending sigma this is max_p rho_p)
      spectral     ||bdiag(L(A))||_2 = max_p sigma_1(L(A)^p)  (Proposition on the
                   spectral norm)
      nuclear      sum_p sum_i sigma_i(L(A)^p)  (Eq. 24 without the 1/alpha factor;
                   alpha = 1 for orthonormal transforms)
    A singular value counts as nonzero when it exceeds max(I1, I2) * u * ||A|| with
    ||A|| the spectral norm above and u the unit roundoff of the arithmetic being
    checked: a slice that is zero in exact arithmetic picks up rounding-level singular
    values from the transforms of the other slices, so the scale is the tensor's, not
    the slice's."""
    I1, I2 = A.shape[:2]
    Ah = slices(transform(A, Ms))
    P = Ah.shape[2]
    sig = [np.linalg.svd(Ah[:, :, p], compute_uv=False) for p in range(P)]
    smax = max(float(s[0]) for s in sig) if P and len(sig[0]) else 0.0
    tol = max(I1, I2) * unit_roundoff * smax
    rho = np.array([int(np.sum(s > tol)) if smax > 0 else 0 for s in sig], dtype=np.int64)
    nuc = float(sum(float(s.sum()) for s in sig))
    return {"multirank": rho, "average": float(rho.mean()), "tubal": int(rho.max()),
            "spectral": smax, "nuclear": nuc}


def nuclear_norm(A: np.ndarray, Ms) -> float:
    """Transform-domain nuclear norm sum_p sum_i sigma_i(L(A)^p) (Theorem 21, Eq. 24,
    without the 1/alpha factor; alpha = 1 for orthonormal transforms)."""
    Ah = slices(transform(A, Ms))
    return float(sum(np.linalg.svd(Ah[:, :, p], compute_uv=False).sum()
                     for p in range(Ah.shape[2])))


# ----------------------------------------------------------------------------------
# The Fourier operator (t-product): M_3 = F_{I3} of Sec. 2, complex
# ----------------------------------------------------------------------------------
def fourier_matrix(n: int) -> np.ndarray:
    """F_n of Sec. 2: (F_n)_{i,j} = omega^{(i-1)(j-1)}, omega = exp(-2 pi i / n)
    (unnormalised; F_n F_n^* = n I)."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def fourier_transform(X: np.ndarray, Ms_rest=()) -> np.ndarray:
    """L(X) with M_3 = F_{I3} (the t-product's transform, Sec. 2) and real M_4..M_K:
    X x_3 F x_4 M_4 ... x_K M_K, complex."""
    Y = mode_product(np.asarray(X, dtype=np.complex128), fourier_matrix(X.shape[2]), 3)
    for k, M in enumerate(Ms_rest, start=4):
        Y = mode_product(Y, np.asarray(M, dtype=np.float64), k)
    return Y


def fourier_inverse(Yh: np.ndarray, Ms_rest=()) -> np.ndarray:
    """L^{-1} of `fourier_transform`; the real part of the result (the imaginary part
    of the inverse of a conjugate-symmetric transform-domain tensor is rounding)."""
    K = len(Ms_rest) + 3
    for k in range(K, 3, -1):
        Yh = mode_product(Yh, np.linalg.inv(np.asarray(Ms_rest[k - 4], dtype=np.float64)), k)
    n = Yh.shape[2]
    return np.real(mode_product(Yh, np.linalg.inv(fourier_matrix(n)), 3))


def tproduct(A: np.ndarray, B: np.ndarray, Ms_rest=()) -> np.ndarray:
    """*_L-product with M_3 = F (the t-product of Kilmer and Martin for third order),
    Algorithm 2 on complex transform-domain slices."""
    Ah = slices(fourier_transform(A, Ms_rest))
    Bh = slices(fourier_transform(B, Ms_rest))
    Ch = np.stack([Ah[:, :, p] @ Bh[:, :, p] for p in range(Ah.shape[2])], axis=2)
    return fourier_inverse(from_slices(Ch, A.shape[2:]), Ms_rest)


def tsvt(A: np.ndarray, tau: float, Ms_rest=()) -> np.ndarray:
    """*_L-SVT with M_3 = F, Algorithm 4: per complex transform-domain slice
    U max(S - tau, 0) V^H, threshold applied unscaled to the slices of L(A)."""
    Ah = slices(fourier_transform(A, Ms_rest))
    Dh = np.empty_like(Ah)
    for p in range(Ah.shape[2]):
        u, s, vh = np.linalg.svd(Ah[:, :, p], full_matrices=False)
        Dh[:, :, p] = (u * np.maximum(s - tau, 0.0)) @ vh
    return fourier_inverse(from_slices(Dh, A.shape[2:]), Ms_rest)


# ----------------------------------------------------------------------------------
# Completion by PGA (Sec. 4: Eqs. 50-53, Algorithm 5)
# ----------------------------------------------------------------------------------
def pga_objective(X, mask, obs, tau, Ms) -> float:
    """F(X) = tau * ||X||_* + 1/2 ||P_Omega(X) - P_Omega(M)||_F^2 (Eq. 11 with
    g = nuclear norm, f of Sec. 4), nuclear norm as in `nuclear_norm`."""
    m = mask.astype(np.float64)
    return tau * nuclear_norm(X, Ms) + 0.5 * float(np.sum((m * (X - obs)) ** 2))


def pga(mask, obs, tau, step, iters, Ms, tol=0.0, X0=None, momentum=True,
        objective=False, mu0=0.0, nu=0.9, fourier=False):
    """Tensor completion by PGA, Algorithm 5.  With mu0 = 0 (default) the threshold is
    the fixed mu = tau; with mu0 > 0 it follows the continuation of Algorithm 5,
    mu_{k+1} = max(nu mu_k, mu_bar), read with mu_bar = tau: iteration k (0-based)
    thresholds at step * max(nu^k mu0, tau).  fourier=True uses M_3 = F (TNN-PGA-F of
    Sec. 5): the SVT is `tsvt` with Ms = [M_4, ..., M_K] (the objective is then not
    available).

        X^0 = X^1 = X0 (zeros by default), t_0 = t_1 = 1
        repeat:  Y^k = X^k + ((t_{k-1} - 1) / t_k) (X^k - X^{k-1})      (Eq. 52)
                 G^k = Y^k - step * P_Omega(Y^k - M)                     (Eq. 51)
                 X^{k+1} = D_{step*tau}(G^k)                            (Eq. 53)
                 t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2
                 r_k = ||Y^k - X^{k+1}||_F / ||X^{k+1}||_F              (Sec. 5)
        until k = iters or (tol > 0 and r_k <= tol).

    `momentum=False` forces the weight to 0 (plain proximal gradient); it exists only so
    that tests can check the monotone decrease of F that this variant guarantees.
    Returns (X_final, info) with info = {"iters", "residual" (list), "objective" (list
    or None), "t" (final t_k)}.
    """
    if fourier and objective:
        raise ValueError("the objective is defined for real transforms only")
    m = np.asarray(mask).astype(np.float64)
    obs = np.asarray(obs, dtype=np.float64)
    X = np.zeros_like(obs) if X0 is None else np.array(X0, dtype=np.float64)
    X_prev = X.copy()
    t_prev, t = 1.0, 1.0
    res, objs = [], ([] if objective else None)
    k_done = 0
    for _ in range(int(iters)):
        beta = (t_prev - 1.0) / t if momentum else 0.0
        Y = X + beta * (X - X_prev)
        G = Y - step * m * (Y - obs)
        mu = max(nu ** k_done * mu0, tau) if mu0 > 0 else tau
        X_new = tsvt(G, step * mu, Ms) if fourier else svt(G, step * mu, Ms)
        nx = float(np.linalg.norm(X_new))
        ny = float(np.linalg.norm(Y - X_new))
        r = ny / nx if nx > 0 else float(np.linalg.norm(Y))
        res.append(r)
        if objective:
            objs.append(pga_objective(X_new, mask, obs, tau, Ms))
        t_prev, t = t, (1.0 + math.sqrt(4.0 * t * t + 1.0)) / 2.0
        X_prev, X = X, X_new
        k_done += 1
        if tol > 0 and r <= tol:
            break
    return X, {"iters": k_done, "residual": res, "objective": objs, "t": t}


# ----------------------------------------------------------------------------------
# Quality measures of Sec. 5 (harness only)
# ----------------------------------------------------------------------------------
def rse(A_ori: np.ndarray, A_obt: np.ndarray) -> float:
    """Relative error ||A_ori - A_obt||_F / ||A_ori||_F.  The printed RSE of Sec. 5 is
    squared and divided by ||A_obt||; the plain relative error is the reading taken."""
    return float(np.linalg.norm(A_ori - A_obt) / np.linalg.norm(A_ori))


def psnr(A_ori: np.ndarray, A_obt: np.ndarray) -> float:
    """PSNR of Sec. 5 read with the per-element mean: 10 log10(max(A_obt)^2 / MSE)."""
    mse = float(np.mean((A_obt - A_ori) ** 2))
    return 10.0 * math.log10(float(np.max(A_obt)) ** 2 / mse)
