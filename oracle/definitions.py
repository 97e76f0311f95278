"""Definitions from the paper that the oracle's fast routes are checked against.

TEST INFRASTRUCTURE ONLY (same rule as `lt_oracle`): these are slow, literal
constructions used to pin the oracle to the paper.  They share nothing with the CUDA
library.

* `matricize(X, n)`       n-mode matricization (Definition in Sec. 2), element by element.
* `btph(X)`               block Toeplitz-plus-Hankel matrix: third order by the matrices
                          of Eq. 3.22, higher orders by the recursive block construction
                          shown for the fourth order in Sec. 3 (Eq. 16).
* `ten(Mat, shape)`       the operator with ten(btph(X)) = X (Sec. 3).
* `cproduct_def(A, B)`    generalized c-product A *_c B = ten(btph(A) btph(B)) (Def. 9).
* `kron_transform(X, Ms)` vec(L(X)) = (M_K kron ... kron M_3 kron I_{I1 I2}) vec(X), the
                          dense-matrix form of L with column-major vec (Eq. 3.5 order).
"""
from __future__ import annotations

import numpy as np


def matricize(X: np.ndarray, n: int) -> np.ndarray:
    """n-mode matricization X_(n) (Sec. 2): element (i_1, ..., i_N) goes to row i_n and
    column j = sum_{k != n} i_k J_k with J_k = prod_{m < k, m != n} I_m (0-based).  The
    printed index formula is garbled (its sum runs over "j != n" and J_k has no upper
    limit); this is the Kolda-Bader reading, which reproduces the paper's third-order
    examples X_(1) = [X^(1), ..., X^(I3)] and X_(2) = [X^(1)T, ..., X^(I3)T]."""
    shape = X.shape
    N = len(shape)
    J = [0] * N
    acc = 1
    for k in range(N):
        if k == n - 1:
            continue
        J[k] = acc
        acc *= shape[k]
    out = np.zeros((shape[n - 1], acc), dtype=X.dtype)
    for idx in np.ndindex(*shape):
        j = sum(idx[k] * J[k] for k in range(N) if k != n - 1)
        out[idx[n - 1], j] = X[idx]
    return out


def _btph_blocks(blocks):
    """Toeplitz-plus-Hankel assembly over one mode.  `blocks[q]` (q = 0..n-1) is the
    matrix standing for the q-th (1-based q+1) sub-tensor along that mode.  With 1-based
    block indices (i, j):
      Toeplitz part: block (i, j) = A_{|i-j|+1};
      Hankel part:   block (i, j) = A_{i+j} if i+j <= n, 0 if i+j = n+1,
                     A_{2n+2-i-j} otherwise.
    (The two matrices of Eq. 3.22.)"""
    n = len(blocks)
    r, c = blocks[0].shape
    out = np.zeros((r * n, c * n), dtype=np.float64)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            blk = blocks[abs(i - j)].copy()
            s = i + j
            if s <= n:
                blk = blk + blocks[s - 1]
            elif s >= n + 2:
                blk = blk + blocks[2 * n + 2 - s - 1]
            out[(i - 1) * r:i * r, (j - 1) * c:j * c] = blk
    return out


def btph(X: np.ndarray) -> np.ndarray:
    """Block Toeplitz-plus-Hankel matrix of an N-th order tensor (N >= 2).  A matrix is
    its own btph; an N-th order tensor is the Toeplitz-plus-Hankel arrangement, over the
    last mode, of the btph matrices of its (N-1)-th order sub-tensors X(..., k_N)."""
    if X.ndim == 2:
        return np.array(X, dtype=np.float64)
    subs = [btph(X[..., q]) for q in range(X.shape[-1])]
    return _btph_blocks(subs)


def ten(Mat: np.ndarray, shape) -> np.ndarray:
    """Inverse of `btph`.  For one mode of size n with sub-tensors A_1..A_n, the first
    block column of the Toeplitz-plus-Hankel matrix is [A_1 + A_2; A_2 + A_3; ...;
    A_{n-1} + A_n; A_n] (read off Eq. 3.22), so the sub-blocks are recovered from the
    bottom up, then recursively."""
    shape = tuple(shape)
    if len(shape) == 2:
        return np.array(Mat[: shape[0], : shape[1]], dtype=np.float64)
    n = shape[-1]
    sub_shape = shape[:-1]
    r = Mat.shape[0] // n
    c = Mat.shape[1] // n
    first_col = [Mat[q * r:(q + 1) * r, 0:c] for q in range(n)]
    subs_btph = [None] * n
    subs_btph[n - 1] = first_col[n - 1]
    for q in range(n - 2, -1, -1):
        subs_btph[q] = first_col[q] - subs_btph[q + 1]
    out = np.empty(shape, dtype=np.float64)
    for q in range(n):
        out[..., q] = ten(subs_btph[q], sub_shape)
    return out


def cproduct_def(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Generalized c-product, Def. 9: A *_c B = ten(btph(A) btph(B))."""
    shape = (A.shape[0], B.shape[1]) + tuple(A.shape[2:])
    return ten(btph(A) @ btph(B), shape)


def kron_transform(X: np.ndarray, Ms) -> np.ndarray:
    """L(X) through one dense matrix: vec(L(X)) = (M_K kron ... kron M_3 kron I) vec(X),
    vec column-major (mode 1 fastest)."""
    big = np.eye(X.shape[0] * X.shape[1])
    for M in Ms:
        big = np.kron(np.asarray(M, dtype=np.float64), big)
    v = X.reshape(-1, order="F")
    return (big @ v).reshape(X.shape, order="F")
