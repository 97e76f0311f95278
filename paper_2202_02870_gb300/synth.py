"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and nothing else: it holds none of the method's
arithmetic (no transform, product, SVD or completion step).  Both the CUDA path and the
CPU oracle consume the arrays it returns, so that they see identical inputs.

Layout: every tensor is returned as a float64 (or uint8) numpy array of shape
(I1, I2, I3, ..., IK) whose memory is column-major (Fortran order, mode 1 fastest), the
layout of the library's device buffers.  The i-th number drawn goes to column-major
linear index i, so `arr.ravel(order="F")` is exactly the draw sequence.

Workload recipes stand in for the paper's colour videos (Sec. 5: xylophone
240x320x3x141, Akiyo/news 144x176x3x300, and the Table 9 videos), which are not
available: low-L-rank tensors X = U *_L V^T with the videos' mode structure
(I3 = 3 colour channels, I4 = frames), Gaussian noise and a Bernoulli observation mask.
The product U *_L V^T itself is formed by the consumer (oracle or library), not here.

Seeds: numpy PCG64, seed = 20220206 + 100 * config + problem; draw order factors U, V,
then noise, then mask, then random transforms.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20220206


def rng_for(config: int, problem: int = 0) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + 100 * int(config) + int(problem))


def _fortran(flat: np.ndarray, shape) -> np.ndarray:
    return np.asfortranarray(flat.reshape(shape, order="F"))


def uniform(rng, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return _fortran(rng.uniform(lo, hi, size=n), shape)


def normal(rng, shape, scale=1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return _fortran(rng.standard_normal(size=n) * scale, shape)


def bernoulli_mask(rng, shape, rho) -> np.ndarray:
    """uint8 mask, 1 = observed, each entry independently with probability rho."""
    n = int(np.prod(shape))
    return _fortran((rng.random(size=n) < rho).astype(np.uint8), shape)


def random_orthogonal(rng, n) -> np.ndarray:
    """Haar-random orthogonal matrix: QR of a Gaussian with the signs of R's diagonal
    moved into Q (Mezzadri, "How to generate random matrices from the classical compact
    groups", 2007)."""
    Z = rng.standard_normal(size=(n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def log_uniform_spectrum(rng, n, cond) -> np.ndarray:
    """d_1 = 1, d_n = cond, the others log-uniform in between (sorted)."""
    if n == 1:
        return np.ones(1)
    inner = np.sort(np.exp(rng.uniform(0.0, np.log(cond), size=max(n - 2, 0))))
    return np.concatenate([[1.0], inner, [float(cond)]])


def conditioned_matrix(rng, n, cond, two_sided=False) -> np.ndarray:
    """Random invertible n x n matrix with 2-norm condition number `cond`:
    Q diag(d) (one-sided) or Q1 diag(d) Q2^T (two-sided)."""
    Q1 = random_orthogonal(rng, n)
    d = log_uniform_spectrum(rng, n, cond)
    if not two_sided:
        return Q1 * d[None, :]
    Q2 = random_orthogonal(rng, n)
    return (Q1 * d[None, :]) @ Q2.T


# --------------------------------------------------------------------------------------
# Workload recipes.  Transforms are described as ("dct", n) -- built by each consumer
# from the paper's definition -- or ("matrix", array) when random.
# --------------------------------------------------------------------------------------
def product_case(config=1, I1=32, l=24, I2=16, trailing=(8,), transforms=None, problem=0):
    """Uniform[-1, 1] operands A (I1 x l x trailing) and B (l x I2 x trailing)."""
    rng = rng_for(config, problem)
    A = uniform(rng, (I1, l) + tuple(trailing))
    B = uniform(rng, (l, I2) + tuple(trailing))
    if transforms is None:
        transforms = [("dct", n) for n in trailing]
    return {"A": A, "B": B, "transforms": transforms}


def completion_case(config, I1, I2, trailing, rank, rho, noise=1e-3, problem=0,
                    transforms=None):
    """Low-L-rank completion problem: factors U (I1 x r x trailing), V (I2 x r x
    trailing) with N(0, 1) entries, noise N(0, noise^2) of the full shape, Bernoulli(rho)
    mask.  The consumer forms X = U *_L V^T (V^T: modes 1 and 2 swapped) and
    obs = mask * (X + noise)."""
    rng = rng_for(config, problem)
    trailing = tuple(trailing)
    U = normal(rng, (I1, rank) + trailing)
    V = normal(rng, (I2, rank) + trailing)
    E = normal(rng, (I1, I2) + trailing, scale=noise)
    mask = bernoulli_mask(rng, (I1, I2) + trailing, rho)
    if transforms is None:
        transforms = [("dct", n) for n in trailing]
    return {"U": U, "V": V, "noise": E, "mask": mask, "transforms": transforms}


def config1():
    """*_L-product, third order: A 32x24x8, B 24x16x8, U[-1, 1], L = DCT-II 8x8."""
    return product_case(config=1, I1=32, l=24, I2=16, trailing=(8,))


def config2():
    """FP64 completion, 144x176x3x32, L-rank 10, sigma = 1e-3, 30% observed,
    L_3 = DCT 3, L_4 = DCT 32, tau = 0.5, step = 1, 100 iterations."""
    c = completion_case(2, 144, 176, (3, 32), rank=10, rho=0.3)
    c.update(tau=0.5, step=1.0, iters=100)
    return c


def config3(I1=256, l=256, I2=128, trailing=(16, 16, 8), cond=1e2):
    """Fifth-order product / L-SVT operands, U[-1, 1]; L_k = Q_k diag(d_k), cond 1e2."""
    rng = rng_for(3)
    A = uniform(rng, (I1, l) + tuple(trailing))
    B = uniform(rng, (l, I2) + tuple(trailing))
    transforms = [("matrix", conditioned_matrix(rng, n, cond)) for n in trailing]
    return {"A": A, "B": B, "transforms": transforms}


def config4_shapes(nprob=64):
    """Shapes of the 64 batched problems: I1 = 16u, I2 = 12u, u ~ U{4..32}, I3 = 3,
    I4 ~ {8, 16, 32, 64}, rank ~ U{5..20}, rho ~ U[0.2, 0.5]."""
    rng = rng_for(4, 999)
    out = []
    for _ in range(nprob):
        u = int(rng.integers(4, 33))
        out.append({"I1": 16 * u, "I2": 12 * u, "trailing": (3, int(rng.choice([8, 16, 32, 64]))),
                    "rank": int(rng.integers(5, 21)), "rho": float(rng.uniform(0.2, 0.5))})
    return out


def config5(I1=540, I2=960, trailing=(3, 120), rank=15, rho=0.2, cond=10.0):
    """Large completion: 540x960x3x120, rank 15, 20% observed, L_3 = DCT 3,
    L_4 = Q1 diag(d) Q2^T with cond 10."""
    c = completion_case(5, I1, I2, trailing, rank=rank, rho=rho)
    rng = rng_for(5, 1)
    c["transforms"] = [("dct", trailing[0]),
                       ("matrix", conditioned_matrix(rng, trailing[1], cond, two_sided=True))]
    c.update(tau=0.5, step=1.0)
    return c
