"""Planted mistakes in the oracle must be caught by the pins (CPU only).

Each case patches one oracle function with a plausible error (a dropped term, a wrong
sign, index or transpose) and asserts that at least one pin of test_oracle_pins fails.
"""
import math

import numpy as np
import pytest

from oracle import lt_oracle as O
from tests import test_oracle_pins as pins


def _dct_delta_ij(n):  # the garbled printed normalisation delta_{i,j}
    C = np.empty((n, n))
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            C[i - 1, j - 1] = math.sqrt((2.0 - (1.0 if i == j else 0.0)) / n) * math.cos(
                (i - 1) * (2 * j - 1) * math.pi / (2 * n))
    return C


def _cprod_no_Z(n):
    C = O.dct_matrix(n)
    return np.linalg.inv(np.diag(C[:, 0])) @ C


def _mode_product_transposed(X, U, n):
    Y = np.tensordot(U.T, X, axes=([1], [n - 1]))
    return np.moveaxis(Y, 0, n - 1)


def _inverse_without_inv(Xh, Ms):
    K = len(Ms) + 2
    for k in range(K, 2, -1):
        Xh = O.mode_product(Xh, np.asarray(Ms[k - 3]).T, k)
    return Xh


def _slices_c_order(X):
    return X.reshape(X.shape[0], X.shape[1], -1, order="C")


def _from_slices_c_order(S, trailing):
    return S.reshape(S.shape[0], S.shape[1], *trailing, order="C")


def _svt_unclamped(A, tau, Ms, return_sigma=False):
    trailing = A.shape[2:]
    Ah = O.slices(O.transform(A, Ms))
    Dh = np.empty_like(Ah)
    sig = []
    for p in range(Ah.shape[2]):
        u, s, vt = np.linalg.svd(Ah[:, :, p], full_matrices=False)
        Dh[:, :, p] = (u * (s - tau)) @ vt
        sig.append(s)
    D = O.inverse_transform(O.from_slices(Dh, trailing), Ms)
    return (D, np.stack(sig, axis=1)) if return_sigma else D


def _pga_wrong_gradient_sign(mask, obs, tau, step, iters, Ms, tol=0.0, X0=None,
                             momentum=True, objective=False):
    return _ORIG_PGA(mask, -np.asarray(obs), tau, step, iters, Ms, tol, X0, momentum, objective)


def _pga_momentum_index(mask, obs, tau, step, iters, Ms, tol=0.0, X0=None,
                        momentum=True, objective=False):
    # beta = (t_k - 1) / t_k instead of (t_{k-1} - 1) / t_k
    m = np.asarray(mask).astype(float)
    X = np.zeros_like(obs, dtype=float)
    Xp = X.copy()
    t = 1.0
    for _ in range(int(iters)):
        tn = (1 + math.sqrt(4 * t * t + 1)) / 2
        beta = (tn - 1) / tn if momentum else 0.0
        Y = X + beta * (X - Xp)
        Xn = O.svt(Y - step * m * (Y - obs), step * tau, Ms)
        t = tn
        Xp, X = X, Xn
    return X, {"iters": iters, "residual": [], "objective": None, "t": t}


_ORIG_PGA = O.pga
_ORIG_TRUNCATE = O.truncate
_ORIG_RANKS = O.ranks_and_norms


def _pga_continuation_late(mask, obs, tau, step, iters, Ms, tol=0.0, X0=None,
                           momentum=True, objective=False, mu0=0.0, nu=0.9):
    # the schedule starts at nu * mu0 instead of mu0
    return _ORIG_PGA(mask, obs, tau, step, iters, Ms, tol, X0, momentum, objective,
                     mu0 * nu, nu)


def _truncate_off_by_one(A, k, Ms):  # keeps k + 1 triplets
    return _ORIG_TRUNCATE(A, k + 1, Ms)


def _ranks_slice_relative(A, Ms, unit_roundoff=2.0 ** -53):
    # tolerance relative to each slice's own largest singular value
    I1, I2 = A.shape[:2]
    Ah = O.slices(O.transform(A, Ms))
    rho = []
    for p in range(Ah.shape[2]):
        s = np.linalg.svd(Ah[:, :, p], compute_uv=False)
        rho.append(int(np.sum(s > max(I1, I2) * unit_roundoff * s[0])) if s[0] > 0 else 0)
    out = _ORIG_RANKS(A, Ms, unit_roundoff)
    out["multirank"] = np.array(rho)
    return out

_ORIG_TSVT = O.tsvt


def _fourier_one_based(n):
    # omega^{ij} with 1-based i, j instead of omega^{(i-1)(j-1)}
    k = np.arange(1, n + 1)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def _tsvt_unitary_threshold(A, tau, Ms_rest=()):
    # threshold the slices of F/sqrt(n)-transformed data instead of F-transformed data
    return _ORIG_TSVT(A, tau * math.sqrt(A.shape[2]), Ms_rest)


MUTATIONS = [
    ("dct_matrix", _dct_delta_ij, [pins.test_dct_matrix_closed_forms_and_scipy]),
    ("cproduct_matrix", _cprod_no_Z, [pins.test_cproduct_matrix_closed_forms]),
    ("mode_product", _mode_product_transposed,
     [lambda: pins.test_mode_product_matricization((3, 4, 2))]),
    ("inverse_transform", _inverse_without_inv,
     [lambda: pins.test_transform_kronecker_brute_force((3, 2))]),
    ("slices", _slices_c_order,
     [pins.test_slice_order_eq_3_5]),
    ("svt", _svt_unclamped, [pins.test_svt_special_cases]),
    ("pga", _pga_wrong_gradient_sign, [pins.test_pga_first_iterates_and_momentum_schedule]),
    ("pga", _pga_momentum_index, [pins.test_pga_first_iterates_and_momentum_schedule]),
    ("pga", _pga_continuation_late, [pins.test_pga_continuation_schedule_and_limit]),
    ("truncate", _truncate_off_by_one, [pins.test_truncate_is_the_eckart_young_product]),
    ("ranks_and_norms", _ranks_slice_relative, [pins.test_ranks_and_norms_on_prescribed_ranks]),
    ("fourier_matrix", _fourier_one_based,
     [pins.test_fourier_matrix_is_numpy_fft_and_scaled_unitary]),
    ("tsvt", _tsvt_unitary_threshold,
     [lambda: pins.test_tsvt_is_the_prox_of_the_fourier_nuclear_norm((4,))]),
]


@pytest.mark.parametrize("name,bad,checks", MUTATIONS,
                         ids=[f"{m[0]}:{m[1].__name__}" for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, bad, checks):
    monkeypatch.setattr(O, name, bad)
    if name == "slices":
        monkeypatch.setattr(O, "from_slices", _from_slices_c_order)
    caught = False
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError):  # a wrong value or a shape error
            caught = True
    assert caught, f"planted mistake in {name} was not caught"
