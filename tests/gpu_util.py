"""Helpers shared by the GPU parity tests: layout conversion between the oracle's
natural-index numpy arrays and the library's column-major device buffers, and context
construction from the generators' transform descriptions.  The DCT matrices of each
side come from that side's own constructor (oracle.dct_matrix vs lt_make_dct)."""
import numpy as np
import torch

from oracle import lt_oracle as O
from paper_2202_02870_gb300 import lt


def to_dev(a, dtype=torch.float64):
    """(I1, I2, ..., IK) numpy -> contiguous CUDA tensor of shape (IK, ..., I2, I1)."""
    a = np.asarray(a)
    flat = np.ascontiguousarray(a.ravel(order="F"))
    t = torch.from_numpy(flat)
    if dtype is not None and a.dtype != np.uint8:
        t = t.to(dtype)
    return t.reshape(tuple(reversed(a.shape))).cuda()


def from_dev(t, shape):
    return t.detach().double().cpu().numpy().reshape(-1).reshape(shape, order="F")


def empty_dev(shape, dtype=torch.float64):
    return torch.empty(tuple(reversed(shape)), dtype=dtype, device="cuda")


def oracle_mats(transforms):
    out = []
    for kind, v in transforms:
        if kind == "dct":
            out.append(O.dct_matrix(v))
        elif kind == "cprod":
            out.append(O.cproduct_matrix(v))
        else:
            out.append(np.asarray(v, dtype=np.float64))
    return out


def lib_mats(transforms):
    out = []
    for kind, v in transforms:
        if kind == "dct":
            out.append(lt.lt_make_dct(v))
        elif kind == "cprod":
            out.append(lt.lt_make_cproduct(v))
        else:
            out.append(np.asarray(v, dtype=np.float64))
    return out


def sizes_of(transforms):
    return [v if kind in ("dct", "cprod") else np.asarray(v).shape[0] for kind, v in transforms]


def make_ctx(transforms, precision=lt.LT_FP64):
    return lt.Context(sizes_of(transforms), lib_mats(transforms), precision)


def dtype_of(precision):
    return torch.float64 if precision == lt.LT_FP64 else torch.float32


def rel(a, b):
    d = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (d if d > 0 else 1.0))
