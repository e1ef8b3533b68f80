"""Helpers shared by the GPU parity tests (marshalling and error metrics only)."""
import numpy as np
import scipy.sparse as sp

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def to_dev(A, dtype=None):
    import torch
    dev = torch.device("cuda", 0)
    val = A.val if dtype is None else A.val.astype(dtype)
    return (torch.from_numpy(np.ascontiguousarray(A.row_ptr)).to(dev),
            torch.from_numpy(np.ascontiguousarray(A.col)).to(dev),
            torch.from_numpy(np.ascontiguousarray(val)).to(dev))


def abs_powers(A, coeffs, x):
    """(|A_theta|^k |x|) for k = 0..p: the denominators of the per-entry error metric, with
    |A_theta| applied as |a_k||A| + |b_k| I (+ |c_k| on the k-2 term)."""
    n = A.n
    M = abs(sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n)))
    out = [np.abs(x)]
    for k, (a, b, c) in enumerate(coeffs, start=1):
        prev = out[-1]
        prev2 = out[-2] if k >= 2 else np.zeros_like(prev)
        out.append(abs(a) * (M @ prev) + abs(b) * prev + abs(c) * prev2)
    return np.array(out)


def max_rel_err(got, ref, den):
    """max_i |got - ref|_i / den_i; entries with den == 0 must match exactly (else inf)."""
    diff = np.abs(got - ref)
    zero = den == 0
    if np.any(diff[zero] != 0):
        return np.inf
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(zero, 0.0, diff / np.where(zero, 1.0, den))
    return float(np.max(r)) if r.size else 0.0
