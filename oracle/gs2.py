"""Two-stage Gauss-Seidel (GS2) preconditioning and the MPK with sub-powers, in FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow and plain on purpose.

Sec. 5.1 (the GS2 part, Alg. GS2): a Gauss-Seidel iteration (L + D) z^{k+1} = v - U z^k
whose triangular solve is replaced by gamma inner Jacobi-Richardson iterations:
    g_0 = D^-1 (v - U z^k);   g_j = g_0 - D^-1 L g_{j-1}  (j = 1..gamma);   z^{k+1} = z^k + g_gamma.
As a preconditioner the paper uses one outer iteration from z^0 = 0, so P^-1 v = g_gamma.
The MPK of the preconditioned operator runs each power as gamma + 2 sub-powers (the GS2
stages, then the product with A):  y_k = a_k A P^-1 y_{k-1} + b_k y_{k-1} + c_k y_{k-2}.

Readings (listed with the design notes):
* L, D, U are the strictly lower part, the diagonal and the strictly upper part of A in the
  caller's row order (the order the matrix is given in), so the preconditioner does not depend
  on the level permutation the blocked kernel uses;
* duplicate entries are summed; a zero or missing diagonal entry is read as 1 (D~), and the
  difference D - D~ joins U, where it multiplies z^0 = 0;
* for a nonzero start the printed pair g_0 = D^-1 (v - U z^k), z^{k+1} = z^k + g_gamma is not a
  Gauss-Seidel step; the residual-correction form g_0 = D~^-1 (v - A z^k) is (with exact inner
  solves it gives z^{k+1} = (L + D~)^-1 (v - (U + D - D~) z^k)).  Both agree for z^0 = 0,
  the only start the paper's preconditioner (and the GPU library) uses.
"""
from __future__ import annotations

import numpy as np

from . import sstep as _sstep

__all__ = ["split_ldu", "gs2_apply", "gs2_mpk", "gs2_gmres"]


def split_ldu(A):
    """Row lists of the strictly lower and strictly upper entries, and the diagonal D~
    (zero or missing diagonal entries read as 1) plus the true diagonal D."""
    n = A.n
    lower = [[] for _ in range(n)]
    upper = [[] for _ in range(n)]
    d = np.zeros(n)
    for i in range(n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = int(A.col[e])
            if j < i:
                lower[i].append((j, float(A.val[e])))
            elif j > i:
                upper[i].append((j, float(A.val[e])))
            else:
                d[i] += A.val[e]
    dt = np.where(d != 0.0, d, 1.0)
    return lower, d, dt, upper


def gs2_apply(A, v, gamma, z0=None, split=None):
    """One outer GS2 iteration (Alg. GS2(a), k = 0) from z0 (default 0) with gamma inner
    Jacobi-Richardson iterations; returns z^1.  With z0 = 0 this is the preconditioner
    P^-1 v of the paper's GS2 experiments."""
    lower, d, dt, upper = split if split is not None else split_ldu(A)
    n = A.n
    z0 = np.zeros(n) if z0 is None else np.asarray(z0, dtype=np.float64)
    # g_0 = D~^-1 (v - A z0): the residual of the start (v itself for z0 = 0)
    az = d * z0
    for i in range(n):
        for j, a in lower[i] + upper[i]:
            az[i] += a * z0[j]
    g0 = (v - az) / dt
    g = g0
    for _ in range(gamma):
        lg = np.zeros(n)
        for i in range(n):
            for j, a in lower[i]:
                lg[i] += a * g[j]
        g = g0 - lg / dt
    return z0 + g


def gs2_mpk(A, p, coeffs, x, gamma):
    """MPK of the GS2-preconditioned operator: y_0 = x,
    y_k = a_k A P^-1 y_{k-1} + b_k y_{k-1} + c_k y_{k-2} (y_{-1} = 0), P^-1 = gs2_apply from
    zero.  Returns an array of shape (p+1, n)."""
    split = split_ldu(A)
    n = A.n
    Y = np.zeros((p + 1, n))
    Y[0] = x
    for k in range(1, p + 1):
        a, b, c = coeffs[k - 1]
        z = gs2_apply(A, Y[k - 1], gamma, split=split)
        y = a * _sstep.spmv(A, z) + b * Y[k - 1]
        if k >= 2:
            y = y + c * Y[k - 2]
        Y[k] = y
    return Y


def gs2_gmres(A, b, gamma, s=8, m=48, tol=1e-8, max_restarts=1000, shifts=None):
    """Right-preconditioned s-step GMRES with P^-1 = one GS2 iteration from zero (Sec. 5.1, GS2
    subsection): the Newton basis of A P^-1, x = x0 + P^-1 (V y); the GMRES residual is the
    true residual b - A x.  Returns the dict of ``sstep.sstep_gmres``."""
    split = split_ldu(A)
    return _sstep.sstep_gmres(A, b, s=s, m=m, tol=tol, max_restarts=max_restarts, shifts=shifts,
                              precond=lambda v: gs2_apply(A, v, gamma, split=split))
