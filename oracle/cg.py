"""Textbook conjugate gradients and s-step (communication-avoiding) CG, in FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow and plain on purpose.

The paper names s-step CG as the short-recurrence Krylov method whose solver speedup should
approach the MPK speedup, since its orthogonalisation cost is minimal (Sec. 4, discussion of
the s-step GMRES results; Sec. 7), and cites Chronopoulos and Gear for the method without
giving its steps.  The form used here is the standard one (Chronopoulos-Gear / Hoemmen /
Carson-Demmel): per outer iteration
  * one MPK on p (s powers) and one on r (s - 1 powers) in the Newton basis give
    Y = [p, rho_1(A) p, .., rho_s(A) p, r, rho_1(A) r, .., rho_{s-1}(A) r], rho_k(A) = prod_{i<k} (A - theta_i I);
  * A Y = Y B for every column but the last of each block, with B the (2s+1) x (2s+1) block
    diagonal change of basis (theta_k on the diagonal, ones below it);
  * the Gram matrix G = Y^T Y;
  * s CG steps on coordinate vectors (p' = e_0, r' = e_{s+1}, x' = 0):
        alpha = r'^T G r' / p'^T G B p';  x' += alpha p';  r'_new = r' - alpha B p';
        beta = r'_new^T G r'_new / r'^T G r';  p' = r'_new + beta p';
  * x += Y x', r = Y r', p = Y p'.
In exact arithmetic the iterates at the end of each outer iteration are those of CG after the
same number of steps.

Readings (listed with the design notes):
* shifts: as for s-step GMRES (Sec. 4: eigenvalue estimates from a few steps of the plain
  method), the Ritz values of a first phase of plain CG (4 s steps from x = 0): the eigenvalues
  of the Lanczos tridiagonal that CG's coefficients give (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
  T_j,j+1 = sqrt(beta_j)/alpha_j), s of them in Leja order; ``cg_shifts`` (Leja points of the
  Gershgorin interval [0, max_i sum_j |a_ij|]) is an alternative that needs no setup phase;
* convergence: the recurrence residual norm sqrt(r'^T G r') is checked after every inner step;
  an outer iteration may stop early, and then recovers x, r, p from the steps taken;
* breakdown: p'^T G B p' <= 0 (A not positive definite, or a numerically singular basis);
* refinement: outer FP64 loop r = b - A x, inner s-step CG on A d = r to inner_tol, x += d;
* residual replacement (``replace`` = k > 0, van der Vorst and Ye; Carson and Demmel for s-step
  methods): at the start of every k-th outer iteration after the first, r is recomputed as
  b - A x (p is kept), which bounds the drift of the recurrence residual in a low-precision
  basis; the inner solve then runs to the overall tolerance.
"""
from __future__ import annotations

import numpy as np

from . import sstep as _sstep

__all__ = ["cg", "gershgorin_bound", "cg_shifts", "lanczos_ritz", "ritz_shifts", "change_of_basis",
           "cacg", "refine_cg", "CGBreakdown"]


class CGBreakdown(RuntimeError):
    """p^T A p <= 0 in the coordinate recurrence."""


def cg(A, b, x0=None, tol=1e-8, max_iters=100000):
    """Textbook CG (Hestenes-Stiefel).  Returns dict(x, iters, hist, converged, alphas,
    betas); hist[k] is ||r_k|| / ||b|| of the recurrence residual."""
    x = np.zeros(A.n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - _sstep.spmv(A, x)
    p = r.copy()
    rr = r @ r
    nb = np.linalg.norm(b)
    hist = [np.sqrt(rr) / nb]
    alphas, betas = [], []
    for k in range(max_iters):
        if np.sqrt(rr) <= tol * nb:
            return dict(x=x, iters=k, hist=hist, converged=True, alphas=alphas, betas=betas)
        q = _sstep.spmv(A, p)
        alpha = rr / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        alphas.append(alpha)
        betas.append(rr_new / rr)
        rr = rr_new
        hist.append(np.sqrt(rr) / nb)
    return dict(x=x, iters=max_iters, hist=hist, converged=bool(np.sqrt(rr) <= tol * nb),
                alphas=alphas, betas=betas)


def lanczos_ritz(alphas, betas):
    """Eigenvalues of the Lanczos tridiagonal of k CG steps (the Ritz values of A on the
    Krylov space), from the CG coefficients alpha_0..alpha_{k-1}, beta_0..beta_{k-2}."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(T)


def ritz_shifts(alphas, betas, s):
    """s Ritz values in Leja order (first = largest modulus)."""
    return _sstep.leja_order(lanczos_ritz(alphas, betas), s)


def gershgorin_bound(A):
    """g = max_i sum_j |a_ij|."""
    s = np.zeros(A.n)
    for i in range(A.n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            s[i] += abs(A.val[e])
    return float(s.max()) if A.n else 0.0


def cg_shifts(A, s):
    """First s Leja points of [0, g] among 10,001 equispaced candidates."""
    g = gershgorin_bound(A)
    return _sstep.leja_order(np.linspace(0.0, g, 10001), s)


def change_of_basis(theta, s):
    """B with A Y[:, c] = Y B[:, c] for every column c of Y but the last of each block."""
    M = 2 * s + 1
    B = np.zeros((M, M))
    for j in range(s):                 # p block: columns 0..s
        B[j, j] = theta[j]
        B[j + 1, j] = 1.0
    for j in range(s - 1):             # r block: columns s+1..2s
        B[s + 1 + j, s + 1 + j] = theta[j]
        B[s + 2 + j, s + 1 + j] = 1.0
    return B


def _basis(A, v, theta, k):
    """[v, (A - theta_0) v, (A - theta_1)(A - theta_0) v, ...], k powers (k + 1 columns)."""
    cols = [v]
    for i in range(k):
        cols.append(_sstep.spmv(A, cols[-1]) - theta[i] * cols[-1])
    return np.array(cols).T


def cacg(A, b, s, theta, x0=None, tol=1e-8, max_iters=100000, stop_abs=None, replace=0):
    """s-step CG (module docstring) from x0.  Stops when the recurrence residual norm is
    <= max(tol * ||b||, stop_abs).  replace = k > 0: r = b - A x at the start of every k-th
    outer iteration after the first.  Returns dict(x, iters, outer, hist, converged) with hist
    the recurrence residual norms / ||b|| after every inner step."""
    n = A.n
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - _sstep.spmv(A, x)
    p = r.copy()
    nb = np.linalg.norm(b)
    target = tol * nb if stop_abs is None else max(tol * nb, stop_abs)
    B = change_of_basis(theta, s)
    hist = [np.linalg.norm(r) / nb]
    iters = 0
    outer = 0
    if np.linalg.norm(r) <= target:
        return dict(x=x, iters=0, outer=0, hist=hist, converged=True)
    while iters < max_iters:
        if replace > 0 and outer > 0 and outer % replace == 0:
            r = b - _sstep.spmv(A, x)
        Y = np.hstack([_basis(A, p, theta, s), _basis(A, r, theta, s - 1)])
        G = Y.T @ Y
        pc = np.zeros(2 * s + 1)
        pc[0] = 1.0
        rc = np.zeros(2 * s + 1)
        rc[s + 1] = 1.0
        xc = np.zeros(2 * s + 1)
        rr = rc @ G @ rc
        done = False
        for _ in range(s):
            Bp = B @ pc
            den = pc @ G @ Bp
            if not den > 0.0:
                raise CGBreakdown("p^T A p = %g" % den)
            alpha = rr / den
            xc = xc + alpha * pc
            rc = rc - alpha * Bp
            rr_new = rc @ G @ rc
            pc = rc + (rr_new / rr) * pc
            rr = rr_new
            iters += 1
            hist.append(np.sqrt(max(rr, 0.0)) / nb)
            if np.sqrt(max(rr, 0.0)) <= target or iters >= max_iters:
                done = True
                break
        x = x + Y @ xc
        r = Y @ rc
        p = Y @ pc
        outer += 1
        if done:
            break
    conv = bool(hist[-1] * nb <= target)
    return dict(x=x, iters=iters, outer=outer, hist=hist, converged=conv)


def refine_cg(A, b, s, theta=None, tol=1e-8, inner_tol=1e-5, max_outer=200, round_inner=None,
              max_iters=100000, replace=0):
    """FP64 iterative refinement around s-step CG: r = b - A x (FP64); s-step CG on A d = r to
    inner_tol relative to ||r|| (to 0.5 tol ||b|| with residual replacement every ``replace``
    outer iterations; ``round_inner`` rounds the inner right-hand side and the correction,
    emulating a lower-precision inner solve); x += d; until ||r|| <= tol ||b||.
    Without ``theta`` a setup phase of 4 s plain CG steps from x = 0 comes first; its Ritz
    values give the shifts.  Returns dict(x, outer, iters, relres, shifts)."""
    x = np.zeros(A.n)
    nb = np.linalg.norm(b)
    iters = 0
    if theta is None:
        setup = cg(A, b, tol=tol, max_iters=4 * s)
        x = setup["x"]
        iters = setup["iters"]
        th = ritz_shifts(setup["alphas"], setup["betas"], s) if setup["iters"] >= s else \
            cg_shifts(A, s)
    else:
        th = np.asarray(theta, dtype=np.float64)
    relres = []
    for k in range(max_outer):
        r = b - _sstep.spmv(A, x)
        relres.append(np.linalg.norm(r) / nb)
        if relres[-1] <= tol:
            return dict(x=x, outer=k, iters=iters, relres=relres, converged=True, shifts=th)
        rin = r if round_inner is None else r.astype(round_inner).astype(np.float64)
        if replace > 0:
            out = cacg(A, rin, s, th, tol=0.0, max_iters=max_iters - iters, stop_abs=0.5 * tol * nb,
                       replace=replace)
        else:
            out = cacg(A, rin, s, th, tol=inner_tol, max_iters=max_iters - iters,
                       stop_abs=tol * nb)
        iters += out["iters"]
        d = out["x"] if round_inner is None else out["x"].astype(round_inner).astype(np.float64)
        x = x + d
    r = b - _sstep.spmv(A, x)
    relres.append(np.linalg.norm(r) / nb)
    return dict(x=x, outer=max_outer, iters=iters, relres=relres, converged=relres[-1] <= tol,
                shifts=th)
