"""GMRES-polynomial preconditioning (Sec. 5.2, Eq. (poly_precon)) in FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper applies P^-1 x = lambda_0 x + lambda_1 A x + ... + lambda_d A^d x with the scalars
taken from d GMRES steps.  Reading used here (the paper gives no formulas for the scalars):

* The polynomial is the GMRES one.  d + 1 steps of GMRES on A from r0 give
  x_{d+1} - x_0 = q(A) r0 with q of degree d, and A q(A) ~ I on the Krylov space.  q is read
  off the Arnoldi relation: with v_1 = r0 / beta and
      h_{j+1,j} v_{j+1} = A v_j - sum_{i<=j} h_{ij} v_i,
  the basis vectors are v_j = phi_j(A) r0 for the Arnoldi polynomials
      phi_1 = 1 / beta,  phi_{j+1}(t) = (t phi_j(t) - sum_{i<=j} h_{ij} phi_i(t)) / h_{j+1,j},
  and q = sum_j y_j phi_j, y the GMRES least-squares coefficients.
* The same polynomial is represented in the Chebyshev basis of an interval [alpha, beta_iv]
  that holds the spectrum (alpha = 0, beta_iv = 1.1 x the largest Ritz value of the setup
  cycle): gamma_k follow from exact interpolation of q at the d + 1 Chebyshev nodes.  This is
  the polynomial of Eq. (poly_precon), evaluated by the stable three-term recurrence instead of
  the monomial sum (which loses all digits at degree 40-80).
* The same q also has a root (product) form: with theta_1..theta_{d+1} the harmonic Ritz values
  of the d + 1 Arnoldi steps (the roots of the GMRES residual polynomial pi, which satisfies
  1 - t q(t) = pi(t) = prod_i (1 - t / theta_i)),
      q(A) x = sum_{k=0}^{d} (1 / theta_{k+1}) prod_{i<=k} (I - A / theta_i) x,
  stable in low precision when the roots are Leja-ordered.  For a symmetric A the harmonic Ritz
  values are the eigenvalues of the pencil Hbar^T Hbar z = theta sym(H_{d+1}) z.
* The solver is restarted GMRES(m) with right preconditioning: the first cycle runs on A and
  supplies the polynomial (its correction is kept); later cycles run on B = A p(A), and their
  correction is x += p(A) V y.
"""
from __future__ import annotations

import numpy as np

from . import mpk as _mpk
from .sstep import chebyshev_coeffs, jacobi_sweeps, spmv

__all__ = ["arnoldi", "arnoldi_poly", "poly_from_arnoldi", "apply_poly", "harmonic_roots",
           "apply_poly_roots", "poly_gmres", "jacobi_sweeps_gmres"]


def arnoldi(A, r0, k):
    """k steps of Arnoldi with modified Gram-Schmidt from r0 (Alg. 3(a)).  Returns
    (V (n x (k+1)), H ((k+1) x k), beta, steps) -- steps < k on a happy breakdown."""
    n = r0.shape[0]
    beta = float(np.linalg.norm(r0))
    V = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    V[:, 0] = r0 / beta
    for j in range(k):
        w = spmv(A, V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return V, H, beta, j + 1
        V[:, j + 1] = w / H[j + 1, j]
    return V, H, beta, k


def arnoldi_poly(H, beta, y, t):
    """q(t) = sum_j y_j phi_j(t) for the Arnoldi polynomials phi_j of H (see the module
    docstring); t: array of points."""
    t = np.asarray(t, dtype=np.float64)
    k = y.shape[0]
    phi = [np.full_like(t, 1.0 / beta)]
    for j in range(k - 1):
        nxt = t * phi[j]
        for i in range(j + 1):
            nxt = nxt - H[i, j] * phi[i]
        phi.append(nxt / H[j + 1, j])
    return sum(y[j] * phi[j] for j in range(k))


def poly_from_arnoldi(H, beta, d, alpha, beta_iv):
    """Chebyshev coefficients gamma_0..gamma_d on [alpha, beta_iv] of the GMRES polynomial of
    degree d built from the leading (d+2) x (d+1) block of the Arnoldi H."""
    Hb = H[: d + 2, : d + 1]
    rhs = np.zeros(d + 2)
    rhs[0] = beta
    y = np.linalg.lstsq(Hb, rhs, rcond=None)[0]
    c0, h = 0.5 * (alpha + beta_iv), 0.5 * (beta_iv - alpha)
    ang = np.pi * (np.arange(d + 1) + 0.5) / (d + 1)
    q = arnoldi_poly(H, beta, y, c0 + h * np.cos(ang))
    gamma = np.array([(2.0 - (k == 0)) / (d + 1) * np.sum(q * np.cos(k * ang)) for k in range(d + 1)])
    return gamma, y


def apply_poly(A, gamma, alpha, beta_iv, x):
    """p(A) x = sum_k gamma_k T_k((A - c0 I) / h) x through the oracle's MPK recurrence."""
    d = gamma.shape[0] - 1
    if d == 0:
        return gamma[0] * x
    Y = _mpk(A, d, chebyshev_coeffs(alpha, beta_iv, d), x)
    return sum(gamma[k] * Y[k] for k in range(d + 1))


def harmonic_roots(H, d):
    """Harmonic Ritz values of the leading d + 1 Arnoldi steps (symmetric A): eigenvalues of
    Hbar^T Hbar z = theta S z with Hbar = H[:d+2, :d+1], S the symmetric part of H[:d+1, :d+1];
    Leja-ordered (sstep.leja_order)."""
    import scipy.linalg
    Hb = H[: d + 2, : d + 1]
    Hs = H[: d + 1, : d + 1]
    th = scipy.linalg.eigh(Hb.T @ Hb, 0.5 * (Hs + Hs.T), eigvals_only=True)
    from .sstep import leja_order
    return leja_order(th, d + 1)


def apply_poly_roots(A, roots, x):
    """q(A) x = sum_k (1 / theta_{k+1}) prod_{i<=k} (I - A / theta_i) x through the oracle MPK
    (three-term recurrence with a_k = -1 / theta_k, b_k = 1, c_k = 0)."""
    d = roots.shape[0] - 1
    if d == 0:
        return x / roots[0]
    coeffs = [(-1.0 / roots[k], 1.0, 0.0) for k in range(d)]
    Y = _mpk(A, d, coeffs, x)
    return sum(Y[k] / roots[k] for k in range(d + 1))


def _gmres_cycle(apply_op, r, m, tol_abs):
    """One GMRES(m) cycle on the operator from residual r (classical Gram-Schmidt applied
    twice, as the GPU's single-column cycles).  Returns (V, y, k, H_arnoldi, beta)."""
    n = r.shape[0]
    beta = float(np.linalg.norm(r))
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    Harn = np.zeros((m + 1, m))
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[:, 0] = r / beta
    k = 0
    for j in range(m):
        w = apply_op(V[:, j])
        h = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h
        h2 = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h2
        H[: j + 1, j] = h + h2
        H[j + 1, j] = np.linalg.norm(w)
        Harn[:, j] = H[:, j]
        if H[j + 1, j] != 0.0:
            V[:, j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        a, b = H[j, j], H[j + 1, j]
        rr = np.hypot(a, b)
        cs[j], sn[j] = (1.0, 0.0) if b == 0.0 else (a / rr, b / rr)
        H[j, j] = cs[j] * a + sn[j] * b
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[j + 1]) <= tol_abs or Harn[j + 1, j] == 0.0:
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    return V[:, :k], y, k, Harn, beta


def poly_gmres(A, b, d, m=48, tol=1e-8, max_restarts=500):
    """Right-preconditioned restarted GMRES(m) with the degree-d GMRES polynomial (module
    docstring).  Returns dict(x, iters, converged, gamma, interval, degree)."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b, dtype=np.float64)
    r = b - spmv(A, x)
    # setup cycle on A
    V, y, k, Harn, beta = _gmres_cycle(lambda v: spmv(A, v), r, m, tol * nb)
    x = x + V @ y
    iters = k
    dd = min(d, k - 1)
    Hk = Harn[:k, :k]
    ritz = np.linalg.eigvalsh(0.5 * (Hk + Hk.T))
    interval = (0.0, 1.1 * float(np.max(np.abs(ritz))))
    gamma, _ = poly_from_arnoldi(Harn, beta, dd, *interval)
    P = lambda v: apply_poly(A, gamma, interval[0], interval[1], v)
    for _ in range(max_restarts):
        r = b - spmv(A, x)
        if np.linalg.norm(r) <= tol * nb:
            return dict(x=x, iters=iters, converged=True, gamma=gamma, interval=interval, degree=dd)
        V, y, k, _, _ = _gmres_cycle(lambda v: spmv(A, P(v)), r, m, tol * nb)
        x = x + P(V @ y)
        iters += k
    return dict(x=x, iters=iters, converged=False, gamma=gamma, interval=interval, degree=dd)


def jacobi_sweeps_gmres(A, b, k, m=48, tol=1e-8, max_restarts=500):
    """Right-preconditioned restarted GMRES(m) with P^-1 = k Jacobi sweeps from zero
    (Sec. 5.1: k Jacobi iterations act as a Neumann-series polynomial preconditioner).
    Cycles as in poly_gmres, every cycle preconditioned; returns dict(x, iters, converged)."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b, dtype=np.float64)
    P = lambda v: jacobi_sweeps(A, v, k)
    iters = 0
    for _ in range(max_restarts):
        r = b - spmv(A, x)
        if np.linalg.norm(r) <= tol * nb:
            return dict(x=x, iters=iters, converged=True)
        V, y, kk, _, _ = _gmres_cycle(lambda v: spmv(A, P(v)), r, m, tol * nb)
        x = x + P(V @ y)
        iters += kk
    return dict(x=x, iters=iters, converged=False)
