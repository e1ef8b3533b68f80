"""Textbook GMRES, s-step GMRES and their building blocks in FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow and plain on purpose: every step
follows the paper's Alg. 3 in order, with the Newton basis of Sec. 4 and the standard
CA-GMRES reconstruction of the Hessenberg matrix from the block QR factors (the paper cites
Hoemmen's thesis for the method and defers details to it).

Readings of points the paper leaves open (all listed with the design notes):
* shifts: Ritz values of the first restart cycle, which is plain GMRES(m); real parts taken;
  the first s of them in Leja order (first = largest modulus, then each next maximises the
  product of distances to those chosen, ties -> smaller value);
* BOrtho: one block classical Gram-Schmidt pass (optionally two); TSQR: CholQR2;
* convergence: checked after every column of each block from the Givens residual estimate.
"""
from __future__ import annotations

import numpy as np

from . import mpk as _mpk

__all__ = [
    "Breakdown", "spmv", "monomial_coeffs", "newton_coeffs", "chebyshev_coeffs", "leja_order",
    "cholqr2", "gmres", "sstep_gmres", "refine_solve", "ritz_values",
]


class Breakdown(RuntimeError):
    """Cholesky of a Gram matrix met a non-positive pivot."""


def spmv(A, x):
    """y = A x through the oracle's plain CSR loop (Alg. 2 with one power)."""
    return _mpk(A, 1, [(1.0, 0.0, 0.0)], x)[1]


def monomial_coeffs(p):
    """Alg. 1: y_k = A y_{k-1}."""
    return [(1.0, 0.0, 0.0)] * p


def newton_coeffs(theta):
    """Sec. 4 Newton basis in product form: y_k = (A - theta_k I) y_{k-1}."""
    return [(1.0, -float(t), 0.0) for t in theta]


def chebyshev_coeffs(alpha, beta, p):
    """Chebyshev basis on [alpha, beta]: y_k = T_k((A - c0 I)/d) x with c0 = (beta+alpha)/2,
    d = (beta-alpha)/2, from T_1(z) = z and T_k(z) = 2 z T_{k-1}(z) - T_{k-2}(z)."""
    c0 = 0.5 * (beta + alpha)
    d = 0.5 * (beta - alpha)
    out = []
    for k in range(1, p + 1):
        if k == 1:
            out.append((1.0 / d, -c0 / d, 0.0))
        else:
            out.append((2.0 / d, -2.0 * c0 / d, -1.0))
    return out


def leja_order(values, count):
    """First ``count`` points of a finite real set in Leja order (ties -> smaller value).
    The product of distances is compared through a sum of logs of absolute differences."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return v
    chosen = []
    mag = np.abs(v)
    first = int(np.flatnonzero(mag == mag.max())[0])
    chosen.append(first)
    score = np.zeros(v.size)
    while len(chosen) < min(count, v.size):
        with np.errstate(divide="ignore"):
            score += np.log(np.abs(v - v[chosen[-1]]))
        s = score.copy()
        s[chosen] = -np.inf
        best = s.max()
        if best == -np.inf:
            break
        chosen.append(int(np.flatnonzero(s == best)[0]))
    out = v[chosen]
    # fewer distinct candidates than requested: repeat the order
    while out.size < count:
        out = np.concatenate([out, out[: count - out.size]])
    return out


def _chol_upper(G):
    """Upper R with R^T R = G (plain Cholesky); raises Breakdown on a pivot <= 0."""
    s = G.shape[0]
    R = np.zeros_like(G)
    for i in range(s):
        d = G[i, i] - R[:i, i] @ R[:i, i]
        if not d > 0.0:
            raise Breakdown("non-positive pivot %d" % i)
        R[i, i] = np.sqrt(d)
        for j in range(i + 1, s):
            R[i, j] = (G[i, j] - R[:i, i] @ R[:i, j]) / R[i, i]
    return R


def cholqr2(W):
    """CholQR applied twice: W = Q R with Q^T Q = I, R upper triangular, positive diagonal.
    (TSQR step of Alg. 3c, replaced by CholQR2.)"""
    R1 = _chol_upper(W.T @ W)
    Q1 = np.linalg.solve(R1.T, W.T).T
    R2 = _chol_upper(Q1.T @ Q1)
    Q = np.linalg.solve(R2.T, Q1.T).T
    return Q, R2 @ R1


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def ritz_values(H, k):
    """Real parts of the eigenvalues of the leading k x k block of an Arnoldi H."""
    if k == 0:
        return np.zeros(0)
    return np.real(np.linalg.eigvals(H[:k, :k]))


def gmres(A, b, x0=None, m=30, tol=1e-8, max_restarts=1000, cgs=False, precond=None):
    """Restarted GMRES(m), Alg. 3(a)+(b): Arnoldi with modified (or classical) Gram-Schmidt,
    Givens rotations, residual check after each column.  Stops when the estimated residual
    norm is <= tol * ||b||.  ``precond`` (a function v -> P^-1 v) makes it right-preconditioned:
    the Arnoldi operator is A P^-1 and the correction is P^-1 (Q y).
    Returns dict(x, iters, hist, H_first, k_first, converged)."""
    M = precond if precond is not None else (lambda v: v)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    nb = np.linalg.norm(b)
    hist = []
    iters = 0
    H_first, k_first = None, 0
    for cycle in range(max_restarts):
        r = b - spmv(A, x)
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta <= tol * nb:
            return dict(x=x, iters=iters, hist=hist, H_first=H_first, k_first=k_first,
                        converged=True)
        Q = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        Harn = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        k = 0
        for j in range(m):
            w = spmv(A, M(Q[:, j]))
            if cgs:
                h = Q[:, : j + 1].T @ w
                w = w - Q[:, : j + 1] @ h
                H[: j + 1, j] = h
            else:
                for i in range(j + 1):
                    H[i, j] = Q[:, i] @ w
                    w = w - H[i, j] * Q[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            Harn[:, j] = H[:, j]
            if H[j + 1, j] != 0.0:
                Q[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            iters += 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) <= tol * nb:
                break
        if cycle == 0:
            H_first, k_first = Harn, k
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + M(Q[:, :k] @ y)
    return dict(x=x, iters=iters, hist=hist, H_first=H_first, k_first=k_first, converged=False)


def sstep_gmres(A, b, x0=None, s=4, m=48, tol=1e-8, max_restarts=1000, shifts=None,
                bcgs_passes=1, basis="newton", precond=None):
    """Restarted s-step GMRES, Alg. 3(a)+(c).

    Per block of s columns starting at basis column j: the MPK builds
    V = [q_j, (A - th_1) q_j, ...] (Newton, Sec. 4) or the monomial basis; BOrtho removes the
    previous basis (block classical Gram-Schmidt, ``bcgs_passes`` sweeps); TSQR = CholQR2
    gives the new orthonormal columns and R; the Hessenberg columns follow from
        H R_s = R_full B,
    with R_full the coefficients of [q_j, v_1..v_s] in the new basis, B the (s+1) x s change
    of basis (shifts on the diagonal, ones below), R_s = R_full without its last row and
    column; then Givens rotations update the least-squares residual.

    Without ``shifts`` the first cycle runs plain GMRES(m) and its Ritz values give the
    shifts (Sec. 4).  ``precond`` (v -> P^-1 v) makes it right-preconditioned: the basis is
    that of A P^-1, y_k = (A P^-1 - theta_k I) y_{k-1}, and x += P^-1 (Q y).
    Returns dict(x, iters, hist, shifts, converged, block_hist, H_cycle, k_cycle): H_cycle is
    the unrotated Arnoldi Hessenberg ((m+1) x m) of the first s-step cycle and k_cycle its
    columns (None, 0 when no s-step cycle ran)."""
    M = precond if precond is not None else (lambda v: v)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    nb = np.linalg.norm(b)
    hist = []
    block_hist = []
    iters = 0
    cycle0 = 0
    H_cycle, k_cycle = None, 0
    if basis == "newton" and shifts is None:
        r0 = gmres(A, b, x, m=m, tol=tol, max_restarts=1, precond=precond)
        x = r0["x"]
        iters += r0["iters"]
        hist.extend(r0["hist"][1:])
        rv = ritz_values(r0["H_first"], r0["k_first"])
        shifts = leja_order(rv, s)
        cycle0 = 1
        if r0["converged"]:
            return dict(x=x, iters=iters, hist=hist, shifts=shifts, converged=True,
                        block_hist=block_hist, H_cycle=H_cycle, k_cycle=k_cycle)
    if basis == "monomial":
        theta = np.zeros(s)
    else:
        theta = np.asarray(shifts, dtype=np.float64)[:s]
    for cycle in range(cycle0, max_restarts):
        r = b - spmv(A, x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            return dict(x=x, iters=iters, hist=hist, shifts=theta, converged=True,
                        block_hist=block_hist, H_cycle=H_cycle, k_cycle=k_cycle)
        Q = np.zeros((n, m + 1))
        Harn = np.zeros((m + 1, m))   # Arnoldi H (kept unrotated for the reconstruction)
        H = np.zeros((m + 1, m))      # H with the Givens rotations applied
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        k = 0
        done = False
        j = 0
        while j < m and not done:
            S = min(s, m - j)
            if precond is None:
                V = _mpk(A, S, newton_coeffs(theta[:S]), Q[:, j])
            else:
                V = np.zeros((S + 1, n))
                V[0] = Q[:, j]
                for i in range(S):
                    V[i + 1] = spmv(A, M(V[i])) - theta[i] * V[i]
            W = V[1:].T.copy()
            C = np.zeros((j + 1, S))
            for _ in range(bcgs_passes):
                Ck = Q[:, : j + 1].T @ W
                W = W - Q[:, : j + 1] @ Ck
                C += Ck
            Qh, Rh = cholqr2(W)
            Q[:, j + 1: j + 1 + S] = Qh
            Rfull = np.zeros((j + 1 + S, S + 1))
            Rfull[j, 0] = 1.0
            Rfull[: j + 1, 1:] = C
            Rfull[j + 1:, 1:] = Rh
            Bm = np.zeros((S + 1, S))
            for i in range(S):
                Bm[i, i] = theta[i]
                Bm[i + 1, i] = 1.0
            Rs = Rfull[: j + S, :S]
            rhs = Rfull @ Bm
            if j > 0:
                rhs -= Harn[: j + S + 1, :j] @ Rs[:j, :]
            T = Rs[j: j + S, :]
            Hnew = np.linalg.solve(T.T, rhs.T).T
            # the columns are Hessenberg: drop what sits below the subdiagonal
            for c in range(S):
                Hnew[j + c + 2:, c] = 0.0
            Harn[: j + S + 1, j: j + S] = Hnew
            H[: j + S + 1, j: j + S] = Hnew
            for c in range(j, j + S):
                for i in range(c):
                    t = cs[i] * H[i, c] + sn[i] * H[i + 1, c]
                    H[i + 1, c] = -sn[i] * H[i, c] + cs[i] * H[i + 1, c]
                    H[i, c] = t
                cs[c], sn[c] = _givens(H[c, c], H[c + 1, c])
                H[c, c] = cs[c] * H[c, c] + sn[c] * H[c + 1, c]
                H[c + 1, c] = 0.0
                g[c + 1] = -sn[c] * g[c]
                g[c] = cs[c] * g[c]
                k = c + 1
                iters += 1
                hist.append(abs(g[c + 1]) / nb)
                if abs(g[c + 1]) <= tol * nb:
                    done = True
                    break
            block_hist.append(abs(g[k]) / nb)
            j += S
        if H_cycle is None:
            H_cycle, k_cycle = Harn.copy(), k
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + M(Q[:, :k] @ y)
    r = b - spmv(A, x)
    return dict(x=x, iters=iters, hist=hist, shifts=theta,
                converged=bool(np.linalg.norm(r) <= tol * nb), block_hist=block_hist,
                H_cycle=H_cycle, k_cycle=k_cycle)


def refine_solve(A, b, tol=1e-8, s=8, m=48, inner_tol=1e-5, max_outer=50, inner_cycles=1,
                 shifts=None, round_inner=None):
    """FP64 iterative refinement around an inner s-step GMRES solve:
    r = b - A x (FP64); solve A d = r to inner_tol (at most ``inner_cycles`` restart cycles);
    x += d; until ||r|| <= tol ||b||.  ``round_inner`` (e.g. np.float32) rounds the inner
    right-hand side and correction to that type, emulating a lower-precision inner solve.
    Returns dict(x, outer, inner_iters, relres, shifts)."""
    n = b.shape[0]
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    inner_iters = 0
    relres = []
    th = shifts
    for outer in range(max_outer):
        r = b - spmv(A, x)
        rr = np.linalg.norm(r) / nb
        relres.append(rr)
        if rr <= tol:
            return dict(x=x, outer=outer, inner_iters=inner_iters, relres=relres, shifts=th)
        rhs = r.astype(round_inner).astype(np.float64) if round_inner else r
        res = sstep_gmres(A, rhs, None, s=s, m=m, tol=inner_tol, max_restarts=inner_cycles,
                          shifts=th)
        th = res["shifts"]
        d = res["x"].astype(round_inner).astype(np.float64) if round_inner else res["x"]
        inner_iters += res["iters"]
        x = x + d
    r = b - spmv(A, x)
    relres.append(np.linalg.norm(r) / nb)
    return dict(x=x, outer=max_outer, inner_iters=inner_iters, relres=relres, shifts=th)


def jacobi_right(A):
    """Sec. 5.1, Eq. (Jacobi) with one iteration from zero: the diagonal preconditioner
    P^-1 = D^-1 applied from the right, as the paper fuses it into the SpMV (A D^-1, a scaling
    along the columns).  Returns (A D^-1 as a CSR with the same pattern, dinv) where dinv_j =
    1 / a_jj, and 1 where the diagonal entry is missing or zero (no scaling of that column)."""
    n = A.n
    d = np.zeros(n)
    for i in range(n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col[e] == i:
                d[i] += A.val[e]
    dinv = np.where(d != 0.0, 1.0 / np.where(d != 0.0, d, 1.0), 1.0)
    val = A.val * dinv[A.col]
    from mpk_inputs import CSR
    return CSR(A.row_ptr.copy(), A.col.copy(), val), dinv


def jacobi_gmres(A, b, s=8, m=48, tol=1e-8, max_restarts=1000):
    """s-step GMRES on A D^-1 u = b, x = D^-1 u (right Jacobi preconditioning: the GMRES
    residual is the true residual)."""
    B, dinv = jacobi_right(A)
    out = sstep_gmres(B, b, s=s, m=m, tol=tol, max_restarts=max_restarts)
    out = dict(out)
    out["x"] = dinv * out["x"]
    return out


def jacobi_sweeps(A, v, k):
    """k Jacobi iterations from z^0 = 0 for P^-1 v (Sec. 5.1, Eq. (Jacobi)):
        z^{j+1} = D^-1 v - D^-1 (L + U) z^j,
    L + U the off-diagonal entries of A, D its diagonal.  Reading for a zero (or missing)
    diagonal entry: D is taken with that entry replaced by 1, i.e. the splitting is
    A = D~ + (A - D~); the extra term (D - D~) z joins L + U there."""
    n = A.n
    d = np.zeros(n)
    for i in range(n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col[e] == i:
                d[i] += A.val[e]
    dt = np.where(d != 0.0, d, 1.0)
    z = np.zeros(n)
    for _ in range(k):
        lu = np.zeros(n)
        for i in range(n):
            for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
                if A.col[e] != i:
                    lu[i] += A.val[e] * z[A.col[e]]
        lu += (d - dt) * z
        z = v / dt - lu / dt
    return z
