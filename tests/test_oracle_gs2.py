"""Pins for the oracle's two-stage Gauss-Seidel (GS2) preconditioner and the MPK of the
GS2-preconditioned operator (Sec. 5.1, GS2 part, Alg. GS2).

Each pin comes from outside the oracle's own loops:
* gamma = 0 is the diagonal scaling D^-1 v (division by the dense diagonal);
* D^-1 L is strictly lower triangular, hence nilpotent, so gamma >= n - 1 inner iterations
  solve (L + D) z = v exactly: a dense triangular solve (SciPy) pins it;
* for any gamma, g_gamma is the truncated Neumann series sum_{i<=gamma} (-D^-1 L)^i D^-1 v
  (dense matrix powers);
* from a nonzero z0 with exact inner solves one GS2 iteration is one Gauss-Seidel sweep
  z1 = (L + D)^-1 (v - U z0);
* the MPK equals the dense recurrence with the dense GS2 matrix;
* right-preconditioned s-step GMRES reaches the FP64 true residual 1e-8 and matches
  numpy.linalg.solve, in fewer iterations than without the preconditioner;
* a planted sign mistake in the inner update is caught by the triangular-solve pin.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import mpk_inputs as mi
from oracle import gs2, sstep


def _dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def _parts(A):
    M = _dense(A)
    d = np.diag(M).copy()
    dt = np.where(d != 0.0, d, 1.0)
    return M, np.tril(M, -1), np.diag(dt), np.triu(M, 1) + np.diag(d - dt)


def _gs2_dense(A, gamma):
    M, L, Dt, _ = _parts(A)
    Di = np.diag(1.0 / np.diag(Dt))
    T = -Di @ L
    G = np.zeros_like(M)
    P = np.eye(A.n)
    for _ in range(gamma + 1):
        G += P @ Di
        P = T @ P
    return G


MATS = [
    ("diff7_5", lambda: mi.diffusion7_lognormal(5)),
    ("rand_nonsym", lambda: mi.random_sparse(50, 0.08, 11, symmetric=False, diag=True)),
    ("rand_zero_diag", lambda: mi.random_sparse(40, 0.1, 5, symmetric=False, diag=False)),
]


def test_gamma0_is_the_diagonal_scaling():
    for _, f in MATS:
        A = f()
        v = mi.uniform_vectors(A.n, 3)[0]
        _, _, Dt, _ = _parts(A)
        assert np.array_equal(gs2.gs2_apply(A, v, 0), v / np.diag(Dt))


def test_enough_inner_iterations_solve_the_lower_triangle_exactly():
    for _, f in MATS:
        A = f()
        v = mi.uniform_vectors(A.n, 4)[0]
        _, L, Dt, _ = _parts(A)
        want = sla.solve_triangular(L + Dt, v, lower=True)
        got = gs2.gs2_apply(A, v, A.n - 1)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_truncated_neumann_series():
    for _, f in MATS:
        A = f()
        v = mi.uniform_vectors(A.n, 5)[0]
        for gamma in (1, 2, 3, 5):
            want = _gs2_dense(A, gamma) @ v
            got = gs2.gs2_apply(A, v, gamma)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), gamma


def test_exact_inner_solve_from_nonzero_start_is_one_gauss_seidel_sweep():
    A = mi.random_sparse(45, 0.1, 9, symmetric=False, diag=True)
    v = mi.uniform_vectors(A.n, 6)[0]
    z0 = mi.uniform_vectors(A.n, 7)[0]
    _, L, Dt, U = _parts(A)
    want = sla.solve_triangular(L + Dt, v - U @ z0, lower=True)
    got = gs2.gs2_apply(A, v, A.n - 1, z0=z0)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_mpk_equals_the_dense_recurrence():
    A = mi.diffusion7_lognormal(5)
    x = mi.uniform_vectors(A.n, 1)[0]
    M = _dense(A)
    for gamma in (0, 1, 2):
        G = _gs2_dense(A, gamma)
        for coeffs in (sstep.newton_coeffs([0.3, 1.7, 0.9, 1.2]), sstep.chebyshev_coeffs(0.1, 2.0, 4)):
            Y = gs2.gs2_mpk(A, 4, coeffs, x, gamma)
            want = [x, None]
            for k in range(1, 5):
                a, b, c = coeffs[k - 1]
                w = a * (M @ (G @ want[k - 1])) + b * want[k - 1]
                if k >= 2:
                    w = w + c * want[k - 2]
                want[k:k + 1] = [w, None]
            for k in range(5):
                assert np.allclose(Y[k], want[k], rtol=1e-12, atol=1e-12 * np.abs(want[k]).max())


def test_gs2_gmres_converges_to_the_solution():
    A = mi.diffusion7_lognormal(8)
    b = mi.uniform_vectors(A.n, 4)[0]
    x_ref = np.linalg.solve(_dense(A), b)
    plain = sstep.sstep_gmres(A, b, s=4, m=24, tol=1e-8)
    for gamma in (1, 2):
        out = gs2.gs2_gmres(A, b, gamma, s=4, m=24, tol=1e-8)
        assert out["converged"]
        assert np.linalg.norm(b - sstep.spmv(A, out["x"])) <= 1e-8 * np.linalg.norm(b)
        kappa = np.linalg.cond(_dense(A))
        assert np.linalg.norm(out["x"] - x_ref) <= kappa * 2e-8 * np.linalg.norm(x_ref)
        assert out["iters"] < plain["iters"]


def test_planted_sign_mistake_is_caught():
    A = mi.random_sparse(30, 0.12, 2, symmetric=False, diag=True)
    v = mi.uniform_vectors(A.n, 8)[0]
    _, L, Dt, _ = _parts(A)
    want = sla.solve_triangular(L + Dt, v, lower=True)
    lower, d, dt, upper = gs2.split_ldu(A)
    # the inner update with + instead of -: g_j = g_0 + D^-1 L g_{j-1}
    g0 = v / dt
    g = g0
    for _ in range(A.n - 1):
        lg = np.zeros(A.n)
        for i in range(A.n):
            for j, a in lower[i]:
                lg[i] += a * g[j]
        g = g0 + lg / dt
    assert not np.allclose(g, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())
