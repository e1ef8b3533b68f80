"""Pins for the oracle's right Jacobi preconditioning (Sec. 5.1, Eq. (Jacobi)).

* A D^-1 equals the dense product A @ diag(1 / diag(A)), with unscaled columns where the
  diagonal is missing or zero;
* the MPK of A D^-1 equals dense matrix powers of that product;
* right-preconditioned s-step GMRES reaches the FP64 true residual 1e-8 on the log-normal
  diffusion matrix in fewer iterations than without the scaling."""
import numpy as np
import scipy.sparse as sp

import mpk_inputs as mi
import oracle
from oracle import sstep


def _dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def test_column_scaling_matches_dense():
    for A in (mi.diffusion7_lognormal(6), mi.random_sparse(70, 0.06, 3, symmetric=False, diag=False)):
        M = _dense(A)
        d = np.diag(M).copy()
        want = M @ np.diag(np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 1.0))
        B, dinv = sstep.jacobi_right(A)
        assert np.allclose(_dense(B), want, rtol=1e-15, atol=0)
        assert np.array_equal(B.col, A.col) and np.array_equal(B.row_ptr, A.row_ptr)


def test_mpk_of_scaled_matrix_matches_dense_powers():
    A = mi.diffusion7_lognormal(5)
    B, _ = sstep.jacobi_right(A)
    x = mi.uniform_vectors(A.n, 1)[0]
    Y = oracle.mpk(B, 4, sstep.monomial_coeffs(4), x)
    Mb = _dense(B)
    for k in range(5):
        want = np.linalg.matrix_power(Mb, k) @ x
        assert np.allclose(Y[k], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_jacobi_gmres_converges_in_fewer_iterations():
    A = mi.diffusion7_lognormal(12)
    b = mi.uniform_vectors(A.n, 4)[0]
    plain = sstep.sstep_gmres(A, b, s=8, m=48, tol=1e-8)
    jac = sstep.jacobi_gmres(A, b, s=8, m=48, tol=1e-8)
    assert jac["converged"]
    assert np.linalg.norm(b - sstep.spmv(A, jac["x"])) <= 1e-8 * np.linalg.norm(b)
    assert jac["iters"] < plain["iters"]


def test_one_sweep_is_the_diagonal_scaling():
    A = mi.random_sparse(60, 0.08, 7, symmetric=False, diag=False)
    v = mi.uniform_vectors(A.n, 2)[0]
    _, dinv = sstep.jacobi_right(A)
    assert np.array_equal(sstep.jacobi_sweeps(A, v, 1), dinv * v)


def test_sweeps_equal_the_neumann_series():
    # k sweeps from zero: z_k = sum_{j<k} B^j D^-1 v with B = I - D^-1 A (Sec. 5.1); the zero
    # diagonal of row 3 is read as 1
    A = _zero_diag_small()
    v = mi.uniform_vectors(A.n, 3)[0]
    M = _dense(A)
    d = np.diag(M).copy()
    dt = np.where(d != 0, d, 1.0)
    B = np.eye(A.n) - M / dt[:, None]
    for k in (1, 2, 5, 9):
        want = sum(np.linalg.matrix_power(B, j) @ (v / dt) for j in range(k))
        got = sstep.jacobi_sweeps(A, v, k)
        assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_many_sweeps_solve_a_diagonally_dominant_system():
    # rows of |off-diagonal| sum <= 0.5 |a_ii|: the iteration contracts by 0.5 per sweep
    rng = np.random.default_rng(11)
    n = 50
    M = np.where(rng.random((n, n)) < 0.1, rng.uniform(-1, 1, (n, n)), 0.0)
    np.fill_diagonal(M, 0.0)
    M += np.diag(2.0 * np.abs(M).sum(axis=1) + rng.uniform(0.5, 1.0, n))
    S = sp.csr_matrix(M)
    A = mi.CSR(S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    v = mi.uniform_vectors(n, 4)[0]
    x = np.linalg.solve(M, v)
    z = sstep.jacobi_sweeps(A, v, 60)
    assert np.abs(z - x).max() <= 2 * 0.5 ** 60 * np.abs(x).max() * n + 1e-14


def test_sweeps_preconditioned_gmres():
    from oracle import poly
    A = mi.diffusion7_lognormal(8)
    b = mi.uniform_vectors(A.n, 4)[0]
    one = sstep.jacobi_gmres(A, b, s=8, m=48, tol=1e-8)
    four = poly.jacobi_sweeps_gmres(A, b, 4, m=48, tol=1e-8)
    assert four["converged"]
    assert np.linalg.norm(b - sstep.spmv(A, four["x"])) <= 1e-8 * np.linalg.norm(b)
    assert four["iters"] < one["iters"]


def _zero_diag_small():
    A = mi.poisson2d_5pt(7)
    val = A.val.copy()
    for e in range(A.row_ptr[3], A.row_ptr[4]):
        if A.col[e] == 3:
            val[e] = 0.0
    return mi.CSR(A.row_ptr, A.col, val)
