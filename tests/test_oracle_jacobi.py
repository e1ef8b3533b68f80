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
