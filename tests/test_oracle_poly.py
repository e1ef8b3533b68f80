"""Pins for the oracle's GMRES polynomial preconditioner (Sec. 5.2).

* the polynomial applied through its Chebyshev coefficients reproduces the (d+1)-step GMRES
  correction V y, built independently by Arnoldi (same vector, two routes);
* on a matrix with d+1 distinct eigenvalues GMRES is exact after d+1 steps, so A p(A) r0 = r0;
* the Chebyshev evaluation matches numpy.polynomial.chebyshev on a diagonal matrix;
* preconditioned GMRES reaches 1e-8 (true residual) in fewer iterations than plain GMRES and
  agrees with numpy.linalg.solve."""
import numpy as np
import scipy.sparse as sp

import mpk_inputs as mi
from oracle import poly, sstep


def _dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def _diag(d):
    n = d.shape[0]
    return mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.astype(np.float64))


def test_polynomial_reproduces_gmres_correction():
    A = mi.poisson2d_5pt(12)
    r0 = mi.uniform_vectors(A.n, 3)[0]
    for d in (4, 9, 15):
        V, H, beta, steps = poly.arnoldi(A, r0, d + 1)
        assert steps == d + 1
        rhs = np.zeros(d + 2)
        rhs[0] = beta
        y = np.linalg.lstsq(H[: d + 2, : d + 1], rhs, rcond=None)[0]
        corr = V[:, : d + 1] @ y                       # x_{d+1} - x_0 of GMRES
        lam = np.linalg.eigvalsh(_dense(A))
        interval = (0.0, 1.1 * lam.max())
        gamma, _ = poly.poly_from_arnoldi(H, beta, d, *interval)
        got = poly.apply_poly(A, gamma, interval[0], interval[1], r0)
        assert np.linalg.norm(got - corr) <= 1e-9 * np.linalg.norm(corr), d


def test_exact_inverse_on_a_small_spectrum():
    ev = np.array([1.0, 2.5, 4.0, 7.0, 9.5])
    A = _diag(np.repeat(ev, 10))
    r0 = mi.uniform_vectors(A.n, 4)[0]
    d = ev.size - 1
    V, H, beta, steps = poly.arnoldi(A, r0, d + 1)
    gamma, _ = poly.poly_from_arnoldi(H, beta, d, 0.0, 11.0)
    z = poly.apply_poly(A, gamma, 0.0, 11.0, r0)
    res = r0 - sstep.spmv(A, z)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(r0)


def test_chebyshev_evaluation_matches_numpy():
    rng = np.random.default_rng(5)
    t = rng.uniform(0.2, 7.8, 40)
    A = _diag(t)
    x = mi.uniform_vectors(A.n, 6)[0]
    gamma = rng.standard_normal(9)
    got = poly.apply_poly(A, gamma, 0.0, 8.0, x)
    want = np.polynomial.chebyshev.chebval((t - 4.0) / 4.0, gamma) * x
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_arnoldi_poly_is_the_krylov_combination():
    """phi_j(A) r0 = v_j for the Arnoldi polynomials (recurrence of the module docstring)."""
    A = mi.random_sparse(80, 0.05, 7, symmetric=True)
    r0 = mi.uniform_vectors(A.n, 8)[0]
    V, H, beta, steps = poly.arnoldi(A, r0, 6)
    M = _dense(A)
    w, Q = np.linalg.eigh(M)
    c = Q.T @ r0
    for j in range(steps):
        e = np.zeros(steps)
        e[j] = 1.0
        vj = Q @ (poly.arnoldi_poly(H, beta, e, w) * c)   # phi_j(A) r0 through the eigenbasis
        assert np.allclose(vj, V[:, j], atol=1e-9)


def test_preconditioned_gmres_converges_faster():
    A = mi.poisson2d_5pt(24)
    b = mi.uniform_vectors(A.n, 2)[0]
    plain = sstep.gmres(A, b, m=20, tol=1e-8)
    pre = poly.poly_gmres(A, b, d=10, m=20, tol=1e-8)
    assert pre["converged"] and plain["converged"]
    assert np.linalg.norm(b - sstep.spmv(A, pre["x"])) <= 1e-8 * np.linalg.norm(b)
    assert pre["iters"] < plain["iters"] / 2
    xs = np.linalg.solve(_dense(A), b)
    assert np.linalg.norm(pre["x"] - xs) <= np.linalg.cond(_dense(A)) * 2e-8 * np.linalg.norm(xs)


def test_root_form_is_the_same_polynomial():
    """The Leja-ordered harmonic-Ritz product form and the Chebyshev form evaluate the same q."""
    for A, d in ((mi.poisson2d_5pt(14), 10), (mi.diffusion7_lognormal(8), 12), (mi.anisotropic(7, 27, 5.0), 8)):
        r0 = mi.uniform_vectors(A.n, 3)[0]
        V, H, beta, steps = poly.arnoldi(A, r0, d + 1)
        lam = np.linalg.eigvalsh(_dense(A))
        interval = (0.0, 1.1 * lam.max())
        gamma, _ = poly.poly_from_arnoldi(H, beta, d, *interval)
        z1 = poly.apply_poly(A, gamma, interval[0], interval[1], r0)
        z2 = poly.apply_poly_roots(A, poly.harmonic_roots(H, d), r0)
        assert np.linalg.norm(z1 - z2) <= 1e-8 * np.linalg.norm(z1), d
        # 1 - A q(A) r0 is the GMRES residual of d + 1 steps
        corr = V[:, : d + 1] @ np.linalg.lstsq(H[: d + 2, : d + 1], np.eye(d + 2)[0] * beta, rcond=None)[0]
        assert np.linalg.norm(z2 - corr) <= 1e-8 * np.linalg.norm(corr)
