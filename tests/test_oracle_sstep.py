"""Pins for the oracle's s-step GMRES pieces (Alg. 3, Sec. 4 Newton basis, CholQR2 for TSQR,
Leja shifts, Chebyshev basis, FP64 refinement).

Checked against: numpy.linalg.qr and numpy.linalg.solve (library special cases), closed forms
on diagonal matrices (T_k(cos phi) = cos(k phi); Newton products), brute-force products of
distances for the Leja order, and the algorithm identities s=1 == classical Gram-Schmidt
GMRES and s-step == GMRES at block boundaries in exact arithmetic."""
import itertools

import numpy as np
import pytest

import mpk_inputs as mi
import oracle
from oracle import sstep


def diag_csr(d):
    n = len(d)
    return mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                  np.asarray(d, dtype=np.float64))


def test_cholqr2_vs_numpy_qr():
    rng = np.random.default_rng(0)
    W = rng.standard_normal((500, 8)) @ np.diag([1, 2, 5, 10, 1e2, 1e3, 1e-1, 3])
    Q, R = sstep.cholqr2(W)
    assert np.linalg.norm(Q.T @ Q - np.eye(8)) <= 1e-12
    assert np.linalg.norm(Q @ R - W) / np.linalg.norm(W) <= 1e-13
    assert np.allclose(np.triu(R), R) and np.all(np.diag(R) > 0)
    Qn, Rn = np.linalg.qr(W)
    sgn = np.sign(np.diag(Rn))
    assert np.allclose(R, sgn[:, None] * Rn, rtol=1e-10, atol=1e-10 * np.abs(Rn).max())


def test_cholqr_breakdown():
    W = np.ones((20, 3))
    with pytest.raises(sstep.Breakdown):
        sstep.cholqr2(W)


def test_chebyshev_closed_form_on_diagonal():
    """A = diag(cos phi_i) on [-1, 1]: y_k = T_k(A) x = cos(k phi) x; and on [alpha, beta] the
    map z = (lambda - c0)/d sends a diagonal entry alpha + d(1 + cos phi) to cos phi."""
    phi = np.linspace(0.05, 3.1, 37)
    x = mi.uniform_vectors(37, 1)[0]
    Y = oracle.mpk(diag_csr(np.cos(phi)), 6, sstep.chebyshev_coeffs(-1.0, 1.0, 6), x)
    for k in range(7):
        assert np.allclose(Y[k], np.cos(k * phi) * x, rtol=1e-13, atol=1e-14)
    alpha, beta = 0.1, 52.0
    d = 0.5 * (beta - alpha)
    Y = oracle.mpk(diag_csr(alpha + d * (1 + np.cos(phi))), 6,
                   sstep.chebyshev_coeffs(alpha, beta, 6), x)
    for k in range(7):
        assert np.allclose(Y[k], np.cos(k * phi) * x, rtol=1e-12, atol=1e-12)


def test_newton_closed_form_on_diagonal():
    dvals = np.linspace(-2, 5, 23)
    th = mi.leja_points_interval(0, 52, 8)
    x = mi.uniform_vectors(23, 2)[0]
    Y = oracle.mpk(diag_csr(dvals), 8, sstep.newton_coeffs(th), x)
    prod = np.ones(23)
    for k in range(8):
        prod = prod * (dvals - th[k])
        assert np.allclose(Y[k + 1], prod * x, rtol=1e-13, atol=0)


def _leja_brute(vals, count):
    """Greedy max-product by direct products (no logs), ties to the smaller value."""
    v = sorted(vals)
    first = max(v, key=lambda t: (abs(t), -t))
    out = [first]
    while len(out) < count:
        best, bestp = None, -1.0
        for t in v:
            if t in out:
                continue
            pr = np.prod([abs(t - u) for u in out])
            if pr > bestp:
                best, bestp = t, pr
        out.append(best)
    return np.array(out)


def test_leja_order_brute_force():
    rng = np.random.default_rng(4)
    for trial in range(5):
        vals = np.unique(np.round(rng.uniform(0.1, 50, size=12), 3))
        assert np.array_equal(sstep.leja_order(vals, 6), _leja_brute(vals, 6))
    # the interval version used for fixed shifts: first point = 52, then 0, then the midpoint
    th = mi.leja_points_interval(0, 52, 3)
    assert th[0] == 52.0 and th[1] == 0.0 and abs(th[2] - 26.0) < 1e-12


def test_gmres_small_vs_solve():
    """n <= 64: restarted GMRES and s-step GMRES reach x = A^-1 b (numpy.linalg.solve) to
    within cond(A) * 1e-8."""
    A = mi.random_sparse(60, 0.1, 3, symmetric=True)
    M = np.zeros((60, 60))
    for i in range(60):
        M[i, A.col[A.row_ptr[i]:A.row_ptr[i + 1]]] = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
    b = mi.uniform_vectors(60, 5)[0]
    xs = np.linalg.solve(M, b)
    kappa = np.linalg.cond(M)
    for res in (sstep.gmres(A, b, m=20, tol=1e-10),
                sstep.sstep_gmres(A, b, s=4, m=20, tol=1e-10),
                sstep.sstep_gmres(A, b, s=5, m=20, tol=1e-10, bcgs_passes=2)):
        assert res["converged"]
        assert np.linalg.norm(res["x"] - xs) <= kappa * 1e-8 * np.linalg.norm(xs)


def test_s1_equals_classical_gs_gmres():
    """s=1 with the monomial basis is classical Gram-Schmidt GMRES: identical residual
    estimates within 1e-10 relative over the first restart cycle."""
    A = mi.stencil7(8, 1, 1, 4.0)
    b = mi.uniform_vectors(A.n, 4)[0]
    r1 = sstep.sstep_gmres(A, b, s=1, m=30, tol=1e-14, max_restarts=1, basis="monomial")
    r2 = sstep.gmres(A, b, m=30, tol=1e-14, max_restarts=1, cgs=True)
    h1 = np.array(r1["hist"])
    h2 = np.array(r2["hist"][1:])
    assert len(h1) == len(h2) == 30
    assert np.max(np.abs(h1 - h2) / h2) <= 1e-10


@pytest.mark.parametrize("s", [2, 4, 8])
def test_sstep_matches_gmres_at_block_boundaries(s):
    """In exact arithmetic s-step GMRES iterates equal GMRES's at iterations j+s; with an FP64
    basis at small n the block-boundary residuals agree within 1e-6 relative."""
    A = mi.stencil7(8, 1, 1, 2.0)
    b = mi.uniform_vectors(A.n, 6)[0]
    th = mi.leja_points_interval(0.1, 16.0, s)
    r1 = sstep.sstep_gmres(A, b, s=s, m=24, tol=1e-14, max_restarts=1, shifts=th)
    r2 = sstep.gmres(A, b, m=24, tol=1e-14, max_restarts=1)
    h2 = np.array(r2["hist"][1:])
    for q, bh in enumerate(r1["block_hist"]):
        it = min((q + 1) * s, 24)
        assert abs(bh - h2[it - 1]) <= 1e-6 * h2[it - 1]


def test_sstep_true_residual_and_shifts_from_ritz():
    """Default path: first cycle = GMRES(m), its Ritz values Leja-ordered become the shifts;
    the final true residual (FP64 oracle SpMV) is <= 1e-8 ||b||."""
    A = mi.diffusion7_lognormal(10, permute=True)
    b = mi.uniform_vectors(A.n, 4)[0]
    res = sstep.sstep_gmres(A, b, s=8, m=48, tol=1e-8)
    assert res["converged"]
    r = b - sstep.spmv(A, res["x"])
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)
    th = res["shifts"]
    assert len(th) == 8 and abs(th[0]) == np.max(np.abs(th))


def test_refinement_reaches_1e8_with_fp32_inner():
    A = mi.anisotropic(10, 27, 10.0)
    b = mi.uniform_vectors(A.n, 9)[0]
    res = sstep.refine_solve(A, b, tol=1e-8, s=8, m=48, round_inner=np.float32)
    assert res["relres"][-1] <= 1e-8
    assert res["outer"] <= 10
