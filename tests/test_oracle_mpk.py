"""Pins for the oracle's MPK (Alg. 1 + Alg. 2, three-term recurrence).

Each check compares the oracle with something it does not compute itself: exact rational
arithmetic, the sine eigenvectors of the Dirichlet Laplacian, a DST-I expansion (library
special case), dense brute force, or the structure of the recurrence.  The planted-mistake
tests show that a plausible bug (dropped term, transposed operand, wrong sign, wrong index)
fails at least one of these checks."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft
import scipy.sparse

import mpk_inputs as mi
import oracle
from oracle import sstep

U = 2.0 ** -53


def dense(A):
    n = A.n
    M = np.zeros((n, n))
    for i in range(n):
        for t in range(A.row_ptr[i], A.row_ptr[i + 1]):
            M[i, A.col[t]] += A.val[t]
    return M


def abs_bound(A, p, coeffs, x):
    """(|A_theta|^k |x|) per power: the denominators of the relative error metric."""
    M = abs(scipy.sparse.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)))
    out = [np.abs(x)]
    for k in range(1, p + 1):
        a, b, c = coeffs[k - 1]
        prev = out[-1]
        prev2 = out[-2] if k >= 2 else np.zeros_like(x)
        out.append(abs(a) * (M @ prev) + abs(b) * prev + abs(c) * prev2)
    return np.array(out)


def exact_mpk(A, p, coeffs, x):
    """Exact rational y_k for dyadic inputs (floats convert to Fraction exactly)."""
    n = A.n
    vals = [Fraction(float(v)) for v in A.val]
    ys = [[Fraction(float(v)) for v in x]]
    cf = [(Fraction(a), Fraction(b), Fraction(c)) for a, b, c in coeffs]
    for k in range(1, p + 1):
        a, b, c = cf[k - 1]
        y1 = ys[-1]
        y2 = ys[-2] if k >= 2 else [Fraction(0)] * n
        yk = []
        for i in range(n):
            acc = Fraction(0)
            for t in range(A.row_ptr[i], A.row_ptr[i + 1]):
                acc += vals[t] * y1[A.col[t]]
            yk.append(a * acc + b * y1[i] + c * y2[i])
        ys.append(yk)
    return ys


def test_c1_exact_rational():
    """2-D Poisson 64x64, p=4 monomial, x ~ U[-1,1) seed 0: the oracle is within
    64*k*2^-53 * (|A|^k|x|)_i of the exact rational A^k x (computed with Fractions)."""
    A = mi.poisson2d_5pt(64)
    x = mi.uniform_vectors(A.n, 0)[0]
    p = 4
    cf = sstep.monomial_coeffs(p)
    Y = oracle.mpk(A, p, cf, x)
    ex = exact_mpk(A, p, cf, x)
    den = abs_bound(A, p, cf, x)
    for k in range(1, p + 1):
        exk = np.array([float(v) for v in ex[k]])
        err = np.abs(Y[k] - exk)
        assert np.all(err <= 64 * k * U * den[k]), k
        # and it is far tighter than the bound: a few ulps of the magnitude
        assert np.max(err / den[k]) < 8 * k * U


def sine_mode(N, j, k):
    r = np.arange(N)
    return np.outer(np.sin(j * np.pi * (r + 1) / (N + 1)), np.sin(k * np.pi * (r + 1) / (N + 1))).ravel()


def test_c1_sine_eigenvectors():
    """A^p v = lambda^p v for the Dirichlet-Laplacian eigenvectors
    v_jk(r,c) = sin(j pi (r+1)/65) sin(k pi (c+1)/65), lambda = 4 - 2cos(j pi/65) - 2cos(k pi/65)."""
    N = 64
    A = mi.poisson2d_5pt(N)
    p = 4
    for (j, k) in [(1, 1), (3, 7), (32, 5), (64, 64), (17, 60)]:
        v = sine_mode(N, j, k)
        lam = 4 - 2 * np.cos(j * np.pi / (N + 1)) - 2 * np.cos(k * np.pi / (N + 1))
        Y = oracle.mpk(A, p, sstep.monomial_coeffs(p), v)
        for q in range(p + 1):
            assert np.allclose(Y[q], lam ** q * v, rtol=0, atol=1e-12 * max(1.0, lam ** q))


def test_c1_dst_expansion_newton_and_chebyshev():
    """A random x expands in the sine basis by a 2-D DST-I (scipy, library special case);
    then p(A) x = sum p(lambda) c v.  Checked for Newton shifts and for the Chebyshev basis."""
    N = 64
    A = mi.poisson2d_5pt(N)
    x = mi.uniform_vectors(A.n, 0)[0]
    cs = np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    lam = 4 - 2 * cs[:, None] - 2 * cs[None, :]
    coef = scipy.fft.dstn(x.reshape(N, N), type=1)
    theta = [7.5, 0.25, 3.0, 6.0]
    Y = oracle.mpk(A, 4, sstep.newton_coeffs(theta), x)
    poly = np.ones_like(lam)
    for k, t in enumerate(theta, start=1):
        poly = poly * (lam - t)
        ref = scipy.fft.idstn(poly * coef, type=1).ravel()
        assert np.max(np.abs(Y[k] - ref)) <= 1e-11 * np.max(np.abs(ref)) + 1e-13
    alpha, beta = 0.1, 8.0
    Yc = oracle.mpk(A, 6, sstep.chebyshev_coeffs(alpha, beta, 6), x)
    z = (lam - 0.5 * (alpha + beta)) / (0.5 * (beta - alpha))
    for k in range(1, 7):
        Tk = np.polynomial.chebyshev.chebval(z, [0] * k + [1])
        ref = scipy.fft.idstn(Tk * coef, type=1).ravel()
        assert np.max(np.abs(Yc[k] - ref)) <= 1e-11 * np.max(np.abs(x)) * 64


@pytest.mark.parametrize("seed,components,symmetric", [(0, 1, True), (1, 2, False), (2, 3, True),
                                                       (3, 1, False)])
def test_dense_brute_force(seed, components, symmetric):
    """n <= 64: the recurrence against dense NumPy matrix products (monomial via
    matrix_power, Newton via explicit products, Chebyshev via the dense three-term loop)."""
    n = 48 + seed * 5
    A = mi.random_sparse(n, 0.1, seed, symmetric=symmetric, components=components)
    M = dense(A)
    x = mi.uniform_vectors(n, seed + 10)[0]
    p = 5
    Y = oracle.mpk(A, p, sstep.monomial_coeffs(p), x)
    for k in range(p + 1):
        ref = np.linalg.matrix_power(M, k) @ x
        assert np.allclose(Y[k], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    th = [0.5, -1.0, 2.0, 0.0, 1.5]
    Y = oracle.mpk(A, p, sstep.newton_coeffs(th), x)
    P = np.eye(n)
    for k in range(1, p + 1):
        P = (M - th[k - 1] * np.eye(n)) @ P
        assert np.allclose(Y[k], P @ x, rtol=1e-12, atol=1e-12 * np.abs(P @ x).max())


def test_exact_integer_matrices():
    """Integer matrices, dyadic x, integer shifts: every intermediate is exact in FP64 here, so
    the oracle must equal the exact rational result bit for bit."""
    A = mi.random_sparse(40, 0.15, 7, symmetric=False, components=2, int_values=True)
    rng = np.random.default_rng(3)
    x = rng.integers(-8, 9, size=A.n).astype(np.float64) / 8.0
    cf = sstep.newton_coeffs([1, -2, 3, 0])
    ex = exact_mpk(A, 4, cf, x)
    Y = oracle.mpk(A, 4, cf, x)
    for k in range(5):
        assert np.array_equal(Y[k], np.array([float(v) for v in ex[k]]))


def test_sampled_equals_full_and_omp_equals_plain():
    """The sampled and OpenMP variants reproduce the plain loop bit for bit."""
    A = mi.stencil27(12, seed=2)
    x = mi.uniform_vectors(A.n, 1)[0]
    cf = sstep.newton_coeffs(mi.leja_points_interval(0, 52, 4))
    Y = oracle.mpk(A, 4, cf, x)
    Yo = oracle.mpk(A, 4, cf, x, threads=True)
    assert np.array_equal(Y, Yo)
    rows = np.array([0, 5, 777, A.n - 1, 1000, 5], dtype=np.int32)
    S = oracle.mpk_sampled(A, 4, cf, x, rows)
    assert np.array_equal(S, Y[:, rows])


def test_generators_nnz_closed_forms():
    """Exact nnz closed forms and symmetry of the generated matrices."""
    assert mi.poisson2d_5pt(64).nnz == 4096 + 4 * 63 * 64
    for N in (5, 9):
        A = mi.stencil27(N, seed=2)
        assert A.nnz == (3 * N - 2) ** 3
        M = dense(A)
        assert np.array_equal(M, M.T)
        # 26 - sum of |off-diagonals| >= -2.6 and == 0 for interior rows before perturbation
        assert np.all(np.diag(M) == 26.0)
        C = mi.diffusion7_lognormal(N)
        assert C.nnz == 7 * N ** 3 - 6 * N ** 2
        Mc = dense(C)
        assert np.allclose(Mc, Mc.T, rtol=0, atol=0)
        # diagonal = sum of face coefficients >= |off-diagonal row sum| (Dirichlet boundary)
        assert np.all(np.diag(Mc) + (Mc.sum(1) - np.diag(Mc)) >= -1e-12)


# ----------------------------------------------------------------------------------------
# Planted mistakes (in a Python copy of the recurrence, never in the GPU path): each one must
# fail at least one of the pins used above.
# ----------------------------------------------------------------------------------------
def _mutant_mpk(A, p, coeffs, x, mutation):
    M = dense(A)
    if mutation == "transpose":
        M = M.T
    Y = [x.copy()]
    for k in range(1, p + 1):
        a, b, c = coeffs[k - 1]
        y1 = Y[-1]
        y2 = Y[-2] if k >= 2 else np.zeros_like(x)
        if mutation == "drop_b":
            b = 0.0
        if mutation == "sign_b":
            b = -b
        if mutation == "c_on_y1":
            y2 = y1
        Y.append(a * (M @ y1) + b * y1 + c * y2)
    return np.array(Y)


@pytest.mark.parametrize("mutation", ["transpose", "drop_b", "sign_b", "c_on_y1"])
def test_planted_mistakes_are_caught(mutation):
    A = mi.random_sparse(40, 0.12, 11, symmetric=False)
    x = mi.uniform_vectors(A.n, 4)[0]
    M = dense(A)
    if mutation == "c_on_y1":
        cf = sstep.chebyshev_coeffs(-3.0, 3.0, 4)
    else:
        cf = sstep.newton_coeffs([0.5, -1.0, 2.0, 1.5])
    bad = _mutant_mpk(A, 4, cf, x, mutation)
    good = oracle.mpk(A, 4, cf, x)
    # the brute-force reference of the pins
    ref = [x]
    for k in range(1, 5):
        a, b, c = cf[k - 1]
        ref.append(a * (M @ ref[-1]) + b * ref[-1] + c * (ref[-2] if k >= 2 else 0 * x))
    ref = np.array(ref)
    assert np.allclose(good, ref, rtol=1e-12, atol=1e-12)
    assert not np.allclose(bad, ref, rtol=1e-6, atol=1e-9)
