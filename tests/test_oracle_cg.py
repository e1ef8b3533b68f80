"""Pins for the oracle's textbook CG and s-step CG (Sec. 4 and Sec. 7 name s-step CG as the
short-recurrence method for the MPK; the method itself is the standard Chronopoulos-Gear /
CA-CG form).

Pinned from outside the loops under test:
* textbook CG reaches numpy.linalg.solve on SPD matrices and, on a diagonal matrix with k
  distinct eigenvalues, terminates after k steps (exact-arithmetic property of CG);
* A Y = Y B holds column by column for the change-of-basis matrix (dense products);
* s-step CG's outer iterates equal textbook CG's after the same number of steps (the method's
  defining property), for the Newton and monomial bases and s = 1 (which is CG itself);
* s-step CG and its FP64 refinement reach the FP64 true residual 1e-8 and numpy.linalg.solve,
  also with an FP32-rounded inner solve;
* the Gershgorin bound is pinned to the largest eigenvalue (eigvalsh) and to a hand value;
* an indefinite matrix raises the breakdown, and a planted mistake in B (a dropped shift) is
  caught by the equivalence with CG.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
from oracle import cg as ocg
from oracle import sstep


def _dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


SPD = {
    "diff7_6": lambda: mi.diffusion7_lognormal(6),
    "poisson2d_12": lambda: mi.poisson2d_5pt(12),
    "s27_5": lambda: mi.stencil27(5, seed=2),
}


@pytest.mark.parametrize("name", sorted(SPD))
def test_textbook_cg_solves(name):
    A = SPD[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    out = ocg.cg(A, b, tol=1e-10)
    assert out["converged"]
    want = np.linalg.solve(_dense(A), b)
    assert np.linalg.norm(out["x"] - want) <= np.linalg.cond(_dense(A)) * 1e-9 * np.linalg.norm(want)


def test_cg_terminates_on_distinct_eigenvalues():
    ev = np.repeat([1.0, 2.5, 4.0, 7.0], 5)
    n = ev.size
    A = mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), ev)
    b = mi.uniform_vectors(n, 1)[0]
    out = ocg.cg(A, b, tol=1e-13)
    assert out["iters"] <= 4 and out["converged"]


def test_change_of_basis_identity():
    A = mi.diffusion7_lognormal(5)
    s = 4
    th = [0.3, 2.0, 1.1, 3.5]
    p = mi.uniform_vectors(A.n, 1)[0]
    r = mi.uniform_vectors(A.n, 2)[0]
    M = _dense(A)
    cols = [p]
    for i in range(s):
        cols.append(M @ cols[-1] - th[i] * cols[-1])
    rc = [r]
    for i in range(s - 1):
        rc.append(M @ rc[-1] - th[i] * rc[-1])
    Y = np.array(cols + rc).T
    B = ocg.change_of_basis(th, s)
    AY = M @ Y
    YB = Y @ B
    for c in range(2 * s + 1):
        if c in (s, 2 * s):
            continue
        assert np.allclose(AY[:, c], YB[:, c], rtol=1e-12, atol=1e-12 * np.abs(AY[:, c]).max())


@pytest.mark.parametrize("s,basis", [(1, "newton"), (3, "newton"), (4, "monomial"), (8, "ritz")])
def test_sstep_iterates_equal_cg(s, basis):
    A = mi.diffusion7_lognormal(8)
    b = mi.uniform_vectors(A.n, 3)[0]
    if basis == "ritz":
        setup = ocg.cg(A, b, tol=0.0, max_iters=4 * s)
        th = ocg.ritz_shifts(setup["alphas"], setup["betas"], s)
    else:
        th = ocg.cg_shifts(A, s) if basis == "newton" else np.zeros(s)
    steps = 3 * s
    ref = ocg.cg(A, b, tol=0.0, max_iters=steps)
    got = ocg.cacg(A, b, s, th, tol=0.0, max_iters=steps)
    assert got["iters"] == steps
    assert np.linalg.norm(got["x"] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    for k in range(steps + 1):
        assert abs(got["hist"][k] - ref["hist"][k]) <= 1e-7 * ref["hist"][0], k


@pytest.mark.parametrize("replace", [1, 2])
def test_residual_replacement_keeps_the_cg_iterates(replace):
    # in FP64 a replaced residual differs from the recurrence one by rounding only, so the
    # iterates stay those of CG
    A = mi.diffusion7_lognormal(8)
    b = mi.uniform_vectors(A.n, 3)[0]
    s = 4
    th = ocg.cg_shifts(A, s)
    ref = ocg.cg(A, b, tol=0.0, max_iters=5 * s)
    got = ocg.cacg(A, b, s, th, tol=0.0, max_iters=5 * s, replace=replace)
    assert np.linalg.norm(got["x"] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    out = ocg.refine_cg(A, b, 8, tol=1e-8, replace=replace)
    assert out["converged"] and out["outer"] <= 2
    assert np.linalg.norm(b - sstep.spmv(A, out["x"])) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("name", sorted(SPD))
def test_sstep_cg_and_refinement_reach_1e8(name):
    A = SPD[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    want = np.linalg.solve(_dense(A), b)
    kappa = np.linalg.cond(_dense(A))
    out = ocg.cacg(A, b, 4, ocg.cg_shifts(A, 4), tol=1e-9)
    assert out["converged"]
    assert np.linalg.norm(b - sstep.spmv(A, out["x"])) <= 1e-8 * np.linalg.norm(b)
    for rnd in (None, np.float32):
        ref = ocg.refine_cg(A, b, 8, tol=1e-8, round_inner=rnd)
        assert ref["converged"]
        assert np.linalg.norm(b - sstep.spmv(A, ref["x"])) <= 1e-8 * np.linalg.norm(b)
        assert np.linalg.norm(ref["x"] - want) <= kappa * 2e-8 * np.linalg.norm(want)


def test_lanczos_ritz_values():
    # after n steps of CG on a diagonal matrix with n distinct eigenvalues, the Ritz values are
    # the eigenvalues; fewer steps give values inside [lambda_min, lambda_max]
    ev = np.array([0.5, 1.0, 2.0, 3.5, 5.0, 8.0])
    n = ev.size
    A = mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), ev)
    b = np.ones(n)
    out = ocg.cg(A, b, tol=0.0, max_iters=n)
    assert np.allclose(np.sort(ocg.lanczos_ritz(out["alphas"], out["betas"])), ev, rtol=1e-10)
    B = mi.diffusion7_lognormal(6)
    lam = np.linalg.eigvalsh(_dense(B))
    o2 = ocg.cg(B, mi.uniform_vectors(B.n, 2)[0], tol=0.0, max_iters=12)
    rz = ocg.lanczos_ritz(o2["alphas"], o2["betas"])
    assert rz.min() >= lam.min() * (1 - 1e-12) and rz.max() <= lam.max() * (1 + 1e-12)
    th = ocg.ritz_shifts(o2["alphas"], o2["betas"], 5)
    assert th[0] == rz.max() and len(set(th)) == 5


def test_gershgorin_bound():
    A = mi.poisson2d_5pt(10)
    assert ocg.gershgorin_bound(A) == 8.0
    B = mi.diffusion7_lognormal(5)
    lmax = np.linalg.eigvalsh(_dense(B)).max()
    g = ocg.gershgorin_bound(B)
    assert lmax <= g * (1 + 1e-14)
    th = ocg.cg_shifts(B, 4)
    assert th[0] == g and np.all((th >= 0) & (th <= g))


def test_indefinite_breaks_down():
    n = 30
    d = np.linspace(-1.0, 3.0, n)
    A = mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = np.ones(n)
    with pytest.raises(ocg.CGBreakdown):
        ocg.cacg(A, b, 4, ocg.cg_shifts(A, 4), tol=1e-12)


def test_planted_basis_mistake_is_caught():
    A = mi.diffusion7_lognormal(5)
    b = mi.uniform_vectors(A.n, 3)[0]
    s = 4
    th = ocg.cg_shifts(A, s)
    ref = ocg.cg(A, b, tol=0.0, max_iters=2 * s)
    orig = ocg.change_of_basis
    try:
        def wrong(theta, s_):
            B = orig(theta, s_)
            B[2, 2] = 0.0          # a dropped (nonzero) shift in the p block
            return B
        ocg.change_of_basis = wrong
        got = ocg.cacg(A, b, s, th, tol=0.0, max_iters=2 * s)
    finally:
        ocg.change_of_basis = orig
    assert np.linalg.norm(got["x"] - ref["x"]) > 1e-6 * np.linalg.norm(ref["x"])
