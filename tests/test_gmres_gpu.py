"""GPU parity for s-step GMRES (Alg. 3(c), Newton basis of Sec. 4) with FP64 refinement.

The oracle (FP64 NumPy s-step GMRES, FP64 CSR SpMV) checks: the final true residual
||b - A x|| / ||b|| <= 1e-8 recomputed on the CPU, the solution against numpy.linalg.solve /
the oracle's solution within cond(A)-scaled bounds, and the Newton shifts against the
oracle's Ritz values in Leja order.  Blocked and unblocked MPK give bit-identical solves."""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
import oracle
from oracle import sstep
from tests.gpu_util import to_dev
from tests.trace_check import trace_problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def _plan(m, A, p=8, both=True, **kw):
    rp, ci, vv = to_dev(A)
    opts = m.mpk_plan_opts_default(keep_f64=1, keep_f32=1 if both else 0, **kw)
    return m.mpk_plan_create(rp, ci, vv, p, opts)


def _solve(m, plan, A, b, **kw):
    import torch
    shifts = kw.pop("shifts", None)
    o = m.mpk_gmres_opts_default(**kw)
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B)
    info = m.sstep_gmres_solve(plan, B, X, o, shifts=shifts, check=False)
    return X.cpu().numpy(), info


def _relres(A, x, b):
    return np.linalg.norm(b - sstep.spmv(A, x)) / np.linalg.norm(b)


MATS = {
    "diff7_12_perm": lambda: mi.diffusion7_lognormal(12),
    "aniso27_10": lambda: mi.anisotropic(10, 27, 20.0),
    "aniso7_14": lambda: mi.anisotropic(14, 7, 50.0),
    "poisson2d_40": lambda: mi.poisson2d_5pt(40),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_solve_reaches_1e8(m, name, basis):
    A = MATS[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    x, info = _solve(m, plan, A, b, basis=m.MPK_F32 if basis == "f32" else m.MPK_F64,
                     s=8, restart=48, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    rr = _relres(A, x, b)
    assert rr <= 1e-8, rr
    assert abs(rr - info["rel_residual"]) <= 1e-9
    # the oracle's FP64 s-step GMRES solution of the same system
    ref = sstep.sstep_gmres(A, b, s=8, m=48, tol=1e-10)
    assert ref["converged"]
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_small_dense_vs_numpy_solve(m):
    A = mi.random_sparse(60, 0.1, 3, symmetric=True)
    b = mi.uniform_vectors(60, 5)[0]
    plan = _plan(m, A, p=4)
    x, info = _solve(m, plan, A, b, s=4, restart=20, tol=1e-10, basis=m.MPK_F64)
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(60, 60)).toarray()
    xs = np.linalg.solve(M, b)
    assert info["status_code"] == m.MPK_OK
    assert np.linalg.norm(x - xs) <= np.linalg.cond(M) * 1e-9 * np.linalg.norm(xs)


def test_shifts_match_oracle_ritz_leja(m):
    """FP64 basis: the shifts the solver derives from its first (plain GMRES) cycle agree with
    the oracle's Ritz values of the same cycle, Leja-ordered."""
    A = mi.anisotropic(10, 7, 4.0)
    b = mi.uniform_vectors(A.n, 9)[0]
    plan = _plan(m, A)
    x, info = _solve(m, plan, A, b, basis=m.MPK_F64, s=8, restart=48, tol=1e-12)
    r0 = sstep.gmres(A, b, m=48, tol=1e-12, max_restarts=1, cgs=True)
    rv = sstep.ritz_values(r0["H_first"], r0["k_first"])
    th = sstep.leja_order(rv, 8)
    assert np.allclose(info["shifts"], th, rtol=1e-6, atol=1e-8 * np.abs(th).max())


def _skewed(A, beta):
    """A plus a skew-symmetric part on its (symmetric) pattern: entries above the diagonal
    gain beta, entries below lose it - a structurally symmetric, numerically unsymmetric
    matrix (as convection adds to diffusion)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    val = A.val + beta * np.sign(A.col - rows)
    return mi.CSR(A.row_ptr, A.col, val)


def test_shifts_match_oracle_ritz_leja_unsymmetric(m):
    """The Ritz values are the real parts of the eigenvalues of the first cycle's Arnoldi H
    on both sides; for an unsymmetric A they are complex, and the reading must still agree."""
    A = _skewed(mi.anisotropic(10, 7, 4.0), 0.6)
    b = mi.uniform_vectors(A.n, 9)[0]
    plan = _plan(m, A)
    x, info = _solve(m, plan, A, b, basis=m.MPK_F64, s=8, restart=48, tol=1e-12, max_outer=1)
    r0 = sstep.gmres(A, b, m=48, tol=1e-12, max_restarts=1, cgs=True)
    H = r0["H_first"][: r0["k_first"], : r0["k_first"]]
    assert np.abs(np.linalg.eigvals(H).imag).max() > 1e-3      # complex Ritz values occur
    rv = sstep.ritz_values(r0["H_first"], r0["k_first"])
    th = sstep.leja_order(rv, 8)
    assert np.allclose(info["shifts"], th, rtol=1e-6, atol=1e-8 * np.abs(th).max())


@pytest.mark.parametrize("name,s,restart", [("aniso27_8", 8, 24), ("skew7_10", 4, 48),
                                            ("poisson2d_40", 6, 36), ("diff7_8", 8, 24)])
def test_cycle_internals_match_oracle(m, name, s, restart):
    """FP64 basis, given shifts, one restart cycle and no refinement: the residual estimate
    after every column's Givens rotation and the cycle's Arnoldi Hessenberg (from the block
    QR factors: H R_s = R_full B) against the oracle's s-step GMRES, within 1e-8 relative
    (tests/trace_check.py; its CPU test shows a wrong Hessenberg column fails it).
    The cases are ones where the s-step basis is well conditioned: the oracle's s-step cycle
    follows textbook GMRES to 1e-10 (checked here).  Where it is not (the log-normal 10^3
    matrix at s = 8: 23 % off textbook GMRES by column 21), two FP64 implementations of the
    same steps legitimately differ by as much, and no tight comparison is well posed."""
    A = {"aniso27_8": lambda: mi.anisotropic(8, 27, 10.0),
         "skew7_10": lambda: _skewed(mi.anisotropic(10, 7, 4.0), 0.6),
         "poisson2d_40": lambda: mi.poisson2d_5pt(40),
         "diff7_8": lambda: mi.diffusion7_lognormal(8)}[name]()
    b = mi.uniform_vectors(A.n, 6)[0]
    r0 = sstep.gmres(A, b, m=restart, tol=1e-14, max_restarts=1, cgs=True)
    th = sstep.leja_order(sstep.ritz_values(r0["H_first"], r0["k_first"]), s)
    tol = 1e-9
    ref = sstep.sstep_gmres(A, b, s=s, m=restart, tol=0.5 * tol, max_restarts=1, shifts=th)
    plain = sstep.gmres(A, b, m=restart, tol=0.5 * tol, max_restarts=1)
    kk = min(len(ref["hist"]), len(plain["hist"]) - 1)
    dev = np.abs(np.array(ref["hist"][:kk]) - np.array(plain["hist"][1: kk + 1])) / np.array(plain["hist"][1: kk + 1])
    assert dev.max() <= 1e-10, dev.max()
    import torch
    plan = _plan(m, A)
    o = m.mpk_gmres_opts_default(s=s, restart=restart, tol=tol, basis=m.MPK_F64, max_outer=1)
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B)
    info = m.sstep_gmres_solve(plan, B, X, o, shifts=th, check=False, trace=True)
    k = info["trace_len"]
    assert k == ref["k_cycle"] and k > 2 * s, (k, ref["k_cycle"])
    problems = trace_problems(info["trace_hist"], info["trace_H"], ref["hist"], ref["H_cycle"], k)
    assert not problems, problems[:5]


def test_blocked_and_unblocked_mpk_give_identical_solves(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    x1, i1 = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8)
    x2, i2 = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8, mpk_flags=m.MPK_UNBLOCKED)
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


def test_given_shifts_and_two_bcgs_sweeps(m):
    A = mi.anisotropic(9, 27, 10.0)
    b = mi.uniform_vectors(A.n, 3)[0]
    plan = _plan(m, A)
    th = mi.leja_points_interval(0.05, float(abs(A.val).max() * 2), 8)
    for passes in (1, 2):
        x, info = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8, shifts=th, bcgs_passes=passes)
        assert info["status_code"] == m.MPK_OK and _relres(A, x, b) <= 1e-8
        assert np.allclose(info["shifts"], th)


def test_breakdown_is_handled(m):
    """A diagonal matrix with two distinct values: the Krylov space has dimension 2, so a block
    of 8 Newton vectors is rank deficient and CholQR breaks down; the solver shrinks s and
    still returns the solution (or reports the breakdown) without a fault."""
    n = 256
    d = np.where(np.arange(n) % 2 == 0, 2.0, 5.0)
    A = mi.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = mi.uniform_vectors(n, 1)[0]
    plan = _plan(m, A)
    x, info = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8, shifts=[4.0, 3.0, 1.0, 6.0, 2.5, 3.5, 5.5, 4.5])
    assert info["status_code"] in (m.MPK_OK, m.MPK_ERR_BREAKDOWN)
    if info["status_code"] == m.MPK_OK:
        assert _relres(A, x, b) <= 1e-8


def test_argument_errors(m):
    import torch
    A = mi.poisson2d_5pt(8)
    rp, ci, vv = to_dev(A)
    plan32 = m.mpk_plan_create(rp, ci, vv.float(), 8)          # FP32 only: no FP64 residual
    B = torch.ones(A.n, dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    info = m.sstep_gmres_solve(plan32, B, X, m.mpk_gmres_opts_default(), check=False)
    assert info["status_code"] == m.MPK_ERR_ARG
    plan = _plan(m, A, p=4)
    info = m.sstep_gmres_solve(plan, B, X, m.mpk_gmres_opts_default(s=8), check=False)
    assert info["status_code"] == m.MPK_ERR_ARG                  # s > p_max of the plan


@pytest.mark.parametrize("name", ["poisson2d_40", "diff7_12_perm", "aniso27_10"])
@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_polynomial_preconditioned_solve(m, name, basis):
    """GMRES-polynomial preconditioning (Sec. 5.2): the solve reaches 1e-8 with fewer Krylov
    columns than without the polynomial, and agrees with the oracle's preconditioned GMRES."""
    from oracle import poly
    A = MATS[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    d = 16
    x, info = _solve(m, plan, A, b, basis=bs, s=8, restart=48, tol=1e-8, poly_degree=d)
    assert info["status_code"] == m.MPK_OK, info
    rr = _relres(A, x, b)
    assert rr <= 1e-8, rr
    assert 1 <= info["poly_degree"] <= d and info["poly_interval"][1] > 0
    _, plain = _solve(m, plan, A, b, basis=bs, s=8, restart=48, tol=1e-8)
    # the first (setup) cycle is plain GMRES: a solve that ends inside it is unchanged
    if plain["iters"] > 48:
        assert info["iters"] < plain["iters"], (info["iters"], plain["iters"])
    else:
        assert info["iters"] <= plain["iters"], (info["iters"], plain["iters"])
    ref = poly.poly_gmres(A, b, d=d, m=48, tol=1e-10)
    assert ref["converged"]
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_polynomial_solve_blocked_equals_unblocked(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    x1, i1 = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8, poly_degree=12)
    x2, i2 = _solve(m, plan, A, b, s=8, restart=48, tol=1e-8, poly_degree=12, mpk_flags=m.MPK_UNBLOCKED)
    assert i1["status_code"] == m.MPK_OK and i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
