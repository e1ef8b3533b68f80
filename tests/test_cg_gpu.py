"""GPU parity for s-step CG with FP64 iterative refinement (the short-recurrence method the paper
names for the MPK, Sec. 4 and Sec. 7), through the C ABI.

* the solve reaches the FP64 true residual 1e-8 (recomputed on the CPU by the oracle's SpMV),
  reports it, and agrees with numpy.linalg.solve and with the oracle's refined s-step CG
  within kappa * 2e-8, in FP32 and FP64 bases, from zero and from a nonzero initial guess;
* the shifts of the setup phase equal the oracle's Ritz values of the same CG steps;
* with given shifts and an FP64 basis the number of CG steps matches the oracle's;
* residual replacement (the default) needs fewer CG steps in an FP32 basis than refinement
  alone;
* the blocked and unblocked MPK give identical solves;
* s = 15 (the largest basis, the Gram kernel's largest shared-memory ring) converges;
* a negative definite matrix reports MPK_ERR_BREAKDOWN, the step limit MPK_ERR_NOT_CONVERGED,
  and invalid options MPK_ERR_ARG."""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
from oracle import cg as ocg
from oracle import sstep
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


MATS = {
    "diff7_12_perm": lambda: mi.diffusion7_lognormal(12),
    "poisson2d_40": lambda: mi.poisson2d_5pt(40),
    "s27_10": lambda: mi.stencil27(10, seed=2),
    "aniso7_12": lambda: mi.anisotropic(12, 7, 30.0),
}


def _dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def _plan(m, A, p=8, **kw):
    rp, ci, vv = to_dev(A)
    return m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(keep_f64=1, keep_f32=1, **kw))


def _solve(m, plan, b, x0=None, shifts=None, **kw):
    import torch
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    info = m.sstep_cg_solve(plan, B, X, m.mpk_cg_opts_default(**kw), shifts=shifts, check=False)
    return X.cpu().numpy(), info


@pytest.mark.parametrize("basis", ["f32", "f64"])
@pytest.mark.parametrize("name", sorted(MATS))
def test_cg_solve_reaches_1e8(m, name, basis):
    A = MATS[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    x, info = _solve(m, plan, b, basis=bs, s=8, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    rr = np.linalg.norm(b - sstep.spmv(A, x)) / np.linalg.norm(b)
    assert rr <= 1e-8, rr
    assert abs(rr - info["rel_residual"]) <= 1e-9
    M = _dense(A)
    kappa = np.linalg.cond(M)
    want = np.linalg.solve(M, b)
    assert np.linalg.norm(x - want) <= kappa * 2e-8 * np.linalg.norm(want)
    ref = ocg.refine_cg(A, b, 8, tol=1e-10)
    assert ref["converged"]
    assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_cg_from_initial_guess(m):
    A = MATS["diff7_12_perm"]()
    b = mi.uniform_vectors(A.n, 5)[0]
    x0 = mi.uniform_vectors(A.n, 6)[0]
    plan = _plan(m, A)
    x, info = _solve(m, plan, b, x0=x0, s=6, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    assert np.linalg.norm(b - sstep.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)


def test_cg_setup_shifts_are_the_oracles_ritz_values(m):
    A = MATS["diff7_12_perm"]()
    b = mi.uniform_vectors(A.n, 4)[0]
    s = 6
    plan = _plan(m, A)
    _, info = _solve(m, plan, b, basis=m.MPK_F64, s=s, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    setup = ocg.cg(A, b, tol=0.0, max_iters=4 * s)
    want = ocg.ritz_shifts(setup["alphas"], setup["betas"], s)
    got = info["shifts"]
    # The setup phase runs CG in s-step form (s = 1: coefficients from the Gram matrix of
    # [p, Ap, r] and coordinate vectors), whose coefficients lose accuracy as the residual
    # falls.  In FP64 NumPy that form's Ritz values differ from textbook CG's by 5.2e-6 of the
    # largest on this matrix, and by up to 2e-5 when the Gram entries are perturbed by 1e-15
    # relative (a change of summation order), so the bound is 5e-5 of the largest shift.
    assert np.allclose(got, want, rtol=0.0, atol=5e-5 * np.abs(want).max()), (got, want)


@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_cg_largest_s(m, basis):
    """s = 15, the largest basis (31 columns, 32 in the pair storage): its Gram kernel's stage
    ring needs more than the default 48 KB of shared memory.  The solve reaches 1e-8."""
    A = MATS["poisson2d_40"]()
    b = mi.uniform_vectors(A.n, 7)[0]
    plan = _plan(m, A, p=15)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    x, info = _solve(m, plan, b, basis=bs, s=15, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    assert np.linalg.norm(b - sstep.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)
    assert 1 <= info["s_used"] <= 15


@pytest.mark.parametrize("s", [1, 4, 8])
def test_cg_steps_match_the_oracle_with_given_shifts(m, s):
    A = MATS["poisson2d_40"]()
    b = mi.uniform_vectors(A.n, 7)[0]
    th = ocg.cg_shifts(A, s)
    plan = _plan(m, A)
    x, info = _solve(m, plan, b, shifts=th, basis=m.MPK_F64, s=s, tol=1e-8)
    assert info["status_code"] == m.MPK_OK, info
    ref = ocg.refine_cg(A, b, s, theta=th, tol=1e-8, inner_tol=1e-8, replace=1)
    assert ref["converged"]
    assert abs(info["iters"] - ref["iters"]) <= max(2, s), (info["iters"], ref["iters"])
    assert np.allclose(info["shifts"], th, rtol=0, atol=0)


def test_cg_residual_replacement_saves_steps_in_fp32(m):
    A = mi.diffusion7_lognormal(20)
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    xr, ir = _solve(m, plan, b, basis=m.MPK_F32, s=8, tol=1e-8, replace=1)
    xn, inn = _solve(m, plan, b, basis=m.MPK_F32, s=8, tol=1e-8, replace=0)
    for x, info in ((xr, ir), (xn, inn)):
        assert info["status_code"] == m.MPK_OK, info
        assert np.linalg.norm(b - sstep.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)
    assert ir["iters"] < inn["iters"], (ir, inn)


def test_cg_blocked_equals_unblocked(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    for bs in (m.MPK_F32, m.MPK_F64):
        x1, i1 = _solve(m, plan, b, basis=bs, s=8, tol=1e-8)
        x2, i2 = _solve(m, plan, b, basis=bs, s=8, tol=1e-8, mpk_flags=m.MPK_UNBLOCKED)
        assert i1["status_code"] == m.MPK_OK, i1
        assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


def test_cg_breakdown_and_limits(m):
    A = mi.poisson2d_5pt(20)
    neg = mi.CSR(A.row_ptr, A.col, -A.val)
    b = mi.uniform_vectors(A.n, 3)[0]
    plan = _plan(m, neg)
    _, info = _solve(m, plan, b, s=4, tol=1e-8)
    assert info["status_code"] == m.MPK_ERR_BREAKDOWN, info
    plan2 = _plan(m, A)
    _, info = _solve(m, plan2, b, s=4, tol=1e-8, max_iters=10)
    assert info["status_code"] == m.MPK_ERR_NOT_CONVERGED, info
    assert info["iters"] <= 10
    for kw in ({"s": 0}, {"s": 16}, {"tol": 0.0}, {"basis": 7}, {"replace": -1}):
        _, info = _solve(m, plan2, b, **kw)
        assert info["status_code"] == m.MPK_ERR_ARG, kw
    small = _plan(m, A, p=4)
    _, info = _solve(m, small, b, s=8)
    assert info["status_code"] == m.MPK_ERR_ARG
    _, info = _solve(m, plan2, b, s=2, shifts=[1.0, float("nan")])
    assert info["status_code"] == m.MPK_ERR_ARG
    rp, ci, vv = to_dev(A)
    f64only = m.mpk_plan_create(rp, ci, vv, 8, m.mpk_plan_opts_default(keep_f64=1, keep_f32=0))
    _, info = _solve(m, f64only, b, basis=m.MPK_F32, s=4)
    assert info["status_code"] == m.MPK_ERR_ARG
