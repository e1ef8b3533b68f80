"""GPU parity for right Jacobi scaling (Sec. 5.1, Eq. (Jacobi): P^-1 = D^-1 fused into the
SpMV as A D^-1).

* mpk_apply(..., MPK_JACOBI) against the oracle's MPK of the explicitly scaled matrix
  (oracle.sstep.jacobi_right), per entry within 64*k*u of (|A D^-1|_theta^k |x|)_i, blocked
  bit-identical to unblocked; rows without a diagonal entry and an explicit zero diagonal
  leave their column unscaled;
* value updates refresh the scaled copy;
* the Jacobi-preconditioned solve reaches the FP64 true residual 1e-8 (recomputed on the CPU)
  with fewer Krylov columns than the plain solve on the log-normal diffusion matrix, and its
  solution agrees with the oracle's right-preconditioned s-step GMRES;
* k Jacobi sweeps (the Neumann polynomial in A D^-1 run by one final-only MPK) equal the
  oracle's sweeps of Eq. (Jacobi), and the solve preconditioned by them needs fewer Krylov
  columns than the diagonal scaling alone and agrees with the oracle's.
All calls go through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
import oracle
from oracle import sstep
from tests.gpu_util import U32, U64, abs_powers, max_rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def _zero_diag():
    """5-point Poisson matrix with the diagonal entries of rows 0 and 17 stored as 0."""
    A = mi.poisson2d_5pt(20)
    val = A.val.copy()
    for i in (0, 17):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col[e] == i:
                val[e] = 0.0
    return mi.CSR(A.row_ptr, A.col, val)


MATS = {
    "diff7_12": lambda: mi.diffusion7_lognormal(12),
    "s27_12": lambda: mi.stencil27(12, seed=2),
    "rand_nonsym_nodiag": lambda: mi.random_sparse(400, 0.01, 5, symmetric=False, components=2,
                                                   diag=False),
    "zero_diag": _zero_diag,
}

BASES = {
    "monomial": lambda p, hi: sstep.monomial_coeffs(p),
    "newton": lambda p, hi: sstep.newton_coeffs(mi.leja_points_interval(0.0, hi, p)),
    "chebyshev": lambda p, hi: sstep.chebyshev_coeffs(0.05, hi, p),
}


def _run(m, plan, n, cf, x, flags, dtype):
    import torch
    p = len(cf)
    X = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)
    Y = torch.full(((p + 1) * n,), float("nan"), dtype=dtype, device="cuda")
    m.mpk_apply(plan, cf, X, Y, flags=flags)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    return Y.cpu().numpy().astype(np.float64).reshape(p + 1, n)


@pytest.mark.parametrize("basis", sorted(BASES))
@pytest.mark.parametrize("name", sorted(MATS))
def test_jacobi_mpk_fp64_vs_oracle(m, name, basis):
    import torch
    A = MATS[name]()
    B, _ = sstep.jacobi_right(A)
    p = 6
    hi = 2.2 * float(np.abs(B.val).max())
    cf = BASES[basis](p, hi)
    x = mi.uniform_vectors(A.n, 3)[0]
    ref = oracle.mpk(B, p, cf, x)
    den = abs_powers(B, cf, x)
    rp, ci, vv = to_dev(A)
    for budget, kern in ((30_000, 0), (60_000, 1), (1 << 30, 2)):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
            l2_budget_bytes=budget, kernel=kern, blocked=1, jacobi=1))
        got = _run(m, plan, A.n, cf, x, m.MPK_JACOBI, torch.float64)
        got_u = _run(m, plan, A.n, cf, x, m.MPK_JACOBI | m.MPK_UNBLOCKED, torch.float64)
        assert np.array_equal(got, got_u)
        assert np.array_equal(got[0], x)
        for k in range(1, p + 1):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64, (k, budget, kern)
        # without the flag the same plan still computes the powers of A
        plain = _run(m, plan, A.n, cf, x, 0, torch.float64)
        refA = oracle.mpk(A, p, cf, x)
        denA = abs_powers(A, cf, x)
        for k in range(1, p + 1):
            assert max_rel_err(plain[k], refA[k], denA[k]) <= 64 * k * U64


@pytest.mark.parametrize("name", ["diff7_12", "s27_12", "rand_nonsym_nodiag"])
def test_jacobi_mpk_fp32_vs_oracle(m, name):
    import torch
    A = MATS[name]()
    B, _ = sstep.jacobi_right(A)
    # the plan rounds b_ij = a_ij / a_jj (formed in FP64) once to FP32
    B32 = mi.CSR(B.row_ptr, B.col, B.val.astype(np.float32).astype(np.float64))
    p = 6
    cf = sstep.chebyshev_coeffs(0.05, 2.2 * float(np.abs(B.val).max()), p)
    x = mi.uniform_vectors(A.n, 5)[0].astype(np.float32).astype(np.float64)
    ref = oracle.mpk(B32, p, cf, x)
    den = abs_powers(B32, cf, x)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
        keep_f32=1, keep_f64=1, l2_budget_bytes=40_000, blocked=1, jacobi=1))
    got = _run(m, plan, A.n, cf, x, m.MPK_JACOBI, torch.float32)
    got_u = _run(m, plan, A.n, cf, x, m.MPK_JACOBI | m.MPK_UNBLOCKED, torch.float32)
    assert np.array_equal(got, got_u)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U32


def test_jacobi_fp32_only_plan(m):
    """A plan built from FP32 values forms D^-1 from them (in FP64)."""
    import torch
    A = mi.diffusion7_lognormal(10)
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    B, _ = sstep.jacobi_right(A32)
    B32 = mi.CSR(B.row_ptr, B.col, B.val.astype(np.float32).astype(np.float64))
    p = 5
    cf = sstep.monomial_coeffs(p)
    x = mi.uniform_vectors(A.n, 6)[0].astype(np.float32).astype(np.float64)
    rp, ci, vv = to_dev(A, np.float32)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(jacobi=1))
    got = _run(m, plan, A.n, cf, x, m.MPK_JACOBI, torch.float32)
    ref = oracle.mpk(B32, p, cf, x)
    den = abs_powers(B32, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U32


def test_jacobi_flag_needs_a_jacobi_plan(m):
    import torch
    A = mi.poisson2d_5pt(16)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, 3)
    x = torch.ones(A.n, dtype=torch.float64, device="cuda")
    Y = torch.zeros(4 * A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MpkError) as e:
        m.mpk_apply(plan, sstep.monomial_coeffs(3), x, Y, flags=m.MPK_JACOBI)
    assert e.value.status == m.MPK_ERR_ARG
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    xs = torch.zeros_like(b)
    o = m.mpk_gmres_opts_default(basis=m.MPK_F64, s=2, restart=8, jacobi=1)
    info = m.sstep_gmres_solve(plan, b, xs, o, check=False)
    assert info["status_code"] == m.MPK_ERR_ARG


def test_jacobi_update_values(m):
    import torch
    A = mi.anisotropic(10, 7, 3.0)
    A2 = mi.anisotropic(10, 7, 50.0)
    B2, _ = sstep.jacobi_right(A2)
    p = 4
    cf = sstep.monomial_coeffs(p)
    x = mi.uniform_vectors(A.n, 2)[0]
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(jacobi=1))
    _, _, v2 = to_dev(A2)
    m.mpk_plan_update_values(plan, rp, ci, v2)
    got = _run(m, plan, A.n, cf, x, m.MPK_JACOBI, torch.float64)
    ref = oracle.mpk(B2, p, cf, x)
    den = abs_powers(B2, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64


def _plan(m, A, p=8, **kw):
    rp, ci, vv = to_dev(A)
    return m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(keep_f64=1, keep_f32=1,
                                                                    jacobi=1, **kw))


def _solve(m, plan, b, **kw):
    import torch
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B)
    info = m.sstep_gmres_solve(plan, B, X, m.mpk_gmres_opts_default(**kw), check=False)
    return X.cpu().numpy(), info


SOLVE_MATS = {
    "diff7_14": lambda: mi.diffusion7_lognormal(14),
    "aniso27_10": lambda: mi.anisotropic(10, 27, 20.0),
    "poisson2d_40": lambda: mi.poisson2d_5pt(40),
}


@pytest.mark.parametrize("name", sorted(SOLVE_MATS))
@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_jacobi_preconditioned_solve(m, name, basis):
    A = SOLVE_MATS[name]()
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    x, info = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8, jacobi=1)
    assert info["status_code"] == m.MPK_OK, info
    rr = np.linalg.norm(b - sstep.spmv(A, x)) / np.linalg.norm(b)
    assert rr <= 1e-8, rr
    assert abs(rr - info["rel_residual"]) <= 1e-9
    _, plain = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8)
    assert plain["status_code"] == m.MPK_OK
    if name == "diff7_14":
        # a strongly varying diagonal: the scaling pays
        assert info["iters"] < plain["iters"], (info["iters"], plain["iters"])
    ref = sstep.jacobi_gmres(A, b, s=8, m=48, tol=1e-10)
    assert ref["converged"]
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_jacobi_with_polynomial_and_blocked_equals_unblocked(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    x1, i1 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, jacobi=1)
    x2, i2 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, jacobi=1, mpk_flags=m.MPK_UNBLOCKED)
    assert i1["status_code"] == m.MPK_OK and i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
    x3, i3 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, jacobi=1, poly_degree=12)
    assert i3["status_code"] == m.MPK_OK, i3
    assert np.linalg.norm(b - sstep.spmv(A, x3)) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [2, 5])
def test_neumann_mpk_equals_jacobi_sweeps(m, k):
    """D^-1 p(A D^-1) v with p(t) = sum_{j<k} (1 - t)^j, one final-only MPK_JACOBI call with
    a = -1, b = 1, gamma = 1, equals k Jacobi sweeps from zero (the oracle runs Eq. (Jacobi)
    itself); compared as p(A D^-1) v = D~ z_k."""
    import torch
    A = MATS["zero_diag"]() if k == 2 else MATS["diff7_12"]()
    B, dinv = sstep.jacobi_right(A)
    cf = [(-1.0, 1.0, 0.0)] * (k - 1)
    v = mi.uniform_vectors(A.n, 8)[0]
    want = sstep.jacobi_sweeps(A, v, k) / dinv
    den = abs_powers(B, cf, v).sum(axis=0)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, max(k - 1, 1), m.mpk_plan_opts_default(jacobi=1, blocked=1))
    X = torch.from_numpy(v).cuda()
    for extra in (0, m.MPK_UNBLOCKED):
        Y = torch.full_like(X, float("nan"))
        m.mpk_apply(plan, m.Coeffs.from_triples(cf, [1.0] * k), X, Y,
                    flags=m.MPK_JACOBI | m.MPK_FINAL_ONLY | extra)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        assert max_rel_err(Y.cpu().numpy(), want, den) <= 64 * k * U64


@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_jacobi_sweeps_preconditioned_solve(m, basis):
    """k Jacobi sweeps as the right preconditioner (Sec. 5.1): the solve reaches 1e-8 in fewer
    Krylov columns than with the diagonal scaling alone, and agrees with the oracle's GMRES
    preconditioned by the sweeps themselves."""
    from oracle import poly
    A = SOLVE_MATS["diff7_14"]()
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    _, one = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8, jacobi=1)
    for k in (2, 4):
        x, info = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8, jacobi=k)
        assert info["status_code"] == m.MPK_OK, info
        assert info["poly_degree"] == k - 1
        rr = np.linalg.norm(b - sstep.spmv(A, x)) / np.linalg.norm(b)
        assert rr <= 1e-8, rr
        assert info["iters"] < one["iters"], (k, info["iters"], one["iters"])
        ref = poly.jacobi_sweeps_gmres(A, b, k, m=48, tol=1e-10)
        assert ref["converged"]
        M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
        kappa = np.linalg.cond(M)
        assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_jacobi_sweeps_blocked_equals_unblocked_and_argument_errors(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    x1, i1 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, jacobi=6)
    x2, i2 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, jacobi=6, mpk_flags=m.MPK_UNBLOCKED)
    assert i1["status_code"] == m.MPK_OK and i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
    for kw in ({"jacobi": 3, "poly_degree": 8}, {"jacobi": 65}, {"jacobi": -1}):
        _, info = _solve(m, plan, b, s=8, restart=48, tol=1e-8, **kw)
        assert info["status_code"] == m.MPK_ERR_ARG, kw
