"""GPU parity for two-stage Gauss-Seidel (GS2) preconditioning as MPK sub-powers (Sec. 5.1, GS2
subsection, Alg. GS2(a) and (b)).

* mpk_apply(..., MPK_GS2 | MPK_GS2_GAMMA(gamma)) against the oracle's MPK of the
  GS2-preconditioned operator (oracle.gs2.gs2_mpk, which runs Alg. GS2 on A's own L, D, U), per
  entry within 64 * k * (gamma + 1) * u of the same recurrence run on absolute values
  (|A| |P^-1|, |P^-1| the truncated Neumann series of |D^-1 L|); blocked (warp tasks with
  dynamic, static and ready-first hand-out, segments that end inside a power) bit-identical to
  unblocked;
  original-order and level-order I/O, final-only with polynomial sums, FP32 and FP64, zero and
  missing diagonal entries;
* flag and plan errors are reported, not run;
* the GS2-preconditioned s-step GMRES reaches the FP64 true residual 1e-8 (recomputed on the
  CPU), needs fewer Krylov columns than the diagonal scaling alone, agrees with the oracle's
  GS2-preconditioned s-step GMRES, and its blocked and unblocked solves are identical.
All calls go through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
from oracle import gs2, sstep
from tests.gpu_util import U32, U64, max_rel_err, to_dev

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
    "diff7_10_perm": lambda: mi.diffusion7_lognormal(10),
    "s27_9": lambda: mi.stencil27(9, seed=2),
    "rand_nonsym_nodiag": lambda: mi.random_sparse(300, 0.012, 5, symmetric=False, components=2,
                                                   diag=False),
    "zero_diag": _zero_diag,
}


def _abs_den(A, coeffs, x, gamma):
    """Denominators: the recurrence on absolute values, |a_k| |A| |P^-1| + |b_k| I (+ |c_k|)."""
    n = A.n
    M = abs(sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n)))
    Lm = sp.tril(M, -1).tocsr()
    d = np.abs(M.diagonal())
    dinv = 1.0 / np.where(d != 0.0, d, 1.0)

    def absP(v):
        g = dinv * v
        acc = g.copy()
        for _ in range(gamma):
            g = dinv * (Lm @ g)
            acc += g
        return acc

    out = [np.abs(x)]
    for k, (a, b, c) in enumerate(coeffs, start=1):
        prev = out[-1]
        prev2 = out[-2] if k >= 2 else np.zeros_like(prev)
        out.append(abs(a) * (M @ absP(prev)) + abs(b) * prev + abs(c) * prev2)
    return np.array(out)


def _run(m, plan, n, cf, x, flags, dtype, gamma=None):
    import torch
    p = len(cf) if not isinstance(cf, m.Coeffs) else cf.p
    X = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)
    nblk = 1 if flags & m.MPK_FINAL_ONLY else p + 1
    Y = torch.full((nblk * n,), float("nan"), dtype=dtype, device="cuda")
    m.mpk_apply(plan, cf, X, Y, flags=flags)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    return Y.cpu().numpy().astype(np.float64).reshape(nblk, n)


def _gs2_flags(m, gamma):
    return m.MPK_GS2 | m.MPK_GS2_GAMMA(gamma)


@pytest.mark.parametrize("gamma", [0, 1, 2, 3])
@pytest.mark.parametrize("name", sorted(MATS))
def test_gs2_mpk_fp64_vs_oracle(m, name, gamma):
    import torch
    A = MATS[name]()
    p = 4
    cf = sstep.newton_coeffs(mi.leja_points_interval(0.0, 2.0, p)) if gamma % 2 else \
        sstep.chebyshev_coeffs(0.05, 2.0, p)
    x = mi.uniform_vectors(A.n, 3)[0]
    ref = gs2.gs2_mpk(A, p, cf, x, gamma)
    den = _abs_den(A, cf, x, gamma)
    fl = _gs2_flags(m, gamma)
    rp, ci, vv = to_dev(A)
    for budget, kern, pblk in ((20_000, 0, 0), (40_000, 2, 3), (1 << 30, 1, 0), (20_000, 3, 3)):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
            l2_budget_bytes=budget, kernel=kern, blocked=1, jacobi=1, p_blk=pblk))
        got = _run(m, plan, A.n, cf, x, fl, torch.float64)
        got_u = _run(m, plan, A.n, cf, x, fl | m.MPK_UNBLOCKED, torch.float64)
        assert np.array_equal(got, got_u), (budget, kern)
        assert np.array_equal(got[0], x)
        for k in range(1, p + 1):
            e = max_rel_err(got[k], ref[k], den[k])
            assert e <= 64 * k * (gamma + 1) * U64, (k, budget, kern, e)


def test_gs2_level_order_io_and_final_only(m):
    import torch
    A = MATS["diff7_10_perm"]()
    p, gamma = 5, 2
    cf = sstep.newton_coeffs(mi.leja_points_interval(0.0, 2.0, p))
    x = mi.uniform_vectors(A.n, 4)[0]
    fl = _gs2_flags(m, gamma)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
        l2_budget_bytes=30_000, blocked=1, jacobi=1))
    full = _run(m, plan, A.n, cf, x, fl, torch.float64)
    perm = m.mpk_plan_perm(plan)["perm"].cpu().numpy()
    lev = _run(m, plan, A.n, cf, x[perm], fl | m.MPK_PERMUTED_IO, torch.float64)
    assert np.array_equal(lev[:, np.argsort(perm)], full)
    gam = [0.5, -1.0, 0.25, 2.0, -0.75, 1.5]
    co = m.Coeffs.from_triples(cf, gam)
    for extra in (0, m.MPK_UNBLOCKED):
        fin = _run(m, plan, A.n, co, x, fl | m.MPK_FINAL_ONLY | extra, torch.float64)[0]
        want = sum(g * full[k] for k, g in enumerate(gam))
        den = np.abs(np.array(gam))[:, None] * _abs_den(A, cf, x, gamma)
        assert max_rel_err(fin, want, den.sum(axis=0)) <= 64 * p * (gamma + 1) * U64
        fin_y = _run(m, plan, A.n, cf, x, fl | m.MPK_FINAL_ONLY | extra, torch.float64)[0]
        assert np.array_equal(fin_y, full[p])


@pytest.mark.parametrize("name", ["diff7_10_perm", "s27_9", "rand_nonsym_nodiag"])
def test_gs2_mpk_fp32_vs_oracle(m, name):
    import torch
    A = MATS[name]()
    p, gamma = 4, 1
    cf = sstep.chebyshev_coeffs(0.05, 2.0, p)
    x = mi.uniform_vectors(A.n, 5)[0].astype(np.float32).astype(np.float64)
    ref = gs2.gs2_mpk(A, p, cf, x, gamma)
    den = _abs_den(A, cf, x, gamma)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
        keep_f32=1, keep_f64=1, l2_budget_bytes=20_000, blocked=1, jacobi=1))
    fl = _gs2_flags(m, gamma)
    got = _run(m, plan, A.n, cf, x, fl, torch.float32)
    got_u = _run(m, plan, A.n, cf, x, fl | m.MPK_UNBLOCKED, torch.float32)
    assert np.array_equal(got, got_u)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * (gamma + 1) * U32


def test_gs2_flag_errors(m):
    import torch
    A = mi.poisson2d_5pt(16)
    rp, ci, vv = to_dev(A)
    x = torch.ones(A.n, dtype=torch.float64, device="cuda")
    Y = torch.zeros(4 * A.n, dtype=torch.float64, device="cuda")
    cf = sstep.monomial_coeffs(3)
    plain = m.mpk_plan_create(rp, ci, vv, 3)
    with pytest.raises(m.MpkError) as e:
        m.mpk_apply(plain, cf, x, Y, flags=_gs2_flags(m, 1))
    assert e.value.status == m.MPK_ERR_ARG
    jp = m.mpk_plan_create(rp, ci, vv, 3, m.mpk_plan_opts_default(jacobi=1))
    with pytest.raises(m.MpkError) as e:
        m.mpk_apply(jp, cf, x, Y, flags=_gs2_flags(m, 1) | m.MPK_JACOBI)
    assert e.value.status == m.MPK_ERR_ARG
    X2 = torch.ones(2 * A.n, dtype=torch.float64, device="cuda")
    Y2 = torch.zeros(8 * A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MpkError) as e:
        m.mpk_apply(jp, cf, X2, Y2, n_rhs=2, flags=_gs2_flags(m, 1))
    assert e.value.status == m.MPK_ERR_UNIMPLEMENTED
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    xs = torch.zeros_like(b)
    info = m.sstep_gmres_solve(plain, b, xs, m.mpk_gmres_opts_default(basis=m.MPK_F64, s=2, restart=8, gs2=1),
                               check=False)
    assert info["status_code"] == m.MPK_ERR_ARG
    for kw in ({"gs2": 1, "jacobi": 1}, {"gs2": 1, "poly_degree": 4}, {"gs2": 1, "gs2_gamma": 16},
               {"gs2": 2}):
        info = m.sstep_gmres_solve(jp, b, xs, m.mpk_gmres_opts_default(basis=m.MPK_F64, s=2, restart=8, **kw),
                                   check=False)
        assert info["status_code"] == m.MPK_ERR_ARG, kw


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


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("basis", ["f32", "f64"])
def test_gs2_preconditioned_solve(m, basis, gamma):
    A = mi.diffusion7_lognormal(12)
    b = mi.uniform_vectors(A.n, 4)[0]
    plan = _plan(m, A)
    bs = m.MPK_F32 if basis == "f32" else m.MPK_F64
    x, info = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8, gs2=1, gs2_gamma=gamma)
    assert info["status_code"] == m.MPK_OK, info
    rr = np.linalg.norm(b - sstep.spmv(A, x)) / np.linalg.norm(b)
    assert rr <= 1e-8, rr
    assert abs(rr - info["rel_residual"]) <= 1e-9
    _, jac = _solve(m, plan, b, basis=bs, s=8, restart=48, tol=1e-8, jacobi=1)
    assert jac["status_code"] == m.MPK_OK
    assert info["iters"] < jac["iters"], (info["iters"], jac["iters"])
    ref = gs2.gs2_gmres(A, b, gamma, s=8, m=48, tol=1e-10)
    assert ref["converged"]
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(x - ref["x"]) <= kappa * 2e-8 * np.linalg.norm(ref["x"])


def test_gs2_solve_blocked_equals_unblocked(m):
    A = mi.diffusion7_lognormal(10)
    b = mi.uniform_vectors(A.n, 2)[0]
    plan = _plan(m, A, l2_budget_bytes=50_000, blocked=1)
    x1, i1 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, gs2=1, gs2_gamma=2)
    x2, i2 = _solve(m, plan, b, s=8, restart=48, tol=1e-8, gs2=1, gs2_gamma=2,
                    mpk_flags=m.MPK_UNBLOCKED)
    assert i1["status_code"] == m.MPK_OK, i1
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
    # gamma = 0 is the diagonal scaling: the same iterates as the Jacobi option
    x3, i3 = _solve(m, plan, b, basis=m.MPK_F64, s=8, restart=48, tol=1e-8, gs2=1, gs2_gamma=0)
    x4, i4 = _solve(m, plan, b, basis=m.MPK_F64, s=8, restart=48, tol=1e-8, jacobi=1)
    assert i3["status_code"] == m.MPK_OK and i4["status_code"] == m.MPK_OK
    assert abs(i3["iters"] - i4["iters"]) <= 8, (i3["iters"], i4["iters"])
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    assert np.linalg.norm(x3 - x4) <= np.linalg.cond(M) * 2e-8 * np.linalg.norm(x4)
