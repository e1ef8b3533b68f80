"""The allocation-free final-power call (mpk_apply_final_noalloc) against the oracle and
against mpk_apply.

mpk_apply_final_noalloc keeps its intermediate vectors in the library's fixed per-device
scratch array.  Each case calls it twice in a row, on different inputs, and compares each
result with the CPU oracle's recurrence (oracle.mpk, on the matrix and vector as the GPU holds
them: FP32-rounded for FP32 cases, level-ordered for level-order I/O) and with
mpk_apply(..., MPK_FINAL_ONLY | MPK_UNBLOCKED) on the same plan.  The tolerance is the MPK's
own, per entry relative to (|A_theta|^p |x|)_i: 64*p*2^-53 in FP64, 64*p*2^-24 in FP32 (one
more power's worth for the gamma sums).  The two GPU calls run the same kernels, so their
results are also expected to be identical.
Also checked: device free memory does not change across calls after the first, and a plan
above the scratch limit is refused before any work.  This file is collected last, so it also
runs after every other GPU test in the same process."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle
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


def _newton(p, lo=0.0, hi=52.0):
    th = mi.leja_points_interval(lo, hi, p)
    return [(1.0, -t, 0.0) for t in th]


def _chebyshev(m, p, lo, hi):
    co = m.mpk_coeffs_chebyshev(lo, hi, p)
    return list(zip(co.a, co.b, co.c))


def _reference(m, plan, coeffs, x, flags, gamma):
    import torch
    y = torch.empty_like(x)
    m.mpk_apply(plan, m.Coeffs.from_triples(coeffs, gamma), x, y,
                flags=flags | m.MPK_FINAL_ONLY | m.MPK_UNBLOCKED)
    return y


def _den(A, coeffs, x, gamma):
    """(|A_theta|^p |x|), or sum_k |gamma_k| (|A_theta|^k |x|), for the matrix A as given."""
    P = abs_powers(A, coeffs, x.cpu().numpy().astype(np.float64))
    if gamma is None:
        return P[-1]
    return (np.abs(np.asarray(gamma))[:, None] * P).sum(axis=0)


CASES = [
    # name, matrix, dtype, p, basis, permuted, gamma
    ("s27_20_f64_newton", lambda: mi.stencil27(20, seed=2), "f64", 8, "newton", False, False),
    ("s27_20_f64_perm", lambda: mi.stencil27(20, seed=2), "f64", 4, "newton", True, False),
    ("diff7_24_f32_cheb", lambda: mi.diffusion7_lognormal(24), "f32", 6, "cheb", False, False),
    ("poisson96_f64_gamma", lambda: mi.poisson2d_5pt(96), "f64", 5, "newton", False, True),
    ("rand_nonsym_f32_perm", lambda: mi.random_sparse(3001, 0.003, 4, symmetric=False, components=2),
     "f32", 3, "newton", True, True),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_mpk_apply_twice(m, case):
    import torch
    name, mk, dt, p, basis, permuted, use_gamma = case
    A = mk()
    tdt = torch.float64 if dt == "f64" else torch.float32
    rp, ci, vv = to_dev(A, np.float64 if dt == "f64" else np.float32)
    plan = m.mpk_plan_create(rp, ci, vv, p)
    if basis == "newton":
        coeffs = _newton(p, 0.0, float(2 * np.abs(A.val).max() * 3))
    else:
        coeffs = _chebyshev(m, p, 0.1, float(np.abs(A.val).max() * 3))
    gamma = list(np.linspace(0.5, -0.25, p + 1)) if use_gamma else None
    flags = m.MPK_PERMUTED_IO if permuted else 0
    co = m.Coeffs.from_triples(coeffs, gamma)
    xs = [torch.from_numpy(mi.uniform_vectors(A.n, seed)[0]).to("cuda", tdt) for seed in (11, 12)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    tol = 64 * p * (U64 if dt == "f64" else U32)
    # the first call sets up the scratch address; after it, nothing may allocate
    m.mpk_apply_final_noalloc(plan, co, xs[0], ys[0], flags=flags)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, y in zip(xs, ys):
        m.mpk_apply_final_noalloc(plan, co, x, y, flags=flags)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for x, y in zip(xs, ys):
        ref = _reference(m, plan, coeffs, x, flags, gamma)
        torch.cuda.synchronize()
        got, want = y.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        if permuted:
            # level-order I/O: measure against the plan's own (level-ordered) matrix
            grp, gci, gval = m.mpk_plan_csr(plan, tdt)
            B = mi.CSR(grp.cpu().numpy(), gci.cpu().numpy(), gval.cpu().numpy().astype(np.float64))
        else:
            B = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64)) if dt == "f32" else A
        den = _den(B, coeffs, x, gamma)
        xo = x.cpu().numpy().astype(np.float64)
        ys_or = oracle.mpk(B, p, coeffs, xo)
        want_or = ys_or[p] if gamma is None else sum(g * ys_or[k] for k, g in enumerate(gamma))
        tol_or = 64 * (p + (1 if gamma is not None else 0)) * (U64 if dt == "f64" else U32)
        assert max_rel_err(got, want_or, den) <= tol_or
        assert max_rel_err(got, want, den) <= tol
        assert np.array_equal(got, want)


def test_noalloc_rejects_plans_above_the_scratch_limit(m):
    import torch
    A = mi.poisson2d_5pt(1000)                    # n = 1,000,000
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, 2)
    co = m.Coeffs.from_triples(_newton(2, 0.0, 8.0))
    x = torch.from_numpy(mi.uniform_vectors(A.n, 3)[0]).cuda()
    y = torch.zeros_like(x)
    # original order needs 5 vectors of 8 MB: above 32 MiB
    with pytest.raises(m.MpkError) as e:
        m.mpk_apply_final_noalloc(plan, co, x, y)
    assert e.value.status == m.MPK_ERR_ARG
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0           # refused before any work
    # level order needs 3 vectors: fits, and matches mpk_apply
    m.mpk_apply_final_noalloc(plan, co, x, y, flags=m.MPK_PERMUTED_IO)
    ref = _reference(m, plan, [(1.0, -t, 0.0) for t in mi.leja_points_interval(0.0, 8.0, 2)], x,
                     m.MPK_PERMUTED_IO, None)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)


def test_noalloc_argument_errors(m):
    import torch
    A = mi.poisson2d_5pt(16)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv.float(), 2)             # FP32 values only
    co = m.Coeffs.from_triples(_newton(2, 0.0, 8.0))
    for dt, flags in ((torch.float64, 0), (torch.float32, m.MPK_FINAL_ONLY),
                      (torch.float32, m.MPK_UNBLOCKED)):
        x = torch.ones(A.n, dtype=dt, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(m.MpkError) as e:
            m.mpk_apply_final_noalloc(plan, co, x, y, flags=flags)   # no FP64 values / bad flag
        assert e.value.status == m.MPK_ERR_ARG


def test_noalloc_jacobi_matches_mpk_apply(m):
    """MPK_JACOBI (powers of A D^-1) through the allocation-free call, both orders."""
    import torch
    A = mi.diffusion7_lognormal(20)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, 6, m.mpk_plan_opts_default(jacobi=1))
    coeffs = _newton(6, 0.0, 2.5)
    co = m.Coeffs.from_triples(coeffs)
    x = torch.from_numpy(mi.uniform_vectors(A.n, 9)[0]).cuda()
    for flags in (m.MPK_JACOBI, m.MPK_JACOBI | m.MPK_PERMUTED_IO):
        y = torch.full_like(x, float("nan"))
        m.mpk_apply_final_noalloc(plan, co, x, y, flags=flags)
        ref = _reference(m, plan, coeffs, x, flags, None)
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
