"""Parity at the benchmark workloads' full sizes, in the configurations bench.py times.

* 27-point 160^3 (n = 4,096,000, nnz = 109,215,352): the plan exactly as the headline creates
  it; Newton p = 2, 4, 8 with Leja shifts on [0, 52], original-order I/O, FP64 and FP32.
  Every power at 2,000 sampled rows (random, plus the corners and both ends of the level
  order) against the oracle evaluated only on those rows' dependency cones
  (oracle.mpk_sampled), within 64 k u of the sampled |A_theta|^k |x| (the same recurrence on
  absolute values); blocked and unblocked bit-identical on the whole vectors; the levels equal
  the closed form (Chebyshev distance to the root's grid point) and the permutation is the
  stable (level, index) sort.
* 7-point log-normal diffusion 256^3 (n = 16,777,216, rows randomly permuted): the levels equal
  the Manhattan distance to the root's grid cell (the level build recovers the grid from the
  permuted rows); FP32 MPK at sampled rows; the GS2-preconditioned s-step GMRES and s-step CG
  reach the FP64 true residual 1e-8, recomputed on the CPU.
* 27-point 128^3 in FP32, Chebyshev p = 6 on [0.1, 52], n_rhs = 8, 16, 32 interleaved in level
  order (the block-MPK leg): sampled rows of several right-hand sides against the oracle.
All calls go through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import mpk_inputs as mi
import oracle
from oracle import sstep
from tests.gpu_util import U32, U64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def _abs(A):
    return mi.CSR(A.row_ptr, A.col, np.abs(A.val))


def _abs_coeffs(cf):
    return [(abs(a), abs(b), abs(c)) for a, b, c in cf]


def _samples(n, extra, count=2000, seed=11):
    rng = np.random.default_rng(seed)
    rows = np.concatenate([rng.choice(n, count, replace=False), np.asarray(extra, dtype=np.int64)])
    return np.unique(rows[(rows >= 0) & (rows < n)]).astype(np.int32)


def _check_sampled(got, A, cf, x, rows, u, p):
    """got: (p+1, n) array on the host; compares rows against the oracle's cones."""
    ref = oracle.mpk_sampled(A, p, cf, x, rows)
    den = oracle.mpk_sampled(_abs(A), p, _abs_coeffs(cf), np.abs(x), rows)
    for k in range(1, p + 1):
        diff = np.abs(got[k][rows] - ref[k])
        zero = den[k] == 0
        assert np.all(diff[zero] == 0), k
        rel = np.max(diff[~zero] / den[k][~zero]) if np.any(~zero) else 0.0
        assert rel <= 64 * k * u, (k, rel)


@pytest.fixture(scope="module")
def s27_160():
    return mi.stencil27(160, seed=2)


def _chebyshev_dist_levels(N, root):
    """Graph distance on the 27-point grid: the Chebyshev distance between grid points
    (row g is grid point (i, j, k) with g = (i N + j) N + k)."""
    g = np.arange(N ** 3, dtype=np.int64)
    i, j, k = np.unravel_index(g, (N, N, N))
    ri, rj, rk = np.unravel_index(int(root), (N, N, N))
    return np.maximum(np.maximum(np.abs(i - ri), np.abs(j - rj)), np.abs(k - rk))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_headline_27pt_160_sampled(m, s27_160, prec):
    import torch
    A = s27_160
    n = A.n
    assert A.nnz == 109_215_352
    dev = torch.device("cuda", 0)
    dt = torch.float64 if prec == "f64" else torch.float32
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vals = A.val if prec == "f64" else A.val.astype(np.float32).astype(np.float64)
    vv = torch.from_numpy(A.val).to(dev).to(dt)
    # the headline's plan
    plan = m.mpk_plan_create(rp, ci, vv, 8, m.mpk_plan_opts_default(assume_symmetric=1, p_blk=4,
                                                                    blocked=1))
    st = m.mpk_plan_stats(plan)
    x = mi.uniform_vectors(n, 0)[0]
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    X = torch.from_numpy(x).to(dev).to(dt)
    theta = mi.leja_points_interval(0.0, 52.0, 8)
    Aref = mi.CSR(A.row_ptr, A.col, vals)
    if prec == "f64":
        # levels: closed form from the root's grid point; the rows inside a level in the
        # oracle's breadth-first order (the plan's default)
        P = m.mpk_plan_perm(plan)
        lev = P["level"].cpu().numpy()
        assert np.array_equal(lev, _chebyshev_dist_levels(160, st["root"]))
        assert st["n_levels"] == int(lev.max()) + 1
        perm = P["perm"].cpu().numpy()
        operm, _, olp = oracle.level_perm_bfs(A, lev, st["n_levels"])
        assert np.array_equal(perm, operm)
        assert np.array_equal(P["level_ptr"].cpu().numpy(), olp)
    lp = None
    for p in (2, 4, 8):
        cf = sstep.newton_coeffs(theta[:p])
        co = m.mpk_coeffs_newton(theta[:p])
        Y = torch.empty((p + 1) * n, dtype=dt, device=dev)
        Yu = torch.empty_like(Y)
        m.mpk_apply(plan, co, X, Y)
        m.mpk_apply(plan, co, X, Yu, flags=m.MPK_UNBLOCKED)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        assert torch.equal(Y, Yu), p
        got = Y.view(p + 1, n).double().cpu().numpy()
        if lp is None:
            lp = m.mpk_plan_perm(plan)["perm"].cpu().numpy()
        rows = _samples(n, [0, n - 1, 159, 160 * 160 - 1, n - 160, int(lp[0]), int(lp[-1]),
                            int(lp[n // 2])])
        _check_sampled(got, Aref, cf, x, rows, U64 if prec == "f64" else U32, p)
        del Y, Yu
    del plan
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def diff256():
    return mi.diffusion7_lognormal(256)


def test_diffusion256_levels_mpk_and_solves(m, diff256):
    import torch
    A = diff256
    n, N = A.n, 256
    assert A.nnz == 117_047_296
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val).to(dev)
    plan = m.mpk_plan_create(rp, ci, vv, 8, m.mpk_plan_opts_default(keep_f64=1, keep_f32=1, jacobi=1))
    st = m.mpk_plan_stats(plan)
    # row r is grid cell cell[r]; the level of r is the Manhattan distance to the root's cell
    cell = np.random.default_rng(1).permutation(n)
    ci_, cj, ck = np.unravel_index(cell, (N, N, N))
    r0 = np.unravel_index(cell[st["root"]], (N, N, N))
    want = np.abs(ci_ - r0[0]) + np.abs(cj - r0[1]) + np.abs(ck - r0[2])
    P = m.mpk_plan_perm(plan)
    lev = P["level"].cpu().numpy()
    assert np.array_equal(lev, want)
    assert st["n_levels"] == int(want.max()) + 1
    # the breadth-first order inside the levels (766 of them, one device sort each)
    operm, _, _ = oracle.level_perm_bfs(A, lev, st["n_levels"])
    assert np.array_equal(P["perm"].cpu().numpy(), operm)
    del P
    # FP32 MPK (the solver's basis precision) at sampled rows
    p = 8
    th = mi.leja_points_interval(0.0, 4.0 * float(np.abs(A.val).max()), p)
    cf = sstep.newton_coeffs(th)
    x = mi.uniform_vectors(n, 4)[0].astype(np.float32).astype(np.float64)
    X = torch.from_numpy(x).to(dev).float()
    Y = torch.empty((p + 1) * n, dtype=torch.float32, device=dev)
    m.mpk_apply(plan, m.mpk_coeffs_newton(th), X, Y)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    got = Y.view(p + 1, n).double().cpu().numpy()
    del Y
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    _check_sampled(got, A32, cf, x, _samples(n, [0, n - 1], count=1000), U32, p)
    # full-size solves: the FP64 true residual recomputed on the CPU
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n))
    b = mi.uniform_vectors(n, 4)[0]
    B = torch.from_numpy(b).to(dev)
    nb = np.linalg.norm(b)
    Xs = torch.zeros_like(B)
    info = m.sstep_gmres_solve(plan, B, Xs, m.mpk_gmres_opts_default(s=8, restart=48, tol=1e-8, gs2=1,
                                                                      gs2_gamma=1), check=False)
    assert info["status_code"] == m.MPK_OK, info
    assert np.linalg.norm(b - M @ Xs.cpu().numpy()) <= 1e-8 * nb
    Xs.zero_()
    info = m.sstep_cg_solve(plan, B, Xs, m.mpk_cg_opts_default(s=8, tol=1e-8), check=False)
    assert info["status_code"] == m.MPK_OK, info
    assert np.linalg.norm(b - M @ Xs.cpu().numpy()) <= 1e-8 * nb
    del plan
    torch.cuda.empty_cache()


def test_block_mpk_128_sampled(m):
    import torch
    A = mi.stencil27(128, seed=5)
    n, p = A.n, 6
    dev = torch.device("cuda", 0)
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val.astype(np.float32)).to(dev)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(assume_symmetric=1, p_blk=p, blocked=1))
    perm = m.mpk_plan_perm(plan)["perm"].cpu().numpy()
    co = m.mpk_coeffs_chebyshev(0.1, 52.0, p)
    cf = list(zip(co.a, co.b, co.c))
    rows = _samples(n, [0, n - 1], count=300, seed=12)
    for n_rhs in (8, 16, 32):
        Xo = mi.uniform_vectors(n, 6, n_rhs).T.astype(np.float32).astype(np.float64)   # n x n_rhs
        X = torch.from_numpy(np.ascontiguousarray(Xo[perm])).to(dev).float()          # level order
        Y = torch.empty((p + 1) * n * n_rhs, dtype=torch.float32, device=dev)
        Yu = torch.empty_like(Y)
        fl = m.MPK_PERMUTED_IO | m.MPK_RHS_INTERLEAVED
        m.mpk_apply(plan, co, X, Y, n_rhs=n_rhs, flags=fl)
        m.mpk_apply(plan, co, X, Yu, n_rhs=n_rhs, flags=fl | m.MPK_UNBLOCKED)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        assert torch.equal(Y, Yu), n_rhs
        lvl = Y.view(p + 1, n, n_rhs).double().cpu().numpy()
        orig = np.empty_like(lvl)
        orig[:, perm, :] = lvl
        for q in sorted({0, n_rhs // 2, n_rhs - 1}):
            _check_sampled(orig[:, :, q], A32, cf, Xo[:, q], rows, U32, p)
        del X, Y, Yu
    del plan
    torch.cuda.empty_cache()
