"""GPU parity: the plan (levels, permutation, groups, permuted CSR) bit-exact against the
oracle, and the MPK within the stated tolerance of the oracle (FP64: 64*k*2^-53, FP32:
64*k*2^-24, per entry relative to (|A_theta|^k |x|)_i), blocked bit-identical to unblocked.

All calls go through the C ABI (ctypes binding)."""
import numpy as np
import pytest

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


def _mats():
    out = {
        "poisson64": mi.poisson2d_5pt(64),
        "s27_12": mi.stencil27(12, seed=2),
        "diff7_10": mi.diffusion7_lognormal(10),
        "rand_nonsym_3c": mi.random_sparse(300, 0.01, 1, symmetric=False, components=3),
        "rand_sym": mi.random_sparse(200, 0.03, 2, symmetric=True),
        "aniso27": mi.anisotropic(9, 27, 30.0),
    }
    return out


MATS = _mats()


def _check_plan(m, A, opts, p_blk, val_bytes=8):
    import torch
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p_blk, opts)
    st = m.mpk_plan_stats(plan)
    lev, root, nl, perm, iperm, lp = oracle.level_structure(A, root_rule=opts.root_rule,
                                                            n_sweeps=opts.n_sweeps,
                                                            level_order=opts.level_order)
    P = m.mpk_plan_perm(plan)
    torch.cuda.synchronize()
    assert st["root"] == root and st["n_levels"] == nl
    assert np.array_equal(P["level"].cpu().numpy(), lev)
    assert np.array_equal(P["perm"].cpu().numpy(), perm)
    assert np.array_equal(P["iperm"].cpu().numpy(), iperm)
    assert np.array_equal(P["level_ptr"].cpu().numpy(), lp)
    brp, bci, bval = oracle.permute_csr(A, perm, iperm)
    grp, gci, gval = m.mpk_plan_csr(plan, torch.float64)
    assert np.array_equal(grp.cpu().numpy(), brp)
    assert np.array_equal(gci.cpu().numpy(), bci)
    assert np.array_equal(gval.cpu().numpy().view(np.uint8), bval.view(np.uint8))
    gp = oracle.level_groups(lp, brp, val_bytes, st["p_blk"], st["l2_budget_bytes"])
    assert np.array_equal(P["group_ptr"].cpu().numpy(), gp)
    return plan


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("root_rule", [0, 1])
@pytest.mark.parametrize("level_order", [0, 1])
def test_plan_bit_exact(m, name, root_rule, level_order):
    A = MATS[name]
    for budget in (20_000, 400_000, 1 << 30):
        opts = m.mpk_plan_opts_default(l2_budget_bytes=budget, root_rule=root_rule, level_order=level_order)
        _check_plan(m, A, opts, 4)


def test_breadth_first_order_large_levels(m):
    """Both sorting paths of the breadth-first order: the randomly permuted log-normal
    diffusion matrix at 48^3 (levels up to about 1700 rows: one-block sorts) and a randomly
    permuted 27-point 48^3 stencil (corner shells up to 6900 rows: radix passes), against the
    oracle's breadth-first order bit for bit; then an MPK on that plan, blocked against
    unblocked and within the oracle's tolerance."""
    import torch
    s27 = mi.stencil27(48, seed=3)
    for A in (mi.diffusion7_lognormal(48),
              mi.symmetric_permute(s27, np.random.default_rng(11).permutation(s27.n))):
        opts = m.mpk_plan_opts_default(level_order=1, assume_symmetric=1, blocked=1)
        plan = _check_plan(m, A, opts, 4)
        cf = BASES["newton"](4)
        x = mi.uniform_vectors(A.n, 2)[0]
        got = _run(m, plan, A, cf, x)
        assert np.array_equal(got, _run(m, plan, A, cf, x, flags=m.MPK_UNBLOCKED))
        ref = oracle.mpk(A, 4, cf, x)
        den = abs_powers(A, cf, x)
        for k in range(1, 5):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64
        del plan
        torch.cuda.empty_cache()


def test_plan_edge_cases(m):
    import torch
    # one row; an empty row; a long row (> 32 entries, block sort path); unsorted columns and
    # duplicate entries; a diagonal matrix (n components)
    cases = []
    cases.append(mi.CSR(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0])))
    n = 70
    rows = [[0, 5, 69], [], list(range(0, 70, 2))[::-1], [3, 3, 1], [4]] + [[i, (i * 7) % n] for i in range(5, n)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], np.int32)
    val = np.arange(1, col.size + 1, dtype=np.float64) * 0.25
    cases.append(mi.CSR(rp, col, val))
    d = 500
    cases.append(mi.CSR(np.arange(d + 1, dtype=np.int32), np.arange(d, dtype=np.int32), np.linspace(1, 2, d)))
    for A in cases:
        opts = m.mpk_plan_opts_default(l2_budget_bytes=4096)
        plan = _check_plan(m, A, opts, 3)
        x = mi.uniform_vectors(A.n, 5)[0]
        cf = sstep.newton_coeffs([0.5, -1.0, 2.0])
        X = torch.from_numpy(x).cuda()
        Y = torch.empty(4 * A.n, dtype=torch.float64, device="cuda")
        m.mpk_apply(plan, cf, X, Y)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        ref = oracle.mpk(A, 3, cf, x)
        den = abs_powers(A, cf, x)
        got = Y.view(4, A.n).cpu().numpy()
        for k in range(4):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * max(k, 1) * U64


def test_empty_matrix(m):
    import torch
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    vv = torch.zeros(0, dtype=torch.float64, device="cuda")
    plan = m.mpk_plan_create(rp, ci, vv, 2)
    st = m.mpk_plan_stats(plan)
    assert st["n"] == 0 and st["n_levels"] == 0
    X = torch.zeros(1, dtype=torch.float64, device="cuda")
    Y = torch.zeros(3, dtype=torch.float64, device="cuda")
    m.mpk_apply(plan, sstep.monomial_coeffs(2), X, Y, ldx=1, ldy=1)


def test_invalid_csr_rejected(m):
    import torch
    A = mi.poisson2d_5pt(8)
    rp, ci, vv = to_dev(A)
    ci[5] = 10_000
    with pytest.raises(m.MpkError) as e:
        m.mpk_plan_create(rp, ci, vv, 2)
    assert e.value.status == m.MPK_ERR_ARG


def _run(m, plan, A, cf, x, flags=0, dtype=None, n_rhs=1):
    import torch
    dt = torch.float64 if dtype is None else dtype
    p = len(cf)
    X = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to("cuda", dt)
    nb = 1 if flags & m.MPK_FINAL_ONLY else p + 1
    Y = torch.full((nb * A.n * n_rhs,), float("nan"), dtype=dt, device="cuda")
    m.mpk_apply(plan, cf, X, Y, n_rhs=n_rhs, flags=flags)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    return Y.cpu().numpy().astype(np.float64).reshape(nb, -1)


BASES = {
    "monomial": lambda p: sstep.monomial_coeffs(p),
    "newton": lambda p: sstep.newton_coeffs(mi.leja_points_interval(0.0, 8.0, p)),
    "chebyshev": lambda p: sstep.chebyshev_coeffs(0.1, 8.0, p),
}


@pytest.mark.parametrize("basis", sorted(BASES))
@pytest.mark.parametrize("name", ["poisson64", "s27_12", "diff7_10", "rand_nonsym_3c"])
def test_mpk_fp64_vs_oracle(m, basis, name):
    A = MATS[name]
    p = 5
    cf = BASES[basis](p)
    x = mi.uniform_vectors(A.n, 0)[0]
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    rp, ci, vv = to_dev(A)
    # kernel 0 = warp tasks with a ticket dispenser, 1 = CTA tasks, 2 = warp tasks in static
    # round robin, 3 = ready-first warp tasks, 4 = lane tasks (lanes sharing rows, sub-slice
    # tasks), 5 = staged warp tasks (slices copied into shared memory), 6 = owner shares (one
    # share of every level group per CTA, warp groups per power); slack 7 makes most warp
    # tasks wait for their dependencies.  The last field is lanes_per_row (the unblocked
    # comparison runs the same row function)
    for budget, cs, stage, sched, kern, slack, lanes in (
            (30_000, 1, -1, 1, 0, 0, 1), (300_000, 2, 0, 1, 1, 0, 1),
            (1 << 30, 8, -1, 0, 0, 0, 1), (100_000, 4, -1, 0, 2, 0, 1),
            (60_000, 1, -1, 1, 0, 7, 1), (60_000, 2, -1, 1, 2, 7, 1),
            (30_000, 1, -1, 1, 1, 0, 1), (30_000, 1, -1, 1, 3, 0, 1),
            (1 << 30, 8, -1, 1, 3, 0, 1),
            (30_000, 1, -1, 1, 4, 0, 1), (60_000, 3, -1, 1, 4, 7, 1),
            (30_000, 1, -1, 1, 4, 0, 2), (60_000, 2, -1, 1, 4, 7, 4),
            (1 << 30, 1, -1, 1, 4, 0, 8), (100_000, 5, -1, 1, 4, 3, 4),
            (30_000, 1, -1, 1, 5, 0, 1), (60_000, 1, -1, 1, 5, 7, 1), (1 << 30, 1, -1, 1, 5, 0, 1),
            (30_000, 1, -1, 1, 6, 0, 1), (1 << 30, 1, -1, 1, 6, 0, 1)):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
            l2_budget_bytes=budget, chunk_slices=cs, stage=stage, schedule=sched, kernel=kern,
            slack_tasks=slack, blocked=1, lanes_per_row=lanes, task_units=cs))
        got_b = _run(m, plan, A, cf, x)
        got_u = _run(m, plan, A, cf, x, flags=m.MPK_UNBLOCKED)
        assert np.array_equal(got_b, got_u)            # blocked == unblocked, bit for bit
        assert np.array_equal(got_b[0], x)
        for k in range(1, p + 1):
            assert max_rel_err(got_b[k], ref[k], den[k]) <= 64 * k * U64, (k, budget)


@pytest.mark.parametrize("name", ["poisson64", "s27_12", "diff7_10"])
def test_mpk_fp32_vs_oracle(m, name):
    import torch
    A = MATS[name]
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    p = 6
    cf = sstep.chebyshev_coeffs(0.1, 8.0, p)
    x = mi.uniform_vectors(A.n, 1)[0].astype(np.float32).astype(np.float64)
    ref = oracle.mpk(A32, p, cf, x)
    den = abs_powers(A32, cf, x)
    rp, ci, vv = to_dev(A, np.float32)
    # lanes_per_row 0 is the automatic choice (4 in FP32)
    for lanes, kern, units in ((0, 0, 1), (1, 0, 1), (1, 4, 2), (2, 4, 1), (4, 4, 3), (8, 4, 1), (1, 5, 1), (1, 6, 1)):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
            l2_budget_bytes=50_000, blocked=1, lanes_per_row=lanes, kernel=kern, task_units=units))
        got = _run(m, plan, A, cf, x, dtype=torch.float32)
        got_u = _run(m, plan, A, cf, x, dtype=torch.float32, flags=m.MPK_UNBLOCKED)
        assert np.array_equal(got, got_u), lanes
        for k in range(1, p + 1):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U32, (lanes, k)


def test_permuted_io_and_y0_is_x(m):
    import torch
    A = MATS["s27_12"]
    p = 4
    cf = BASES["newton"](p)
    x = mi.uniform_vectors(A.n, 3)[0]
    ref = oracle.mpk(A, p, cf, x)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=100_000, blocked=1))
    perm = m.mpk_plan_perm(plan)["perm"].cpu().numpy()
    got = _run(m, plan, A, cf, x[perm], flags=m.MPK_PERMUTED_IO)
    full = _run(m, plan, A, cf, x)
    assert np.array_equal(got, full[:, perm])
    Y = torch.empty((p + 1) * A.n, dtype=torch.float64, device="cuda")
    Y[: A.n] = torch.from_numpy(x[perm]).cuda()
    m.mpk_apply(plan, cf, None, Y, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    assert np.array_equal(Y.view(p + 1, -1).cpu().numpy(), got)
    den = abs_powers(A, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(full[k], ref[k], den[k]) <= 64 * k * U64


@pytest.mark.parametrize("n_rhs", [1, 2, 3, 8, 16, 32])
@pytest.mark.parametrize("interleaved", [False, True])
def test_block_mpk_n_rhs(m, n_rhs, interleaved):
    import torch
    A = MATS["s27_12"]
    p = 6
    cf = sstep.chebyshev_coeffs(0.1, 52.0, p)
    Xc = mi.uniform_vectors(A.n, 6, n_rhs=n_rhs).astype(np.float32).astype(np.float64)  # (n_rhs, n)
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    rp, ci, vv = to_dev(A, np.float32)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=200_000, blocked=1))
    flags = m.MPK_RHS_INTERLEAVED if interleaved else 0
    xin = Xc.T.copy() if interleaved else Xc   # row-major n x n_rhs, or column-major
    got = _run(m, plan, A, cf, xin, dtype=torch.float32, n_rhs=n_rhs, flags=flags)
    got_u = _run(m, plan, A, cf, xin, dtype=torch.float32, n_rhs=n_rhs, flags=flags | m.MPK_UNBLOCKED)
    assert np.array_equal(got, got_u)
    got = got.reshape(p + 1, A.n, n_rhs) if interleaved else got.reshape(p + 1, n_rhs, A.n).transpose(0, 2, 1)
    for q in range(n_rhs):
        ref = oracle.mpk(A32, p, cf, Xc[q])
        den = abs_powers(A32, cf, Xc[q])
        for k in range(1, p + 1):
            assert max_rel_err(got[k, :, q], ref[k], den[k]) <= 64 * k * U32


@pytest.mark.parametrize("kern,lanes", [(0, 1), (1, 1), (2, 1), (3, 1), (4, 1), (4, 4), (5, 1), (6, 1)])
def test_final_only_gamma_and_segments(m, kern, lanes):
    import torch
    A = MATS["diff7_10"]
    p = 9
    cf = sstep.chebyshev_coeffs(0.05, 12.0, p)
    gamma = np.linspace(1.0, -0.5, p + 1)
    x = mi.uniform_vectors(A.n, 8)[0]
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    rp, ci, vv = to_dev(A)
    # p_blk = 4 -> segments of 4, 4, 1 powers (the remainder launch)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=60_000, p_blk=4,
                                                                     kernel=kern, slack_tasks=5, blocked=1,
                                                                     lanes_per_row=lanes))
    full = _run(m, plan, A, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(full[k], ref[k], den[k]) <= 64 * k * U64
    fin = _run(m, plan, A, cf, x, flags=m.MPK_FINAL_ONLY)
    assert np.array_equal(fin[0], full[p])
    co = m.Coeffs.from_triples(cf, gamma=gamma)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    for fl in (m.MPK_FINAL_ONLY, m.MPK_FINAL_ONLY | m.MPK_UNBLOCKED):
        m.mpk_apply(plan, co, X, Y, flags=fl)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        poly = Y.cpu().numpy()
        want = sum(gamma[k] * ref[k] for k in range(p + 1))
        dsum = sum(abs(gamma[k]) * den[k] for k in range(p + 1))
        assert max_rel_err(poly, want, dsum) <= 64 * (p + 1) * U64


def test_host_io(m):
    import torch
    A = MATS["poisson64"]
    p = 4
    cf = BASES["newton"](p)
    x = mi.uniform_vectors(A.n, 0)[0]
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p)
    Xh = torch.from_numpy(x.copy()).pin_memory()
    Yh = torch.empty((p + 1) * A.n, dtype=torch.float64).pin_memory()
    m.mpk_apply(plan, cf, Xh, Yh, flags=m.MPK_HOST_IO)
    dev = _run(m, plan, A, cf, x)
    assert np.array_equal(Yh.numpy().reshape(p + 1, -1), dev)


@pytest.mark.parametrize("kern,lanes", [(0, 1), (1, 1), (2, 1), (3, 1), (4, 1), (4, 4), (5, 1), (6, 1)])
def test_timeout_is_reported_and_plan_recovers(m, kern, lanes):
    """A completion that nothing publishes: the waits on it run out (short bound), the call
    reports MPK_ERR_TIMEOUT, and the plan works again afterwards."""
    A = MATS["s27_12"]
    p = 3
    cf = BASES["monomial"](p)
    x = mi.uniform_vectors(A.n, 0)[0]
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=30_000, wait_timeout_us=20_000,
                                                                     kernel=kern, blocked=1, lanes_per_row=lanes))
    import torch
    X = torch.from_numpy(x).cuda()
    Y = torch.empty((p + 1) * A.n, dtype=torch.float64, device="cuda")
    m.mpk_apply(plan, cf, X, Y, flags=m.MPK_DEBUG_DROP_FLAG)
    assert m.mpk_plan_sync(plan) == m.MPK_ERR_TIMEOUT
    got = _run(m, plan, A, cf, x)
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64


def test_update_values_keeps_structure(m):
    import torch
    A = mi.anisotropic(10, 7, 3.0)
    B = mi.anisotropic(10, 7, 50.0)
    p = 4
    cf = BASES["monomial"](p)
    x = mi.uniform_vectors(A.n, 2)[0]
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p)
    _, _, vb = to_dev(B)
    m.mpk_plan_update_values(plan, rp, ci, vb)
    got = _run(m, plan, B, cf, x)
    ref = oracle.mpk(B, p, cf, x)
    den = abs_powers(B, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64


def test_automatic_blocked_choice(m):
    """Default plans choose between the blocked and unblocked kernel by themselves: a matrix
    larger than the L2 cache is timed both ways on the first call, a small one runs unblocked.
    Every call returns the unblocked kernel's values bit for bit."""
    import torch
    for A, p in ((mi.stencil27(96, seed=2), 4), (MATS["s27_12"], 4)):
        x = mi.uniform_vectors(A.n, 1)[0]
        rp, ci, vv = to_dev(A)
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(assume_symmetric=1))
        cf = BASES["newton"](p)
        ref = _run(m, plan, A, cf, x, flags=m.MPK_UNBLOCKED)
        first = _run(m, plan, A, cf, x)           # may time both kernels
        again = _run(m, plan, A, cf, x)           # the cached choice
        assert np.array_equal(first, ref) and np.array_equal(again, ref)
        del plan
        torch.cuda.empty_cache()


@pytest.mark.parametrize("kern,lanes", [(0, 1), (3, 1), (4, 4), (5, 1), (6, 1)])
def test_graph_capture_replays_the_blocked_kernel(m, kern, lanes):
    """A blocked mpk_apply captured in a CUDA graph (after one ordinary call, which builds the
    schedule) replays correctly: the per-power launch counts the dependency waits compare
    against live in device memory, so each replay is a fresh launch.  Each replay's result
    equals the unblocked kernel's bit for bit."""
    import torch
    A = MATS["s27_12"]
    p = 5
    cf = BASES["newton"](p)
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=40_000, blocked=1,
                                                                     slack_tasks=5, kernel=kern,
                                                                     lanes_per_row=lanes))
    X = torch.from_numpy(mi.uniform_vectors(A.n, 2)[0]).cuda()
    Y = torch.empty((p + 1) * A.n, dtype=torch.float64, device="cuda")
    m.mpk_apply(plan, cf, X, Y)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        m.mpk_apply(plan, cf, X, Y)
    for seed in (3, 4, 5):
        xs = mi.uniform_vectors(A.n, seed)[0]
        X.copy_(torch.from_numpy(xs))
        g.replay()
        torch.cuda.synchronize()
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        ref = _run(m, plan, A, cf, xs, flags=m.MPK_UNBLOCKED)
        assert np.array_equal(Y.cpu().numpy().reshape(p + 1, -1), ref)


def test_maximum_power_count_and_rhs_block(m):
    """p = 63 (MPK_MAX_P, Chebyshev basis so the powers stay bounded) through one blocked
    launch of 63 local powers, bit-identical to 63 SpMVs and within the tolerance of the oracle;
    n_rhs = 1024 (the largest block) in FP32, interleaved and column-major, against the oracle
    column by column on a sample of right-hand sides."""
    import torch
    A = MATS["diff7_10"]
    p = 63
    cf = sstep.chebyshev_coeffs(0.0, 2.2 * float(np.abs(A.val).max()), p)
    x = mi.uniform_vectors(A.n, 9)[0]
    rp, ci, vv = to_dev(A)
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    for lanes in (1, 4):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=40_000, blocked=1,
                                                                         lanes_per_row=lanes))
        assert m.mpk_plan_stats(plan)["p_blk"] == p
        got = _run(m, plan, A, cf, x)
        got_u = _run(m, plan, A, cf, x, flags=m.MPK_UNBLOCKED)
        assert np.array_equal(got, got_u)
        for k in range(1, p + 1):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64, (lanes, k)
    # the largest block of right-hand sides
    B = mi.random_sparse(300, 0.02, 4, symmetric=True, diag=True)
    B32 = mi.CSR(B.row_ptr, B.col, B.val.astype(np.float32).astype(np.float64))
    nr, p2 = 1024, 2
    cf2 = sstep.newton_coeffs([0.5, -0.25])
    Xh = mi.uniform_vectors(B.n, 3, nr).astype(np.float32)            # nr x n
    rpb, cib, vb = to_dev(B, np.float32)
    plan2 = m.mpk_plan_create(rpb, cib, vb, p2, m.mpk_plan_opts_default(blocked=1))
    cols = [0, 1, 511, 1023]
    for fl, X, unpack in (
            (m.MPK_RHS_INTERLEAVED, torch.from_numpy(np.ascontiguousarray(Xh.T)).cuda(),
             lambda Y: Y.view(p2 + 1, B.n, nr).permute(0, 2, 1)),
            (0, torch.from_numpy(np.ascontiguousarray(Xh)).cuda().view(-1),
             lambda Y: Y.view(p2 + 1, nr, B.n))):
        Y = torch.full(((p2 + 1) * B.n * nr,), float("nan"), dtype=torch.float32, device="cuda")
        m.mpk_apply(plan2, cf2, X, Y, n_rhs=nr, flags=fl)
        assert m.mpk_plan_sync(plan2) == m.MPK_OK
        out = unpack(Y).double().cpu().numpy()          # (p+1, nr, n)
        for q in cols:
            xq = Xh[q].astype(np.float64)
            ref2 = oracle.mpk(B32, p2, cf2, xq)
            den2 = abs_powers(B32, cf2, xq)
            for k in range(1, p2 + 1):
                assert max_rel_err(out[k, q], ref2[k], den2[k]) <= 64 * k * 2.0 ** -24, (fl, q, k)
