"""GPU parity of the owner-share blocked kernel (opts.kernel = 6): the level-group wavefront of
Sec. 3 with every group split into one share per CTA and a warp group per power.

Each case is bit-identical to p back-to-back SpMVs on the same plan (the same row function) and
within the oracle's tolerance (FP64 64*k*2^-53, FP32 64*k*2^-24 per entry, relative to
(|A_theta|^k |x|)_i).  The cases vary what the kernel's schedule depends on: the lag between
powers, the L2 prefetch distance, power counts above the eight warp groups of a CTA (powers
share a warp group round robin), several launches per call (segments of p_blk powers), the
final-only ring of three vectors on an unsymmetric pattern (the dependency closure over A^T),
level groups smaller than the CTA count (empty shares), and one group for the whole matrix."""
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


def _run(m, plan, n, cf, x, flags=0, dtype=None):
    import torch
    dt = torch.float64 if dtype is None else dtype
    p = len(cf)
    X = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
    nb = 1 if flags & m.MPK_FINAL_ONLY else p + 1
    Y = torch.full((nb * n,), float("nan"), dtype=dt, device="cuda")
    m.mpk_apply(plan, cf, X, Y, flags=flags)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    return Y.cpu().numpy().astype(np.float64).reshape(nb, -1)


MATS = {
    "s27_14": lambda: mi.stencil27(14, seed=2),
    "diff7_12": lambda: mi.diffusion7_lognormal(12),
    "rand_nonsym_3c": lambda: mi.random_sparse(400, 0.01, 1, symmetric=False, components=3),
    "aniso27": lambda: mi.anisotropic(11, 27, 30.0),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("p,p_blk,lag,pf", [(4, 0, 1, 1), (2, 0, 1, 0), (3, 0, 2, 2), (8, 0, 1, 1),
                                             (11, 0, 1, 1), (9, 4, 3, 1), (5, 2, 1, 0)])
def test_owner_fp64_bit_exact_and_oracle(m, name, p, p_blk, lag, pf):
    A = MATS[name]()
    cf = sstep.newton_coeffs(mi.leja_points_interval(0.0, 8.0, p))
    x = mi.uniform_vectors(A.n, 3)[0]
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    rp, ci, vv = to_dev(A)
    for budget in (20_000, 1 << 30):
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
            l2_budget_bytes=budget, p_blk=p_blk, kernel=6, blocked=1, owner_lag=lag, owner_prefetch=pf))
        got = _run(m, plan, A.n, cf, x)
        got_u = _run(m, plan, A.n, cf, x, flags=m.MPK_UNBLOCKED)
        assert np.array_equal(got, got_u), (budget, p, lag)
        assert np.array_equal(got[0], x)
        for k in range(1, p + 1):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64, (budget, k)


@pytest.mark.parametrize("name", ["s27_14", "rand_nonsym_3c"])
def test_owner_fp32_and_final_only(m, name):
    import torch
    A = MATS[name]()
    A32 = mi.CSR(A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    p = 6
    cf = sstep.chebyshev_coeffs(0.1, 8.0, p)
    gamma = np.linspace(1.0, -0.5, p + 1)
    x = mi.uniform_vectors(A.n, 5)[0].astype(np.float32).astype(np.float64)
    ref = oracle.mpk(A32, p, cf, x)
    den = abs_powers(A32, cf, x)
    rp, ci, vv = to_dev(A, np.float32)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(
        l2_budget_bytes=30_000, p_blk=4, kernel=6, blocked=1))
    got = _run(m, plan, A.n, cf, x, dtype=torch.float32)
    got_u = _run(m, plan, A.n, cf, x, dtype=torch.float32, flags=m.MPK_UNBLOCKED)
    assert np.array_equal(got, got_u)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U32, k
    # the ring of three vectors (final only) and the gamma sum, blocked against unblocked
    fin = _run(m, plan, A.n, cf, x, dtype=torch.float32, flags=m.MPK_FINAL_ONLY)
    assert np.array_equal(fin[0], got[p])
    co = m.Coeffs.from_triples(cf, gamma=gamma)
    X = torch.from_numpy(x).to("cuda", torch.float32)
    outs = []
    for fl in (m.MPK_FINAL_ONLY, m.MPK_FINAL_ONLY | m.MPK_UNBLOCKED):
        Y = torch.empty(A.n, dtype=torch.float32, device="cuda")
        m.mpk_apply(plan, co, X, Y, flags=fl)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        outs.append(Y.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_owner_repeated_calls_and_level_order_io(m):
    """Counters accumulate over launches: many calls in a row, in level order and in the
    original order, each equal to the unblocked kernel's values."""
    import torch
    A = mi.stencil27(16, seed=4)
    p = 4
    cf = sstep.newton_coeffs(mi.leja_points_interval(0.0, 52.0, p))
    rp, ci, vv = to_dev(A)
    plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=60_000, kernel=6, blocked=1))
    perm = m.mpk_plan_perm(plan)["perm"].cpu().numpy()
    for seed in range(6):
        x = mi.uniform_vectors(A.n, seed)[0]
        flags = m.MPK_PERMUTED_IO if seed % 2 else 0
        xin = x[perm] if seed % 2 else x
        got = _run(m, plan, A.n, cf, xin, flags=flags)
        ref = _run(m, plan, A.n, cf, xin, flags=flags | m.MPK_UNBLOCKED)
        assert np.array_equal(got, ref), seed
