"""GPU parity of the batched MPK (mpk_batch_*): many uneven systems in one persistent launch.

Every system's powers equal its own mpk_apply's bit for bit (the same row function) and the
oracle's recurrence on that system's level-ordered matrix within the MPK tolerance, per entry
relative to (|A_theta|^k |x|)_i: 64 k 2^-53 in FP64, 64 k 2^-24 in FP32.  Also: a captured
CUDA graph of a batch call replays correctly on new inputs, and MPK_UNBLOCKED gives the same
values.  All calls go through the C ABI."""
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


def _systems():
    return [
        mi.stencil27(12, seed=2),
        mi.diffusion7_lognormal(10),
        mi.poisson2d_5pt(40),
        mi.anisotropic(9, 27, 30.0),
        mi.random_sparse(300, 0.02, 1, symmetric=False, components=3),
        mi.CSR(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0])),   # one row
        mi.anisotropic(14, 7, 5.0),
        mi.stencil27(7, seed=4),
    ]


def _coeffs(i, A, p):
    hi = 2.2 * float(np.abs(A.val).max()) * 3
    if i % 2:
        return sstep.chebyshev_coeffs(0.0, hi, p)
    return sstep.newton_coeffs(mi.leja_points_interval(0.0, hi, p))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_batch_matches_each_system_and_the_oracle(m, dt):
    import torch
    tdt = torch.float64 if dt == "f64" else torch.float32
    npdt = np.float64 if dt == "f64" else np.float32
    p = 6
    mats = _systems()
    plans, cfs, xs, Ys = [], [], [], []
    for i, A in enumerate(mats):
        rp, ci, vv = to_dev(A, npdt)
        plans.append(m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(l2_budget_bytes=40_000)))
        cfs.append(_coeffs(i, A, p))
        x = mi.uniform_vectors(A.n, 20 + i)[0].astype(npdt).astype(np.float64)
        xs.append(torch.from_numpy(x).to("cuda", tdt))
        Ys.append(torch.full(((p + 1) * A.n,), float("nan"), dtype=tdt, device="cuda"))
    B = m.Batch(plans, p, tdt)
    B.apply(cfs, xs, Ys)
    assert B.sync() == m.MPK_OK
    u = U64 if dt == "f64" else U32
    for i, (A, plan) in enumerate(zip(mats, plans)):
        got = Ys[i].view(p + 1, A.n).double().cpu().numpy()
        # alone: the plan's own call (blocked, level order) - the same values bit for bit
        Yo = torch.full_like(Ys[i], float("nan"))
        m.mpk_apply(plan, cfs[i], xs[i], Yo, flags=m.MPK_PERMUTED_IO)
        Yu = torch.full_like(Ys[i], float("nan"))
        m.mpk_apply(plan, cfs[i], xs[i], Yu, flags=m.MPK_PERMUTED_IO | m.MPK_UNBLOCKED)
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        assert np.array_equal(got, Yo.view(p + 1, A.n).double().cpu().numpy()), i
        assert np.array_equal(got, Yu.view(p + 1, A.n).double().cpu().numpy()), i
        # the oracle on the system's level-ordered matrix as the GPU holds it
        grp, gci, gval = m.mpk_plan_csr(plan, tdt)
        Bm = mi.CSR(grp.cpu().numpy(), gci.cpu().numpy(), gval.double().cpu().numpy())
        x = xs[i].double().cpu().numpy()
        ref = oracle.mpk(Bm, p, cfs[i], x)
        den = abs_powers(Bm, cfs[i], x)
        for k in range(1, p + 1):
            assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * u, (i, k)


def test_batch_many_uneven_systems_and_unblocked(m):
    """40 systems of grid edges 8..28 (7- and 27-point, anisotropic): batch == unblocked."""
    import torch
    p = 8
    rng = np.random.default_rng(5)
    plans, cfs, xs, Ys, ns = [], [], [], [], []
    for i in range(40):
        N = int(rng.integers(8, 29))
        A = mi.anisotropic(N, 7 if i % 2 else 27, float(rng.uniform(1.0, 100.0)))
        rp, ci, vv = to_dev(A, np.float32)
        plans.append(m.mpk_plan_create(rp, ci, vv, p))
        cfs.append(_coeffs(i, A, p))
        xs.append(torch.from_numpy(mi.uniform_vectors(A.n, 100 + i)[0]).to("cuda", torch.float32))
        Ys.append(torch.empty(((p + 1) * A.n,), dtype=torch.float32, device="cuda"))
        ns.append(A.n)
    B = m.Batch(plans, p, torch.float32)
    B.apply(cfs, xs, Ys)
    assert B.sync() == m.MPK_OK
    got = [y.clone() for y in Ys]
    B.apply(cfs, xs, Ys, flags=m.MPK_PERMUTED_IO | m.MPK_UNBLOCKED)
    assert B.sync() == m.MPK_OK
    for a, b in zip(got, Ys):
        assert torch.equal(a, b)


def test_batch_graph_capture_replays(m):
    import torch
    p = 5
    mats = [mi.stencil27(10, seed=1), mi.diffusion7_lognormal(9), mi.poisson2d_5pt(30)]
    plans, cfs, Ys = [], [], []
    for i, A in enumerate(mats):
        rp, ci, vv = to_dev(A)
        plans.append(m.mpk_plan_create(rp, ci, vv, p))
        cfs.append(_coeffs(i, A, p))
        Ys.append(torch.zeros(((p + 1) * A.n,), dtype=torch.float64, device="cuda"))
    B = m.Batch(plans, p, torch.float64)
    fl = m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X
    B.apply(cfs, None, Ys, flags=fl)                  # uploads the records, builds the schedule
    assert B.sync() == m.MPK_OK
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        B.apply(cfs, None, Ys, flags=fl)
    for seed in (3, 4):
        xs = []
        for i, A in enumerate(mats):
            x = torch.from_numpy(mi.uniform_vectors(A.n, seed * 10 + i)[0]).cuda()
            Ys[i][: A.n].copy_(x)
            xs.append(x)
        g.replay()
        torch.cuda.synchronize()
        assert B.sync() == m.MPK_OK
        for i, (A, plan) in enumerate(zip(mats, plans)):
            Yo = torch.empty_like(Ys[i])
            m.mpk_apply(plan, cfs[i], xs[i], Yo, flags=m.MPK_PERMUTED_IO | m.MPK_UNBLOCKED)
            torch.cuda.synchronize()
            assert torch.equal(Ys[i], Yo), (seed, i)
