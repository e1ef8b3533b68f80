"""GPU checks of the autotuner (mpk_autotune, an addition without a counterpart in the paper,
which tunes p_opt and its cache size by hand): it times every candidate, returns options that
build a working plan whose results equal p back-to-back SpMVs bit for bit, never reports a best
slower than the base options, works for blocks of right-hand sides, and rejects invalid calls.
All calls go through the C ABI."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle
from oracle import sstep
from tests.gpu_util import U64, abs_powers, max_rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def test_autotune_fp64(m):
    import torch
    A = mi.stencil27(40, seed=2)
    p = 4
    cf = sstep.newton_coeffs(mi.leja_points_interval(0.0, 52.0, p))
    rp, ci, vv = to_dev(A)
    best, info = m.mpk_autotune(rp, ci, vv, cf, reps=3)
    assert info["n_trials"] == 9
    assert 0 <= info["best_index"] < 9
    assert 0 < info["best_ms"] <= info["base_ms"]
    plan = m.mpk_plan_create(rp, ci, vv, p, best)
    x = mi.uniform_vectors(A.n, 0)[0]
    X = torch.from_numpy(x).cuda()
    Y = torch.empty((p + 1) * A.n, dtype=torch.float64, device="cuda")
    Yu = torch.empty_like(Y)
    m.mpk_apply(plan, cf, X, Y)
    m.mpk_apply(plan, cf, X, Yu, flags=m.MPK_UNBLOCKED)
    assert m.mpk_plan_sync(plan) == m.MPK_OK
    assert torch.equal(Y, Yu)
    got = Y.view(p + 1, A.n).cpu().numpy()
    ref = oracle.mpk(A, p, cf, x)
    den = abs_powers(A, cf, x)
    for k in range(1, p + 1):
        assert max_rel_err(got[k], ref[k], den[k]) <= 64 * k * U64


def test_autotune_block_rhs_fp32(m):
    A = mi.stencil27(32, seed=5)
    p = 6
    co = m.mpk_coeffs_chebyshev(0.1, 52.0, p)
    rp, ci, _ = to_dev(A)
    _, _, v32 = to_dev(A, np.float32)
    fl = m.MPK_PERMUTED_IO | m.MPK_RHS_INTERLEAVED
    best, info = m.mpk_autotune(rp, ci, v32, co, n_rhs=8, flags=fl, reps=2)
    assert info["n_trials"] == 9 and info["best_ms"] <= info["base_ms"]
    best2, info2 = m.mpk_autotune(rp, ci, v32, co, n_rhs=8, flags=fl | m.MPK_FINAL_ONLY, reps=2)
    assert info2["n_trials"] == 9
    assert m.mpk_plan_create(rp, ci, v32, p, best).n == A.n


def test_autotune_rejects_invalid_calls(m):
    A = mi.poisson2d_5pt(16)
    rp, ci, vv = to_dev(A)
    cf = sstep.monomial_coeffs(3)
    for kw in ({"flags": m.MPK_HOST_IO}, {"flags": m.MPK_UNBLOCKED}, {"reps": 0}, {"n_rhs": 0}):
        _, info = m.mpk_autotune(rp, ci, vv, cf, check=False, **kw)
        assert info["status_code"] == m.MPK_ERR_ARG, kw
