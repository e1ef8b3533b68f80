"""GPU tests of the solve server (continuous batching under an HBM budget).

Each request's solution is bitwise identical whether it runs alone or mixed with others
(every reduction in the solve has a fixed order), also with GS2-preconditioned solves, every
solution reaches the 1e-8 true
residual, a request larger than the budget is refused, and a budget that fits one request at
a time serialises admission."""
import time

import numpy as np
import pytest

import mpk_inputs as mi
from oracle import sstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def _requests(k=10):
    reqs = []
    for r in mi.solve_stream(k, seed=7, n_min=8, n_max=16):
        A = mi.anisotropic(r["N"], r["stencil"], min(r["a"], 20.0))
        b = mi.uniform_vectors(A.n, r["b_seed"] % 100000)[0]
        reqs.append((A, b))
    return reqs


def _drain(srv, expect, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < expect:
        for res in srv.poll(64):
            out[res["id"]] = res
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.001)
    return out


@pytest.mark.parametrize("precond", ["none", "gs2"])
def test_alone_vs_mixed_bitwise(m, precond):
    reqs = _requests(10)

    def opts(**kw):
        o = m.mpk_server_opts_default(**kw)
        if precond == "gs2":   # two-stage Gauss-Seidel sub-powers (Sec. 5.1) in every solve
            o.gmres.gs2 = 1
            o.gmres.gs2_gamma = 1
        return o
    srv = m.Server(opts(max_active=1))
    alone = []
    for A, b in reqs:
        rid, x = srv.submit(A.row_ptr, A.col, A.val, b)
        res = _drain(srv, 1)[rid]
        assert res["status"] == m.MPK_OK, res
        alone.append(res["x"].copy())
    srv.close()
    srv = m.Server(opts(max_active=4))
    ids = [srv.submit(A.row_ptr, A.col, A.val, b)[0] for A, b in reqs]
    got = _drain(srv, len(ids))
    srv.close()
    for i, (A, b) in enumerate(reqs):
        res = got[ids[i]]
        assert res["status"] == m.MPK_OK
        assert np.array_equal(res["x"], alone[i])
        rr = np.linalg.norm(b - sstep.spmv(A, res["x"])) / np.linalg.norm(b)
        assert rr <= 1e-8, rr
        assert res["t_submit_ms"] <= res["t_start_ms"] <= res["t_done_ms"]


def test_budget_refusal_and_serialised_admission(m):
    A = mi.anisotropic(12, 27, 5.0)
    b = mi.uniform_vectors(A.n, 1)[0]
    srv = m.Server(m.mpk_server_opts_default(hbm_budget_bytes=1 << 20))
    with pytest.raises(m.MpkError) as e:
        srv.submit(A.row_ptr, A.col, A.val, b)
    assert e.value.status == m.MPK_ERR_BUDGET
    srv.close()
    # a budget a bit above one request's estimate: requests run one after the other
    probe = m.Server(m.mpk_server_opts_default())
    est = None
    probe.close()
    nnz, n = A.nnz, A.n
    o = m.mpk_server_opts_default(max_active=4)
    est = 12 * nnz + 4 * (n + 1) + 2 * 12 * nnz + 16 * nnz + 64 * n + (8 << 20) \
        + (o.gmres.restart + 1) * 4 * ((n + 31) // 32 * 32) + 24 * n + (16 << 20)
    srv = m.Server(m.mpk_server_opts_default(max_active=4, hbm_budget_bytes=int(est * 1.5)))
    ids = [srv.submit(A.row_ptr, A.col, A.val, b)[0] for _ in range(3)]
    got = _drain(srv, 3)
    srv.close()
    ts = sorted((got[i]["t_start_ms"], got[i]["t_done_ms"]) for i in ids)
    for (s0, d0), (s1, d1) in zip(ts, ts[1:]):
        assert s1 >= d0 - 1e-6
    for i in ids:
        assert got[i]["status"] == m.MPK_OK
