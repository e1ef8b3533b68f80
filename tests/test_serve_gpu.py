"""GPU tests of the solve server (continuous batching under an HBM budget).

Each request's solution is bitwise identical whether it runs alone or mixed with others
(every reduction in the solve has a fixed order), also with GS2-preconditioned solves, every
solution reaches the 1e-8 true residual, solves run concurrently (their [start, done]
intervals overlap), a request submitted while others run is admitted before they all finish,
a request larger than the budget is refused, and a budget that fits one request at a time
serialises admission."""
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


def test_concurrent_solves_and_admission_mid_run(m):
    """Three solves submitted together run concurrently (their [start, done] intervals
    overlap); a fourth submitted while they run is admitted (started) before all three have
    finished; every result is the same as the request's solve alone."""
    reqs = []
    # the first three are large enough (a few hundred thousand rows, anisotropy up to 40) to
    # run for well over the 10 ms before the fourth is submitted; the fourth is small
    for N, st, a in ((64, 27, 5.0), (60, 27, 12.0), (72, 7, 40.0), (20, 27, 3.0)):
        A = mi.anisotropic(N, st, a)
        reqs.append((A, mi.uniform_vectors(A.n, N)[0]))
    srv = m.Server(m.mpk_server_opts_default(max_active=4))
    ids = [srv.submit(A.row_ptr, A.col, A.val, b)[0] for A, b in reqs[:3]]
    time.sleep(0.01)
    late, _ = srv.submit(reqs[3][0].row_ptr, reqs[3][0].col, reqs[3][0].val, reqs[3][1])
    got = _drain(srv, 4)
    srv.close()
    first = [got[i] for i in ids]
    for r in first + [got[late]]:
        assert r["status"] == m.MPK_OK, r
    spans = [(r["t_start_ms"], r["t_done_ms"]) for r in first]
    overlap = any(min(d0, d1) > max(s0, s1) for i, (s0, d0) in enumerate(spans)
                  for (s1, d1) in spans[i + 1:])
    assert overlap, spans
    lr = got[late]
    assert min(s for s, _ in spans) < lr["t_submit_ms"] < max(d for _, d in spans), (lr, spans)
    assert lr["t_start_ms"] < max(d for _, d in spans), (lr, spans)   # admitted before all done
    # the same solutions alone
    srv = m.Server(m.mpk_server_opts_default(max_active=1))
    for (A, b), rid in zip(reqs, ids + [late]):
        aid, _ = srv.submit(A.row_ptr, A.col, A.val, b)
        alone = _drain(srv, 1)[aid]
        assert np.array_equal(alone["x"], got[rid]["x"])
    srv.close()


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
