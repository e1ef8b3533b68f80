"""The cycle-internals comparison (tests/trace_check.py) accepts the oracle's own cycle and
rejects it with one planted mistake: a wrong Hessenberg column, or a wrong estimate."""
import numpy as np

import mpk_inputs as mi
from oracle import sstep
from tests.trace_check import trace_problems


def _cycle():
    A = mi.diffusion7_lognormal(8)
    b = mi.uniform_vectors(A.n, 3)[0]
    th = mi.leja_points_interval(0.5, 12.0, 4)
    r = sstep.sstep_gmres(A, b, s=4, m=24, tol=1e-9, max_restarts=1, shifts=th)
    return np.asarray(r["hist"]), r["H_cycle"], r["k_cycle"]


def test_own_cycle_passes():
    hist, H, k = _cycle()
    assert k > 8
    assert trace_problems(hist, H, hist, H, k) == []


def test_planted_wrong_hessenberg_column_fails():
    hist, H, k = _cycle()
    for col in (0, k // 2, k - 1):
        bad = H.copy()
        bad[: col + 2, col] *= 1.0 + 1e-6     # one column 1e-6 off
        assert trace_problems(hist, bad, hist, H, k)
        bad = H.copy()
        bad[col + 1, col] = -bad[col + 1, col]   # a wrong sign on the subdiagonal
        assert trace_problems(hist, bad, hist, H, k)


def test_planted_wrong_estimate_fails():
    hist, H, k = _cycle()
    bad = hist.copy()
    bad[3] *= 1.0 + 1e-7
    assert trace_problems(bad, H, hist, H, k)
    short = hist[: k - 1]
    assert trace_problems(short, H, hist, H, k)
