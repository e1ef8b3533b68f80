"""Comparison of one s-step GMRES cycle's internals (the residual estimate after each column's
Givens rotation, and the unrotated Arnoldi Hessenberg) with the oracle's.  Host-side only; used
by the GPU parity test and pinned by a CPU test that plants wrong values."""
import numpy as np

RTOL = 1e-8          # relative to the estimate, or to the largest Hessenberg entry
EST_FLOOR = 1e-6     # below this relative residual an estimate is compared absolutely
EST_ATOL = 1e-14


def trace_problems(hist, H, ref_hist, ref_H, k):
    """Mismatches (list of strings) between the first k estimates / Hessenberg columns of a
    cycle and the oracle's; empty when they agree."""
    out = []
    hist = np.asarray(hist, dtype=np.float64)
    ref_hist = np.asarray(ref_hist, dtype=np.float64)
    if hist.shape[0] < k or ref_hist.shape[0] < k:
        return ["fewer than %d estimates" % k]
    for c in range(k):
        r = ref_hist[c]
        tol = RTOL * r if r >= EST_FLOOR else EST_ATOL
        if not abs(hist[c] - r) <= tol:
            out.append("estimate %d: %.17g vs %.17g" % (c, hist[c], r))
    Hk = np.asarray(H, dtype=np.float64)[: k + 1, :k]
    Rk = np.asarray(ref_H, dtype=np.float64)[: k + 1, :k]
    scale = np.abs(Rk).max() if Rk.size else 0.0
    bad = np.argwhere(~(np.abs(Hk - Rk) <= RTOL * scale))
    for i, j in bad[:10]:
        out.append("H[%d, %d]: %.17g vs %.17g" % (i, j, Hk[i, j], Rk[i, j]))
    return out
