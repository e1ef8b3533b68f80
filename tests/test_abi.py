"""The C ABI: the library builds, loads, and exports every function include/mpk.h declares;
the binding declares the same set.  Host-only helpers (no GPU involved) are checked against
the oracle's independent versions."""
import ctypes
import os
import re

import numpy as np
import pytest

import mpk_inputs as mi
from oracle import sstep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as m
    return m


def test_library_exports_every_declared_symbol(built):
    decl = declared_functions()
    assert {"mpk_plan_create", "mpk_apply", "sstep_gmres_solve", "mpk_plan_destroy"} <= decl
    L = ctypes.CDLL(built.LIB_PATH)
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(built.exported_symbols()) == decl


def test_host_helpers_match_oracle(built):
    m = built
    co = m.mpk_coeffs_chebyshev(0.1, 52.0, 6)
    ref = np.array(sstep.chebyshev_coeffs(0.1, 52.0, 6))
    assert np.array_equal(np.stack([co.a, co.b, co.c], 1), ref)
    th = mi.leja_points_interval(0, 52, 8)
    co = m.mpk_coeffs_newton(th)
    assert np.array_equal(np.stack([co.a, co.b, co.c], 1), np.array(sstep.newton_coeffs(th)))
    rng = np.random.default_rng(3)
    for _ in range(5):
        v = np.unique(np.round(rng.uniform(0.05, 60, size=40), 4))
        assert np.array_equal(m.mpk_leja_order(v, 8), sstep.leja_order(v, 8))
    assert m.mpk_version().startswith("mpk_gb300")
    assert m.status_name(m.MPK_ERR_TIMEOUT) == "MPK_ERR_TIMEOUT"


def test_argument_errors_without_gpu(built):
    """Invalid arguments are rejected before any device work."""
    m = built
    h = ctypes.c_void_p(0)
    assert m.lib().mpk_plan_create(None, 4, None, None, ctypes.byref(h)) == m.MPK_ERR_ARG
    A = m.mpk_csr(10, 0, 0, 0, 0, m.MPK_F64)
    assert m.lib().mpk_plan_create(ctypes.byref(A), 0, None, None, ctypes.byref(h)) == m.MPK_ERR_ARG
    assert m.lib().mpk_plan_create(ctypes.byref(A), 64, None, None, ctypes.byref(h)) == m.MPK_ERR_ARG
    assert m.lib().mpk_coeffs_chebyshev(1.0, 0.5, 3, None, None, None) == m.MPK_ERR_ARG


def _match(got, ref):
    """Largest distance between two eigenvalue multisets (greedy nearest matching)."""
    used = np.zeros(len(got), bool)
    worst = 0.0
    for z in ref:
        d = np.abs(got - z)
        d[used] = np.inf
        i = int(np.argmin(d))
        used[i] = True
        worst = max(worst, float(d[i]))
    return worst


def test_hessenberg_eigenvalues_match_numpy(built):
    """The Ritz values' eigen solver (mpk_hessenberg_eigvals, host QR iteration) against
    numpy.linalg.eigvals (LAPACK): random upper Hessenberg matrices (complex pairs), split
    subdiagonals, symmetric tridiagonals, a Jordan-like defective block, and k up to 128."""
    m = built
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 4, 7, 16, 48, 128):
        cases = [np.triu(rng.standard_normal((n, n)), -1)]
        if n > 3:
            H = np.triu(rng.standard_normal((n, n)), -1)
            H[n // 2, n // 2 - 1] = 0.0
            H[1, 0] = 0.0
            cases.append(H)
        d = rng.uniform(-5, 5, n)
        e = rng.standard_normal(max(n - 1, 0))
        cases.append(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))
        for H in cases:
            got = m.mpk_hessenberg_eigvals(H)
            ref = np.linalg.eigvals(H)
            assert _match(got, ref) <= 1e-10 * max(1.0, np.linalg.norm(H)), n
            # complex pairs come as (a + bi, a - bi)
            for i in np.nonzero(got.imag > 0)[0]:
                assert got[i + 1] == np.conj(got[i])
    # a 2 x 2 rotation block inside a triangular matrix: eigenvalues 3 +- 2i, 1, 5
    H = np.array([[3.0, 2.0, 1.0, 0.5], [-2.0, 3.0, 0.2, 0.1], [0.0, 0.0, 1.0, 4.0], [0.0, 0.0, 0.0, 5.0]])
    got = np.sort_complex(m.mpk_hessenberg_eigvals(H))
    assert np.allclose(got, np.sort_complex(np.array([1.0, 5.0, 3 + 2j, 3 - 2j])), atol=1e-13)
    # defective: a Jordan block of size 4 (eigenvalue 2, sensitive as eps^(1/4))
    J = 2.0 * np.eye(4) + np.diag(np.ones(3), 1)
    assert _match(m.mpk_hessenberg_eigvals(J), np.full(4, 2.0)) <= 1e-3
    with pytest.raises(m.MpkError):
        m.mpk_hessenberg_eigvals(np.full((3, 3), np.nan))
