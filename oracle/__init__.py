"""CPU oracle for the level-blocked MPK and s-step GMRES path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2309_02228_gb300``) and never imports it.

* ``mpk_oracle.c`` (built into ``_liboracle.so``): plain FP64 MPK (Alg. 1 + Alg. 2, with the
  Newton / Chebyshev three-term recurrence), BFS levels, level permutation, permuted CSR and
  level groups.  ``build()`` compiles it with gcc.
* ``sstep.py``: textbook GMRES and s-step GMRES (Alg. 3), CholQR2, Leja ordering, Chebyshev
  coefficients, FP64 iterative refinement, in NumPy.
* ``poly.py``: the GMRES polynomial preconditioner (Sec. 5.2) and right-preconditioned GMRES.
* ``gs2.py``: two-stage Gauss-Seidel (GS2) preconditioning, the MPK of the GS2-preconditioned
  operator (powers made of sub-powers) and s-step GMRES with it.
* ``cg.py``: textbook CG, s-step CG (Newton basis, Gram matrix, coordinate recurrences) and
  FP64 refinement around it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpk_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, no FP contraction) into oracle/_liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        I32, I64, VP = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_mpk.argtypes = [I32, i32p, i32p, f64p, I32, f64p, f64p, f64p, f64p, f64p]
        lib.oracle_mpk.restype = None
        lib.oracle_mpk_omp.argtypes = lib.oracle_mpk.argtypes
        lib.oracle_mpk_omp.restype = None
        lib.oracle_omp_threads.argtypes = []
        lib.oracle_omp_threads.restype = I32
        lib.oracle_mpk_sampled.argtypes = [I32, i32p, i32p, f64p, I32, f64p, f64p, f64p, f64p,
                                           I32, i32p, f64p]
        lib.oracle_mpk_sampled.restype = I32
        lib.oracle_levels.argtypes = [I32, i32p, i32p, I32, I32, i32p, ctypes.POINTER(I32)]
        lib.oracle_levels.restype = I32
        lib.oracle_level_perm.argtypes = [I32, i32p, I32, i32p, i32p, i32p]
        lib.oracle_level_perm.restype = None
        lib.oracle_level_perm_bfs.argtypes = [I32, i32p, i32p, i32p, I32, i32p, i32p, i32p]
        lib.oracle_level_perm_bfs.restype = I32
        lib.oracle_permute_csr.argtypes = [I32, i32p, i32p, VP, I32, i32p, i32p, i32p, i32p, VP]
        lib.oracle_permute_csr.restype = None
        lib.oracle_level_groups.argtypes = [I32, i32p, i32p, I32, I32, I64, i32p]
        lib.oracle_level_groups.restype = I32
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _coeff_arrays(p, coeffs):
    """coeffs: sequence of p (a_k, b_k, c_k) triples, k = 1..p."""
    c = np.asarray(coeffs, dtype=np.float64).reshape(p, 3)
    return _f64(c[:, 0]), _f64(c[:, 1]), _f64(c[:, 2])


def mpk(A, p, coeffs, x, threads: bool = False):
    """Y[k] = y_k for k = 0..p, y_0 = x, y_k = a_k A y_{k-1} + b_k y_{k-1} + c_k y_{k-2}
    (Alg. 1 with the Alg. 2 row loop; Newton shifts of Sec. 4 as b_k = -theta_k).
    A: object with row_ptr/col/val.  Returns an array of shape (p+1, n), float64."""
    lib = _load()
    n = int(A.row_ptr.shape[0] - 1)
    a, b, c = _coeff_arrays(p, coeffs)
    Y = np.empty((p + 1, n), dtype=np.float64)
    fn = lib.oracle_mpk_omp if threads else lib.oracle_mpk
    fn(n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), int(p), a, b, c, _f64(x), Y)
    return Y


def mpk_sampled(A, p, coeffs, x, rows):
    """The values y_k[rows] of ``mpk`` (k = 0..p), computing only the rows they depend on.
    Returns shape (p+1, len(rows))."""
    lib = _load()
    n = int(A.row_ptr.shape[0] - 1)
    rows = _i32(rows)
    a, b, c = _coeff_arrays(p, coeffs)
    out = np.empty((p + 1, rows.shape[0]), dtype=np.float64)
    rc = lib.oracle_mpk_sampled(n, _i32(A.row_ptr), _i32(A.col), _f64(A.val), int(p), a, b, c,
                                _f64(x), int(rows.shape[0]), rows, out)
    if rc != 0:
        raise MemoryError("oracle_mpk_sampled")
    return out


def omp_threads() -> int:
    return int(_load().oracle_omp_threads())


def levels(A, root_rule: int = 0, n_sweeps: int = 2):
    """BFS levels of the symmetrised graph of A (Sec. 3).  Returns (level[n], root, n_levels)."""
    lib = _load()
    n = int(A.row_ptr.shape[0] - 1)
    lev = np.empty(n, dtype=np.int32)
    root = ctypes.c_int32(0)
    nl = lib.oracle_levels(n, _i32(A.row_ptr), _i32(A.col), int(root_rule), int(n_sweeps), lev,
                           ctypes.byref(root))
    if nl < 0:
        raise MemoryError("oracle_levels")
    return lev, int(root.value), int(nl)


def level_perm(level, n_levels):
    """Stable order of rows by (level, index).  Returns (perm, iperm, level_ptr)."""
    lib = _load()
    n = int(level.shape[0])
    perm = np.empty(n, dtype=np.int32)
    iperm = np.empty(n, dtype=np.int32)
    lp = np.empty(n_levels + 1, dtype=np.int32)
    lib.oracle_level_perm(n, _i32(level), int(n_levels), perm, iperm, lp)
    return perm, iperm, lp


def level_perm_bfs(A, level, n_levels):
    """Rows by level, and inside a level in breadth-first order: by the position of the row's
    earliest-placed neighbour (in G(A + A^T)) one level down, then by index (see
    mpk_oracle.c).  Returns (perm, iperm, level_ptr)."""
    lib = _load()
    n = int(level.shape[0])
    perm = np.empty(n, dtype=np.int32)
    iperm = np.empty(n, dtype=np.int32)
    lp = np.empty(n_levels + 1, dtype=np.int32)
    if lib.oracle_level_perm_bfs(n, _i32(A.row_ptr), _i32(A.col), _i32(level), int(n_levels),
                                 perm, iperm, lp) != 0:
        raise MemoryError("oracle_level_perm_bfs")
    return perm, iperm, lp


def permute_csr(A, perm, iperm, val_dtype=np.float64):
    """B = P A P^T with columns ascending per row; values moved bit-exactly.
    Returns (row_ptr, col, val)."""
    lib = _load()
    n = int(A.row_ptr.shape[0] - 1)
    val = np.ascontiguousarray(A.val, dtype=val_dtype)
    nnz = int(A.col.shape[0])
    rp = np.empty(n + 1, dtype=np.int32)
    ci = np.empty(nnz, dtype=np.int32)
    vo = np.empty(nnz, dtype=val_dtype)
    lib.oracle_permute_csr(n, _i32(A.row_ptr), _i32(A.col), val.ctypes.data, val.itemsize,
                           _i32(perm), _i32(iperm), rp, ci, vo.ctypes.data)
    return rp, ci, vo


def level_groups(level_ptr, rp_perm, val_bytes: int, p: int, budget: int):
    """Consecutive levels grouped under the byte budget (see mpk_oracle.c).  Returns group_ptr
    (indices into the level list, n_groups+1 entries)."""
    lib = _load()
    nl = int(level_ptr.shape[0] - 1)
    gp = np.empty(nl + 1, dtype=np.int32)
    ng = lib.oracle_level_groups(nl, _i32(level_ptr), _i32(rp_perm), int(val_bytes), int(p),
                                 int(budget), gp)
    return gp[: ng + 1].copy()


def level_structure(A, root_rule: int = 0, n_sweeps: int = 2, level_order: int = 0):
    """levels + the level permutation in one call: (level, root, n_levels, perm, iperm,
    level_ptr).  level_order 0: index order inside a level; 1: breadth-first order."""
    lev, root, nl = levels(A, root_rule, n_sweeps)
    if level_order == 1:
        perm, iperm, lp = level_perm_bfs(A, lev, nl)
    else:
        perm, iperm, lp = level_perm(lev, nl)
    return lev, root, nl, perm, iperm, lp
