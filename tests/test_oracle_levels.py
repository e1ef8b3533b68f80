"""Pins for the oracle's level construction (Sec. 3: BFS levels of the matrix graph), the
level permutation, the permuted matrix and the level groups.

Closed forms on grids from a corner root (5-point: i+j; 7-point: i+j+k; 27-point:
max(i,j,k)), unweighted shortest paths from scipy.sparse.csgraph (library special case) on
random graphs, scipy's own sparse indexing for P A P^T, and invariants that hold for any
graph.  The hand-drawn fixture under tests/golden/ is worked out by hand from the definition."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path, connected_components

import mpk_inputs as mi
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def grid_coords3(N):
    idx = np.arange(N ** 3)
    i, r = np.divmod(idx, N * N)
    j, k = np.divmod(r, N)
    return i, j, k


def check_invariants(A, lev, root, nl):
    n = A.n
    assert lev.min() == 0 and lev.max() == nl - 1
    assert set(np.unique(lev)) == set(range(nl))          # levels partition the rows
    assert lev[root] == 0 and np.count_nonzero(lev == 0) == 1
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    assert np.all(np.abs(lev[rows] - lev[A.col]) <= 1)    # every nonzero spans <= 1 level


@pytest.mark.parametrize("N", [1, 2, 7, 16])
def test_grid_closed_forms(N):
    A5 = mi.poisson2d_5pt(N)
    lev, root, nl = oracle.levels(A5, root_rule=1)
    i, j = np.divmod(np.arange(N * N), N)
    assert root == 0 and np.array_equal(lev, i + j) and nl == 2 * N - 1
    A7 = mi.stencil7(N)
    lev, root, nl = oracle.levels(A7, root_rule=0)
    i, j, k = grid_coords3(N)
    assert root == 0 and np.array_equal(lev, i + j + k) and nl == 3 * N - 2
    A27 = mi.stencil27(N, seed=2)
    lev, root, nl = oracle.levels(A27, root_rule=0)
    assert root == 0 and np.array_equal(lev, np.maximum(np.maximum(i, j), k)) and nl == N
    # level sizes of the 27-point shells: 3L^2 + 3L + 1
    sizes = np.bincount(lev)
    L = np.arange(N)
    assert np.array_equal(sizes, 3 * L * L + 3 * L + 1)


def test_permuted_grid_recovers_manhattan_distance():
    """A randomly permuted 7-point grid: the George-Liu root is a grid corner and the levels
    are the Manhattan distances from it."""
    N = 9
    A = mi.diffusion7_lognormal(N, permute=True)
    perm = np.random.default_rng(1).permutation(N ** 3)   # row r of A is grid cell perm[r]
    lev, root, nl = oracle.levels(A, root_rule=0)
    check_invariants(A, lev, root, nl)
    i, j, k = grid_coords3(N)
    ci, cj, ck = i[perm[root]], j[perm[root]], k[perm[root]]
    assert {ci, cj, ck} <= {0, N - 1}                      # a corner
    man = np.abs(i[perm] - ci) + np.abs(j[perm] - cj) + np.abs(k[perm] - ck)
    assert np.array_equal(lev, man) and nl == 3 * N - 2


@pytest.mark.parametrize("seed,comp,sym", [(0, 1, True), (1, 3, True), (2, 1, False),
                                           (3, 4, False), (4, 2, True)])
def test_random_graphs_vs_shortest_path(seed, comp, sym):
    A = mi.random_sparse(60, 0.05, seed, symmetric=sym, components=comp)
    n = A.n
    S = sp.csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(n, n))
    G = ((S + S.T) > 0).astype(np.float64)
    G.setdiag(0)
    G.eliminate_zeros()
    for rule in (0, 1):
        lev, root, nl = oracle.levels(A, root_rule=rule)
        check_invariants(A, lev, root, nl)
        dist = shortest_path(G, unweighted=True, directed=False, indices=root)
        reach = np.isfinite(dist)
        assert np.array_equal(lev[reach], dist[reach].astype(np.int32))
        # other components: each starts at its lowest-index row, one level above the last
        ncomp, lab = connected_components(G, directed=False)
        top = int(dist[reach].max())
        done = set(np.flatnonzero(reach))
        while len(done) < n:
            start = min(set(range(n)) - done)
            d2 = shortest_path(G, unweighted=True, directed=False, indices=start)
            r2 = np.isfinite(d2)
            assert np.array_equal(lev[r2], (top + 1 + d2[r2]).astype(np.int32))
            top = int(top + 1 + d2[r2].max())
            done |= set(np.flatnonzero(r2))
        assert nl == top + 1
        if rule == 1:
            assert root == 0


def test_george_liu_root_properties():
    """The George-Liu root never has smaller eccentricity than row 0 and lies in row 0's
    component; on a path graph it is an end point (eccentricity = diameter)."""
    n = 31
    rows, cols = [], []
    order = np.random.default_rng(5).permutation(n)
    for t in range(n - 1):
        a, b = order[t], order[t + 1]
        rows += [a, b]
        cols += [b, a]
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    M.setdiag(1.0)
    M = M.tocsr()
    M.sort_indices()
    A = mi.CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    lev, root, nl = oracle.levels(A, root_rule=0)
    assert root in (order[0], order[-1]) and nl == n
    for seed in range(6):
        B = mi.random_sparse(50, 0.06, seed + 20, symmetric=True, components=1)
        S = sp.csr_matrix((np.ones(B.nnz), B.col, B.row_ptr), shape=(50, 50))
        D = shortest_path(S, unweighted=True, directed=False)
        lev, root, nl = oracle.levels(B, root_rule=0)
        if np.isfinite(D[0]).all():
            assert D[root].max() >= D[0].max()


def test_golden_hand_worked_levels():
    """Hand-worked BFS levels, permutation and groups of a 10-row graph (tests/golden)."""
    with open(os.path.join(GOLD, "levels_small.json")) as f:
        g = json.load(f)
    A = mi.CSR(np.array(g["row_ptr"], dtype=np.int32), np.array(g["col"], dtype=np.int32),
               np.ones(len(g["col"])))
    lev, root, nl = oracle.levels(A, root_rule=g["root_rule"])
    assert root == g["root"] and lev.tolist() == g["level"] and nl == g["n_levels"]
    perm, iperm, lp = oracle.level_perm(lev, nl)
    assert perm.tolist() == g["perm"] and lp.tolist() == g["level_ptr"]
    rp, ci, vv = oracle.permute_csr(A, perm, iperm)
    gp = oracle.level_groups(lp, rp, 8, g["groups_p"], g["groups_budget"])
    assert gp.tolist() == g["group_ptr"]


def test_level_perm_matches_lexsort():
    A = mi.diffusion7_lognormal(8)
    lev, root, nl = oracle.levels(A)
    perm, iperm, lp = oracle.level_perm(lev, nl)
    ref = np.lexsort((np.arange(A.n), lev))                 # by level, then index
    assert np.array_equal(perm, ref)
    assert np.array_equal(iperm[perm], np.arange(A.n))
    assert np.array_equal(lp, np.concatenate([[0], np.cumsum(np.bincount(lev, minlength=nl))]))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_permute_csr_matches_scipy(dtype):
    A = mi.stencil27(7, seed=2)
    lev, root, nl = oracle.levels(A)
    perm, iperm, lp = oracle.level_perm(lev, nl)
    rp, ci, vv = oracle.permute_csr(A, perm, iperm, val_dtype=dtype)
    S = sp.csr_matrix((A.val.astype(dtype), A.col, A.row_ptr), shape=(A.n, A.n))
    B = S[perm][:, perm].tocsr()
    B.sort_indices()
    assert np.array_equal(rp, B.indptr) and np.array_equal(ci, B.indices)
    assert np.array_equal(vv.view(np.uint8), B.data.astype(dtype).view(np.uint8))


def test_permute_csr_keeps_duplicate_order():
    """Duplicate column entries keep their stored order (stable), values moved bit-exactly."""
    rp = np.array([0, 3, 5], dtype=np.int32)
    col = np.array([1, 0, 1, 1, 0], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    A = mi.CSR(rp, col, val)
    perm = np.array([1, 0], dtype=np.int32)
    iperm = np.array([1, 0], dtype=np.int32)
    r2, c2, v2 = oracle.permute_csr(A, perm, iperm)
    # new row 0 = old row 1: cols [1,0] -> [0,1]; new row 1 = old row 0: cols [1,0,1] -> [0,1,0]
    assert r2.tolist() == [0, 2, 5]
    assert c2.tolist() == [0, 1, 0, 0, 1]
    assert v2.tolist() == [4.0, 5.0, 1.0, 3.0, 2.0]


def test_level_groups_rule():
    """Groups partition the levels; every multi-level group fits the budget; adding the next
    level to any group would exceed it (maximality of the greedy walk)."""
    A = mi.stencil27(12, seed=2)
    lev, root, nl = oracle.levels(A)
    perm, iperm, lp = oracle.level_perm(lev, nl)
    rp, ci, vv = oracle.permute_csr(A, perm, iperm)
    w, p = 8, 4

    def cost(l0, l1):
        R = int(lp[l1] - lp[l0])
        Z = int(rp[lp[l1]] - rp[lp[l0]])
        return p * (4 * R + (4 + w) * Z) + (p + 1) * w * R

    for budget in (10_000, 200_000, 1_000_000, 10 ** 12):
        gp = oracle.level_groups(lp, rp, w, p, budget)
        assert gp[0] == 0 and gp[-1] == nl and np.all(np.diff(gp) >= 1)
        for g in range(len(gp) - 1):
            if gp[g + 1] - gp[g] > 1:
                assert cost(gp[g], gp[g + 1]) <= budget
            if gp[g + 1] < nl:
                assert cost(gp[g], gp[g + 1] + 1) > budget
        if budget == 10 ** 12:
            assert gp.tolist() == [0, nl]


# ---- breadth-first order inside levels (the plan's level_order = 1)

def _queue_bfs_order(A, lev):
    """The same order by its other definition: a queue breadth-first search from each
    component's root (the row alone on the first level of its component), every row taken
    from the queue appending its not yet placed next-level neighbours (in G(A + A^T)) in
    ascending index.  Plain Python, for small graphs."""
    n = A.n
    nb = [set() for _ in range(n)]
    for i in range(n):
        for j in A.col[A.row_ptr[i]:A.row_ptr[i + 1]]:
            if j != i:
                nb[i].add(int(j))
                nb[int(j)].add(i)
    roots = sorted((int(lev[i]), i) for i in range(n)
                   if not any(lev[j] == lev[i] - 1 for j in nb[i]))
    order, placed = [], np.zeros(n, bool)
    for _, r in roots:
        q = [r]
        placed[r] = True
        order.append(r)
        h = 0
        while h < len(q):
            i = q[h]
            h += 1
            for j in sorted(nb[i]):
                if lev[j] == lev[i] + 1 and not placed[j]:
                    placed[j] = True
                    order.append(j)
                    q.append(j)
    return np.array(order, dtype=np.int32)


def test_bfs_order_golden_hand_worked():
    with open(os.path.join(GOLD, "level_order_bfs_small.json")) as f:
        g = json.load(f)
    A = mi.CSR(np.array(g["row_ptr"], dtype=np.int32), np.array(g["col"], dtype=np.int32),
               np.ones(len(g["col"])))
    lev, root, nl = oracle.levels(A, root_rule=g["root_rule"])
    assert lev.tolist() == g["level"] and nl == g["n_levels"]
    perm, iperm, lp = oracle.level_perm(lev, nl)
    assert perm.tolist() == g["perm_index"] and lp.tolist() == g["level_ptr"]
    perm, iperm, lp = oracle.level_perm_bfs(A, lev, nl)
    assert perm.tolist() == g["perm_bfs"] and lp.tolist() == g["level_ptr"]
    assert np.array_equal(iperm[perm], np.arange(A.n))


@pytest.mark.parametrize("seed,comp,sym", [(0, 1, True), (1, 3, False), (2, 1, False), (3, 5, True)])
def test_bfs_order_matches_queue_definition(seed, comp, sym):
    A = mi.random_sparse(400, 0.01, seed, symmetric=sym, components=comp)
    lev, root, nl = oracle.levels(A)
    perm, iperm, lp = oracle.level_perm_bfs(A, lev, nl)
    assert np.array_equal(perm, _queue_bfs_order(A, lev))
    assert np.array_equal(iperm[perm], np.arange(A.n))
    assert np.array_equal(lp, oracle.level_perm(lev, nl)[2])     # the same levels and sizes


def test_bfs_order_on_permuted_grid_matches_queue_and_keys():
    """A randomly relabelled 7-point grid (the solver workload's structure): the queue
    definition, levels still contiguous, and inside each level the keys (earliest lower
    neighbour's position) non-decreasing with ties in ascending index."""
    A = mi.diffusion7_lognormal(7)
    lev, root, nl = oracle.levels(A)
    perm, iperm, lp = oracle.level_perm_bfs(A, lev, nl)
    assert np.array_equal(perm, _queue_bfs_order(A, lev))
    assert np.all(np.diff(lev[perm]) >= 0)
    S = sp.csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(A.n, A.n))
    S = (S + S.T).tocsr()
    for q in range(1, A.n):
        if lev[perm[q]] != lev[perm[q - 1]] or lev[perm[q]] == 0:
            continue
        def key(r):
            nbr = S.indices[S.indptr[r]:S.indptr[r + 1]]
            return min(iperm[j] for j in nbr if lev[j] == lev[r] - 1)
        a, b = perm[q - 1], perm[q]
        assert (key(a), a) < (key(b), b)


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_bfs_order_on_natural_2d_grid_is_index_order(N):
    """On a 5-point grid numbered row by row, from the corner root, the earliest lower
    neighbour of (i, j) is (i-1, j) (or (0, j-1) on the first row, which shares its key with
    (1, j-1) and wins the tie by index), so the breadth-first order inside each anti-diagonal
    is the index order."""
    A = mi.poisson2d_5pt(N)
    lev, root, nl = oracle.levels(A, root_rule=1)
    pb = oracle.level_perm_bfs(A, lev, nl)
    pi = oracle.level_perm(lev, nl)
    for a, b in zip(pb, pi):
        assert np.array_equal(a, b)


def test_bfs_order_planted_mistakes_fail_the_queue_check():
    """Plausible mistakes in the breadth-first key (the latest lower neighbour instead of the
    earliest; ties by descending index) give another order on a permuted grid."""
    A = mi.diffusion7_lognormal(6)
    lev, root, nl = oracle.levels(A)
    want = _queue_bfs_order(A, lev)
    S = sp.csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(A.n, A.n))
    S = (S + S.T).tocsr()
    perm0, _, lp = oracle.level_perm(lev, nl)
    for variant in ("latest", "desc"):
        pos = np.empty(A.n, np.int64)
        out = []
        for l in range(nl):
            rows = perm0[lp[l]:lp[l + 1]]
            keys = []
            for r in rows:
                ks = [pos[j] for j in S.indices[S.indptr[r]:S.indptr[r + 1]] if lev[j] == l - 1]
                k = -1 if not ks else (max(ks) if variant == "latest" else min(ks))
                keys.append((k, -r if variant == "desc" else r))
            for q, (_, r) in enumerate(sorted(zip(keys, rows))):
                pos[r] = lp[l] + q
                out.append(r)
        assert not np.array_equal(np.array(out), want), variant
