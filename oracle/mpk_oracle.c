/*
 * CPU oracle for the level-blocked matrix power kernel path.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct C in FP64 (values are doubles,
 * indices 32-bit as in the paper's Sec. 2.2).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library; the GPU library never links it, and this
 * file includes nothing from the GPU side.
 *
 * Built with -ffp-contract=off so that "acc += v * x" rounds the product and the sum
 * separately on every host (x86 and Arm alike).
 *
 * Contents (each function cites the passage it follows):
 *   oracle_mpk            Alg. 1 (back-to-back SpMV) with the Alg. 2 row loop, generalised to
 *                         the three-term recurrence used for Newton (Sec. 4) and Chebyshev
 *                         bases: y_k = a_k (A y_{k-1}) + b_k y_{k-1} + c_k y_{k-2}.
 *   oracle_mpk_omp        the same arithmetic with a static OpenMP row loop (Alg. 2's
 *                         "schedule(static)"), used only to time the CPU baseline.
 *   oracle_mpk_sampled    the same recurrence evaluated only on the rows a set of sampled
 *                         outputs depends on (for full-size checks).
 *   oracle_levels         BFS levels of the graph of A (Sec. 3: RACE's level structure).
 *   oracle_level_perm     rows sorted by (level, original index), and the level pointer.
 *   oracle_level_perm_bfs rows by level, and inside a level in breadth-first order (the
 *                         earliest-placed neighbour one level down, then the index).
 *   oracle_permute_csr    B = P A P^T in the level order, columns ascending per row.
 *   oracle_level_groups   consecutive levels grouped under a cache budget (Sec. 3 / Sec. 4:
 *                         the cache size parameter C).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------------
 * MPK, Alg. 1 + Alg. 2.  Y holds p+1 vectors of length n back to back; Y[0..n) = x.
 * For k = 1: the c term multiplies y_{-1} := 0.
 * ------------------------------------------------------------------------------------- */
void oracle_mpk(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, int32_t p,
                const double *a, const double *b, const double *c, const double *x, double *Y)
{
    memcpy(Y, x, (size_t)n * sizeof(double));
    for (int32_t k = 1; k <= p; k++) {
        double *yk = Y + (size_t)k * n;
        const double *y1 = Y + (size_t)(k - 1) * n;
        const double *y2 = (k >= 2) ? Y + (size_t)(k - 2) * n : NULL;
        for (int32_t i = 0; i < n; i++) {
            double acc = 0.0;
            for (int32_t t = rp[i]; t < rp[i + 1]; t++)
                acc += val[t] * y1[ci[t]];
            double prev2 = y2 ? y2[i] : 0.0;
            yk[i] = a[k - 1] * acc + b[k - 1] * y1[i] + c[k - 1] * prev2;
        }
    }
}

/* Same arithmetic as oracle_mpk, rows split statically over OpenMP threads. */
void oracle_mpk_omp(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, int32_t p,
                    const double *a, const double *b, const double *c, const double *x, double *Y)
{
    memcpy(Y, x, (size_t)n * sizeof(double));
    for (int32_t k = 1; k <= p; k++) {
        double *yk = Y + (size_t)k * n;
        const double *y1 = Y + (size_t)(k - 1) * n;
        const double *y2 = (k >= 2) ? Y + (size_t)(k - 2) * n : NULL;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; i++) {
            double acc = 0.0;
            for (int32_t t = rp[i]; t < rp[i + 1]; t++)
                acc += val[t] * y1[ci[t]];
            double prev2 = y2 ? y2[i] : 0.0;
            yk[i] = a[k - 1] * acc + b[k - 1] * y1[i] + c[k - 1] * prev2;
        }
    }
}

int32_t oracle_omp_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------
 * The recurrence of oracle_mpk evaluated only where sampled outputs need it.
 * need_k = rows whose y_k is required: need_p = the samples, need_{k-1} = need_k plus the
 * column indices of need_k's rows.  out[k*n_s + s] = y_k[rows[s]], k = 0..p.
 * Returns 0, or -1 when memory runs out.
 * ------------------------------------------------------------------------------------- */
int32_t oracle_mpk_sampled(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                           int32_t p, const double *a, const double *b, const double *c,
                           const double *x, int32_t n_s, const int32_t *rows, double *out)
{
    int32_t *mark = (int32_t *)malloc((size_t)n * sizeof(int32_t)); /* smallest k needing row */
    int32_t **lists = (int32_t **)calloc((size_t)p + 1, sizeof(int32_t *));
    int64_t *lens = (int64_t *)calloc((size_t)p + 1, sizeof(int64_t));
    double *Y = (double *)malloc((size_t)(p + 1) * n * sizeof(double));
    if (!mark || !lists || !lens || !Y) { free(mark); free(lists); free(lens); free(Y); return -1; }
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    /* list[k] = rows needing y_k (k = p .. 0); each list contains the next one */
    int32_t *cur = (int32_t *)malloc((size_t)(n_s > 0 ? n_s : 1) * sizeof(int32_t));
    int64_t cur_len = 0;
    for (int32_t s = 0; s < n_s; s++) {
        int32_t r = rows[s];
        if (mark[r] != p) { mark[r] = p; cur[cur_len++] = r; }
    }
    lists[p] = cur; lens[p] = cur_len;
    for (int32_t k = p; k >= 1; k--) {
        /* need_{k-1} = need_k + cols(need_k) (+ need_k for the b and c terms) */
        int64_t cap = lens[k];
        for (int64_t q = 0; q < lens[k]; q++) { int32_t r = lists[k][q]; cap += rp[r + 1] - rp[r]; }
        int32_t *nxt = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
        if (!nxt) return -1;
        int64_t m = 0;
        for (int64_t q = 0; q < lens[k]; q++) {
            int32_t r = lists[k][q];
            if (mark[r] != k - 1) { mark[r] = k - 1; nxt[m++] = r; }
            for (int32_t t = rp[r]; t < rp[r + 1]; t++) {
                int32_t j = ci[t];
                if (mark[j] != k - 1) { mark[j] = k - 1; nxt[m++] = j; }
            }
        }
        lists[k - 1] = nxt; lens[k - 1] = m;
    }
    for (int64_t q = 0; q < lens[0]; q++) { int32_t r = lists[0][q]; Y[r] = x[r]; }
    for (int32_t k = 1; k <= p; k++) {
        double *yk = Y + (size_t)k * n;
        const double *y1 = Y + (size_t)(k - 1) * n;
        const double *y2 = (k >= 2) ? Y + (size_t)(k - 2) * n : NULL;
        for (int64_t q = 0; q < lens[k]; q++) {
            int32_t i = lists[k][q];
            double acc = 0.0;
            for (int32_t t = rp[i]; t < rp[i + 1]; t++)
                acc += val[t] * y1[ci[t]];
            double prev2 = y2 ? y2[i] : 0.0;
            yk[i] = a[k - 1] * acc + b[k - 1] * y1[i] + c[k - 1] * prev2;
        }
    }
    for (int32_t k = 0; k <= p; k++)
        for (int32_t s = 0; s < n_s; s++)
            out[(size_t)k * n_s + s] = Y[(size_t)k * n + rows[s]];
    for (int32_t k = 0; k <= p; k++) free(lists[k]);
    free(lists); free(lens); free(mark); free(Y);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Levels (Sec. 3).  level(i) = BFS distance from the root in the undirected graph with an
 * edge {i, j} for every stored entry (i, j) or (j, i), i != j.
 *
 * Root (the paper defers the choice to RACE; the reading used here):
 *   root_rule 0 - George-Liu pseudo-peripheral search: r = row 0; BFS(r); then up to n_sweeps
 *                 times: c = the row of minimum degree in r's last level (ties: smallest
 *                 index), BFS(c); if ecc(c) > ecc(r) then r = c, else stop.
 *                 degree(i) = (entries in row i) + (entries in column i).
 *   root_rule 1 - r = row 0.
 * Rows not reached from r: when the queue empties, the BFS restarts at the lowest-index
 * unvisited row, one level above the last level used.
 * Returns the number of levels; *root_out = r.  -1 on allocation failure.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int64_t *ptr;   /* n+1 */
    int32_t *adj;   /* neighbours: row entries followed by column entries */
} sym_graph;

static int build_sym(int32_t n, const int32_t *rp, const int32_t *ci, sym_graph *g)
{
    int64_t nnz = rp[n];
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc((size_t)(2 * nnz > 0 ? 2 * nnz : 1) * sizeof(int32_t));
    if (!cnt || !g->ptr || !g->adj) { free(cnt); return -1; }
    for (int32_t i = 0; i < n; i++) {
        cnt[i] += rp[i + 1] - rp[i];
        for (int32_t t = rp[i]; t < rp[i + 1]; t++) cnt[ci[t]] += 1;
    }
    g->ptr[0] = 0;
    for (int32_t i = 0; i < n; i++) g->ptr[i + 1] = g->ptr[i] + cnt[i];
    int64_t *fill = cnt;
    for (int32_t i = 0; i < n; i++) fill[i] = g->ptr[i];
    for (int32_t i = 0; i < n; i++)
        for (int32_t t = rp[i]; t < rp[i + 1]; t++) g->adj[fill[i]++] = ci[t];
    for (int32_t i = 0; i < n; i++)
        for (int32_t t = rp[i]; t < rp[i + 1]; t++) g->adj[fill[ci[t]]++] = i;
    free(cnt);
    return 0;
}

/* BFS from r over unvisited rows (level[] == -1 marks unvisited), assigning base + distance.
   Returns the highest level assigned; the rows of that level are left in queue[*last_lo ..
   *last_hi). */
static int32_t bfs_from(const sym_graph *g, int32_t r, int32_t base, int32_t *level,
                        int32_t *queue, int64_t *last_lo, int64_t *last_hi, int64_t *visited)
{
    int64_t head = 0, tail = 0;
    level[r] = base;
    queue[tail++] = r;
    int64_t lev_lo = 0, lev_hi = 1;
    int32_t cur = base;
    while (head < tail) {
        int32_t i = queue[head++];
        for (int64_t t = g->ptr[i]; t < g->ptr[i + 1]; t++) {
            int32_t j = g->adj[t];
            if (level[j] == -1) { level[j] = level[i] + 1; queue[tail++] = j; }
        }
        if (head == lev_hi && tail > lev_hi) { lev_lo = lev_hi; lev_hi = tail; cur++; }
    }
    *last_lo = lev_lo; *last_hi = lev_hi;
    *visited += tail;
    return cur;
}

int32_t oracle_levels(int32_t n, const int32_t *rp, const int32_t *ci, int32_t root_rule,
                      int32_t n_sweeps, int32_t *level, int32_t *root_out)
{
    if (n == 0) { *root_out = -1; return 0; }
    sym_graph g;
    if (build_sym(n, rp, ci, &g)) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    int64_t lo, hi, vis = 0;
    for (int32_t i = 0; i < n; i++) level[i] = -1;
    int32_t r = 0;
    int32_t ecc = bfs_from(&g, r, 0, level, queue, &lo, &hi, &vis);
    if (root_rule == 0) {
        for (int32_t sw = 0; sw < n_sweeps; sw++) {
            int32_t best = -1;
            int64_t best_deg = 0;
            for (int64_t q = lo; q < hi; q++) {
                int32_t v = queue[q];
                int64_t d = g.ptr[v + 1] - g.ptr[v];
                if (best < 0 || d < best_deg || (d == best_deg && v < best)) { best = v; best_deg = d; }
            }
            /* BFS from the candidate restricted to the same component */
            int32_t *lev2 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
            int32_t *q2 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
            for (int32_t i = 0; i < n; i++) lev2[i] = -1;
            int64_t lo2, hi2, vis2 = 0;
            int32_t ecc2 = bfs_from(&g, best, 0, lev2, q2, &lo2, &hi2, &vis2);
            if (ecc2 > ecc) {
                memcpy(level, lev2, (size_t)n * sizeof(int32_t));
                memcpy(queue, q2, (size_t)n * sizeof(int32_t));
                r = best; ecc = ecc2; lo = lo2; hi = hi2; vis = vis2;
                free(lev2); free(q2);
            } else {
                free(lev2); free(q2);
                break;
            }
        }
    }
    *root_out = r;
    int32_t top = ecc;
    /* remaining components: lowest-index unvisited row, one level above the last */
    int32_t scan = 0;
    while (vis < n) {
        while (level[scan] != -1) scan++;
        top = bfs_from(&g, scan, top + 1, level, queue, &lo, &hi, &vis);
    }
    free(queue); free(g.ptr); free(g.adj);
    return top + 1;
}

/* Rows sorted by (level, original index): perm[r] = original row at position r,
   iperm[perm[r]] = r, level_ptr[l] = first position of level l (n_levels+1 entries). */
void oracle_level_perm(int32_t n, const int32_t *level, int32_t n_levels, int32_t *perm,
                       int32_t *iperm, int32_t *level_ptr)
{
    for (int32_t l = 0; l <= n_levels; l++) level_ptr[l] = 0;
    for (int32_t i = 0; i < n; i++) level_ptr[level[i] + 1]++;
    for (int32_t l = 0; l < n_levels; l++) level_ptr[l + 1] += level_ptr[l];
    int32_t *pos = (int32_t *)malloc((size_t)(n_levels > 0 ? n_levels : 1) * sizeof(int32_t));
    if (n_levels > 0) memcpy(pos, level_ptr, (size_t)n_levels * sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) perm[pos[level[i]]++] = i;
    for (int32_t r = 0; r < n; r++) iperm[perm[r]] = r;
    free(pos);
}

/* Breadth-first order inside levels (the plan's level_order = 1).  The paper fixes the levels
   but not the order of the rows inside one; this reading places level l's rows, levels in
   ascending order, by the key (position of the row's earliest-placed neighbour in level l - 1,
   row index), the neighbours taken in G(A + A^T).  A row with no neighbour in level l - 1 (a
   component's root, alone in its level) takes key -1.  The result is the queue order of a
   breadth-first search from each root in which every row, taken from the queue in order,
   appends its not yet placed neighbours of the next level in ascending index: Cuthill-McKee
   without its degree sort.  perm, iperm, level_ptr as in oracle_level_perm.  Returns 0, or -1
   on allocation failure. */
typedef struct { int32_t key, row; } key_row;

static int cmp_key_row(const void *a, const void *b)
{
    const key_row *x = (const key_row *)a, *y = (const key_row *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->row > y->row) - (x->row < y->row);
}

int32_t oracle_level_perm_bfs(int32_t n, const int32_t *rp, const int32_t *ci, const int32_t *level,
                              int32_t n_levels, int32_t *perm, int32_t *iperm, int32_t *level_ptr)
{
    /* rows grouped by level, ascending index inside a level (the index order) */
    oracle_level_perm(n, level, n_levels, perm, iperm, level_ptr);
    if (n == 0) return 0;
    sym_graph g;
    if (build_sym(n, rp, ci, &g)) return -1;
    key_row *buf = (key_row *)malloc((size_t)n * sizeof(key_row));
    if (!buf) { free(g.ptr); free(g.adj); return -1; }
    for (int32_t l = 0; l < n_levels; l++) {
        int32_t lo = level_ptr[l], hi = level_ptr[l + 1];
        for (int32_t q = lo; q < hi; q++) {
            int32_t i = perm[q], key = -1;
            for (int64_t t = g.ptr[i]; t < g.ptr[i + 1]; t++) {
                int32_t j = g.adj[t];
                /* level l - 1 is already in its final order: iperm[j] is j's new position */
                if (level[j] == l - 1 && (key < 0 || iperm[j] < key)) key = iperm[j];
            }
            buf[q - lo].key = key;
            buf[q - lo].row = i;
        }
        qsort(buf, (size_t)(hi - lo), sizeof(key_row), cmp_key_row);
        for (int32_t q = lo; q < hi; q++) {
            perm[q] = buf[q - lo].row;
            iperm[perm[q]] = q;
        }
    }
    free(buf); free(g.ptr); free(g.adj);
    return 0;
}

/* B = P A P^T: row r of B is row perm[r] of A with each column j replaced by iperm[j];
   entries are then ordered by new column, equal columns keeping their stored order.
   Values are moved as raw bytes of width val_bytes, so FP32 and FP64 inputs come out
   bit-identical.  rp_out has n+1 entries. */
void oracle_permute_csr(int32_t n, const int32_t *rp, const int32_t *ci, const void *val,
                        int32_t val_bytes, const int32_t *perm, const int32_t *iperm,
                        int32_t *rp_out, int32_t *ci_out, void *val_out)
{
    const unsigned char *vin = (const unsigned char *)val;
    unsigned char *vout = (unsigned char *)val_out;
    rp_out[0] = 0;
    for (int32_t r = 0; r < n; r++) {
        int32_t o = perm[r];
        rp_out[r + 1] = rp_out[r] + (rp[o + 1] - rp[o]);
    }
    for (int32_t r = 0; r < n; r++) {
        int32_t o = perm[r];
        int32_t base = rp_out[r];
        int32_t len = rp[o + 1] - rp[o];
        /* insertion sort by new column; strict comparison keeps equal columns in order */
        for (int32_t q = 0; q < len; q++) {
            int32_t t = rp[o] + q;
            int32_t cnew = iperm[ci[t]];
            int32_t pos = q;
            while (pos > 0 && ci_out[base + pos - 1] > cnew) {
                ci_out[base + pos] = ci_out[base + pos - 1];
                memcpy(vout + (size_t)(base + pos) * val_bytes,
                       vout + (size_t)(base + pos - 1) * val_bytes, (size_t)val_bytes);
                pos--;
            }
            ci_out[base + pos] = cnew;
            memcpy(vout + (size_t)(base + pos) * val_bytes, vin + (size_t)t * val_bytes,
                   (size_t)val_bytes);
        }
    }
}

/* Level groups.  Walk the levels in order; a level joins the current group while
     p * (4*rows + (4 + val_bytes)*nnz) + (p + 1) * val_bytes * rows  <=  budget
   holds for the group with the level added; otherwise the group is closed and the level
   starts the next one (a level over budget on its own is a group by itself).
   level_ptr indexes rows of the level-ordered matrix whose row pointer is rp_perm.
   group_ptr[g] = first level of group g (n_groups+1 entries).  Returns n_groups. */
int32_t oracle_level_groups(int32_t n_levels, const int32_t *level_ptr, const int32_t *rp_perm,
                            int32_t val_bytes, int32_t p, int64_t budget, int32_t *group_ptr)
{
    int32_t ng = 0;
    int64_t rows = 0, nnz = 0;
    int32_t open = 0;
    for (int32_t l = 0; l < n_levels; l++) {
        int64_t r = (int64_t)level_ptr[l + 1] - level_ptr[l];
        int64_t z = (int64_t)rp_perm[level_ptr[l + 1]] - rp_perm[level_ptr[l]];
        if (open) {
            int64_t R = rows + r, Z = nnz + z;
            int64_t cost = (int64_t)p * (4 * R + (4 + (int64_t)val_bytes) * Z)
                         + (int64_t)(p + 1) * val_bytes * R;
            if (cost <= budget) { rows = R; nnz = Z; continue; }
        }
        group_ptr[ng++] = l;
        rows = r; nnz = z; open = 1;
    }
    group_ptr[ng] = n_levels;
    return ng;
}
