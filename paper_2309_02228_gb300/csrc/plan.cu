// Plan construction: the paper's pre-processing (Sec. 3) done on the GPU.
//
//   BFS levels of the graph of A + A^T (Sec. 3: RACE analyses the matrix graph by a BFS),
//   George-Liu root search, rows sorted by (level, index), B = P A P^T, level groups under a
//   byte budget (the cache-size parameter C of Sec. 4), SELL-32 slices inside each group,
//   blocked tasks (chunks of slices) with their dependency ranges.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <numeric>

#include "mpk_internal.cuh"

// The library's memory pool of each device (stream-ordered allocations), created once; freed
// blocks stay in the pool for reuse instead of going back to the driver at every sync.
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static mpk_status mpk_pool(cudaMemPool_t *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MPK_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return MPK_OK;
    }
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return MPK_ERR_CUDA;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    *out = pool;
    return MPK_OK;
}

mpk_status DevBuf::alloc_on(size_t b, cudaStream_t s) {
    release();
    if (b == 0) b = 16;
    cudaMemPool_t pool;
    MPK_TRY(mpk_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(&p, b, pool, s);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA;
    }
    bytes = b;
    stream = s;
    ordered = true;
    return MPK_OK;
}

void mpk_log_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    fprintf(stderr, "[mpk] CUDA error %s (%d) in %s at %s:%d\n", cudaGetErrorString(e), (int)e,
            what, file, line);
}

// ============================================================================================
// Exclusive scan (int32 or int64 output, 64-bit accumulation), three phases.
// ============================================================================================
static constexpr int SCAN_BLOCK = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <typename TI>
__global__ void scan_partials_kernel(const TI *in, int64_t n, long long *part) {
    __shared__ long long sh[SCAN_BLOCK];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_BLOCK + threadIdx.x;
        if (idx < n) s += (long long)in[idx];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = SCAN_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// single block: exclusive scan of part[0..m) in place, total into part[m]
__global__ void scan_top_kernel(long long *part, int64_t m) {
    __shared__ long long sh[SCAN_BLOCK];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += SCAN_BLOCK) {
        int64_t idx = base + threadIdx.x;
        long long v = idx < m ? part[idx] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
            long long t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (idx < m) part[idx] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += sh[SCAN_BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[m] = carry;
}

template <typename TI, typename TO>
__global__ void scan_final_kernel(const TI *in, TO *out, int64_t n, const long long *part) {
    __shared__ long long sh[SCAN_TILE];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // load tile (coalesced), then each thread scans SCAN_ITEMS consecutive entries
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_BLOCK + threadIdx.x;
        sh[i * SCAN_BLOCK + threadIdx.x] = idx < n ? (long long)in[idx] : 0;
    }
    __syncthreads();
    long long loc[SCAN_ITEMS];
    long long s = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        loc[i] = s;
        s += sh[threadIdx.x * SCAN_ITEMS + i];
    }
    __shared__ long long tsum[SCAN_BLOCK];
    tsum[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        long long t = threadIdx.x >= off ? tsum[threadIdx.x - off] : 0;
        __syncthreads();
        tsum[threadIdx.x] += t;
        __syncthreads();
    }
    long long excl = tsum[threadIdx.x] - s + part[blockIdx.x];
    __syncthreads();
    for (int i = 0; i < SCAN_ITEMS; i++) sh[threadIdx.x * SCAN_ITEMS + i] = excl + loc[i];
    __syncthreads();
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * SCAN_BLOCK + threadIdx.x;
        if (idx < n) out[idx] = (TO)sh[i * SCAN_BLOCK + threadIdx.x];
    }
}

template <typename TO> __global__ void scan_total_kernel(TO *out, int64_t n, const long long *part, int64_t m) {
    out[n] = (TO)part[m];
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)(ceil_div(n, SCAN_TILE) + 2) * sizeof(long long); }

template <typename TI, typename TO>
static mpk_status exclusive_scan(const TI *in, TO *out, int64_t n, void *tmp, cudaStream_t s) {
    int64_t m = ceil_div(n, SCAN_TILE);
    long long *part = (long long *)tmp;
    if (m > 0) scan_partials_kernel<TI><<<(unsigned)m, SCAN_BLOCK, 0, s>>>(in, n, part);
    scan_top_kernel<<<1, SCAN_BLOCK, 0, s>>>(part, m);
    if (m > 0) scan_final_kernel<TI, TO><<<(unsigned)m, SCAN_BLOCK, 0, s>>>(in, out, n, part);
    scan_total_kernel<TO><<<1, 1, 0, s>>>(out, n, part, m);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

mpk_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, void *tmp,
                              cudaStream_t s) {
    return exclusive_scan<int32_t, int32_t>(in, out, n, tmp, s);
}

// ============================================================================================
// Small element-wise kernels
// ============================================================================================
__global__ void fill_i32_kernel(int32_t *p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void iota_kernel(int32_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
static unsigned grid_for(int64_t n, int block = 256) {
    int64_t g = ceil_div(n, block);
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)std::max<int64_t>(g, 1);
}

// CSR validation: row_ptr monotone, row_ptr[0] = 0, row_ptr[n] = nnz, cols in range.
__global__ void validate_kernel(const int32_t *rp, const int32_t *ci, int64_t n, int64_t nnz,
                                unsigned *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rp[i], b = rp[i + 1];
        if (a > b || a < 0 || (int64_t)b > nnz) { atomicOr(bad, 1u); continue; }
        for (int32_t t = a; t < b; t++) {
            int32_t c = ci[t];
            if (c < 0 || (int64_t)c >= n) { atomicOr(bad, 2u); break; }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0 || (int64_t)rp[n] != nnz) atomicOr(bad, 4u);
    }
}

// ============================================================================================
// Transpose pattern (for the BFS on A + A^T when the pattern may be unsymmetric)
// ============================================================================================
__global__ void col_count_kernel(const int32_t *ci, int64_t nnz, int32_t *cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[t]], 1);
}
__global__ void transpose_fill_kernel(const int32_t *rp, const int32_t *ci, int64_t n,
                                      int32_t *cursor, int32_t *ciT) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int32_t t = rp[i]; t < rp[i + 1]; t++) {
            int32_t pos = atomicAdd(&cursor[ci[t]], 1);
            ciT[pos] = (int32_t)i;
        }
}

// ============================================================================================
// BFS: one cooperative persistent kernel per component, level-synchronous, warp per frontier
// vertex, with a bounded grid barrier (the wait gives up after timeout_ns and raises error).
// ============================================================================================
struct BfsCtl {
    int32_t qsize[2];
    uint32_t bar_count;
    uint32_t bar_gen;
    uint32_t error;
    int32_t top;             // highest level assigned
    long long visited;       // rows labelled by this BFS
    unsigned long long argmin;   // (degree << 32) | row, minimum over the last level
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// returns false (on every thread of the block) if the barrier timed out
__device__ bool grid_barrier_bounded(BfsCtl *ctl, unsigned nblocks, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        uint32_t gen = ld_acquire_u32(&ctl->bar_gen);
        __threadfence();
        uint32_t arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == nblocks - 1) {
            ctl->bar_count = 0;
            __threadfence();
            st_release_u32(&ctl->bar_gen, gen + 1);
        } else {
            uint64_t t0 = globaltimer_ns();
            unsigned backoff = 32;
            while (ld_acquire_u32(&ctl->bar_gen) == gen) {
                if (ld_acquire_u32(&ctl->error)) { ok = 0; break; }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicOr(&ctl->error, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(backoff);
                if (backoff < 1024) backoff <<= 1;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct BfsArgs {
    int64_t n;
    const int32_t *rp, *ci;      // A
    const int32_t *rpT, *ciT;    // A^T (nullable: symmetric pattern)
    int32_t *level;
    int32_t *q0, *q1;
    BfsCtl *ctl;
    int32_t base;                // level of the root
    uint64_t timeout_ns;
};

__device__ __forceinline__ long long degree_of(const BfsArgs &a, int32_t v) {
    long long d = a.rp[v + 1] - a.rp[v];
    if (a.rpT) d += a.rpT[v + 1] - a.rpT[v];
    else d *= 2;   // symmetric pattern: column count equals row count
    return d;
}

__device__ __forceinline__ void expand_list(const BfsArgs &a, const int32_t *adj, int32_t beg,
                                            int32_t end, int32_t next_level, int32_t *out,
                                            int32_t *out_size, int lane) {
    for (int32_t t0 = beg; t0 < end; t0 += 32) {
        int32_t t = t0 + lane;
        bool push = false;
        int32_t j = 0;
        if (t < end) {
            j = adj[t];
            if (a.level[j] == -1) push = (atomicCAS(&a.level[j], -1, next_level) == -1);
        }
        unsigned m = __ballot_sync(0xffffffffu, push);
        if (m) {
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(out_size, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (push) out[base + __popc(m & ((1u << lane) - 1))] = j;
        }
    }
}

__global__ void bfs_kernel(BfsArgs a) {
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int cur = 0;
    int32_t L = a.base;
    int32_t last_f = 0;
    int last_buf = 0;
    long long visited = 0;
    while (true) {
        int32_t f = *(volatile int32_t *)&a.ctl->qsize[cur];
        if (f == 0) break;
        visited += f;
        last_f = f;
        last_buf = cur;
        const int32_t *in = cur ? a.q1 : a.q0;
        int32_t *out = cur ? a.q0 : a.q1;
        int32_t *osz = &a.ctl->qsize[cur ^ 1];
        for (int64_t i = gwarp; i < f; i += nwarps) {
            int32_t v = in[i];
            expand_list(a, a.ci, a.rp[v], a.rp[v + 1], L + 1, out, osz, lane);
            if (a.rpT) expand_list(a, a.ciT, a.rpT[v], a.rpT[v + 1], L + 1, out, osz, lane);
        }
        if (!grid_barrier_bounded(a.ctl, nblocks, a.timeout_ns)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->qsize[cur] = 0;
        // the reset must be visible before the next level's pushes into this buffer's counter
        if (!grid_barrier_bounded(a.ctl, nblocks, a.timeout_ns)) return;
        cur ^= 1;
        L++;
    }
    // L is one past the last level; the last frontier sits in buffer last_buf
    const int32_t *lastq = last_buf ? a.q1 : a.q0;
    int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = gtid; i < last_f; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = lastq[i];
        unsigned long long key = ((unsigned long long)degree_of(a, v) << 32) | (uint32_t)v;
        atomicMin(&a.ctl->argmin, key);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->top = L - 1;
        a.ctl->visited = visited;
    }
}

__global__ void bfs_init_kernel(BfsCtl *ctl, int32_t *level, int32_t *q0, int32_t root,
                                int32_t base) {
    ctl->qsize[0] = 1;
    ctl->qsize[1] = 0;
    ctl->bar_count = 0;
    ctl->bar_gen = 0;
    ctl->error = 0;
    ctl->top = base;
    ctl->visited = 0;
    ctl->argmin = ~0ull;
    level[root] = base;
    q0[0] = root;
}

// first index >= from with level == -1 inside [from, to); result via atomicMin
__global__ void first_unvisited_kernel(const int32_t *level, int64_t from, int64_t to,
                                       unsigned long long *res) {
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to;
         i += (int64_t)gridDim.x * blockDim.x)
        if (level[i] == -1) { atomicMin(res, (unsigned long long)i); return; }
}

struct BfsResult {
    int32_t top;
    long long visited;
    int32_t argmin_row;
};

struct BfsRunner {
    BfsArgs args{};
    DevBuf ctl_buf;
    int grid = 0, block = 256;
    mpk_status run(int32_t root, int32_t base, int32_t *level, cudaStream_t s, BfsResult *res) {
        BfsCtl *ctl = ctl_buf.as<BfsCtl>();
        bfs_init_kernel<<<1, 1, 0, s>>>(ctl, level, args.q0, root, base);
        MPK_CUDA(cudaGetLastError());
        BfsArgs a = args;
        a.level = level;
        a.ctl = ctl;
        a.base = base;
        void *kargs[] = {&a};
        MPK_CUDA(cudaLaunchCooperativeKernel((void *)bfs_kernel, dim3(grid), dim3(block), kargs,
                                             0, s));
        BfsCtl h;
        MPK_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        if (h.error) return MPK_ERR_TIMEOUT;
        res->top = h.top;
        res->visited = h.visited;
        res->argmin_row = (int32_t)(h.argmin & 0xffffffffull);
        return MPK_OK;
    }
};

// ============================================================================================
// Stable LSD radix sort of (key = level, value = row) by 8-bit digits.
// ============================================================================================
static constexpr int RS_BLOCK = 256;
static constexpr int RS_ITEMS = 8;
static constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;

__global__ void rs_hist_kernel(const int32_t *keys, int64_t n, int shift, int32_t *hist,
                               int64_t n_tiles) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = base + (int64_t)i * RS_BLOCK + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// order inside a tile: round r handles items base + r*256 + tid, so the tile is visited in
// index order; ranks among equal digits come from warp match masks and per-warp counts.
__global__ void rs_scatter_kernel(const int32_t *keys, const int32_t *vals, int64_t n, int shift,
                                  const int32_t *offs, int64_t n_tiles, int32_t *keys_out,
                                  int32_t *vals_out) {
    __shared__ int32_t wcnt[RS_BLOCK / 32][256];
    __shared__ int32_t run[256];
    __shared__ int32_t tot[256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = offs[(int64_t)tid * n_tiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; r++) {
        for (int q = 0; q < RS_BLOCK / 32; q++) wcnt[q][tid] = 0;
        __syncthreads();
        int64_t idx = base + (int64_t)r * RS_BLOCK + tid;
        bool valid = idx < n;
        int32_t key = valid ? keys[idx] : 0;
        int32_t val = valid ? vals[idx] : 0;
        unsigned d = valid ? (unsigned)((key >> shift) & 255) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1));
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {   // exclusive prefix over warps for digit tid
            int32_t acc = 0;
            for (int q = 0; q < RS_BLOCK / 32; q++) {
                int32_t t = wcnt[q][tid];
                wcnt[q][tid] = acc;
                acc += t;
            }
            tot[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int32_t pos = run[d] + wcnt[w][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        run[tid] += tot[tid];
        __syncthreads();
    }
}

// ============================================================================================
// Permutation, level pointer, permuted CSR
// ============================================================================================
__global__ void iperm_kernel(const int32_t *perm, int64_t n, int32_t *iperm) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        iperm[perm[r]] = (int32_t)r;
}

// ============================================================================================
// Breadth-first order inside levels (opts.level_order = 1).  Level l's rows are ordered by the
// key (position of the row's earliest-placed neighbour in level l - 1, row index), neighbours
// taken in G(A + A^T); a row without a neighbour one level down (a component's root) takes the
// smallest key.  Levels are placed in ascending order, each after the one below it is final.
// The rows of a level enter in ascending index (the stable sort by level), so a stable sort by
// the neighbour position alone gives the (position, index) order.
// ============================================================================================
// key of the level's rows: 0 for no neighbour one level down, else 1 + that neighbour's
// position relative to the start of level l - 1
__global__ void bfs_order_key_kernel(const int32_t *rp, const int32_t *ci, const int32_t *rpT,
                                     const int32_t *ciT, const int32_t *level, const int32_t *perm,
                                     const int32_t *iperm, int32_t lo, int32_t m, int32_t l,
                                     int32_t prev_lo, int32_t *keys, int32_t *rows) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int32_t i = perm[lo + t];
        int32_t key = 0x7fffffff;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            const int32_t j = ci[e];
            if (level[j] == l - 1) key = min(key, iperm[j]);
        }
        if (rpT)
            for (int32_t e = rpT[i]; e < rpT[i + 1]; e++) {
                const int32_t j = ciT[e];
                if (level[j] == l - 1) key = min(key, iperm[j]);
            }
        keys[t] = key == 0x7fffffff ? 0 : key - prev_lo + 1;
        rows[t] = i;
    }
}

static constexpr int BOS_MAX = 4096;   // rows a level may hold for the one-block sort

// One block: sort (key, row) of m <= BOS_MAX rows (bitonic network on the packed 64-bit
// pairs in shared memory) and place them at positions lo .. lo + m - 1.
__global__ void __launch_bounds__(512) bfs_order_small_kernel(const int32_t *keys, const int32_t *rows, int32_t m,
                                                              int32_t lo, int32_t *perm, int32_t *iperm) {
    __shared__ unsigned long long v[BOS_MAX];
    int32_t np = 1;
    while (np < m) np <<= 1;
    for (int32_t t = threadIdx.x; t < np; t += blockDim.x)
        v[t] = t < m ? (((unsigned long long)(uint32_t)keys[t] << 32) | (uint32_t)rows[t]) : ~0ull;
    __syncthreads();
    for (int32_t k = 2; k <= np; k <<= 1) {
        for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (int32_t t = threadIdx.x; t < np; t += blockDim.x) {
                const int32_t u = t ^ jj;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    const unsigned long long a = v[t], b = v[u];
                    if ((a > b) == up) {
                        v[t] = b;
                        v[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int32_t t = threadIdx.x; t < m; t += blockDim.x) {
        const int32_t r = (int32_t)(v[t] & 0xffffffffull);
        perm[lo + t] = r;
        iperm[r] = lo + t;
    }
}

__global__ void bfs_order_place_kernel(const int32_t *rows, int32_t m, int32_t lo, int32_t *perm, int32_t *iperm) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int32_t r = rows[t];
        perm[lo + t] = r;
        iperm[r] = lo + t;
    }
}
__global__ void level_hist_kernel(const int32_t *level, int64_t n, int32_t *cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[level[i]], 1);
}
__global__ void perm_rowlen_kernel(const int32_t *rp, const int32_t *perm, int64_t n, int32_t *len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = perm[r];
        len[r] = rp[o + 1] - rp[o];
    }
}

// warp per row of length <= 32: bitonic sort of (new column, stored position) keys
template <typename TV>
__global__ void permute_rows_warp_kernel(const int32_t *rp, const int32_t *ci, const TV *val,
                                         const int32_t *perm, const int32_t *iperm,
                                         const int32_t *rp_new, int64_t n, int32_t *ci_new,
                                         double *v64, float *v32, int32_t *entry_map,
                                         int32_t *long_rows, int32_t *n_long) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t o = perm[r];
        int32_t beg = rp[o], len = rp[o + 1] - beg;
        if (len > 32) {
            if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int32_t)r;
            continue;
        }
        unsigned long long key = ~0ull;
        if (lane < len) key = ((unsigned long long)(uint32_t)iperm[ci[beg + lane]] << 32) | (uint32_t)lane;
        // bitonic sort ascending across the warp
        for (int k = 2; k <= 32; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                unsigned long long other = __shfl_xor_sync(0xffffffffu, key, j);
                bool up = ((lane & k) == 0);
                bool lower = ((lane & j) == 0);
                unsigned long long mn = key < other ? key : other;
                unsigned long long mx = key < other ? other : key;
                key = (lower == up) ? mn : mx;
            }
        }
        if (lane < len) {
            int32_t src = beg + (int32_t)(key & 0xffffffffull);
            int32_t dst = rp_new[r] + lane;
            ci_new[dst] = (int32_t)(key >> 32);
            TV v = val[src];
            if (v64) v64[dst] = (double)v;
            if (v32) v32[dst] = (float)v;
            entry_map[src] = dst;
        }
    }
}

// block per long row: rank of each entry among (new column, stored position) by counting
template <typename TV>
__global__ void permute_rows_long_kernel(const int32_t *rp, const int32_t *ci, const TV *val,
                                         const int32_t *perm, const int32_t *iperm,
                                         const int32_t *rp_new, const int32_t *long_rows,
                                         int32_t *ci_new, double *v64, float *v32,
                                         int32_t *entry_map) {
    int32_t r = long_rows[blockIdx.x];
    int32_t o = perm[r];
    int32_t beg = rp[o], len = rp[o + 1] - beg;
    for (int32_t t = threadIdx.x; t < len; t += blockDim.x) {
        int32_t ct = iperm[ci[beg + t]];
        int32_t rank = 0;
        for (int32_t u = 0; u < len; u++) {
            int32_t cu = iperm[ci[beg + u]];
            rank += (cu < ct) || (cu == ct && u < t);
        }
        int32_t dst = rp_new[r] + rank;
        ci_new[dst] = ct;
        TV v = val[beg + t];
        if (v64) v64[dst] = (double)v;
        if (v32) v32[dst] = (float)v;
        entry_map[beg + t] = dst;
    }
}

template <typename TV>
__global__ void update_values_kernel(const TV *val, const int32_t *entry_map, int64_t nnz,
                                     double *v64, float *v32) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = entry_map[t];
        TV v = val[t];
        if (v64) v64[d] = (double)v;
        if (v32) v32[d] = (float)v;
    }
}

__global__ void gather_rp_kernel(const int32_t *rp, const int32_t *idx, int64_t m, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = rp[idx[i]];
}

// ============================================================================================
// SELL-32 slices, chunks, dependency ranges
// ============================================================================================
__global__ void slice_len_kernel(const int32_t *rp, const int32_t *slice_row, int64_t n_slices,
                                 int32_t *slice_len) {
    const int lane = threadIdx.x & 31;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_slices;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t r0 = slice_row[s], r1 = slice_row[s + 1];
        int32_t r = r0 + lane;
        int32_t len = r < r1 ? rp[r + 1] - rp[r] : 0;
        for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
        if (lane == 0) slice_len[s] = len;
    }
}

__global__ void sell_fill_kernel(const int32_t *rp, const int32_t *ci, const double *v64,
                                 const float *v32, const int32_t *slice_row,
                                 const int32_t *slice_len, const long long *slice_ptr,
                                 int64_t n_slices, int32_t *s_col, double *s64, float *s32) {
    const int lane = threadIdx.x & 31;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_slices;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t r0 = slice_row[s], r1 = slice_row[s + 1];
        int32_t r = r0 + lane;
        int32_t beg = 0, len = 0;
        if (r < r1) { beg = rp[r]; len = rp[r + 1] - beg; }
        int32_t L = slice_len[s];
        long long p0 = 32ll * slice_ptr[s];
        for (int32_t j = 0; j < L; j++) {
            long long d = p0 + 32ll * j + lane;
            if (j < len) {
                s_col[d] = ci[beg + j];
                if (s64) s64[d] = v64[beg + j];
                if (s32) s32[d] = v32[beg + j];
            } else {
                s_col[d] = -1;
                if (s64) s64[d] = 0.0;
                if (s32) s32[d] = 0.0f;
            }
        }
    }
}

// Right Jacobi scaling (Sec. 5.1, Eq. (Jacobi)).  D^-1 of the level-order matrix:
// d_i = the sum of row i's entries in column i (columns ascend inside a row), dinv_i = 1 / d_i,
// or 1 where d_i is zero or the entry is missing (that column is left unscaled).
template <typename TV>
__global__ void jacobi_dinv_kernel(const int32_t *rp, const int32_t *ci, const TV *val, int64_t n,
                                   double *dinv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = rp[i], hi = rp[i + 1];
        while (lo < hi) {   // first entry with column >= i
            const int32_t mid = lo + (hi - lo) / 2;
            if (ci[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        double d = 0.0;
        for (int32_t t = lo; t < rp[i + 1] && ci[t] == i; t++) d += (double)val[t];
        dinv[i] = d != 0.0 ? 1.0 / d : 1.0;
    }
}

// SELL values of A D^-1: b_e = a_e * dinv[col(e)], formed in FP64 and rounded once to each
// kept precision; padding (col -1) stays 0
__global__ void jacobi_scale_kernel(const int32_t *s_col, const double *s64, const float *s32,
                                    int64_t ne, const double *dinv, double *j64, float *j32) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = s_col[e];
        double b = 0.0;
        if (c >= 0) b = (s64 ? s64[e] : (double)s32[e]) * dinv[c];
        if (j64) j64[e] = b;
        if (j32) j32[e] = (float)b;
    }
}

// Strictly lower entries of the caller's row order, for the two-stage Gauss-Seidel sub-powers
// (Sec. 5.1, Alg. GS2): bit `lane` of word slice_ptr[s] + j is set when lane's entry j of slice
// s is stored (column >= 0), its row is inside the slice, and the column's original index is
// below the row's (perm maps level order to the original order).  One warp per slice.
__global__ void gs2_lower_mask_kernel(const int32_t *s_col, const long long *slice_ptr,
                                      const int32_t *slice_row, const int32_t *slice_len,
                                      int64_t n_slices, const int32_t *perm, uint32_t *lmask) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = w0; sl < n_slices; sl += nw) {
        const int32_t row = slice_row[sl] + lane;
        const bool in = row < slice_row[sl + 1];
        const int32_t orow = in ? perm[row] : 0;
        const long long sp = slice_ptr[sl];
        const int32_t L = slice_len[sl];
        for (int32_t j = 0; j < L; j++) {
            const int32_t c = s_col[32 * (sp + j) + lane];
            const bool low = in && c >= 0 && perm[c] < orow;
            const uint32_t m = __ballot_sync(0xffffffffu, low);
            if (lane == 0) lmask[sp + j] = m;
        }
    }
}

// The strictly lower entries of every row, packed in their stored order into slices of their
// own (the GS2 inner stages read only them, Sec. 5.1): slice s keeps the rows of the full
// slice; its length is the largest lower count among those rows.  One warp per slice.
__global__ void gs2_lower_len_kernel(const int32_t *slice_row, const int32_t *slice_len,
                                     const long long *slice_ptr, int64_t n_slices,
                                     const uint32_t *lmask, int32_t *l_len) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = w0; sl < n_slices; sl += nw) {
        const long long sp = slice_ptr[sl];
        int32_t cnt = 0;
        for (int32_t j = 0; j < slice_len[sl]; j++) cnt += (lmask[sp + j] >> lane) & 1u;
        for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
        if (lane == 0) l_len[sl] = cnt;
    }
}

// Fill the packed lower slices: lane l of slice s copies its row's lower entries (columns and
// the Jacobi-scaled values b_ij) in stored order to 32 * l_ptr[s] + 32 * j + l; the rest of the
// slice length is padding (column -1, value 0).
__global__ void gs2_lower_fill_kernel(const int32_t *slice_len, const long long *slice_ptr,
                                      const long long *l_ptr, const int32_t *l_len, int64_t n_slices,
                                      const uint32_t *lmask, const int32_t *s_col, const double *j64,
                                      const float *j32, int32_t *l_col, double *l64, float *l32) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = w0; sl < n_slices; sl += nw) {
        const long long sp = slice_ptr[sl], lp = l_ptr[sl];
        int32_t cnt = 0;
        for (int32_t j = 0; j < slice_len[sl]; j++) {
            if (!((lmask[sp + j] >> lane) & 1u)) continue;
            const long long src = 32ll * (sp + j) + lane, dst = 32ll * (lp + cnt) + lane;
            l_col[dst] = s_col[src];
            if (l64) l64[dst] = j64[src];
            if (l32) l32[dst] = j32[src];
            cnt++;
        }
        for (; cnt < l_len[sl]; cnt++) {
            const long long dst = 32ll * (lp + cnt) + lane;
            l_col[dst] = -1;
            if (l64) l64[dst] = 0.0;
            if (l32) l32[dst] = 0.0f;
        }
    }
}

static mpk_status gs2_lower_fill(mpk_plan_s *P, cudaStream_t s) {
    if (!P->l_col.p || P->n_slices == 0) return MPK_OK;
    gs2_lower_fill_kernel<<<grid_for((int64_t)P->n_slices * 32), 256, 0, s>>>(
        P->slice_len.as<int32_t>(), P->slice_ptr.as<long long>(), P->l_slice_ptr.as<long long>(),
        P->l_slice_len.as<int32_t>(), P->n_slices, P->s_lmask.as<uint32_t>(), P->s_col.as<int32_t>(),
        P->has64 ? P->s_jval64.as<double>() : nullptr, P->has32 ? P->s_jval32.as<float>() : nullptr,
        P->l_col.as<int32_t>(), P->has64 ? P->l_val64.as<double>() : nullptr,
        P->has32 ? P->l_val32.as<float>() : nullptr);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

__global__ void row_chunk_kernel(const int32_t *chunk_row, int64_t n_chunks, int32_t *row_chunk) {
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x)
        for (int32_t r = chunk_row[c] + threadIdx.x; r < chunk_row[c + 1]; r += blockDim.x)
            row_chunk[r] = (int32_t)c;
}

// dependency range of a chunk: the chunks holding any column of its rows (and itself); with
// `sym_close` also the chunks whose rows reference it (closure over A^T), which the 3-buffer
// ring of MPK_FINAL_ONLY needs for unsymmetric patterns.
__global__ void dep_kernel(const int32_t *rp, const int32_t *ci, const int32_t *row_chunk,
                           int64_t n, int sym_close, int32_t *dep_lo, int32_t *dep_hi) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = row_chunk[r];
        int32_t lo = c, hi = c;
        int32_t beg = rp[r], end = rp[r + 1];
        if (end > beg) {
            // columns are ascending inside each row
            lo = min(lo, row_chunk[ci[beg]]);
            hi = max(hi, row_chunk[ci[end - 1]]);
        }
        atomicMin(&dep_lo[c], lo);
        atomicMax(&dep_hi[c], hi);
        if (sym_close)
            for (int32_t t = beg; t < end; t++) {
                int32_t cc = row_chunk[ci[t]];
                atomicMin(&dep_lo[cc], c);
                atomicMax(&dep_hi[cc], c);
            }
    }
}

// ============================================================================================
// Host orchestration
// ============================================================================================
extern "C" mpk_status mpk_plan_opts_default(mpk_plan_opts *o) {
    if (!o) return MPK_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->l2_budget_bytes = 0;
    o->p_blk = 0;
    o->root_rule = 0;
    o->n_sweeps = 2;
    o->assume_symmetric = 0;
    o->chunk_slices = 8;
    o->keep_f32 = 0;
    o->keep_f64 = 0;
    o->ctas_per_sm = 0;
    o->wait_timeout_us = 2000000u;
    o->schedule = 1;
    o->slack_tasks = 0;
    o->block_threads = 256;
    o->stage = -1;
    o->kernel = 4;
    o->blocked = -1;
    o->jacobi = 0;
    o->owner_lag = 1;
    o->owner_prefetch = 1;
    o->level_order = 1;
    return MPK_OK;
}

template <typename T> static mpk_status upload(DevBuf &b, const std::vector<T> &h, cudaStream_t s) {
    MPK_TRY(b.alloc(std::max<size_t>(h.size(), 1) * sizeof(T)));
    if (!h.empty())
        MPK_CUDA(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return MPK_OK;
}

static mpk_status plan_create_impl(const mpk_csr *A, int32_t p_max, const mpk_plan_opts *opts,
                                   cudaStream_t s, mpk_plan_s *P) {
    auto t0 = std::chrono::steady_clock::now();
    if (opts) P->opts = *opts;
    else mpk_plan_opts_default(&P->opts);
    mpk_plan_opts &o = P->opts;
    if (o.n_sweeps < 0 || o.chunk_slices <= 0 || o.root_rule < 0 || o.root_rule > 1 ||
        o.level_order < 0 || o.level_order > 1)
        return MPK_ERR_ARG;
    const int64_t n = A->n, nnz = A->nnz;
    P->n = n;
    P->nnz = nnz;
    P->p_max = p_max;
    P->p_blk = (o.p_blk > 0 && o.p_blk < p_max) ? o.p_blk : p_max;
    if (!o.keep_f32 && !o.keep_f64) {
        if (A->dtype == MPK_F64) o.keep_f64 = 1;
        else o.keep_f32 = 1;
    }
    P->has64 = o.keep_f64 != 0;
    P->has32 = o.keep_f32 != 0;
    P->jacobi = o.jacobi != 0;
    // the groups are sized for the MPK precision: FP32 whenever an FP32 copy is kept (the
    // FP64 copy then only serves residuals), else FP64
    P->group_dtype = P->has32 ? MPK_F32 : MPK_F64;

    MPK_CUDA(cudaGetDevice(&P->device));
    MPK_CUDA(cudaDeviceGetAttribute(&P->n_sm, cudaDevAttrMultiProcessorCount, P->device));
    int l2 = 0;
    MPK_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, P->device));
    P->l2_bytes = l2;
    if (o.l2_budget_bytes <= 0) o.l2_budget_bytes = P->l2_bytes / 2;
    if (o.wait_timeout_us == 0) o.wait_timeout_us = 2000000u;

    // ---- control block and flags allocated early so an empty matrix still has them
    MPK_TRY(P->ctrl.alloc(sizeof(MpkCtrl)));
    MPK_CUDA(cudaMemsetAsync(P->ctrl.p, 0, sizeof(MpkCtrl), s));
    {
        uint32_t one = 1;   // epoch starts at 1 so that zeroed flags are below every target
        MPK_CUDA(cudaMemcpyAsync(P->ctrl.p, &one, sizeof(one), cudaMemcpyHostToDevice, s));
    }

    // ---- validation (row pointer monotone and consistent, columns in range)
    if (n > 0) {
        DevBuf bad;
        MPK_TRY(bad.alloc_on(sizeof(unsigned), s));
        MPK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
        validate_kernel<<<grid_for(n), 256, 0, s>>>(A->row_ptr, A->col, n, nnz, bad.as<unsigned>());
        MPK_CUDA(cudaGetLastError());
        unsigned hbad = 0;
        MPK_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(hbad), cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        if (hbad) return MPK_ERR_ARG;
    }

    const size_t tmp_bytes = std::max(scan_tmp_bytes(n + 1), scan_tmp_bytes(nnz + 1));
    DevBuf tmp;
    MPK_TRY(tmp.alloc_on(std::max<size_t>(tmp_bytes, 256 * 8192 * 8), s));

    // ---- transpose pattern (unless the caller states the pattern is symmetric)
    DevBuf rpT, ciT, cursor;
    const bool sym = o.assume_symmetric != 0;
    if (!sym) {
        MPK_TRY(cursor.alloc_on((n + 1) * sizeof(int32_t), s));
        MPK_TRY(rpT.alloc_on((n + 1) * sizeof(int32_t), s));
        MPK_TRY(ciT.alloc_on(std::max<int64_t>(nnz, 1) * sizeof(int32_t), s));
        MPK_CUDA(cudaMemsetAsync(cursor.p, 0, (n + 1) * sizeof(int32_t), s));
        col_count_kernel<<<grid_for(nnz), 256, 0, s>>>(A->col, nnz, cursor.as<int32_t>());
        MPK_TRY(exclusive_scan<int32_t, int32_t>(cursor.as<int32_t>(), rpT.as<int32_t>(), n, tmp.p, s));
        MPK_CUDA(cudaMemcpyAsync(cursor.p, rpT.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        transpose_fill_kernel<<<grid_for(n), 256, 0, s>>>(A->row_ptr, A->col, n, cursor.as<int32_t>(), ciT.as<int32_t>());
        MPK_CUDA(cudaGetLastError());
    }

    // ---- BFS levels + George-Liu root
    MPK_TRY(P->level.alloc(n * sizeof(int32_t)));
    DevBuf lev2, q0, q1;
    MPK_TRY(lev2.alloc_on(n * sizeof(int32_t), s));
    MPK_TRY(q0.alloc_on(n * sizeof(int32_t), s));
    MPK_TRY(q1.alloc_on(n * sizeof(int32_t), s));
    BfsRunner bfs;
    MPK_TRY(bfs.ctl_buf.alloc_on(sizeof(BfsCtl), s));
    {
        int occ = 0;
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfs_kernel, bfs.block, 0));
        // sized to the matrix: a cooperative launch holds every SM it spans until it ends, so a
        // small matrix takes a few CTAs and leaves the rest of the GPU to concurrent work
        bfs.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)P->n_sm * std::max(1, std::min(occ, 4)),
                                                               ceil_div(n, 2048)));
        bfs.args.n = n;
        bfs.args.rp = A->row_ptr;
        bfs.args.ci = A->col;
        bfs.args.rpT = sym ? nullptr : rpT.as<int32_t>();
        bfs.args.ciT = sym ? nullptr : ciT.as<int32_t>();
        bfs.args.q0 = q0.as<int32_t>();
        bfs.args.q1 = q1.as<int32_t>();
        bfs.args.timeout_ns = (uint64_t)o.wait_timeout_us * 1000ull;
    }
    int32_t n_levels = 0;
    if (n > 0) {
        int32_t *levA = P->level.as<int32_t>(), *levB = lev2.as<int32_t>();
        fill_i32_kernel<<<grid_for(n), 256, 0, s>>>(levA, n, -1);
        BfsResult cur;
        MPK_TRY(bfs.run(0, 0, levA, s, &cur));
        P->bfs_sweeps = 1;
        int32_t root = 0;
        if (o.root_rule == 0) {
            for (int sw = 0; sw < o.n_sweeps; sw++) {
                int32_t cand = cur.argmin_row;
                fill_i32_kernel<<<grid_for(n), 256, 0, s>>>(levB, n, -1);
                BfsResult nxt;
                MPK_TRY(bfs.run(cand, 0, levB, s, &nxt));
                P->bfs_sweeps++;
                if (nxt.top > cur.top) {
                    std::swap(levA, levB);
                    root = cand;
                    cur = nxt;
                } else {
                    break;
                }
            }
        }
        if (levA != P->level.as<int32_t>())
            MPK_CUDA(cudaMemcpyAsync(P->level.p, levA, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        levA = P->level.as<int32_t>();
        P->root = root;
        // remaining components: lowest-index unvisited row, one level above the last
        long long visited = cur.visited;
        int32_t top = cur.top;
        int64_t scan_pos = 0;
        const int64_t W = 1 << 20;
        DevBuf resb;
        MPK_TRY(resb.alloc_on(sizeof(unsigned long long), s));
        unsigned long long *res = resb.as<unsigned long long>();
        while (visited < n) {
            unsigned long long h = ~0ull;
            while (h == ~0ull && scan_pos < n) {
                MPK_CUDA(cudaMemsetAsync(res, 0xff, sizeof(*res), s));
                int64_t to = std::min<int64_t>(n, scan_pos + W);
                first_unvisited_kernel<<<grid_for(to - scan_pos), 256, 0, s>>>(levA, scan_pos, to, res);
                MPK_CUDA(cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
                MPK_CUDA(cudaStreamSynchronize(s));
                if (h == ~0ull) scan_pos = to;
            }
            if (h == ~0ull) return MPK_ERR_CUDA;   // visited count and labels disagree
            scan_pos = (int64_t)h;
            BfsResult cr;
            MPK_TRY(bfs.run((int32_t)h, top + 1, levA, s, &cr));
            visited += cr.visited;
            top = cr.top;
        }
        n_levels = top + 1;
    }
    P->n_levels = n_levels;
    q1.release();

    // ---- stable sort of rows by level: perm, iperm, level_ptr
    MPK_TRY(P->perm.alloc(n * sizeof(int32_t)));
    MPK_TRY(P->iperm.alloc(n * sizeof(int32_t)));
    MPK_TRY(P->level_ptr.alloc((n_levels + 1) * sizeof(int32_t)));
    if (n > 0) {
        DevBuf kA, kB, vA, vB, hist;
        MPK_TRY(kA.alloc_on(n * 4, s));
        MPK_TRY(kB.alloc_on(n * 4, s));
        MPK_TRY(vA.alloc_on(n * 4, s));
        MPK_TRY(vB.alloc_on(n * 4, s));
        int64_t n_tiles = ceil_div(n, RS_TILE);
        MPK_TRY(hist.alloc_on((256 * n_tiles + 1) * sizeof(int32_t), s));
        DevBuf offs;
        MPK_TRY(offs.alloc_on((256 * n_tiles + 1) * sizeof(int32_t), s));
        DevBuf stmp;
        MPK_TRY(stmp.alloc_on(scan_tmp_bytes(256 * n_tiles + 1), s));
        MPK_CUDA(cudaMemcpyAsync(kA.p, P->level.p, n * 4, cudaMemcpyDeviceToDevice, s));
        iota_kernel<<<grid_for(n), 256, 0, s>>>(vA.as<int32_t>(), n);
        int32_t *ki = kA.as<int32_t>(), *ko = kB.as<int32_t>();
        int32_t *vi = vA.as<int32_t>(), *vo = vB.as<int32_t>();
        for (int shift = 0; shift == 0 || (shift < 31 && ((int64_t)1 << shift) < n_levels); shift += 8) {
            rs_hist_kernel<<<(unsigned)n_tiles, RS_BLOCK, 0, s>>>(ki, n, shift, hist.as<int32_t>(), n_tiles);
            MPK_TRY(exclusive_scan<int32_t, int32_t>(hist.as<int32_t>(), offs.as<int32_t>(), 256 * n_tiles, stmp.p, s));
            rs_scatter_kernel<<<(unsigned)n_tiles, RS_BLOCK, 0, s>>>(ki, vi, n, shift, offs.as<int32_t>(), n_tiles, ko, vo);
            MPK_CUDA(cudaGetLastError());
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        MPK_CUDA(cudaMemcpyAsync(P->perm.p, vi, n * 4, cudaMemcpyDeviceToDevice, s));
        iperm_kernel<<<grid_for(n), 256, 0, s>>>(P->perm.as<int32_t>(), n, P->iperm.as<int32_t>());
        DevBuf cnt;
        MPK_TRY(cnt.alloc_on((n_levels + 1) * 4, s));
        MPK_CUDA(cudaMemsetAsync(cnt.p, 0, (n_levels + 1) * 4, s));
        level_hist_kernel<<<grid_for(n), 256, 0, s>>>(P->level.as<int32_t>(), n, cnt.as<int32_t>());
        MPK_TRY(exclusive_scan<int32_t, int32_t>(cnt.as<int32_t>(), P->level_ptr.as<int32_t>(), n_levels, tmp.p, s));
    } else {
        MPK_CUDA(cudaMemsetAsync(P->level_ptr.p, 0, 4, s));
    }
    // ---- breadth-first order inside levels (level_order = 1), one level after another
    if (o.level_order == 1 && n > 0 && n_levels > 1) {
        std::vector<int32_t> lp(n_levels + 1);
        MPK_CUDA(cudaMemcpyAsync(lp.data(), P->level_ptr.p, (n_levels + 1) * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        int32_t maxm = 0;
        for (int32_t l = 0; l < n_levels; l++) maxm = std::max(maxm, lp[l + 1] - lp[l]);
        const int64_t tiles = ceil_div(maxm, RS_TILE);
        DevBuf kA, kB, vA, vB, hist, offs, stmp;
        MPK_TRY(kA.alloc_on((size_t)maxm * 4, s));
        MPK_TRY(kB.alloc_on((size_t)maxm * 4, s));
        MPK_TRY(vA.alloc_on((size_t)maxm * 4, s));
        MPK_TRY(vB.alloc_on((size_t)maxm * 4, s));
        MPK_TRY(hist.alloc_on((256 * tiles + 1) * sizeof(int32_t), s));
        MPK_TRY(offs.alloc_on((256 * tiles + 1) * sizeof(int32_t), s));
        MPK_TRY(stmp.alloc_on(scan_tmp_bytes(256 * tiles + 1), s));
        const int32_t *rT = sym ? nullptr : rpT.as<int32_t>();
        const int32_t *cT = sym ? nullptr : ciT.as<int32_t>();
        for (int32_t l = 1; l < n_levels; l++) {
            const int32_t lo = lp[l], m = lp[l + 1] - lp[l];
            if (m <= 1) continue;
            bfs_order_key_kernel<<<grid_for(m), 256, 0, s>>>(A->row_ptr, A->col, rT, cT, P->level.as<int32_t>(),
                                                             P->perm.as<int32_t>(), P->iperm.as<int32_t>(), lo, m, l,
                                                             lp[l - 1], kA.as<int32_t>(), vA.as<int32_t>());
            if (m <= BOS_MAX) {
                bfs_order_small_kernel<<<1, 512, 0, s>>>(kA.as<int32_t>(), vA.as<int32_t>(), m, lo,
                                                         P->perm.as<int32_t>(), P->iperm.as<int32_t>());
            } else {
                // stable radix sort by key (the rows are in ascending index within the level)
                const int64_t nt = ceil_div(m, RS_TILE);
                const int32_t maxkey = lp[l] - lp[l - 1];
                int32_t *ki = kA.as<int32_t>(), *ko = kB.as<int32_t>();
                int32_t *vi = vA.as<int32_t>(), *vo = vB.as<int32_t>();
                for (int shift = 0; shift == 0 || (shift < 31 && ((int64_t)1 << shift) <= maxkey); shift += 8) {
                    rs_hist_kernel<<<(unsigned)nt, RS_BLOCK, 0, s>>>(ki, m, shift, hist.as<int32_t>(), nt);
                    MPK_TRY(exclusive_scan<int32_t, int32_t>(hist.as<int32_t>(), offs.as<int32_t>(), 256 * nt, stmp.p, s));
                    rs_scatter_kernel<<<(unsigned)nt, RS_BLOCK, 0, s>>>(ki, vi, m, shift, offs.as<int32_t>(), nt, ko, vo);
                    std::swap(ki, ko);
                    std::swap(vi, vo);
                }
                bfs_order_place_kernel<<<grid_for(m), 256, 0, s>>>(vi, m, lo, P->perm.as<int32_t>(), P->iperm.as<int32_t>());
            }
            MPK_CUDA(cudaGetLastError());
        }
    }
    rpT.release();
    ciT.release();
    cursor.release();
    lev2.release();

    // ---- permuted CSR B = P A P^T, columns ascending per row
    MPK_TRY(P->rp.alloc((n + 1) * 4));
    MPK_TRY(P->ci.alloc(std::max<int64_t>(nnz, 1) * 4));
    MPK_TRY(P->entry_map.alloc(std::max<int64_t>(nnz, 1) * 4));
    if (P->has64) MPK_TRY(P->val64.alloc(std::max<int64_t>(nnz, 1) * 8));
    if (P->has32) MPK_TRY(P->val32.alloc(std::max<int64_t>(nnz, 1) * 4));
    if (n > 0) {
        DevBuf len;
        MPK_TRY(len.alloc_on(n * 4, s));
        perm_rowlen_kernel<<<grid_for(n), 256, 0, s>>>(A->row_ptr, P->perm.as<int32_t>(), n, len.as<int32_t>());
        MPK_TRY(exclusive_scan<int32_t, int32_t>(len.as<int32_t>(), P->rp.as<int32_t>(), n, tmp.p, s));
        DevBuf longr, nlong;
        MPK_TRY(longr.alloc_on(n * 4, s));
        MPK_TRY(nlong.alloc_on(4, s));
        MPK_CUDA(cudaMemsetAsync(nlong.p, 0, 4, s));
        double *v64 = P->has64 ? P->val64.as<double>() : nullptr;
        float *v32 = P->has32 ? P->val32.as<float>() : nullptr;
        unsigned g = grid_for(n * 32);
        if (A->dtype == MPK_F64)
            permute_rows_warp_kernel<double><<<g, 256, 0, s>>>(A->row_ptr, A->col, (const double *)A->val, P->perm.as<int32_t>(), P->iperm.as<int32_t>(), P->rp.as<int32_t>(), n, P->ci.as<int32_t>(), v64, v32, P->entry_map.as<int32_t>(), longr.as<int32_t>(), nlong.as<int32_t>());
        else
            permute_rows_warp_kernel<float><<<g, 256, 0, s>>>(A->row_ptr, A->col, (const float *)A->val, P->perm.as<int32_t>(), P->iperm.as<int32_t>(), P->rp.as<int32_t>(), n, P->ci.as<int32_t>(), v64, v32, P->entry_map.as<int32_t>(), longr.as<int32_t>(), nlong.as<int32_t>());
        MPK_CUDA(cudaGetLastError());
        int32_t hlong = 0;
        MPK_CUDA(cudaMemcpyAsync(&hlong, nlong.p, 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        if (hlong > 0) {
            if (A->dtype == MPK_F64)
                permute_rows_long_kernel<double><<<hlong, 256, 0, s>>>(A->row_ptr, A->col, (const double *)A->val, P->perm.as<int32_t>(), P->iperm.as<int32_t>(), P->rp.as<int32_t>(), longr.as<int32_t>(), P->ci.as<int32_t>(), v64, v32, P->entry_map.as<int32_t>());
            else
                permute_rows_long_kernel<float><<<hlong, 256, 0, s>>>(A->row_ptr, A->col, (const float *)A->val, P->perm.as<int32_t>(), P->iperm.as<int32_t>(), P->rp.as<int32_t>(), longr.as<int32_t>(), P->ci.as<int32_t>(), v64, v32, P->entry_map.as<int32_t>());
            MPK_CUDA(cudaGetLastError());
        }
    } else {
        MPK_CUDA(cudaMemsetAsync(P->rp.p, 0, 4, s));
    }

    // ---- level groups (host, integer-exact): per-level rows and nnz from level_ptr and rp
    P->h_level_ptr.assign(n_levels + 1, 0);
    std::vector<int32_t> h_rp_at(n_levels + 1, 0);
    if (n > 0) {
        MPK_CUDA(cudaMemcpyAsync(P->h_level_ptr.data(), P->level_ptr.p, (n_levels + 1) * 4, cudaMemcpyDeviceToHost, s));
        DevBuf at;
        MPK_TRY(at.alloc_on((n_levels + 1) * 4, s));
        gather_rp_kernel<<<grid_for(n_levels + 1), 256, 0, s>>>(P->rp.as<int32_t>(), P->level_ptr.as<int32_t>(), n_levels + 1, at.as<int32_t>());
        MPK_CUDA(cudaMemcpyAsync(h_rp_at.data(), at.p, (n_levels + 1) * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
    }
    {
        const int64_t w = P->group_dtype == MPK_F64 ? 8 : 4;
        const int64_t pb = P->p_blk;
        const int64_t budget = o.l2_budget_bytes;
        std::vector<int32_t> gp;
        int64_t rows = 0, z = 0;
        bool open = false;
        for (int32_t l = 0; l < n_levels; l++) {
            int64_t r = (int64_t)P->h_level_ptr[l + 1] - P->h_level_ptr[l];
            int64_t zz = (int64_t)h_rp_at[l + 1] - h_rp_at[l];
            P->max_level_rows = std::max<int32_t>(P->max_level_rows, (int32_t)r);
            if (open) {
                int64_t R = rows + r, Z = z + zz;
                int64_t cost = pb * (4 * R + (4 + w) * Z) + (pb + 1) * w * R;
                if (cost <= budget) { rows = R; z = Z; continue; }
            }
            gp.push_back(l);
            rows = r;
            z = zz;
            open = true;
        }
        gp.push_back(n_levels);
        P->h_group_ptr = gp;
        P->n_groups = (int32_t)gp.size() - 1;
        MPK_TRY(upload(P->group_ptr, gp, s));
    }

    // ---- SELL-32 slices inside groups
    std::vector<int32_t> h_slice_row, h_slice_group;
    for (int32_t g = 0; g < P->n_groups; g++) {
        int32_t r0 = P->h_level_ptr[P->h_group_ptr[g]];
        int32_t r1 = P->h_level_ptr[P->h_group_ptr[g + 1]];
        for (int32_t r = r0; r < r1; r += 32) {
            h_slice_row.push_back(r);
            h_slice_group.push_back(g);
        }
    }
    P->n_slices = (int32_t)h_slice_row.size();
    h_slice_row.push_back((int32_t)n);
    MPK_TRY(upload(P->slice_row, h_slice_row, s));
    MPK_TRY(P->slice_len.alloc((P->n_slices + 1) * 4));
    MPK_TRY(P->slice_ptr.alloc((P->n_slices + 1) * 8));
    std::vector<long long> h_sp(P->n_slices + 1, 0);
    if (P->n_slices > 0) {
        slice_len_kernel<<<grid_for((int64_t)P->n_slices * 32), 256, 0, s>>>(P->rp.as<int32_t>(), P->slice_row.as<int32_t>(), P->n_slices, P->slice_len.as<int32_t>());
        DevBuf st;
        MPK_TRY(st.alloc_on(scan_tmp_bytes(P->n_slices + 1), s));
        MPK_TRY((exclusive_scan<int32_t, long long>(P->slice_len.as<int32_t>(), P->slice_ptr.as<long long>(), P->n_slices, st.p, s)));
        MPK_CUDA(cudaMemcpyAsync(h_sp.data(), P->slice_ptr.p, (P->n_slices + 1) * 8, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        P->sell_nnz = h_sp[P->n_slices] * 32;
    }
    if (P->sell_nnz >= (1ll << 31)) return MPK_ERR_UNIMPLEMENTED;   // 32-bit entry offsets
    // ---- chunks: up to chunk_slices consecutive slices of one group, and no more SELL entries
    // than one shared-memory slot holds (two slots of FP64 entries, 12 bytes each, in the
    // opt-in shared memory)
    MPK_CUDA(cudaDeviceGetAttribute(&P->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
    const long long slot_entries = ((long long)P->smem_optin - 1024) / (2 * 12) / 32 * 32;
    P->stage_smem = o.stage != 0;
    std::vector<int32_t> h_chunk_slice, h_chunk_row;
    std::vector<long long> h_ce;
    P->h_group_chunk.assign(P->n_groups + 1, 0);
    P->h_chunk_group.clear();
    P->max_chunk_entries = 0;
    {
        int32_t sl = 0;
        for (int32_t g = 0; g < P->n_groups; g++) {
            P->h_group_chunk[g] = (int32_t)h_chunk_slice.size();
            while (sl < P->n_slices && h_slice_group[sl] == g) {
                const int32_t first = sl;
                long long ents = 32ll * (h_sp[sl + 1] - h_sp[sl]);
                sl++;
                while (sl < P->n_slices && h_slice_group[sl] == g && sl - first < o.chunk_slices &&
                       ents + 32ll * (h_sp[sl + 1] - h_sp[sl]) <= slot_entries) {
                    ents += 32ll * (h_sp[sl + 1] - h_sp[sl]);
                    sl++;
                }
                if (ents > slot_entries) P->stage_smem = 0;   // one slice exceeds a slot
                h_chunk_slice.push_back(first);
                h_chunk_row.push_back(h_slice_row[first]);
                h_ce.push_back(32ll * h_sp[first]);
                P->h_chunk_group.push_back(g);
                P->max_chunk_entries = std::max<int64_t>(P->max_chunk_entries, ents);
            }
        }
        P->h_group_chunk[P->n_groups] = (int32_t)h_chunk_slice.size();
    }
    P->n_chunks = (int32_t)h_chunk_slice.size();
    h_chunk_slice.push_back(P->n_slices);
    h_chunk_row.push_back((int32_t)n);
    h_ce.push_back(P->sell_nnz);
    MPK_TRY(upload(P->chunk_slice, h_chunk_slice, s));
    MPK_TRY(upload(P->chunk_row, h_chunk_row, s));
    MPK_TRY(upload(P->chunk_entry, h_ce, s));
    P->h_chunk_entry = h_ce;
    MPK_CUDA(cudaStreamSynchronize(s));
    MPK_TRY(P->s_col.alloc(std::max<int64_t>(P->sell_nnz, 1) * 4));
    if (P->has64) MPK_TRY(P->s_val64.alloc(std::max<int64_t>(P->sell_nnz, 1) * 8));
    if (P->has32) MPK_TRY(P->s_val32.alloc(std::max<int64_t>(P->sell_nnz, 1) * 4));
    if (P->jacobi) {
        MPK_TRY(P->dinv64.alloc(std::max<int64_t>(n, 1) * 8));
        if (P->has64) MPK_TRY(P->s_jval64.alloc(std::max<int64_t>(P->sell_nnz, 1) * 8));
        if (P->has32) MPK_TRY(P->s_jval32.alloc(std::max<int64_t>(P->sell_nnz, 1) * 4));
        MPK_TRY(P->s_lmask.alloc(std::max<int64_t>(P->sell_nnz / 32, 1) * 4));
    }
    mpk_status st = mpk_build_blocks(P, s);
    if (st != MPK_OK) return st;
    if (P->jacobi && P->n_slices > 0) {   // needs the SELL columns filled above
        gs2_lower_mask_kernel<<<grid_for((int64_t)P->n_slices * 32), 256, 0, s>>>(
            P->s_col.as<int32_t>(), P->slice_ptr.as<long long>(), P->slice_row.as<int32_t>(),
            P->slice_len.as<int32_t>(), P->n_slices, P->perm.as<int32_t>(),
            P->s_lmask.as<uint32_t>());
        MPK_CUDA(cudaGetLastError());
        // packed lower slices for the GS2 inner stages
        DevBuf llen;
        MPK_TRY(llen.alloc(P->n_slices * 4));
        gs2_lower_len_kernel<<<grid_for((int64_t)P->n_slices * 32), 256, 0, s>>>(
            P->slice_row.as<int32_t>(), P->slice_len.as<int32_t>(), P->slice_ptr.as<long long>(),
            P->n_slices, P->s_lmask.as<uint32_t>(), llen.as<int32_t>());
        MPK_CUDA(cudaGetLastError());
        std::vector<int32_t> h_len(P->n_slices);
        MPK_CUDA(cudaMemcpyAsync(h_len.data(), llen.p, P->n_slices * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
        std::vector<long long> h_lp(P->n_slices + 1, 0);
        for (int64_t i = 0; i < P->n_slices; i++) h_lp[i + 1] = h_lp[i] + h_len[i];
        P->l_sell_nnz = 32ll * h_lp[P->n_slices];
        MPK_TRY(upload(P->l_slice_ptr, h_lp, s));
        MPK_TRY(upload(P->l_slice_len, h_len, s));
        MPK_TRY(P->l_col.alloc(std::max<int64_t>(P->l_sell_nnz, 1) * 4));
        if (P->has64) MPK_TRY(P->l_val64.alloc(std::max<int64_t>(P->l_sell_nnz, 1) * 8));
        if (P->has32) MPK_TRY(P->l_val32.alloc(std::max<int64_t>(P->l_sell_nnz, 1) * 4));
        MPK_TRY(gs2_lower_fill(P, s));
    }

    // ---- blocked-task dependency ranges and flags
    MPK_TRY(P->dep_lo.alloc((P->n_chunks + 1) * 4));
    MPK_TRY(P->dep_hi.alloc((P->n_chunks + 1) * 4));
    MPK_TRY(P->flags.alloc((P->n_chunks + 1) * 4));
    MPK_CUDA(cudaMemsetAsync(P->flags.p, 0, (P->n_chunks + 1) * 4, s));
    if (P->n_chunks > 0) {
        DevBuf row_chunk;
        MPK_TRY(row_chunk.alloc_on(n * 4, s));
        row_chunk_kernel<<<(unsigned)std::min<int64_t>(P->n_chunks, 65535), 256, 0, s>>>(P->chunk_row.as<int32_t>(), P->n_chunks, row_chunk.as<int32_t>());
        fill_i32_kernel<<<grid_for(P->n_chunks), 256, 0, s>>>(P->dep_lo.as<int32_t>(), P->n_chunks, 0x7fffffff);
        fill_i32_kernel<<<grid_for(P->n_chunks), 256, 0, s>>>(P->dep_hi.as<int32_t>(), P->n_chunks, -1);
        dep_kernel<<<grid_for(n), 256, 0, s>>>(P->rp.as<int32_t>(), P->ci.as<int32_t>(), row_chunk.as<int32_t>(), n, sym ? 0 : 1, P->dep_lo.as<int32_t>(), P->dep_hi.as<int32_t>());
        MPK_CUDA(cudaGetLastError());
        P->h_dep_hi.assign(P->n_chunks, 0);
        MPK_CUDA(cudaMemcpyAsync(P->h_dep_hi.data(), P->dep_hi.p, P->n_chunks * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
    }
    // ---- warp-task counter blocks: up to 32 consecutive chunks of one group
    {
        std::vector<int32_t> h_cbs, h_blast;
        P->h_chunk_blk.assign(P->n_chunks, 0);
        for (int32_t g = 0; g < P->n_groups; g++) {
            for (int32_t c = P->h_group_chunk[g]; c < P->h_group_chunk[g + 1]; c++) {
                if (c == P->h_group_chunk[g] || h_cbs.back() == 32) {
                    h_cbs.push_back(0);
                    h_blast.push_back(c);
                }
                h_cbs.back()++;
                h_blast.back() = c;
                P->h_chunk_blk[c] = (int32_t)h_cbs.size() - 1;
            }
        }
        P->n_cblk = (int32_t)h_cbs.size();
        P->h_wait_blk.assign(P->n_chunks, 0);
        P->h_dep_hi_blk.assign(P->n_chunks, 0);
        for (int32_t c = 0; c < P->n_chunks; c++) {
            const int32_t hi = std::max(P->h_dep_hi[c], c);
            P->h_wait_blk[c] = P->h_chunk_blk[hi];
            P->h_dep_hi_blk[c] = h_blast[P->h_wait_blk[c]];
        }
        MPK_TRY(upload(P->cblk_size, h_cbs, s));
        MPK_TRY(P->wave_cnt.alloc((size_t)(P->p_blk + 1) * std::max(P->n_cblk, 1) * 4));
        MPK_CUDA(cudaMemsetAsync(P->wave_cnt.p, 0, P->wave_cnt.bytes, s));
        MPK_TRY(P->wave_kep.alloc((MPK_MAX_P + 1) * 4));
        MPK_CUDA(cudaMemsetAsync(P->wave_kep.p, 0, P->wave_kep.bytes, s));
        // ready-first cursors: (local power, shard), at most one shard per resident warp
        P->max_shards = P->n_sm * 64;
        MPK_TRY(P->wave_cur.alloc((size_t)(MPK_MAX_P + 1) * P->max_shards * 4));
        MPK_CUDA(cudaMemsetAsync(P->wave_cur.p, 0, P->wave_cur.bytes, s));
        MPK_TRY(upload(P->chunk_blk_d, P->h_chunk_blk, s));
        MPK_TRY(upload(P->wait_blk_d, P->h_wait_blk, s));
    }
    MPK_TRY(P->prefix.alloc((MPK_MAX_P + 2) * sizeof(unsigned long long)));
    MPK_CUDA(cudaMemsetAsync(P->prefix.p, 0, P->prefix.bytes, s));
    P->ctas_per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 3;
    // compute warps + one control warp
    P->blocked_block = ((o.block_threads == 128 || o.block_threads == 256) ? o.block_threads : 256) + 32;
    P->sched_type = o.schedule == 0 ? 0 : 1;
    // lag-greedy slack: about the tasks in flight (two slots per resident CTA)
    P->sched_slack = o.slack_tasks > 0 ? o.slack_tasks : 2ll * P->n_sm * P->ctas_per_sm;
    P->wave = o.kernel == 1 ? 0 : 1;
    P->ready_first = o.kernel == 3 ? 1 : 0;
    P->shard_warps = o.shard_warps > 0 ? o.shard_warps : 4;
    P->short_rows = (P->n_slices > 0 && P->sell_nnz <= 12ll * 32 * P->n_slices) ? 1 : 0;
    P->wave_dynamic = o.kernel == 2 ? 0 : 1;
    // warp tasks: four tasks per resident warp (32 per SM) - measured best on the 27-point
    // 160^3 matrix in FP32 and FP64; smaller slack makes warps wait for their dependencies
    P->wave_slack = o.slack_tasks > 0 ? o.slack_tasks : 4ll * 32 * P->n_sm;
    // lane tasks: lanes per row of the single-rhs kernels (automatic: 1 - sharing rows
    // measured slower in both precisions on the 27-point 160^3 matrix, unblocked and blocked)
    if (o.lanes_per_row == 0) P->lanes = 1;
    else if (o.lanes_per_row == 1 || o.lanes_per_row == 2 || o.lanes_per_row == 4 || o.lanes_per_row == 8)
        P->lanes = o.lanes_per_row;
    else return MPK_ERR_ARG;
    if (o.task_units < 0 || o.kernel < 0 || o.kernel > 6 || o.task_dispatch < 0 || o.task_dispatch > 2 ||
        o.owner_lag < 0 || o.owner_lag > 4 || o.owner_prefetch < 0 || o.owner_prefetch > 4 ||
        o.level_order < 0 || o.level_order > 1)
        return MPK_ERR_ARG;
    P->lane_kernel = (o.kernel == 4 || o.kernel == 5 || o.kernel == 6 || P->lanes > 1) ? 1 : 0;
    P->lane_slack = o.slack_tasks > 0 ? o.slack_tasks : 0;
    MPK_CUDA(cudaStreamSynchronize(s));
    auto t1 = std::chrono::steady_clock::now();
    P->create_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    return MPK_OK;
}

// ---- lane-task graph: units = sub-slices of 32 / lpr rows, chunks of `units` units inside
// one level group, dependency ranges over the rows (as for the slice chunks), counter blocks
// of up to 32 chunks of one group
mpk_status mpk_get_lane_graph(mpk_plan_s *P, int lpr, int units, LaneGraph **out, cudaStream_t s) {
    if (lpr != 1 && lpr != 2 && lpr != 4 && lpr != 8) return MPK_ERR_ARG;
    if (units < 1) units = 1;
    const int key = lpr * 65536 + units;
    auto it = P->lane_graphs.find(key);
    if (it != P->lane_graphs.end()) {
        *out = it->second.get();
        return MPK_OK;
    }
    std::unique_ptr<LaneGraph> G(new LaneGraph());
    G->lpr = lpr;
    G->units = units;
    const int64_t n = P->n;
    const int R = 32 / lpr;
    std::vector<int32_t> sr(P->n_slices + 1, 0), slen(P->n_slices + 1, 0);
    std::vector<long long> sp(P->n_slices + 1, 0);
    if (P->n_slices > 0) {
        MPK_CUDA(cudaMemcpyAsync(sr.data(), P->slice_row.p, (P->n_slices + 1) * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaMemcpyAsync(slen.data(), P->slice_len.p, P->n_slices * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaMemcpyAsync(sp.data(), P->slice_ptr.p, (P->n_slices + 1) * 8, cudaMemcpyDeviceToHost, s));
    }
    MPK_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> code, cu, crow, cgroup;
    std::vector<int4> meta;
    int32_t sl = 0;
    for (int32_t g = 0; g < P->n_groups; g++) {
        const int32_t gend = P->h_level_ptr[P->h_group_ptr[g + 1]];
        int in_chunk = 0;
        for (; sl < P->n_slices && sr[sl] < gend; sl++) {
            const int32_t rows = sr[sl + 1] - sr[sl];
            for (int h = 0; h * R < rows; h++) {
                if (in_chunk == 0 || in_chunk == units) {
                    cu.push_back((int32_t)code.size());
                    crow.push_back(sr[sl] + h * R);
                    cgroup.push_back(g);
                    in_chunk = 0;
                }
                code.push_back(sl * lpr + h);
                meta.push_back(make_int4((int)(32ll * sp[sl] + h * R), slen[sl], sr[sl] + h * R, sr[sl + 1]));
                G->max_len = std::max(G->max_len, slen[sl]);
                in_chunk++;
            }
        }
    }
    G->n_units = (int32_t)code.size();
    G->n_chunks = (int32_t)cu.size();
    cu.push_back(G->n_units);
    crow.push_back((int32_t)n);
    MPK_TRY(upload(G->unit_code, code, s));
    MPK_TRY(upload(G->unit_meta, meta, s));
    G->h_meta = meta;
    MPK_TRY(upload(G->chunk_unit, cu, s));
    G->h_chunk_unit = cu;
    std::vector<int32_t> dep_hi(G->n_chunks, 0);
    if (G->n_chunks > 0) {
        DevBuf d_crow, row_chunk, dlo, dhi;
        MPK_TRY(upload(d_crow, crow, s));
        MPK_TRY(row_chunk.alloc_on(n * 4, s));
        MPK_TRY(dlo.alloc_on((size_t)G->n_chunks * 4, s));
        MPK_TRY(dhi.alloc_on((size_t)G->n_chunks * 4, s));
        row_chunk_kernel<<<(unsigned)std::min<int64_t>(G->n_chunks, 65535), 256, 0, s>>>(d_crow.as<int32_t>(), G->n_chunks, row_chunk.as<int32_t>());
        fill_i32_kernel<<<grid_for(G->n_chunks), 256, 0, s>>>(dlo.as<int32_t>(), G->n_chunks, 0x7fffffff);
        fill_i32_kernel<<<grid_for(G->n_chunks), 256, 0, s>>>(dhi.as<int32_t>(), G->n_chunks, -1);
        dep_kernel<<<grid_for(n), 256, 0, s>>>(P->rp.as<int32_t>(), P->ci.as<int32_t>(), row_chunk.as<int32_t>(), n,
                                               P->opts.assume_symmetric ? 0 : 1, dlo.as<int32_t>(), dhi.as<int32_t>());
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaMemcpyAsync(dep_hi.data(), dhi.p, (size_t)G->n_chunks * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<int32_t> cbs, blast;
    G->h_chunk_blk.assign(G->n_chunks, 0);
    for (int32_t c = 0; c < G->n_chunks; c++) {
        if (c == 0 || cgroup[c] != cgroup[c - 1] || cbs.back() == 32) {
            cbs.push_back(0);
            blast.push_back(c);
        }
        cbs.back()++;
        blast.back() = c;
        G->h_chunk_blk[c] = (int32_t)cbs.size() - 1;
    }
    G->n_cblk = (int32_t)cbs.size();
    G->h_wait_blk.assign(G->n_chunks, 0);
    G->h_dep_hi_blk.assign(G->n_chunks, 0);
    for (int32_t c = 0; c < G->n_chunks; c++) {
        const int32_t hi = std::max(dep_hi[c], c);
        G->h_wait_blk[c] = G->h_chunk_blk[hi];
        G->h_dep_hi_blk[c] = blast[G->h_wait_blk[c]];
    }
    MPK_TRY(upload(G->cblk_size, cbs, s));
    G->h_cblk_size = cbs;
    MPK_TRY(G->cnt.alloc((size_t)(P->p_blk + 1) * std::max(G->n_cblk, 1) * 4));
    MPK_CUDA(cudaMemsetAsync(G->cnt.p, 0, G->cnt.bytes, s));
    MPK_TRY(G->kep.alloc((MPK_MAX_P + 1) * 4));
    MPK_CUDA(cudaMemsetAsync(G->kep.p, 0, G->kep.bytes, s));
    MPK_CUDA(cudaStreamSynchronize(s));   // host vectors above outlive their copies
    *out = G.get();
    P->lane_graphs[key] = std::move(G);
    return MPK_OK;
}

// Owner-kernel dependencies (one thread per row): the CTA range and last group of the shares
// holding the row's columns, merged into the row's share; with `sym_close` also the row's
// share merged into each of those shares (closure over A^T).  dlo / dhi / dg start at the
// share's own CTA and group.
__global__ void owner_dep_kernel(const int32_t *rp, const int32_t *ci, const int32_t *row_share, int64_t n,
                                 int G, int sym_close, int32_t *dlo, int32_t *dhi, int32_t *dg) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t sh = row_share[r];
        const int32_t c = sh % G, g = sh / G;
        int32_t lo = c, hi = c, gd = g;
        for (int32_t t = rp[r]; t < rp[r + 1]; t++) {
            const int32_t s2 = row_share[ci[t]];
            const int32_t c2 = s2 % G, g2 = s2 / G;
            lo = min(lo, c2);
            hi = max(hi, c2);
            gd = max(gd, g2);
            if (sym_close) {
                atomicMin(&dlo[s2], c);
                atomicMax(&dhi[s2], c);
                atomicMax(&dg[s2], g);
            }
        }
        atomicMin(&dlo[sh], lo);
        atomicMax(&dhi[sh], hi);
        atomicMax(&dg[sh], gd);
    }
}

__global__ void owner_dep_init_kernel(int64_t n_shares, int G, int32_t *dlo, int32_t *dhi, int32_t *dg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_shares;
         i += (int64_t)gridDim.x * blockDim.x) {
        dlo[i] = (int32_t)(i % G);
        dhi[i] = (int32_t)(i % G);
        dg[i] = (int32_t)(i / G);
    }
}

__global__ void owner_dep_pack_kernel(int64_t n_shares, const int32_t *dlo, const int32_t *dhi,
                                      const int32_t *dg, int4 *dep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_shares;
         i += (int64_t)gridDim.x * blockDim.x)
        dep[i] = make_int4(dlo[i], dhi[i], dg[i], 0);
}

mpk_status mpk_get_owner_graph(mpk_plan_s *P, int G, OwnerGraph **out, cudaStream_t s) {
    if (G < 1) return MPK_ERR_ARG;
    auto it = P->owner_graphs.find(G);
    if (it != P->owner_graphs.end()) {
        *out = it->second.get();
        return MPK_OK;
    }
    std::unique_ptr<OwnerGraph> O(new OwnerGraph());
    O->G = G;
    const int64_t n = P->n;
    const int64_t n_shares = (int64_t)P->n_groups * G;
    if (n_shares >= (1ll << 31)) return MPK_ERR_UNIMPLEMENTED;
    std::vector<int32_t> sr(P->n_slices + 1, 0), slen(P->n_slices + 1, 0);
    if (P->n_slices > 0) {
        MPK_CUDA(cudaMemcpyAsync(sr.data(), P->slice_row.p, (P->n_slices + 1) * 4, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaMemcpyAsync(slen.data(), P->slice_len.p, P->n_slices * 4, cudaMemcpyDeviceToHost, s));
    }
    MPK_CUDA(cudaStreamSynchronize(s));
    // split each group's slices into G shares of about equal work: a slice weighs its stored
    // entries per row plus two (the per-slice cost of the row epilogue)
    std::vector<int32_t> share((size_t)n_shares + 1, 0), share_row((size_t)n_shares + 1, 0);
    int32_t sl = 0;
    for (int32_t g = 0; g < P->n_groups; g++) {
        const int32_t gend = P->h_level_ptr[P->h_group_ptr[g + 1]];
        const int32_t g0 = sl;
        while (sl < P->n_slices && sr[sl] < gend) sl++;
        const int32_t g1 = sl;
        int64_t wsum = 0;
        for (int32_t t = g0; t < g1; t++) wsum += slen[t] + 2;
        int32_t cur = g0;
        int64_t acc = 0;
        for (int c = 0; c < G; c++) {
            const int64_t target = wsum * c / G;
            while (cur < g1 && acc < target) acc += slen[cur++] + 2;
            share[(size_t)g * G + c] = cur;
        }
        for (int c = 0; c < G; c++) {
            const int32_t a = share[(size_t)g * G + c];
            const int32_t b = c + 1 < G ? share[(size_t)g * G + c + 1] : g1;
            O->max_share_slices = std::max(O->max_share_slices, b - a);
        }
    }
    share[(size_t)n_shares] = P->n_slices;
    for (int64_t i = 0; i <= n_shares; i++) share_row[i] = share[i] < P->n_slices ? sr[share[i]] : (int32_t)n;
    MPK_TRY(upload(O->share, share, s));
    MPK_TRY(O->dep.alloc((size_t)std::max<int64_t>(n_shares, 1) * sizeof(int4)));
    if (n_shares > 0 && n > 0) {
        DevBuf d_srow, row_share, dlo, dhi, dg;
        MPK_TRY(upload(d_srow, share_row, s));
        MPK_TRY(row_share.alloc_on(n * 4, s));
        MPK_TRY(dlo.alloc_on((size_t)n_shares * 4, s));
        MPK_TRY(dhi.alloc_on((size_t)n_shares * 4, s));
        MPK_TRY(dg.alloc_on((size_t)n_shares * 4, s));
        row_chunk_kernel<<<(unsigned)std::min<int64_t>(n_shares, 65535), 256, 0, s>>>(d_srow.as<int32_t>(), n_shares, row_share.as<int32_t>());
        owner_dep_init_kernel<<<grid_for(n_shares), 256, 0, s>>>(n_shares, G, dlo.as<int32_t>(), dhi.as<int32_t>(), dg.as<int32_t>());
        owner_dep_kernel<<<grid_for(n), 256, 0, s>>>(P->rp.as<int32_t>(), P->ci.as<int32_t>(), row_share.as<int32_t>(), n, G,
                                                     P->opts.assume_symmetric ? 0 : 1, dlo.as<int32_t>(), dhi.as<int32_t>(), dg.as<int32_t>());
        owner_dep_pack_kernel<<<grid_for(n_shares), 256, 0, s>>>(n_shares, dlo.as<int32_t>(), dhi.as<int32_t>(), dg.as<int32_t>(), O->dep.as<int4>());
        MPK_CUDA(cudaGetLastError());
    }
    MPK_TRY(O->prog.alloc((size_t)(P->p_blk + 1) * G * 4));
    MPK_CUDA(cudaMemsetAsync(O->prog.p, 0, O->prog.bytes, s));
    MPK_TRY(O->kep.alloc((MPK_MAX_P + 1) * 4));
    MPK_CUDA(cudaMemsetAsync(O->kep.p, 0, O->kep.bytes, s));
    MPK_CUDA(cudaStreamSynchronize(s));   // host vectors above outlive their copies
    *out = O.get();
    P->owner_graphs[G] = std::move(O);
    return MPK_OK;
}

// SELL fill (shared with value updates)
mpk_status mpk_build_blocks(mpk_plan_s *P, cudaStream_t s) {
    if (P->n_slices == 0) return MPK_OK;
    sell_fill_kernel<<<grid_for((int64_t)P->n_slices * 32), 256, 0, s>>>(
        P->rp.as<int32_t>(), P->ci.as<int32_t>(), P->has64 ? P->val64.as<double>() : nullptr,
        P->has32 ? P->val32.as<float>() : nullptr, P->slice_row.as<int32_t>(),
        P->slice_len.as<int32_t>(), P->slice_ptr.as<long long>(), P->n_slices,
        P->s_col.as<int32_t>(), P->has64 ? P->s_val64.as<double>() : nullptr,
        P->has32 ? P->s_val32.as<float>() : nullptr);
    MPK_CUDA(cudaGetLastError());
    if (P->jacobi) {
        if (P->has64)
            jacobi_dinv_kernel<double><<<grid_for(P->n), 256, 0, s>>>(
                P->rp.as<int32_t>(), P->ci.as<int32_t>(), P->val64.as<double>(), P->n,
                P->dinv64.as<double>());
        else
            jacobi_dinv_kernel<float><<<grid_for(P->n), 256, 0, s>>>(
                P->rp.as<int32_t>(), P->ci.as<int32_t>(), P->val32.as<float>(), P->n,
                P->dinv64.as<double>());
        MPK_CUDA(cudaGetLastError());
        jacobi_scale_kernel<<<grid_for(P->sell_nnz), 256, 0, s>>>(
            P->s_col.as<int32_t>(), P->has64 ? P->s_val64.as<double>() : nullptr,
            P->has64 ? nullptr : P->s_val32.as<float>(), P->sell_nnz,
            P->dinv64.as<double>(), P->has64 ? P->s_jval64.as<double>() : nullptr,
            P->has32 ? P->s_jval32.as<float>() : nullptr);
        MPK_CUDA(cudaGetLastError());
        MPK_TRY(gs2_lower_fill(P, s));   // value updates: refresh the packed lower slices
    }
    return MPK_OK;
}

// slice_ptr holds the running sum of slice lengths: entry (j, lane) of slice s lives at
// 32*slice_ptr[s] + 32*j + lane in s_col / s_val*.

extern "C" mpk_status mpk_plan_create(const mpk_csr *A, int32_t p_max, const mpk_plan_opts *opts,
                                      cudaStream_t stream, mpk_plan_t *out) {
    if (!out) return MPK_ERR_ARG;
    *out = nullptr;
    if (!A || A->n < 0 || A->nnz < 0 || A->n >= (1ll << 31) - 1 || A->nnz >= (1ll << 31) - 1)
        return MPK_ERR_ARG;
    if (p_max < 1 || p_max > MPK_MAX_P) return MPK_ERR_ARG;
    if (A->dtype != MPK_F32 && A->dtype != MPK_F64) return MPK_ERR_ARG;
    if (A->n > 0 && !A->row_ptr) return MPK_ERR_ARG;
    if (A->nnz > 0 && (!A->col || !A->val)) return MPK_ERR_ARG;
    if (A->n == 0 && A->nnz != 0) return MPK_ERR_ARG;
    mpk_plan_s *P = new (std::nothrow) mpk_plan_s();
    if (!P) return MPK_ERR_OOM;
    mpk_status st = plan_create_impl(A, p_max, opts, stream, P);
    if (st != MPK_OK) {
        cudaStreamSynchronize(stream);
        cudaGetLastError();
        delete P;
        return st;
    }
    *out = P;
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_destroy(mpk_plan_t plan) {
    if (!plan) return MPK_ERR_ARG;
    cudaDeviceSynchronize();
    delete plan;
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_stats(mpk_plan_t P, mpk_plan_info *st) {
    if (!P || !st) return MPK_ERR_ARG;
    memset(st, 0, sizeof(*st));
    st->n = P->n;
    st->nnz = P->nnz;
    st->n_levels = P->n_levels;
    st->n_groups = P->n_groups;
    st->n_slices = P->n_slices;
    st->n_chunks = P->n_chunks;
    st->root = P->root;
    st->p_blk = P->p_blk;
    st->l2_budget_bytes = P->opts.l2_budget_bytes;
    st->sell_nnz = P->sell_nnz;
    size_t b = 0;
    for (const DevBuf *d : {&P->perm, &P->iperm, &P->level, &P->level_ptr, &P->group_ptr, &P->rp,
                            &P->ci, &P->val64, &P->val32, &P->entry_map, &P->slice_row,
                            &P->slice_ptr, &P->slice_len, &P->s_col, &P->s_val64, &P->s_val32,
                            &P->s_jval64, &P->s_jval32, &P->dinv64, &P->s_lmask, &P->l_slice_ptr, &P->l_slice_len, &P->l_col, &P->l_val64, &P->l_val32, &P->chunk_slice, &P->chunk_row, &P->chunk_entry, &P->dep_lo, &P->dep_hi, &P->flags,
                            &P->ctrl, &P->ws_x, &P->ws_y})
        b += d->bytes;
    st->device_bytes = (int64_t)b;
    st->create_ms = P->create_ms;
    st->bfs_sweeps = P->bfs_sweeps;
    st->max_level_rows = P->max_level_rows;
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_perm(mpk_plan_t P, int32_t *perm, int32_t *iperm, int32_t *level,
                                    int32_t *level_ptr, int32_t *group_ptr, cudaStream_t s) {
    if (!P) return MPK_ERR_ARG;
    const size_t nb = P->n * sizeof(int32_t);
    if (perm && nb) MPK_CUDA(cudaMemcpyAsync(perm, P->perm.p, nb, cudaMemcpyDeviceToDevice, s));
    if (iperm && nb) MPK_CUDA(cudaMemcpyAsync(iperm, P->iperm.p, nb, cudaMemcpyDeviceToDevice, s));
    if (level && nb) MPK_CUDA(cudaMemcpyAsync(level, P->level.p, nb, cudaMemcpyDeviceToDevice, s));
    if (level_ptr)
        MPK_CUDA(cudaMemcpyAsync(level_ptr, P->level_ptr.p, (P->n_levels + 1) * 4, cudaMemcpyDeviceToDevice, s));
    if (group_ptr)
        MPK_CUDA(cudaMemcpyAsync(group_ptr, P->group_ptr.p, (P->n_groups + 1) * 4, cudaMemcpyDeviceToDevice, s));
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_csr(mpk_plan_t P, mpk_dtype dtype, int32_t *row_ptr, int32_t *col,
                                   void *val, cudaStream_t s) {
    if (!P) return MPK_ERR_ARG;
    if (dtype == MPK_F64 && val && !P->has64) return MPK_ERR_ARG;
    if (dtype == MPK_F32 && val && !P->has32) return MPK_ERR_ARG;
    if (row_ptr) MPK_CUDA(cudaMemcpyAsync(row_ptr, P->rp.p, (P->n + 1) * 4, cudaMemcpyDeviceToDevice, s));
    if (col && P->nnz) MPK_CUDA(cudaMemcpyAsync(col, P->ci.p, P->nnz * 4, cudaMemcpyDeviceToDevice, s));
    if (val && P->nnz)
        MPK_CUDA(cudaMemcpyAsync(val, dtype == MPK_F64 ? P->val64.p : P->val32.p,
                                 P->nnz * (dtype == MPK_F64 ? 8 : 4), cudaMemcpyDeviceToDevice, s));
    return MPK_OK;
}

extern "C" mpk_status mpk_plan_update_values(mpk_plan_t P, const mpk_csr *A, cudaStream_t s) {
    if (!P || !A || A->n != P->n || A->nnz != P->nnz) return MPK_ERR_ARG;
    if (P->nnz == 0) return MPK_OK;
    if (!A->val) return MPK_ERR_ARG;
    double *v64 = P->has64 ? P->val64.as<double>() : nullptr;
    float *v32 = P->has32 ? P->val32.as<float>() : nullptr;
    if (A->dtype == MPK_F64)
        update_values_kernel<double><<<grid_for(P->nnz), 256, 0, s>>>((const double *)A->val, P->entry_map.as<int32_t>(), P->nnz, v64, v32);
    else
        update_values_kernel<float><<<grid_for(P->nnz), 256, 0, s>>>((const float *)A->val, P->entry_map.as<int32_t>(), P->nnz, v64, v32);
    MPK_CUDA(cudaGetLastError());
    return mpk_build_blocks(P, s);
}
