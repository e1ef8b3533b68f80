// Internal declarations of the GB300 MPK library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <memory>
#include <vector>

#include "../../include/mpk.h"

#define MPK_MAX_P 63

// -------------------------------------------------------------------------------------------
// Error plumbing: every CUDA call is checked; failures become an mpk_status.
// -------------------------------------------------------------------------------------------
#define MPK_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError(); /* clear the thread's non-sticky error state */          \
            mpk_log_cuda_error(e_, #call, __FILE__, __LINE__);                           \
            return e_ == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA;         \
        }                                                                                \
    } while (0)

#define MPK_TRY(...)                                                                     \
    do {                                                                                 \
        mpk_status s_ = (__VA_ARGS__);                                                   \
        if (s_ != MPK_OK) return s_;                                                     \
    } while (0)

void mpk_log_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Device buffer owned by the library (freed on destruction).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;   // stream-ordered buffers: the stream that owns them
    bool ordered = false;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (ordered) cudaFreeAsync(p, stream);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        ordered = false;
    }
    // Stream-ordered allocation from the library's memory pool: allocated and freed in the
    // order of stream s, so neither waits for work on other streams (cudaFree synchronises the
    // whole device).  Only for buffers that work on s alone uses.
    mpk_status alloc_on(size_t b, cudaStream_t s);
    mpk_status alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA;
        }
        bytes = b;
        return MPK_OK;
    }
    // grow-only
    mpk_status ensure(size_t b) { return (bytes >= b && p) ? MPK_OK : alloc(b); }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Control block of the blocked MPK launches (device memory, one per plan).
struct MpkCtrl {
    uint32_t epoch;       // increments once per completed blocked launch
    uint32_t ticket;      // task dispenser (reset by the last CTA)
    uint32_t done_ctas;   // CTAs finished in this launch (reset by the last CTA)
    uint32_t error;       // latched: 1 = a dependency wait ran out
    uint32_t err_task;    // first task that timed out (diagnostics)
    uint32_t pad[3];
};

// Cached blocked schedule for one (segment length) value.
struct Schedule {
    int32_t p = 0;
    int64_t slack = 0;
    int64_t n_tasks = 0;
    DevBuf desc;    // int4 per ticket: {chunk | (k << 24), first SELL entry, entries, 0}
};

// Task graph of the lane-task kernel (opts.kernel = 4, or lanes_per_row > 1): units are
// sub-slices of 32 / lpr rows of the SELL-32 slices (only those holding a row); a chunk is up
// to `units` consecutive units of one level group; chunks are counted in blocks of up to 32
// consecutive chunks of one group.  A task (chunk c, power k) waits until every block up to
// the one holding max(dep_hi(c), c) has finished power k-1.  Built on first use per
// (lpr, units) and kept by the plan.
struct LaneGraph {
    int lpr = 1, units = 1;
    int32_t n_units = 0, n_chunks = 0, n_cblk = 0;
    int32_t max_len = 0;               // longest slice (entries per row)
    DevBuf unit_code;                  // int32 per unit: slice * lpr + sub-slice, ascending
    DevBuf unit_meta;                  // int4 per unit: {first SELL entry, slice length,
                                       // first row, end of the slice's rows}
    DevBuf chunk_unit;                 // int32 [n_chunks + 1]: first unit of each chunk
    DevBuf cblk_size;                  // chunks per counter block
    DevBuf cnt;                        // uint32 [(p_blk + 1) * n_cblk]: counters [(k) * n_cblk + b]
    DevBuf kep;                        // uint32 per local power: launches that ran it
    std::vector<int4> h_meta;          // unit_meta on the host
    std::vector<int32_t> h_cblk_size;  // cblk_size on the host
    std::vector<int32_t> h_chunk_unit; // first unit of each chunk (n_chunks + 1)
    std::vector<int32_t> h_chunk_blk;  // counter block of each chunk
    std::vector<int32_t> h_wait_blk;   // last block a chunk's task waits for
    std::vector<int32_t> h_dep_hi_blk; // last chunk of that block (the schedule's bound)
    std::map<int64_t, std::unique_ptr<struct Schedule>> schedules;   // key: p and slack
};

// Share graph of the owner kernel (opts.kernel = 6): every level group's slices split into G
// contiguous shares balanced by stored entries, share (g, c) = slices [share[g G + c],
// share[g G + c + 1]) owned by CTA c for every power.  dep holds, per share, the range of
// CTAs [clo, chi] owning any share its rows read (and, unless the pattern is declared
// symmetric, any share whose rows read it: the closure over A^T that the 3-buffer ring of
// MPK_FINAL_ONLY needs) and the last group among them.  prog counts, per (local power, CTA),
// the groups finished, accumulating over launches against kep.  Built on first use per G.
struct OwnerGraph {
    int32_t G = 0;
    int32_t max_share_slices = 0;
    DevBuf share;      // int32 [n_groups * G + 1]
    DevBuf dep;        // int4 per share {clo, chi, gdep, 0}
    DevBuf prog;       // uint32 [(p_blk + 1) * G]
    DevBuf kep;        // uint32 per local power: launches that ran it
};

// The plan: level structure, permuted matrix in SELL-32 form, blocked-task metadata.
struct mpk_plan_s {
    int device = 0;
    int n_sm = 0;
    int64_t l2_bytes = 0;
    mpk_plan_opts opts{};
    int32_t p_max = 0;
    int32_t p_blk = 0;
    mpk_dtype group_dtype = MPK_F64;   // precision the groups were sized for

    int64_t n = 0, nnz = 0;
    int32_t n_levels = 0, n_groups = 0, n_slices = 0, n_chunks = 0, root = 0;
    int32_t bfs_sweeps = 0, max_level_rows = 0;
    int64_t sell_nnz = 0;
    double create_ms = 0.0;

    // level structure
    DevBuf perm, iperm, level, level_ptr, group_ptr;
    std::vector<int32_t> h_level_ptr, h_group_ptr;

    // permuted CSR (level order)
    DevBuf rp, ci, val64, val32;
    bool has64 = false, has32 = false;
    // map from original CSR entry to permuted entry (for value updates)
    DevBuf entry_map;

    // SELL-32: slice s covers rows [slice_row[s], slice_row[s+1]) (<= 32 rows); entry (j, lane)
    // at slice_ptr[s] + 32*j + lane; padding has col = -1.
    DevBuf slice_row, slice_ptr, slice_len, s_col, s_val64, s_val32;
    // right Jacobi scaling (opts.jacobi): SELL values of A D^-1 in the same layout, and
    // D^-1 in level order (FP64; 1 where the diagonal entry is missing or zero)
    bool jacobi = false;
    DevBuf s_jval64, s_jval32, dinv64;
    // two-stage Gauss-Seidel sub-powers (MPK_GS2, built with opts.jacobi): bit lane of word
    // slice_ptr[s] + j marks a strictly lower entry in the caller's row order
    DevBuf s_lmask;
    // the strictly lower entries packed per row into slices of their own (same rows as the
    // full slices; l_slice_ptr in units of 32 entries), with the Jacobi-scaled values
    DevBuf l_slice_ptr, l_slice_len, l_col, l_val64, l_val32;
    int64_t l_sell_nnz = 0;

    // blocked tasks: chunk c = slices [chunk_slice[c], chunk_slice[c+1]) inside one group
    DevBuf chunk_slice, chunk_row, chunk_entry, dep_lo, dep_hi;
    int64_t max_chunk_entries = 0;    // SELL entries of the largest chunk
    int smem_optin = 0;               // opt-in shared memory per CTA (bytes)
    int stage_smem = 1;               // stage task matrix blocks in shared memory
    std::vector<long long> h_chunk_entry;
    std::vector<int32_t> h_chunk_group;   // group of each chunk
    std::vector<int32_t> h_group_chunk;   // first chunk of each group (n_groups+1)
    DevBuf flags;     // uint32 per chunk
    DevBuf prefix;    // uint64 per power: epoch-tagged count of leading chunks done
    std::vector<int32_t> h_dep_hi;
    int sched_type = 1;       // 0 = level-group wavefront, 1 = lag-greedy
    int64_t sched_slack = 0;  // lag-greedy slack in tasks
    // warp-task kernel (wave): chunks are counted in blocks of up to 32 consecutive chunks of
    // one group; a task waits until every block up to the one holding max(dep_hi(c), c) has
    // finished the previous power.  Counters accumulate over launches: after the j-th launch
    // that ran local power k, block b's counter reads j * cblk_size[b] (mod 2^32).
    int wave = 1;                     // 1: warp-task kernel, 0: CTA-task kernel
    int wave_dynamic = 1;             // warp tasks: 1 dynamic tickets, 0 static round robin
    int short_rows = 0;               // stored rows average <= 12 entries: two slices per warp
    int32_t n_cblk = 0;
    std::vector<int32_t> h_chunk_blk; // counter block of each chunk
    std::vector<int32_t> h_wait_blk;  // last block a chunk's task waits for
    std::vector<int32_t> h_dep_hi_blk;// dep_hi rounded up to the end of its block
    DevBuf cblk_size, wave_cnt;       // chunks per block; counters [(k) * n_cblk + b]
    DevBuf wave_kep;                  // uint32 per local power: launches that ran it
    // ready-first hand-out (opts.kernel = 3): per local power the next chunk not yet handed
    // out (reset by each launch's last CTA), and per chunk its counter block and the last
    // block its task depends on
    int ready_first = 0;
    int32_t shard_warps = 4, max_shards = 1;   // warps per shard; cursor rows allocated
    DevBuf wave_cur, chunk_blk_d, wait_blk_d;
    int64_t wave_slack = 0;
    // automatic blocked / unblocked choice per (precision, p, n_rhs) (opts.blocked = -1)
    std::map<int, bool> auto_blocked;
    DevBuf ctrl;      // MpkCtrl
    uint64_t launches_since_reset = 0;
    int ctas_per_sm = 0;
    int blocked_block = 256;
    std::map<int, std::unique_ptr<Schedule>> schedules;

    // lane tasks: lanes per row of the single-rhs kernels (1, 2, 4, 8), whether the blocked
    // single-rhs path runs the lane-task kernel, and its graphs per (lpr, units)
    int lanes = 1;
    int lane_kernel = 0;
    int64_t lane_slack = 0;            // lag-greedy slack of the lane tasks (0: resident warps)
    std::map<int, std::unique_ptr<LaneGraph>> lane_graphs;
    // owner kernel: share graphs per grid size
    std::map<int, std::unique_ptr<OwnerGraph>> owner_graphs;

    // workspace for permuted / interleaved vectors; ws_h: the GS2 inner iterates (2 vectors)
    DevBuf ws_x, ws_y, ws_host, ws_h;
    uint32_t latched_error = 0;
};

// -------------------------------------------------------------------------------------------
// Helpers implemented in the .cu files
// -------------------------------------------------------------------------------------------
// exclusive scan of int32 in[0..n) into out[0..n] (out[n] = total); 64-bit accumulation,
// error if the total does not fit int32.  tmp: device scratch >= scan_tmp_bytes(n).
size_t scan_tmp_bytes(int64_t n);
mpk_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, void *tmp,
                              cudaStream_t s);

mpk_status mpk_get_schedule(mpk_plan_s *P, int p, Schedule **out, cudaStream_t s);
// Lag-greedy task order (tickets: chunk | power << 24) over nc chunks and p powers, each
// power's chunks ascending; a chunk of power k is emitted once every chunk up to dh[c] has
// been emitted at power k-1 at least `slack` tickets earlier.
mpk_status mpk_lag_greedy_order(int p, int32_t nc, const std::vector<int32_t> &dh, int64_t slack,
                                std::vector<uint32_t> &out);
// The lane-task graph of a plan for (lpr, units), built on first use (plan.cu).
mpk_status mpk_get_lane_graph(mpk_plan_s *P, int lpr, int units, LaneGraph **out, cudaStream_t s);
mpk_status mpk_build_blocks(mpk_plan_s *P, cudaStream_t s);
// The owner kernel's share graph of a plan for G CTAs, built on first use (plan.cu).
mpk_status mpk_get_owner_graph(mpk_plan_s *P, int G, OwnerGraph **out, cudaStream_t s);

// Row-sum kernels shared by the MPK and the solver (apply.cu)
mpk_status mpk_launch_residual(mpk_plan_s *P, const double *x, const double *b, double *r,
                               cudaStream_t s);
// h_gamma of one GS2 application from zero to v (level order, one vector, precision dtype):
// h_0 = v, h_j = v - L_B h_{j-1}; the preconditioned vector is D~^-1 h_gamma.  out and tmp
// are n-vectors; gamma >= 1.
mpk_status mpk_gs2_inner(mpk_plan_s *P, mpk_dtype dtype, int gamma, const void *v, void *out,
                         void *tmp, cudaStream_t s);
mpk_status mpk_apply_internal(mpk_plan_s *P, const mpk_coeffs *co, mpk_dtype dtype,
                              const void *X, int64_t ldx, void *Y, int64_t ldy, int32_t n_rhs,
                              uint32_t flags, cudaStream_t stream);

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
