// The matrix power kernel (Sec. 3, Alg. 1 with the Alg. 2 row kernel) on the level-ordered
// SELL-32 matrix of a plan, unblocked (one launch per power) and level-blocked (one persistent
// launch running the level-group wavefront with per-chunk dependency flags).
//
// Both paths call the same row function, so their results are bit-identical (the paper's
// observation that cache blocking leaves the numerics unchanged, Sec. 1 and Sec. 4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mpk_internal.cuh"

namespace {

struct Coefs {
    double a[MPK_MAX_P + 1], b[MPK_MAX_P + 1], c[MPK_MAX_P + 1], g[MPK_MAX_P + 2];
};

// Vector set of one launch.  Power k (absolute) lives at vec(k); element (row r, rhs q) at
// vec(k)[r * ld_row + q] with ld_row = n_rhs.
struct VecSet {
    const void *x;        // y_0
    void *ybase;          // all-powers mode: y_k = ybase + k * bstride (k >= 1)
    void *ring[3];        // final-only mode: y_k in ring[k % 3]
    void *final_out;      // final-only mode: y_p (or sum gamma_k y_k)
    int64_t bstride;      // elements between power blocks (all-powers mode)
    int final_only;
    int use_gamma;
    int p_total;          // last absolute power of the whole call
};

template <typename T> __device__ __forceinline__ const T *vec_ro(const VecSet &v, int k) {
    if (k == 0) return reinterpret_cast<const T *>(v.x);
    if (v.final_only) return reinterpret_cast<const T *>(v.ring[k % 3]);
    return reinterpret_cast<const T *>(v.ybase) + (int64_t)k * v.bstride;
}
template <typename T> __device__ __forceinline__ T *vec_rw(const VecSet &v, int k) {
    if (v.final_only) {
        if (k == v.p_total && !v.use_gamma) return reinterpret_cast<T *>(v.final_out);
        return reinterpret_cast<T *>(v.ring[k % 3]);
    }
    return reinterpret_cast<T *>(v.ybase) + (int64_t)k * v.bstride;
}

struct SellView {
    const long long *slice_ptr;
    const int32_t *slice_row;
    const int32_t *slice_len;
    const int32_t *col;
    const void *val;
};

// ------------------------------------------------------------------------------------------
// The row function: power k of rows [slice_row[s], slice_row[s+1]) for rhs block [q0, q0+NR).
// Thread `lane` owns row slice_row[s] + lane.  The row sum runs over the stored entries in
// ascending column order with one fused multiply-add per entry; then
//     y_k = a_k * sum + b_k * y_{k-1} + c_k * y_{k-2}   (terms with a zero coefficient skipped)
// ------------------------------------------------------------------------------------------
template <typename T, int NR> struct VecLoad;
template <> struct VecLoad<float, 1> { static __device__ __forceinline__ void ld(const float *p, float *o) { o[0] = p[0]; } };
template <> struct VecLoad<float, 2> { static __device__ __forceinline__ void ld(const float *p, float *o) { float2 v = *reinterpret_cast<const float2 *>(p); o[0] = v.x; o[1] = v.y; } };
template <int NR> struct VecLoadF4 {
    static __device__ __forceinline__ void ld(const float *p, float *o) {
#pragma unroll
        for (int i = 0; i < NR / 4; i++) {
            float4 v = reinterpret_cast<const float4 *>(p)[i];
            o[4 * i] = v.x; o[4 * i + 1] = v.y; o[4 * i + 2] = v.z; o[4 * i + 3] = v.w;
        }
    }
};
template <> struct VecLoad<float, 4> : VecLoadF4<4> {};
template <> struct VecLoad<float, 8> : VecLoadF4<8> {};
template <> struct VecLoad<float, 16> : VecLoadF4<16> {};
template <> struct VecLoad<float, 32> : VecLoadF4<32> {};
template <> struct VecLoad<double, 1> { static __device__ __forceinline__ void ld(const double *p, double *o) { o[0] = p[0]; } };
template <int NR> struct VecLoadD2 {
    static __device__ __forceinline__ void ld(const double *p, double *o) {
#pragma unroll
        for (int i = 0; i < NR / 2; i++) {
            double2 v = reinterpret_cast<const double2 *>(p)[i];
            o[2 * i] = v.x; o[2 * i + 1] = v.y;
        }
    }
};
template <> struct VecLoad<double, 2> : VecLoadD2<2> {};
template <> struct VecLoad<double, 4> : VecLoadD2<4> {};
template <> struct VecLoad<double, 8> : VecLoadD2<8> {};
template <> struct VecLoad<double, 16> : VecLoadD2<16> {};

template <typename T, int NR>
__device__ __forceinline__ void row_power(const SellView &A, int64_t s, int lane, int n_rhs,
                                          const VecSet &V, int k, const Coefs &cf) {
    const int32_t r0 = __ldg(A.slice_row + s), r1 = __ldg(A.slice_row + s + 1);
    const int32_t row = r0 + lane;
    if (row >= r1) return;
    const int32_t L = __ldg(A.slice_len + s);
    const long long base = 32ll * __ldg(A.slice_ptr + s) + lane;
    const T *__restrict__ val = reinterpret_cast<const T *>(A.val);
    const T *y1 = vec_ro<T>(V, k - 1);
    const T *y2 = k >= 2 ? vec_ro<T>(V, k - 2) : nullptr;
    T *yk = vec_rw<T>(V, k);
    const T a = (T)cf.a[k], b = (T)cf.b[k], c = (T)cf.c[k];
    for (int q0 = 0; q0 < n_rhs; q0 += NR) {
        T acc[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) acc[q] = (T)0;
#pragma unroll 4
        for (int32_t j = 0; j < L; j++) {
            const long long d = base + 32ll * j;
            const int32_t cidx = __ldg(A.col + d);
            const T v = __ldg(val + d);
            if (cidx >= 0) {
                T xv[NR];
                VecLoad<T, NR>::ld(y1 + (int64_t)cidx * n_rhs + q0, xv);
#pragma unroll
                for (int q = 0; q < NR; q++) acc[q] = fma(v, xv[q], acc[q]);
            }
        }
        const int64_t o = (int64_t)row * n_rhs + q0;
        T res[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) res[q] = a * acc[q];
        if (b != (T)0) {
            T yv[NR];
            VecLoad<T, NR>::ld(y1 + o, yv);
#pragma unroll
            for (int q = 0; q < NR; q++) res[q] = fma(b, yv[q], res[q]);
        }
        if (c != (T)0 && y2) {
            T yv[NR];
            VecLoad<T, NR>::ld(y2 + o, yv);
#pragma unroll
            for (int q = 0; q < NR; q++) res[q] = fma(c, yv[q], res[q]);
        }
#pragma unroll
        for (int q = 0; q < NR; q++) yk[o + q] = res[q];
        if (V.use_gamma) {
            // running polynomial sum_k gamma_k y_k (eq. (3)); tasks of one chunk run in order
            T *acc_out = reinterpret_cast<T *>(V.final_out);
            const T gk = (T)cf.g[k];
            if (k == 1) {
                const T *x = reinterpret_cast<const T *>(V.x);
                const T g0 = (T)cf.g[0];
#pragma unroll
                for (int q = 0; q < NR; q++) acc_out[o + q] = fma(gk, res[q], g0 * x[o + q]);
            } else {
#pragma unroll
                for (int q = 0; q < NR; q++) acc_out[o + q] = fma(gk, res[q], acc_out[o + q]);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Unblocked: one launch per power (Alg. 1), warp per slice.
// ------------------------------------------------------------------------------------------
template <typename T, int NR>
__global__ void __launch_bounds__(256) mpk_power_kernel(SellView A, int64_t n_slices, int n_rhs,
                                                        VecSet V, int k, Coefs cf) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = w0; s < n_slices; s += nw) row_power<T, NR>(A, s, lane, n_rhs, V, k, cf);
}

// ------------------------------------------------------------------------------------------
// Blocked: persistent CTAs take tasks (chunk c, power k) from a ticket counter in the order of
// the level-group wavefront.  Before computing, a task waits until every chunk in its
// dependency range has published power k-1; after computing it publishes power k.
// Flags are monotone per launch: value epoch*64 + k.  Every wait is bounded in time.
// ------------------------------------------------------------------------------------------
struct BlockedArgs {
    const int32_t *chunk_slice;
    const int32_t *dep_lo, *dep_hi;
    const uint32_t *tasks;
    int64_t n_tasks;
    uint32_t *flags;
    MpkCtrl *ctrl;
    int k0;                 // absolute power before this segment
    uint64_t timeout_ns;
    uint32_t debug_drop;    // 1: task (chunk 0, power 1) does not publish
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

template <typename T, int NR>
__global__ void __launch_bounds__(256) mpk_blocked_kernel(SellView A, int n_rhs, VecSet V,
                                                          Coefs cf, BlockedArgs B) {
    __shared__ uint32_t s_task, s_next, s_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    if (tid == 0) {
        s_base = *(volatile uint32_t *)&B.ctrl->epoch * 64u;
        s_task = atomicAdd(&B.ctrl->ticket, 1u);
        s_abort = 0;
    }
    __syncthreads();
    const uint32_t base = s_base;
    while (true) {
        const uint32_t t = s_task;
        if (t >= B.n_tasks || s_abort) break;
        const uint32_t code = __ldg(B.tasks + t);
        const int32_t c = (int32_t)(code & 0xffffffu);
        const int k = (int)(code >> 24);
        if (tid == 0) s_next = atomicAdd(&B.ctrl->ticket, 1u);   // overlap with the task
        if (k > 1) {
            const int32_t lo = __ldg(B.dep_lo + c), hi = __ldg(B.dep_hi + c);
            const uint32_t target = base + (uint32_t)(k - 1);
            int fail = 0;
            for (int32_t i = lo + tid; i <= hi; i += blockDim.x) {
                if (ld_acquire_u32(B.flags + i) >= target) continue;
                const uint64_t t0 = globaltimer_ns();
                unsigned backoff = 64;
                while (ld_acquire_u32(B.flags + i) < target) {
                    if (globaltimer_ns() - t0 > B.timeout_ns ||
                        *(volatile uint32_t *)&B.ctrl->error) {
                        fail = 1;
                        break;
                    }
                    __nanosleep(backoff);
                    if (backoff < 2048) backoff <<= 1;
                }
                if (fail) break;
            }
            if (__syncthreads_or(fail)) {
                if (tid == 0) {
                    if (atomicOr(&B.ctrl->error, 1u) == 0u) B.ctrl->err_task = t;
                }
                break;
            }
        }
        const int32_t s0 = __ldg(B.chunk_slice + c), s1 = __ldg(B.chunk_slice + c + 1);
        for (int32_t s = s0 + warp; s < s1; s += nwarp)
            row_power<T, NR>(A, s, lane, n_rhs, V, B.k0 + k, cf);
        __syncthreads();
        if (tid == 0) {
            if (!(B.debug_drop && c == 0 && k == 1)) {
                __threadfence();
                st_release_u32(B.flags + c, base + (uint32_t)k);
            }
            s_task = s_next;
        }
        __syncthreads();
    }
    // the last CTA out re-arms the control block for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&B.ctrl->done_ctas, 1u);
        if (done == gridDim.x - 1) {
            B.ctrl->ticket = 0;
            B.ctrl->done_ctas = 0;
            atomicAdd(&B.ctrl->epoch, 1u);
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Staging: user layout (original or level order, column-major or interleaved) <-> the
// kernel's interleaved level-order layout.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void gather_in_kernel(const T *X, int64_t ldx, int interleaved, const int32_t *perm,
                                 int64_t n, int n_rhs, T *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = perm ? perm[r] : r;
        for (int q = 0; q < n_rhs; q++)
            out[r * n_rhs + q] = interleaved ? X[src * n_rhs + q] : X[src + q * ldx];
    }
}
template <typename T>
__global__ void scatter_out_kernel(const T *in, const int32_t *iperm, int64_t n, int n_rhs,
                                   T *Y, int64_t ldy, int interleaved) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = iperm ? iperm[i] : i;
        for (int q = 0; q < n_rhs; q++) {
            const T v = in[r * n_rhs + q];
            if (interleaved) Y[i * n_rhs + q] = v;
            else Y[i + q * ldy] = v;
        }
    }
}

static unsigned grid_n(int64_t n, int block = 256) {
    int64_t g = ceil_div(std::max<int64_t>(n, 1), block);
    return (unsigned)std::min<int64_t>(g, 152 * 16);
}

template <typename T, int NR>
mpk_status launch_powers(mpk_plan_s *P, const SellView &A, int n_rhs, const VecSet &V,
                         const Coefs &cf, int p, bool blocked, uint32_t flags, cudaStream_t s) {
    if (!blocked) {
        const int64_t warps = P->n_slices;
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(warps, 1), 8), 152 * 64);
        for (int k = 1; k <= p; k++) {
            mpk_power_kernel<T, NR><<<grid, 256, 0, s>>>(A, P->n_slices, n_rhs, V, k, cf);
        }
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }
    // blocked, in segments of at most p_blk powers (the paper's p_opt and remainder, Sec. 3)
    int k0 = 0;
    while (k0 < p) {
        const int seg = std::min(P->p_blk, p - k0);
        Schedule *sch = nullptr;
        MPK_TRY(mpk_get_schedule(P, seg, &sch, s));
        BlockedArgs B;
        B.chunk_slice = P->chunk_slice.as<int32_t>();
        B.dep_lo = P->dep_lo.as<int32_t>();
        B.dep_hi = P->dep_hi.as<int32_t>();
        B.tasks = sch->tasks.as<uint32_t>();
        B.n_tasks = sch->n_tasks;
        B.flags = P->flags.as<uint32_t>();
        B.ctrl = P->ctrl.as<MpkCtrl>();
        B.k0 = k0;
        B.timeout_ns = (uint64_t)P->opts.wait_timeout_us * 1000ull;
        B.debug_drop = (flags & MPK_DEBUG_DROP_FLAG) && k0 == 0 ? 1u : 0u;
        // epochs advance by one per launch; re-arm the flags long before they could wrap
        if (++P->launches_since_reset >= (1ull << 25)) {
            MPK_CUDA(cudaMemsetAsync(P->flags.p, 0, (P->n_chunks + 1) * 4, s));
            uint32_t one = 1;
            MPK_CUDA(cudaMemcpyAsync(P->ctrl.p, &one, 4, cudaMemcpyHostToDevice, s));
            P->launches_since_reset = 1;
        }
        int occ = 0;
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mpk_blocked_kernel<T, NR>, 256, 0));
        const int per_sm = std::max(1, std::min(occ, P->ctas_per_sm));
        const int64_t grid = std::min<int64_t>((int64_t)P->n_sm * per_sm, std::max<int64_t>(sch->n_tasks, 1));
        mpk_blocked_kernel<T, NR><<<(unsigned)grid, 256, 0, s>>>(A, n_rhs, V, cf, B);
        MPK_CUDA(cudaGetLastError());
        k0 += seg;
    }
    return MPK_OK;
}

template <typename T>
mpk_status dispatch_nr(mpk_plan_s *P, const SellView &A, int n_rhs, const VecSet &V,
                       const Coefs &cf, int p, bool blocked, uint32_t flags, cudaStream_t s) {
    const int maxnr = sizeof(T) == 4 ? 32 : 16;
    int nr = 1;
    while (nr * 2 <= maxnr && n_rhs % (nr * 2) == 0) nr *= 2;
    switch (nr) {
    case 1: return launch_powers<T, 1>(P, A, n_rhs, V, cf, p, blocked, flags, s);
    case 2: return launch_powers<T, 2>(P, A, n_rhs, V, cf, p, blocked, flags, s);
    case 4: return launch_powers<T, 4>(P, A, n_rhs, V, cf, p, blocked, flags, s);
    case 8: return launch_powers<T, 8>(P, A, n_rhs, V, cf, p, blocked, flags, s);
    case 16: return launch_powers<T, 16>(P, A, n_rhs, V, cf, p, blocked, flags, s);
    default:
        if constexpr (sizeof(T) == 4) return launch_powers<T, 32>(P, A, n_rhs, V, cf, p, blocked, flags, s);
        return MPK_ERR_ARG;
    }
}

}  // namespace

// ============================================================================================
// Schedule: the level-group wavefront.  Step t runs powers k = 1..p on groups g = t-(k-1),
// ascending in k; inside (g, k) the chunks ascend.  A chunk's rows lie in one group, so its
// dependencies lie in groups g-1..g+1, all of which the order places earlier.
// ============================================================================================
mpk_status mpk_get_schedule(mpk_plan_s *P, int p, Schedule **out, cudaStream_t s) {
    auto it = P->schedules.find(p);
    if (it != P->schedules.end()) {
        *out = it->second.get();
        return MPK_OK;
    }
    std::vector<uint32_t> h;
    h.reserve((size_t)p * P->n_chunks);
    const int G = P->n_groups;
    for (int t = 0; t <= G + p - 2; t++)
        for (int k = 1; k <= p; k++) {
            const int g = t - (k - 1);
            if (g < 0 || g >= G) continue;
            for (int32_t c = P->h_group_chunk[g]; c < P->h_group_chunk[g + 1]; c++)
                h.push_back((uint32_t)c | ((uint32_t)k << 24));
        }
    std::unique_ptr<Schedule> sch(new Schedule());
    sch->p = p;
    sch->n_tasks = (int64_t)h.size();
    MPK_TRY(sch->tasks.alloc(std::max<size_t>(h.size(), 1) * 4));
    if (!h.empty())
        MPK_CUDA(cudaMemcpyAsync(sch->tasks.p, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
    // the host vector must outlive the copy
    MPK_CUDA(cudaStreamSynchronize(s));
    *out = sch.get();
    P->schedules[p] = std::move(sch);
    return MPK_OK;
}

mpk_status mpk_apply_internal(mpk_plan_s *P, const mpk_coeffs *co, mpk_dtype dtype,
                              const void *X, int64_t ldx, void *Y, int64_t ldy, int32_t n_rhs,
                              uint32_t flags, cudaStream_t s) {
    if (!P || !co || !Y) return MPK_ERR_ARG;
    const int p = co->p;
    if (p < 1 || p > MPK_MAX_P || !co->a || !co->b || !co->c) return MPK_ERR_ARG;
    if (n_rhs < 1 || n_rhs > 1024) return MPK_ERR_ARG;
    if (dtype == MPK_F64 && !P->has64) return MPK_ERR_ARG;
    if (dtype == MPK_F32 && !P->has32) return MPK_ERR_ARG;
    const bool interleaved = (flags & MPK_RHS_INTERLEAVED) != 0;
    const bool permuted = (flags & MPK_PERMUTED_IO) != 0;
    const bool final_only = (flags & MPK_FINAL_ONLY) != 0;
    const bool host_io = (flags & MPK_HOST_IO) != 0;
    const bool y0x = (flags & MPK_Y0_IS_X) != 0;
    const bool blocked = (flags & MPK_UNBLOCKED) == 0;
    if (y0x && (!permuted || final_only || host_io)) return MPK_ERR_ARG;
    if (!y0x && !X) return MPK_ERR_ARG;
    const int64_t n = P->n;
    if (!interleaved && (ldx < n && !y0x)) return MPK_ERR_ARG;
    if (ldy < n) return MPK_ERR_ARG;
    if (n == 0) return MPK_OK;
    const size_t es = dtype == MPK_F64 ? 8 : 4;
    const int64_t blk = n * n_rhs;                    // elements of one interleaved block
    const int64_t ublk = ldy * n_rhs;                 // elements between user output blocks
    const int64_t nout_blocks = final_only ? 1 : (p + 1);

    Coefs cf;
    memset(&cf, 0, sizeof(cf));
    for (int k = 1; k <= p; k++) {
        cf.a[k] = co->a[k - 1];
        cf.b[k] = co->b[k - 1];
        cf.c[k] = co->c[k - 1];
    }
    const bool use_gamma = final_only && co->gamma;
    if (use_gamma)
        for (int k = 0; k <= p; k++) cf.g[k] = co->gamma[k];

    // host I/O: stage X in and Y out through device buffers
    const void *Xd = X;
    void *Yd = Y;
    if (host_io) {
        const int64_t xin = interleaved ? blk : ldx * n_rhs;
        const int64_t yout = nout_blocks * ublk;
        MPK_TRY(P->ws_host.ensure((size_t)(xin + yout) * es));
        char *base = P->ws_host.as<char>();
        MPK_CUDA(cudaMemcpyAsync(base, X, (size_t)xin * es, cudaMemcpyHostToDevice, s));
        Xd = base;
        Yd = base + (size_t)xin * es;
    }

    // The kernels work on interleaved level-order blocks.  Direct mode: the user's buffers
    // already are (level order with one rhs or interleaved), so no staging is needed.
    // Vector loads of several right-hand sides need 16-byte aligned blocks; other callers'
    // buffers go through the staging path.
    const bool aligned16 = ((uintptr_t)Yd % 16 == 0) && (y0x || (uintptr_t)Xd % 16 == 0) &&
                           ((size_t)ublk * es) % 16 == 0;
    const bool direct = permuted && !host_io && (n_rhs == 1 || (interleaved && aligned16));
    const int32_t *perm = permuted ? nullptr : P->perm.as<int32_t>();
    const int32_t *iperm = permuted ? nullptr : P->iperm.as<int32_t>();

    VecSet V;
    memset(&V, 0, sizeof(V));
    V.final_only = final_only ? 1 : 0;
    V.use_gamma = use_gamma ? 1 : 0;
    V.p_total = p;
    const unsigned g = grid_n(n);

    if (direct) {
        if (final_only) {
            MPK_TRY(P->ws_y.ensure((size_t)3 * blk * es));
            V.x = Xd;
            for (int i = 0; i < 3; i++) V.ring[i] = P->ws_y.as<char>() + (size_t)i * blk * es;
            V.final_out = Yd;
        } else {
            if (!y0x) {
                // y_0 = x into block 0 of Y
                if (n_rhs == 1 || interleaved)
                    MPK_CUDA(cudaMemcpyAsync(Yd, Xd, (size_t)blk * es, cudaMemcpyDeviceToDevice, s));
            }
            V.x = Yd;
            V.ybase = Yd;
            V.bstride = ublk;
        }
    } else {
        // stage: ws_x = x (level order, interleaved); outputs in ws_y
        MPK_TRY(P->ws_x.ensure((size_t)blk * es));
        const int64_t nb = final_only ? 4 : (p + 1);
        MPK_TRY(P->ws_y.ensure((size_t)nb * blk * es));
        if (dtype == MPK_F64)
            gather_in_kernel<double><<<g, 256, 0, s>>>((const double *)Xd, ldx, interleaved, perm, n, n_rhs, P->ws_x.as<double>());
        else
            gather_in_kernel<float><<<g, 256, 0, s>>>((const float *)Xd, ldx, interleaved, perm, n, n_rhs, P->ws_x.as<float>());
        MPK_CUDA(cudaGetLastError());
        if (final_only) {
            V.x = P->ws_x.p;
            for (int i = 0; i < 3; i++) V.ring[i] = P->ws_y.as<char>() + (size_t)i * blk * es;
            V.final_out = P->ws_y.as<char>() + (size_t)3 * blk * es;
        } else {
            MPK_CUDA(cudaMemcpyAsync(P->ws_y.p, P->ws_x.p, (size_t)blk * es, cudaMemcpyDeviceToDevice, s));
            V.x = P->ws_y.p;
            V.ybase = P->ws_y.p;
            V.bstride = blk;
        }
    }

    SellView A;
    A.slice_ptr = P->slice_ptr.as<long long>();
    A.slice_row = P->slice_row.as<int32_t>();
    A.slice_len = P->slice_len.as<int32_t>();
    A.col = P->s_col.as<int32_t>();
    A.val = dtype == MPK_F64 ? P->s_val64.p : P->s_val32.p;

    if (dtype == MPK_F64) MPK_TRY(dispatch_nr<double>(P, A, n_rhs, V, cf, p, blocked, flags, s));
    else MPK_TRY(dispatch_nr<float>(P, A, n_rhs, V, cf, p, blocked, flags, s));

    if (!direct) {
        // un-stage every output block into the user's layout / order
        for (int64_t b = 0; b < nout_blocks; b++) {
            const char *src = final_only ? (const char *)V.final_out : P->ws_y.as<char>() + (size_t)b * blk * es;
            char *dst = (char *)Yd + (size_t)b * ublk * es;
            if (dtype == MPK_F64)
                scatter_out_kernel<double><<<g, 256, 0, s>>>((const double *)src, iperm, n, n_rhs, (double *)dst, ldy, interleaved);
            else
                scatter_out_kernel<float><<<g, 256, 0, s>>>((const float *)src, iperm, n, n_rhs, (float *)dst, ldy, interleaved);
        }
        MPK_CUDA(cudaGetLastError());
    }
    if (host_io) {
        MPK_CUDA(cudaMemcpyAsync(Y, Yd, (size_t)nout_blocks * ublk * es, cudaMemcpyDeviceToHost, s));
        MPK_CUDA(cudaStreamSynchronize(s));
    }
    return MPK_OK;
}

extern "C" mpk_status mpk_apply(mpk_plan_t plan, const mpk_coeffs *co, mpk_dtype dtype,
                                const void *X, int64_t ldx, void *Y, int64_t ldy, int32_t n_rhs,
                                uint32_t flags, cudaStream_t stream) {
    return mpk_apply_internal(plan, co, dtype, X, ldx, Y, ldy, n_rhs, flags, stream);
}

extern "C" mpk_status mpk_plan_sync(mpk_plan_t P, cudaStream_t s) {
    if (!P) return MPK_ERR_ARG;
    MPK_CUDA(cudaStreamSynchronize(s));
    MpkCtrl h;
    MPK_CUDA(cudaMemcpy(&h, P->ctrl.p, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.error) {
        // clear the latched error; the flags of the aborted launch sit below every later
        // launch's targets because each launch uses a new epoch
        uint32_t zero[2] = {0, 0};
        MPK_CUDA(cudaMemcpy(&P->ctrl.as<MpkCtrl>()->error, zero, 8, cudaMemcpyHostToDevice));
        return MPK_ERR_TIMEOUT;
    }
    return MPK_OK;
}

// ============================================================================================
// Host helpers
// ============================================================================================
extern "C" mpk_status mpk_coeffs_chebyshev(double alpha, double beta, int32_t p, double *a,
                                           double *b, double *c) {
    if (p < 1 || !a || !b || !c || !(beta > alpha)) return MPK_ERR_ARG;
    const double c0 = 0.5 * (alpha + beta), d = 0.5 * (beta - alpha);
    for (int k = 1; k <= p; k++) {
        // T_1(z) = z ; T_k(z) = 2 z T_{k-1}(z) - T_{k-2}(z), z = (A - c0 I)/d
        a[k - 1] = (k == 1 ? 1.0 : 2.0) / d;
        b[k - 1] = -(k == 1 ? 1.0 : 2.0) * c0 / d;
        c[k - 1] = k == 1 ? 0.0 : -1.0;
    }
    return MPK_OK;
}

extern "C" mpk_status mpk_coeffs_newton(const double *theta, int32_t p, double *a, double *b,
                                        double *c) {
    if (p < 1 || !theta || !a || !b || !c) return MPK_ERR_ARG;
    for (int k = 0; k < p; k++) {
        a[k] = 1.0;
        b[k] = -theta[k];
        c[k] = 0.0;
    }
    return MPK_OK;
}

extern "C" mpk_status mpk_leja_order(const double *values, int32_t n, int32_t count, double *out) {
    if (!values || !out || n < 1 || count < 1) return MPK_ERR_ARG;
    std::vector<double> v(values, values + n);
    std::sort(v.begin(), v.end());
    std::vector<char> used(n, 0);
    std::vector<double> score(n, 0.0);
    std::vector<double> chosen;
    // first: largest modulus, ties to the smaller value (v is ascending)
    int first = 0;
    for (int i = 1; i < n; i++)
        if (std::fabs(v[i]) > std::fabs(v[first])) first = i;
    chosen.push_back(v[first]);
    used[first] = 1;
    int last = first;
    while ((int)chosen.size() < std::min(count, n)) {
        int best = -1;
        double bests = -INFINITY;
        for (int i = 0; i < n; i++) {
            score[i] += std::log(std::fabs(v[i] - v[last]));
            if (used[i]) continue;
            if (score[i] > bests) { bests = score[i]; best = i; }
        }
        if (best < 0 || bests == -INFINITY) break;
        used[best] = 1;
        chosen.push_back(v[best]);
        last = best;
    }
    const int m = (int)chosen.size();
    for (int i = 0; i < count; i++) out[i] = chosen[i % m];
    return MPK_OK;
}

extern "C" const char *mpk_status_str(mpk_status s) {
    switch (s) {
    case MPK_OK: return "MPK_OK";
    case MPK_ERR_ARG: return "MPK_ERR_ARG";
    case MPK_ERR_CUDA: return "MPK_ERR_CUDA";
    case MPK_ERR_OOM: return "MPK_ERR_OOM";
    case MPK_ERR_TIMEOUT: return "MPK_ERR_TIMEOUT";
    case MPK_ERR_BREAKDOWN: return "MPK_ERR_BREAKDOWN";
    case MPK_ERR_NOT_CONVERGED: return "MPK_ERR_NOT_CONVERGED";
    case MPK_ERR_UNIMPLEMENTED: return "MPK_ERR_UNIMPLEMENTED";
    case MPK_ERR_BUDGET: return "MPK_ERR_BUDGET";
    case MPK_ERR_NOT_READY: return "MPK_ERR_NOT_READY";
    }
    return "MPK_ERR_UNKNOWN";
}

extern "C" const char *mpk_version(void) { return "mpk_gb300 1 sm_103a"; }
