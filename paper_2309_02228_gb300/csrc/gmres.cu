// s-step GMRES (Sec. 4, Alg. 3(a)+(c)) on the device, with FP64 iterative refinement.
//
// One restart cycle, block j (s columns):
//   MPK (Newton basis, Sec. 4):   V[:, j+1..j+s] from V[:, j] through the level-blocked kernel
//   BOrtho (block CGS):            C = Q^T W,  W <- W - Q C
//   TSQR (CholQR2):                R1 = chol(W^T W - C^T C), W <- W R1^-1, R2 = chol(W^T W),
//                                  W <- W R2^-1  (or a second BCGS sweep instead of CholQR2's
//                                  plain second pass)
//   Hessenberg columns from H R_s = R_full B (change of basis B: shifts on the diagonal, ones
//   below), Givens rotations, residual estimate per column, convergence check.
// Refinement: r = b - A x in FP64 with the FP64 matrix; each outer step runs one cycle on
// A d = r in the basis precision and adds d to x.  With an FP64 basis this is plain restarted
// s-step GMRES whose restart residual is the true one.
//
// Precision: the tall-skinny products accumulate FP32 (or FP64) products per thread in the
// basis precision and combine per-thread partial sums in FP64 in a fixed order (FP64 FMAs run
// at 1/64 of the FP32 rate on this part, so per-product FP64 accumulation would dominate);
// all small dense work (Gram reductions, Cholesky, Hessenberg, Givens, least squares, Ritz
// values) is FP64 on one CTA.  Every reduction has a fixed order: results do not depend on
// scheduling.
#include <cuda.h>
#include <map>
#include <mutex>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "mpk_internal.cuh"

namespace {

constexpr int SMAX = 16;       // largest block size s
constexpr int MMAX = 128;      // largest restart length m
constexpr int RED_BLOCK = 256;

unsigned grid_rows(int64_t n, int per_sm = 4) {
    int64_t g = ceil_div(std::max<int64_t>(n, 1), RED_BLOCK);
    return (unsigned)std::min<int64_t>(g, 152 * per_sm);
}

// ------------------------------------------------------------------------------------------
// Vector kernels (level order <-> original order, conversions, scalings)
// ------------------------------------------------------------------------------------------
__global__ void gather_f64_kernel(const double *src, const int32_t *perm, int64_t n, double *dst) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        dst[r] = src[perm[r]];
}
__global__ void scatter_f64_kernel(const double *src, const int32_t *perm, int64_t n, double *dst) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        dst[perm[r]] = src[r];
}
// v = r / nrm (nrm read on the device), converted to the basis type
template <typename T>
__global__ void normalize_kernel(const double *r, const double *nrm, int64_t n, T *v) {
    const double inv = 1.0 / *nrm;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (T)(r[i] * inv);
}

// ------------------------------------------------------------------------------------------
// Deterministic FP64 reductions: per-CTA partials in a fixed tree, then one CTA sums the
// partials in order.
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(RED_BLOCK) sumsq_partial_kernel(const T *v, int64_t n, double *part) {
    __shared__ double sh[RED_BLOCK];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)v[i];
        s = fma(x, x, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// out[e] = sum over b of part[b * stride + e], e < m; optional sqrt
// out[e] = sum_b part[b * stride + e], e < m: one warp per output, lane l adds partials l,
// l + 32, ... in order, then a fixed shuffle tree (the result does not depend on the grid)
static constexpr int REDP_WARPS = 8;
__global__ void __launch_bounds__(32 * REDP_WARPS) reduce_partials_kernel(const double *part, int nb, int m,
                                                                         int64_t stride, double *out, int take_sqrt) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * REDP_WARPS + (threadIdx.x >> 5);
    if (e >= m) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(int64_t)b * stride + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = take_sqrt ? sqrt(s) : s;
}
static inline unsigned redp_grid(int m) { return (unsigned)((m + REDP_WARPS - 1) / REDP_WARPS); }

// ------------------------------------------------------------------------------------------
// Tall-skinny Gram G = X^T Y (X: n x K, Y: n x S, column-major), G col-major K x S.
// A warp owns a tile of CT columns of X and streams 32 rows per step straight from global
// memory (lane l takes row r0 + l: every column load is one coalesced 128-byte line); each lane
// keeps the CT x S products of its rows in registers (64 FMAs per CT + S loads).  With fewer
// tiles than warps, the warps of a tile split the steps.
// Precision (FP32 basis): a lane sums its products in FP32 over one visit of the CTA to a
// range of GRAM_RANGE rows, i.e. at most GRAM_RANGE / 32 = 32 terms; the 32 lanes' block sums
// are then added by a fixed five-level FP32 tree (lane_halve) and the result is added to FP64
// totals in shared memory; the totals of the warps of a tile and of the CTAs are summed in
// FP64 in a fixed order (reduce_partials_kernel).  So |G^ - G| <= (37 u32 + m u64) |X|^T |Y|
// entrywise (u32 = 2^-24, m the number of FP64 additions), about 2.2e-6 relative to |X|^T|Y|.
// ------------------------------------------------------------------------------------------
constexpr int GRAM_RANGE = 1024;       // rows a CTA takes per visit

// Sum over the 32 lanes of each of the N values of every lane, by recursive halving: at the
// level of offset o a lane keeps one half of its values (the upper half when lane & o), adds
// its partner's copy of that half, and sends the other half.  After the five levels lane l
// holds N / 32 values, the sums of entries base .. base + N/32 - 1 over all lanes, each a fixed
// five-level tree.  62 shuffles for N = 64 instead of 320 for one butterfly per value.
template <typename T, int N>
__device__ __forceinline__ int lane_halve(T (&v)[N], int lane) {
    static_assert(N >= 32 && (N & (N - 1)) == 0, "power of two, at least one value per lane");
    int base = 0;
#pragma unroll
    for (int o = 16, c = N; o >= 1; o >>= 1, c >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < c / 2; i++) {
            const T keep = up ? v[i + c / 2] : v[i];
            const T send = up ? v[i] : v[i + c / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) base += c / 2;
    }
    return base;
}

template <typename T, int SB>
__global__ void __launch_bounds__(256, 2) gram_kernel(const T *X, int64_t ldx, int K, const T *Y,
                                                      int64_t ldy, int S, int64_t n, double *part) {
    constexpr int ACC = sizeof(T) == 4 ? 64 : 32;   // accumulators per lane
    constexpr int CT = ACC / SB;                     // X columns per tile
    // FP64 totals per warp group: slot[rpart][a][b] (a < K, b < S); rsplit * K * S <= 8 * ACC fits
    __shared__ double slot[(MMAX + 1 + SMAX) * SMAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = (K + CT - 1) / CT;
    const bool many = ntiles >= 8;
    const int rsplit = many ? 1 : 8 / ntiles;        // warps per tile
    const int active = many ? 8 : ntiles * rsplit;
    const int rpart = many ? 0 : warp / ntiles;
    for (int e = tid; e < (MMAX + 1 + SMAX) * SMAX; e += 256) slot[e] = 0.0;
    __syncthreads();
    if (warp < active) {
        for (int tile = many ? warp : warp % ntiles; tile < ntiles; tile += many ? 8 : ntiles) {
            const int c0 = tile * CT;
            for (int64_t base = (int64_t)blockIdx.x * GRAM_RANGE; base < n; base += (int64_t)gridDim.x * GRAM_RANGE) {
                T acc[ACC];   // acc[a * SB + b]
#pragma unroll
                for (int e = 0; e < ACC; e++) acc[e] = (T)0;
                // the values of one step (32 rows of the tile's columns); the next step's are
                // loaded before this step's FMAs, so two steps' loads are in flight per lane
                auto load = [&](int st, T (&xv)[CT], T (&yv)[SB]) {
                    const int64_t r = base + st * 32 + lane;
                    const bool in = st < GRAM_RANGE / 32 && r < n;
#pragma unroll
                    for (int a = 0; a < CT; a++) xv[a] = (in && c0 + a < K) ? X[(int64_t)(c0 + a) * ldx + r] : (T)0;
#pragma unroll
                    for (int b = 0; b < SB; b++) yv[b] = (in && b < S) ? Y[(int64_t)b * ldy + r] : (T)0;
                };
                T xv[CT], yv[SB];
                load(rpart, xv, yv);
                for (int st = rpart; st < GRAM_RANGE / 32; st += rsplit) {
                    if (base + st * 32 >= n) break;
                    T xn[CT], yn[SB];
                    load(st + rsplit, xn, yn);
#pragma unroll
                    for (int a = 0; a < CT; a++)
#pragma unroll
                        for (int b = 0; b < SB; b++) acc[a * SB + b] = fma(xv[a], yv[b], acc[a * SB + b]);
#pragma unroll
                    for (int a = 0; a < CT; a++) xv[a] = xn[a];
#pragma unroll
                    for (int b = 0; b < SB; b++) yv[b] = yn[b];
                }
                // this visit's block sums over the lanes, then into the FP64 totals (each entry
                // has one owner lane, so no two lanes add to the same slot)
                const int e0 = lane_halve<T, ACC>(acc, lane);
#pragma unroll
                for (int j = 0; j < ACC / 32; j++) {
                    const int a = (e0 + j) / SB, b = (e0 + j) % SB;
                    if (c0 + a < K && b < S) slot[((int64_t)rpart * K + c0 + a) * S + b] += (double)acc[j];
                }
            }
        }
    }
    __syncthreads();
    const int KS = K * S;
    for (int e = tid; e < KS; e += 256) {
        const int a = e % K, b = e / K;
        double t = 0.0;
        for (int ph = 0; ph < rsplit; ph++) t += slot[((int64_t)ph * K + a) * S + b];
        part[(int64_t)blockIdx.x * KS + e] = t;   // G column-major [b * K + a]
    }
}


// ------------------------------------------------------------------------------------------
// W <- (W - Q C) Rinv, row by row, and (optionally) the Gram of the new W for the next step.
// Q: n x K1, W: n x S (in place), C: K1 x S, Rinv: S x S (FP64, converted to T).
// ------------------------------------------------------------------------------------------
template <typename T, int SB>
__global__ void __launch_bounds__(256) update_kernel(const T *Q, int64_t ldq, int K1, T *W, int64_t ldw,
                                                     int S, const double *C, const double *Rinv, int64_t n,
                                                     double *gpart) {
    // fused Gram of the new block only up to s = 8 (register budget); larger blocks take a
    // separate Gram pass.  Precision of the fused Gram (FP32 basis): a lane sums its rows'
    // products in FP32 over at most 32 rows, the lanes' block sums are added by a five-level
    // FP32 butterfly, and the result goes into FP64 totals per warp (shared memory), summed over
    // the warps and CTAs in FP64 in a fixed order: the bound of gram_kernel, (37 u32 + m u64)
    // times |W|^T |W| entrywise.
    constexpr bool FUSE = SB <= 8;
    constexpr int NG = FUSE ? SB * (SB + 1) / 2 : 1;
    __shared__ T cs[MMAX + 1][SB];
    __shared__ T ri[SB][SB];
    __shared__ double red[SB * SB];
    __shared__ double wred[8][NG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < K1 * S; e += blockDim.x) cs[e % K1][e / K1] = (T)C[e];
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) ri[e % S][e / S] = (T)Rinv[e];
    for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) red[e] = 0.0;
    for (int e = threadIdx.x; e < 8 * NG; e += blockDim.x) wred[e / NG][e % NG] = 0.0;
    __syncthreads();
    T g2[NG];
#pragma unroll
    for (int e = 0; e < NG; e++) g2[e] = (T)0;
    const bool gram = FUSE && gpart != nullptr;
    // the lanes' FP32 block sums into this warp's FP64 totals (entry e by lane e % 32)
    auto flush = [&]() {
#pragma unroll
        for (int e = 0; e < NG; e++) {
            T v = g2[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == (e & 31) && warp < 8) wred[warp][e] += (double)v;
            g2[e] = (T)0;
        }
    };
    int since = 0;
    // warp-uniform rounds of 32 consecutive rows (the flush needs every lane)
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + warp * 32; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + lane;
        if (i < n) {
            T w[SB];
#pragma unroll
            for (int b = 0; b < SB; b++) w[b] = b < S ? W[(int64_t)b * ldw + i] : (T)0;
            // groups of eight basis columns; the next group's loads are issued before this
            // group's FMAs (ascending order of the FMAs kept)
            T q[8];
#pragma unroll
            for (int u = 0; u < 8; u++) q[u] = u < K1 ? Q[(int64_t)u * ldq + i] : (T)0;
            for (int a0 = 0; a0 < K1; a0 += 8) {
                T qn[8];
#pragma unroll
                for (int u = 0; u < 8; u++) qn[u] = a0 + 8 + u < K1 ? Q[(int64_t)(a0 + 8 + u) * ldq + i] : (T)0;
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (a0 + u < K1) {
#pragma unroll
                        for (int b = 0; b < SB; b++)
                            if (b < S) w[b] = fma(-q[u], cs[a0 + u][b], w[b]);
                    }
#pragma unroll
                for (int u = 0; u < 8; u++) q[u] = qn[u];
            }
            T wn[SB];
#pragma unroll
            for (int b = 0; b < SB; b++) {
                T v = (T)0;
#pragma unroll
                for (int c = 0; c < SB; c++)
                    if (c <= b && b < S) v = fma(w[c], ri[c][b], v);
                wn[b] = v;
            }
#pragma unroll
            for (int b = 0; b < SB; b++)
                if (b < S) W[(int64_t)b * ldw + i] = wn[b];
            if (gram) {
                int e = 0;
#pragma unroll
                for (int b = 0; b < SB; b++)
#pragma unroll
                    for (int c = 0; c <= b; c++) {
                        if (b < S && e < NG) g2[e] = fma(wn[b], wn[c], g2[e]);
                        e++;
                    }
            }
        }
        if (gram && ++since == 32) {
            flush();
            since = 0;
        }
    }
    if (!gram) return;
    flush();
    __syncthreads();
    for (int e = threadIdx.x; e < NG; e += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw && w < 8; w++) t += wred[w][e];
        // packed lower triangle (b >= c) -> red[b * S + c]
        int b = 0, c = e;
        while (c > b) { c -= b + 1; b++; }
        if (b < S) red[b * S + c] = t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        const int b = e / S, c = e % S;
        // symmetric S x S, column-major: G[b + c*S]
        gpart[(int64_t)blockIdx.x * S * S + b + c * S] = b >= c ? red[b * S + c] : red[c * S + b];
    }
}

// ------------------------------------------------------------------------------------------
// Staged streaming for the tall-skinny products: row blocks of R rows (R <= 256) of every
// column are copied into a ring of shared-memory stages by the tensor memory accelerator, one
// 2-D tensor copy (cp.async.bulk.tensor.2d) per box of R rows x 8 columns, completion on the
// stage's mbarrier.  Each SM keeps several blocks of every column in flight whatever the
// register tiling of the arithmetic.  (One 1-D bulk copy per column chunk instead measured
// 0.9-1.9 TB/s, scaling with the copy's size; 2-D boxes of 8 columns stream at about 7 TB/s.)
// The tensor maps cover n rows: rows past n and columns past the block are filled with zeros,
// so they add nothing.  Every wait is bounded; a CTA whose copy does not land within the bound
// sets *err, waits (bounded) for its other copies in flight, and writes NaN partial sums.
// ------------------------------------------------------------------------------------------
constexpr int ST_MAXST = 8;                     // stages per CTA at most
constexpr int ST_BOXC = 8;                      // columns per tensor box
constexpr uint64_t ST_WAIT_NS = 2000000000ull;  // bound of one stage wait (2 s)

__device__ __forceinline__ void st_mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void st_mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool st_mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// box of the tensor map at (row x, column y) into shared memory (x a multiple of R >= 32, so
// x * sizeof(T) is a multiple of 16 bytes)
__device__ __forceinline__ void st_tma2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(map), "r"(x), "r"(y),
                   "r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ uint64_t st_now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true when the phase with this parity has completed; false after the time bound
__device__ __forceinline__ bool st_wait(uint64_t *bar, uint32_t parity) {
    if (st_mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = st_now_ns();
    while (!st_mbar_try_wait(bar, parity)) {
        if (st_now_ns() - t0 > ST_WAIT_NS) return false;
        __nanosleep(64);
    }
    return true;
}

// The staged Gram's X columns in a stage: K rounded up to whole register tiles (CT columns)
// and whole boxes, so every tile column lies inside the stage; columns past K arrive as zeros
// (boxes past the tensor map's last column are filled by the copy engine), so the tiles read
// them without a guard.
template <typename T, int SB> __host__ __device__ constexpr int gram_ct() { return (sizeof(T) == 4 ? 64 : 32) / SB; }
template <typename T, int SB> __host__ __device__ inline int gram_kp(int K) {
    const int m = gram_ct<T, SB>() > ST_BOXC ? gram_ct<T, SB>() : ST_BOXC;
    return (K + m - 1) / m * m;
}

// The ring of one CTA: blocks b = blockIdx.x + i * gridDim.x (i = 0 .. nmine - 1) of R rows;
// block i lands in stage i % nst, which holds the first map's KP columns, then the second's.
struct StageRing {
    unsigned char *base;
    uint64_t *full;
    int KP, NCP, R, nst;   // KP, NCP: padded to whole boxes
    int64_t n, nmine;
    template <typename T> __device__ __forceinline__ T *col(int st, int c) const {
        return reinterpret_cast<T *>(base) + ((int64_t)st * NCP + c) * R;
    }
    __device__ __forceinline__ int64_t row0(int64_t i) const { return ((int64_t)blockIdx.x + i * gridDim.x) * R; }
    // one thread: the copies of this CTA's block i (the second map may be absent: KP == NCP)
    template <typename T> __device__ __forceinline__ void issue(int64_t i, const CUtensorMap *m1, const CUtensorMap *m2) const {
        const int st = (int)(i % nst);
        const int x = (int)row0(i);
        st_mbar_expect_tx(&full[st], (uint32_t)((int64_t)NCP * R * sizeof(T)));
        for (int c = 0; c < KP; c += ST_BOXC) st_tma2d(col<T>(st, c), m1, x, c, &full[st]);
        for (int c = KP; c < NCP; c += ST_BOXC) st_tma2d(col<T>(st, c), m2, x, c - KP, &full[st]);
    }
    // after a timeout: wait (bounded) for the copies still in flight, blocks i0 .. i1 - 1
    __device__ __forceinline__ void drain(int64_t i0, int64_t i1) const {
        for (int64_t i = i0; i < i1 && i < nmine; i++) st_wait(&full[i % nst], (uint32_t)((i / nst) & 1));
    }
};

// Wait for the phase with this parity, bounded, and give up early when another warp of the
// CTA has latched an error in *bad.
__device__ __forceinline__ bool st_wait_or_bad(uint64_t *bar, uint32_t parity, const volatile int *bad) {
    if (st_mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = st_now_ns();
    while (!st_mbar_try_wait(bar, parity)) {
        if (*bad || st_now_ns() - t0 > ST_WAIT_NS) return false;
        __nanosleep(64);
    }
    return true;
}
__device__ __forceinline__ void st_mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}

// G = X^T Y with staged rows (gram_kernel's register tiles and precision).  Warp 7 produces:
// it refills a stage once the stage's "empty" mbarrier shows that every consumer warp has left
// it.  Warps 0..6 consume, each owning one tile of columns (or several, when there are more
// tiles than warps), waiting only for their next stage's data - no CTA-wide barrier per stage.
// A lane sums at most 32 of its rows in FP32 before folding them by lane_halve into FP64 totals
// in shared memory (a warp with several tiles folds at the end of every tile visit); CTAs'
// totals are summed by reduce_partials_kernel.  Bound as gram_kernel's: (40 u32 + m u64)
// |X|^T |Y| entrywise.
constexpr int GS_CONSUMERS = 7;
template <typename T, int SB>
__global__ void __launch_bounds__(256, 2) gram_stage_kernel(const __grid_constant__ CUtensorMap mx,
                                                            const __grid_constant__ CUtensorMap my, int K,
                                                            int S, int64_t n, int R, int nst, double *part,
                                                            uint32_t *err) {
    constexpr int ACC = sizeof(T) == 4 ? 64 : 32;
    constexpr int CT = ACC / SB;
    extern __shared__ __align__(128) unsigned char gs_dyn[];
    __shared__ double slot[(MMAX + 1 + SMAX) * SMAX];
    __shared__ uint64_t full[ST_MAXST], empty[ST_MAXST];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = (K + CT - 1) / CT;
    const bool many = ntiles >= GS_CONSUMERS;
    const int rsplit = many ? 1 : GS_CONSUMERS / ntiles;
    const int active = many ? GS_CONSUMERS : ntiles * rsplit;
    const int rpart = many ? 0 : warp / ntiles;
    StageRing ring;
    ring.base = gs_dyn;
    ring.full = full;
    ring.KP = gram_kp<T, SB>(K);
    ring.NCP = ring.KP + (S + ST_BOXC - 1) / ST_BOXC * ST_BOXC;
    ring.R = R;
    ring.nst = nst;
    ring.n = n;
    const int64_t nblk = (n + R - 1) / R;
    ring.nmine = (int64_t)blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    for (int e = tid; e < (MMAX + 1 + SMAX) * SMAX; e += 256) slot[e] = 0.0;
    if (tid < nst) {
        st_mbar_init(&full[tid], 1);
        st_mbar_init(&empty[tid], (uint32_t)active);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const volatile int *vbad = &s_bad;
    if (warp == GS_CONSUMERS) {
        // producer: block i into stage i % nst once the consumers released block i - nst
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t i = 0; i < ring.nmine; i++) {
                const int st = (int)(i % nst);
                if (i >= nst && !st_wait_or_bad(&empty[st], (uint32_t)(((i / nst) - 1) & 1), vbad)) {
                    s_bad = 1;
                    atomicOr(err, 1u);
                    break;
                }
                ring.issue<T>(i, &mx, &my);
                issued = i + 1;
            }
            if (*vbad) ring.drain(issued > nst ? issued - nst : 0, issued);   // copies still in flight
        }
    } else if (warp < active) {
        using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        T acc[ACC];
#pragma unroll
        for (int e = 0; e < ACC; e++) acc[e] = (T)0;
        int cnt = 0;                              // rows per lane in acc since the last fold
        const int rpl = 2 * ((R + 64 * rsplit - 1) / (64 * rsplit));   // rows per lane per stage
        // the lanes' FP32 sums of tile c0 by lane_halve, into the FP64 totals; acc restarts at 0
        auto flush = [&](int c0) {
            const int e0 = lane_halve<T, ACC>(acc, lane);
#pragma unroll
            for (int jj = 0; jj < ACC / 32; jj++) {
                const int a = (e0 + jj) / SB, b = (e0 + jj) % SB;
                if (c0 + a < K && b < S) slot[((int64_t)rpart * K + c0 + a) * S + b] += (double)acc[jj];
            }
#pragma unroll
            for (int e = 0; e < ACC; e++) acc[e] = (T)0;
        };
        const int KP = ring.KP;
        for (int64_t i = 0; i < ring.nmine; i++) {
            const int st = (int)(i % nst);
            const bool ok = st_wait_or_bad(&full[st], (uint32_t)((i / nst) & 1), vbad);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    s_bad = 1;
                    atomicOr(err, 1u);
                }
                break;
            }
            const int rows = (int)min((int64_t)R, n - ring.row0(i));
            for (int tile = many ? warp : warp % ntiles; tile < ntiles; tile += many ? GS_CONSUMERS : ntiles) {
                const int c0 = tile * CT;
                if (!many && cnt + rpl > 32) {
                    flush(c0);
                    cnt = 0;
                }
                const T *xc = ring.col<T>(st, c0);
                const T *yc = ring.col<T>(st, KP);
                // lane l takes the row pairs (2 l, 2 l + 1) + 64 rsplit k of its part; rows past
                // n are zeros (the copy's fill), so a pair may run past the block's last row
                for (int rr = 2 * (rpart * 32 + lane); rr < rows; rr += 64 * rsplit) {
                    T x0[CT], x1[CT], y0[SB], y1[SB];
                    // no guards: columns past K and past S are zeros in the stage (see gram_kp;
                    // the S boxes are padded to 8 >= SB or to SB = 16)
#pragma unroll
                    for (int a = 0; a < CT; a++) {
                        const V2 v = *reinterpret_cast<const V2 *>(xc + a * R + rr);
                        x0[a] = v.x;
                        x1[a] = v.y;
                    }
#pragma unroll
                    for (int b = 0; b < SB; b++) {
                        const V2 v = *reinterpret_cast<const V2 *>(yc + b * R + rr);
                        y0[b] = v.x;
                        y1[b] = v.y;
                    }
#pragma unroll
                    for (int a = 0; a < CT; a++)
#pragma unroll
                        for (int b = 0; b < SB; b++) {
                            acc[a * SB + b] = fma(x0[a], y0[b], acc[a * SB + b]);
                            acc[a * SB + b] = fma(x1[a], y1[b], acc[a * SB + b]);
                        }
                }
                if (many) flush(c0);
                else cnt += rpl;
            }
            // this warp is done with stage st: one arrival on its empty barrier
            __syncwarp();
            if (lane == 0) st_mbar_arrive(&empty[st]);
        }
        if (!many && cnt > 0) flush((warp % ntiles) * CT);
    }
    __syncthreads();
    const int KS = K * S;
    for (int e = tid; e < KS; e += 256) {
        const int a = e % K, b = e / K;
        double t = 0.0;
        for (int ph = 0; ph < rsplit; ph++) t += slot[((int64_t)ph * K + a) * S + b];
        part[(int64_t)blockIdx.x * KS + e] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : t;
    }
}

// SB values of a 16-byte aligned shared-memory row in 16-byte loads
template <typename T, int SB> __device__ __forceinline__ void vec_row(const T *p, T (&o)[SB]) {
    if constexpr (sizeof(T) == 4 && SB % 4 == 0) {
#pragma unroll
        for (int v = 0; v < SB / 4; v++) {
            const float4 t = reinterpret_cast<const float4 *>(p)[v];
            o[4 * v] = t.x;
            o[4 * v + 1] = t.y;
            o[4 * v + 2] = t.z;
            o[4 * v + 3] = t.w;
        }
    } else if constexpr (sizeof(T) == 8 && SB % 2 == 0) {
#pragma unroll
        for (int v = 0; v < SB / 2; v++) {
            const double2 t = reinterpret_cast<const double2 *>(p)[v];
            o[2 * v] = t.x;
            o[2 * v + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int b = 0; b < SB; b++) o[b] = p[b];
    }
}

// W <- (W - Q C) Rinv with Q and W staged (update_kernel's arithmetic, row by row: the same
// FMAs in the same order), the new W stored straight from registers, and (S <= 8) the Gram of
// the new W: per lane FP32 sums over at most 32 of its rows, a five-level butterfly, FP64 per
// warp, the warps and CTAs in FP64 in a fixed order - update_kernel's bound.  Warp 7 produces
// (refills a stage once every consumer warp has released it); warps 0..6 take the stage's rows
// one per thread, the rows past 224 going to a different warp in each stage.
template <typename T, int SB>
__global__ void __launch_bounds__(256, 2) update_stage_kernel(const __grid_constant__ CUtensorMap mq,
                                                              const __grid_constant__ CUtensorMap mw, int K1, T *W,
                                                              int64_t ldw, int S, const double *C, const double *Rinv,
                                                              int64_t n, int R, int nst, double *gpart, uint32_t *err) {
    constexpr bool FUSE = SB <= 8;
    constexpr int NG = FUSE ? SB * (SB + 1) / 2 : 1;
    constexpr int NCW = GS_CONSUMERS;
    extern __shared__ __align__(128) unsigned char us_dyn[];
    __shared__ __align__(16) T cs[MMAX + 1][SB];
    __shared__ __align__(16) T ri[SB][SB];
    __shared__ double red[SB * SB];
    __shared__ double wred[8][NG];
    __shared__ uint64_t full[ST_MAXST], empty[ST_MAXST];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // coefficients past S (and the tables' unused rows) are zeros, so the FMAs run over all SB
    // columns without a guard: a column past S stays 0 (its staged values are zeros too)
    for (int e = tid; e < (MMAX + 1) * SB; e += 256) cs[e / SB][e % SB] = (T)0;
    for (int e = tid; e < SB * SB; e += 256) ri[e % SB][e / SB] = (T)0;
    __syncthreads();
    for (int e = tid; e < K1 * S; e += 256) cs[e % K1][e / K1] = (T)C[e];
    for (int e = tid; e < S * S; e += 256) ri[e % S][e / S] = (T)Rinv[e];
    for (int e = tid; e < SB * SB; e += 256) red[e] = 0.0;
    for (int e = tid; e < 8 * NG; e += 256) wred[e / NG][e % NG] = 0.0;
    StageRing ring;
    ring.base = us_dyn;
    ring.full = full;
    ring.KP = (K1 + ST_BOXC - 1) / ST_BOXC * ST_BOXC;
    ring.NCP = ring.KP + (S + ST_BOXC - 1) / ST_BOXC * ST_BOXC;
    ring.R = R;
    ring.nst = nst;
    ring.n = n;
    const int64_t nblk = (n + R - 1) / R;
    ring.nmine = (int64_t)blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int KP = ring.KP;
    if (tid < nst) {
        st_mbar_init(&full[tid], 1);
        st_mbar_init(&empty[tid], (uint32_t)NCW);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const volatile int *vbad = &s_bad;
    const bool gram = FUSE && gpart != nullptr;
    if (warp == NCW) {
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t i = 0; i < ring.nmine; i++) {
                const int st = (int)(i % nst);
                if (i >= nst && !st_wait_or_bad(&empty[st], (uint32_t)(((i / nst) - 1) & 1), vbad)) {
                    s_bad = 1;
                    atomicOr(err, 1u);
                    break;
                }
                ring.issue<T>(i, &mq, &mw);
                issued = i + 1;
            }
            if (*vbad) ring.drain(issued > nst ? issued - nst : 0, issued);
        }
    } else {
        T g2[NG];
#pragma unroll
        for (int e = 0; e < NG; e++) g2[e] = (T)0;
        auto flush = [&]() {
#pragma unroll
            for (int e = 0; e < NG; e++) {
                T v = g2[e];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == (e & 31)) wred[warp][e] += (double)v;
                g2[e] = (T)0;
            }
        };
        int since = 0;          // rows this thread has summed into g2 since the last flush
        for (int64_t i = 0; i < ring.nmine; i++) {
            const int st = (int)(i % nst);
            const bool ok = st_wait_or_bad(&full[st], (uint32_t)((i / nst) & 1), vbad);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    s_bad = 1;
                    atomicOr(err, 1u);
                }
                break;
            }
            const int64_t r0 = ring.row0(i);
            const int rows = (int)min((int64_t)R, n - r0);
            // this stage's virtual warp: the rows past 32 NCW rotate over the warps
            const int vw = (int)((warp + i) % NCW);
            for (int rb = 0; rb < R; rb += 32 * NCW) {
                const int rr = rb + vw * 32 + lane;
                if (rb + vw * 32 >= R) break;   // warp-uniform: no rows of this round for this warp
                if (rr < rows) {
                    T w[SB];
                    // all SB columns without a guard: the staged W columns past S (within the
                    // padded boxes) are zeros and so are their coefficients
#pragma unroll
                    for (int b = 0; b < SB; b++) w[b] = ring.col<T>(st, KP + b)[rr];
                    // the coefficients of row a of C (and of R^-1) as 16-byte vector loads from
                    // shared memory; the FMAs as in update_kernel
                    for (int a = 0; a < K1; a++) {
                        const T q = ring.col<T>(st, a)[rr];
                        T cr[SB];
                        vec_row<T, SB>(&cs[a][0], cr);
#pragma unroll
                        for (int b = 0; b < SB; b++) w[b] = fma(-q, cr[b], w[b]);
                    }
                    T wn[SB];
#pragma unroll
                    for (int b = 0; b < SB; b++) wn[b] = (T)0;
#pragma unroll
                    for (int c = 0; c < SB; c++) {
                        T rr_[SB];
                        vec_row<T, SB>(&ri[c][0], rr_);
#pragma unroll
                        for (int b = c; b < SB; b++) wn[b] = fma(w[c], rr_[b], wn[b]);
                    }
#pragma unroll
                    for (int b = 0; b < SB; b++)
                        if (b < S) W[(int64_t)b * ldw + r0 + rr] = wn[b];
                    if (gram) {
                        int e = 0;
#pragma unroll
                        for (int b = 0; b < SB; b++)
#pragma unroll
                            for (int c = 0; c <= b; c++) {
                                if (b < S && e < NG) g2[e] = fma(wn[b], wn[c], g2[e]);
                                e++;
                            }
                    }
                }
                if (gram && ++since == 32) {
                    flush();
                    since = 0;
                }
            }
            __syncwarp();
            if (lane == 0) st_mbar_arrive(&empty[st]);
        }
        if (gram) flush();
    }
    __syncthreads();
    if (!gram) return;
    for (int e = tid; e < NG; e += 256) {
        double t = 0.0;
        for (int w = 0; w < NCW; w++) t += wred[w][e];
        int b = 0, c = e;
        while (c > b) { c -= b + 1; b++; }
        if (b < S) red[b * S + c] = t;
    }
    __syncthreads();
    for (int e = tid; e < S * S; e += 256) {
        const int b = e / S, c = e % S;
        const double v = b >= c ? red[b * S + c] : red[c * S + b];
        gpart[(int64_t)blockIdx.x * S * S + b + c * S] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
    }
}

// Host side of the staged kernels.  Tensor maps are encoded with the driver's
// cuTensorMapEncodeTiled, reached through the runtime (no link against the driver library);
// without it the callers run the register-streaming kernels.  R rows per stage and the ring
// depth come from the kernel's shared-memory budget (stage_budget): the largest R (at most
// 256, a box's limit) that leaves three stages, else two, then as many stages of that size as
// the budget holds, so that narrow stages (the CholQR normalisation, short blocks) get a
// deeper ring.
constexpr size_t ST_BUDGET = 96 * 1024;   // dynamic shared memory per CTA at most

typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static TmapEncodeFn tmap_encoder() {
    static TmapEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TmapEncodeFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D map of `cols` columns of n rows, column stride ld elements, boxes of R rows x ST_BOXC
// columns; false when the columns do not meet the copy engine's alignment (16-byte base and
// stride) or no encoder is available
template <typename T> static bool make_tmap(CUtensorMap *m, const T *base, int64_t ld, int64_t n, int cols, int R) {
    TmapEncodeFn enc = tmap_encoder();
    if (!enc || !base || cols < 1 || n < 1 || ld < n || n >= (1ll << 31)) return false;
    if ((uintptr_t)base % 16 != 0 || ((int64_t)ld * (int64_t)sizeof(T)) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * (int64_t)sizeof(T))};
    cuuint32_t box[2] = {(cuuint32_t)R, (cuuint32_t)ST_BOXC};
    cuuint32_t es[2] = {1, 1};
    return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
               const_cast<T *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The dynamic shared memory a CTA of `kern` may take while two CTAs stay resident on an SM:
// half the SM's shared memory, less the per-CTA reservation and the kernel's static arrays, at
// most ST_BUDGET.  Computed once per (kernel, device), when the kernel's dynamic limit is also
// raised to ST_BUDGET: setting it per launch raced between host threads that launch the same
// kernel with different stage sizes (the server runs one solve per thread).
static std::mutex g_smem_attr_mu;
static std::map<std::pair<const void *, int>, size_t> g_stage_budget;
template <typename F> static mpk_status stage_budget(F kern, size_t *budget) {
    int dev = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_smem_attr_mu);
    const auto key = std::make_pair(reinterpret_cast<const void *>(kern), dev);
    const auto it = g_stage_budget.find(key);
    if (it != g_stage_budget.end()) {
        *budget = it->second;
        return MPK_OK;
    }
    int sm_bytes = 0, reserved = 0;
    MPK_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    MPK_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    cudaFuncAttributes fa;
    MPK_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(kern)));
    const int64_t half = (int64_t)sm_bytes / 2 - reserved - (int64_t)fa.sharedSizeBytes;
    MPK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ST_BUDGET));
    const size_t b = (size_t)std::max<int64_t>(0, std::min<int64_t>(half, (int64_t)ST_BUDGET));
    g_stage_budget.emplace(key, b);
    *budget = b;
    return MPK_OK;
}

static bool stage_choice(int NCP, size_t es, size_t budget, int *R, int *nst) {
    static const int rs[4] = {256, 128, 64, 32};
    for (int q = 3; q >= 2; q--)
        for (int r : rs) {
            const size_t sb = (size_t)NCP * r * es;
            if (sb * q <= budget) {
                *R = r;
                *nst = (int)std::min<size_t>(ST_MAXST, budget / sb);
                return true;
            }
        }
    return false;
}
static inline int box_pad(int c) { return (c + ST_BOXC - 1) / ST_BOXC * ST_BOXC; }

// G partials (grid x K x S, part) of X^T Y by the staged kernel on at most max_grid CTAs (one
// per SM); MPK_ERR_UNIMPLEMENTED when the columns or sizes do not allow it.
template <typename T>
static mpk_status gram_stage_launch(const T *X, int64_t ldx, int K, const T *Y, int64_t ldy, int S, int64_t n,
                                    int nsm, int max_grid, double *part, uint32_t *err, int *grid, cudaStream_t s) {
    int R = 0, nst = 0;
    // FP32 bases only: an FP64 Gram is bound by the FP64 pipe however its rows arrive
    if (sizeof(T) != 4 || n <= 0 || K < 1 || S < 1 || S > SMAX || K > MMAX + 1 + SMAX) return MPK_ERR_UNIMPLEMENTED;
    // the stage's padded X columns, as the kernel instantiated for this S computes them
    const int kp = S <= 4 ? gram_kp<T, 4>(K) : (S <= 8 ? gram_kp<T, 8>(K) : gram_kp<T, 16>(K));
    auto kern = S <= 4 ? gram_stage_kernel<T, 4> : (S <= 8 ? gram_stage_kernel<T, 8> : gram_stage_kernel<T, 16>);
    size_t budget = 0;
    MPK_TRY(stage_budget(kern, &budget));
    if (!stage_choice(kp + box_pad(S), sizeof(T), budget, &R, &nst)) return MPK_ERR_UNIMPLEMENTED;
    CUtensorMap mx, my;
    if (!make_tmap<T>(&mx, X, ldx, n, K, R) || !make_tmap<T>(&my, Y, ldy, n, S, R)) return MPK_ERR_UNIMPLEMENTED;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(2 * nsm, max_grid), ceil_div(n, R)));
    const size_t dsm = (size_t)(kp + box_pad(S)) * R * sizeof(T) * nst;
    kern<<<g, 256, dsm, s>>>(mx, my, K, S, n, R, nst, part, err);
    MPK_CUDA(cudaGetLastError());
    *grid = g;
    return MPK_OK;
}

// W <- (W - Q C) Rinv (and the S x S Gram partials of the new W in gpart when S <= 8 and gpart
// is given) by the staged kernel; MPK_ERR_UNIMPLEMENTED when not applicable.
template <typename T>
static mpk_status update_stage_launch(const T *Q, int64_t ldq, int K1, T *W, int64_t ldw, int S, const double *C,
                                      const double *Rinv, int64_t n, int nsm, int max_grid, double *gpart,
                                      uint32_t *err, int *grid, cudaStream_t s) {
    int R = 0, nst = 0;
    // FP32 bases
    if (sizeof(T) != 4 || n <= 0 || S < 1 || S > SMAX || K1 < 0 || K1 > MMAX + 1) return MPK_ERR_UNIMPLEMENTED;
    auto kern = S <= 4 ? update_stage_kernel<T, 4> : (S <= 8 ? update_stage_kernel<T, 8> : update_stage_kernel<T, 16>);
    size_t budget = 0;
    MPK_TRY(stage_budget(kern, &budget));
    if (!stage_choice(box_pad(K1) + box_pad(S), sizeof(T), budget, &R, &nst)) return MPK_ERR_UNIMPLEMENTED;
    CUtensorMap mq, mw;
    if (!make_tmap<T>(&mw, W, ldw, n, S, R)) return MPK_ERR_UNIMPLEMENTED;
    if (K1 > 0) {
        if (!make_tmap<T>(&mq, Q, ldq, n, K1, R)) return MPK_ERR_UNIMPLEMENTED;
    } else {
        mq = mw;   // not read: no Q columns
    }
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(2 * nsm, max_grid), ceil_div(n, R)));
    const size_t dsm = (size_t)(box_pad(K1) + box_pad(S)) * R * sizeof(T) * nst;
    kern<<<g, 256, dsm, s>>>(mq, mw, K1, W, ldw, S, C, Rinv, n, R, nst, S <= 8 ? gpart : nullptr, err);
    MPK_CUDA(cudaGetLastError());
    *grid = g;
    return MPK_OK;
}

// x[i] += sum_a V[i, a] y[a]  (correction in the basis precision, added to FP64 x); with
// right Jacobi scaling (dinv != nullptr) x[i] += dinv[i] * (V y)[i] in FP64 (Sec. 5.1)
template <typename T>
__global__ void xupdate_kernel(const T *V, int64_t ldv, int k, const double *y, int64_t n,
                               const double *dinv, double *x) {
    __shared__ T ys[MMAX + 1];
    for (int a = threadIdx.x; a < k; a += blockDim.x) ys[a] = (T)y[a];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T d = (T)0;
        for (int a = 0; a < k; a++) d = fma(V[(int64_t)a * ldv + i], ys[a], d);
        x[i] += dinv ? dinv[i] * (double)d : (double)d;
    }
}

// out[i] = sum_a V[i, a] y[a] in the basis precision (a correction before the polynomial
// preconditioner is applied to it); x[i] += d[i] in FP64
template <typename T>
__global__ void vy_kernel(const T *V, int64_t ldv, int k, const double *y, int64_t n, T *out) {
    __shared__ T ys[MMAX + 1];
    for (int a = threadIdx.x; a < k; a += blockDim.x) ys[a] = (T)y[a];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T d = (T)0;
        for (int a = 0; a < k; a++) d = fma(V[(int64_t)a * ldv + i], ys[a], d);
        out[i] = d;
    }
}
template <typename A, typename B>
__global__ void cvt_kernel(const A *in, int64_t n, B *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}
template <typename T>
__global__ void add_f64_kernel(const T *d, int64_t n, const double *dinv, double *x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += dinv ? dinv[i] * (double)d[i] : (double)d[i];
}

// ------------------------------------------------------------------------------------------
// Small dense FP64 work, one CTA
// ------------------------------------------------------------------------------------------
struct CycleState {            // device memory, one per solve
    double H[(MMAX + 1) * MMAX];      // Arnoldi H (unrotated), column-major, ld MMAX+1
    double Hr[(MMAX + 1) * MMAX];     // rotated
    double cs[MMAX], sn[MMAX], g[MMAX + 1];
    double C[(MMAX + 1) * SMAX];      // BCGS coefficients of the current block (K1 x S)
    double C2[(MMAX + 1) * SMAX];
    double R1[SMAX * SMAX], R2[SMAX * SMAX], Rinv[SMAX * SMAX];
    double y[MMAX + 1];
    double hist[MMAX];                // |g_{c+1}| after column c's rotation (residual estimate)
    double nrm[4];
    // scratch of the single-thread kernels (kept here: device memory, not per-thread stack)
    double A[SMAX * SMAX];
    double Ct[(MMAX + 1) * SMAX], Rt[SMAX * SMAX];
    double RF[(MMAX + 1 + SMAX) * (SMAX + 1)];
    double RHS[(MMAX + 1 + SMAX) * SMAX], Hn[(MMAX + 1 + SMAX) * SMAX];
    int status;                 // 0 ok, 1 breakdown
    int conv_k;                 // columns done when converged (0: not yet)
    int kdone;                  // columns in the basis so far
    double est;                 // latest residual estimate |g[k]|
};

// The small dense steps below run on one CTA each.  On this GPU a dependent chain of FP64
// operations in a single thread costs tens of cycles per operation, so every step spreads its
// independent work over the threads and keeps only true recurrences sequential.  Each keeps
// the summation order of the plain algorithm, so results do not depend on the thread count.

// Cholesky of an S x S SPD matrix A (col-major, shared memory) into upper R with R^T R = A,
// and Rinv = R^-1, by one warp: lane 0 takes the pivot, lanes j > i the rest of row i; then
// lane j back-substitutes column j of the inverse.  False (on every lane) on a non-positive
// pivot.
__device__ bool chol_inv_warp(const double *A, int S, double *R, double *Rinv, int lane) {
    for (int e = lane; e < S * S; e += 32) {
        R[e] = 0.0;
        Rinv[e] = 0.0;
    }
    __syncwarp();
    for (int i = 0; i < S; i++) {
        double d = 0.0;
        if (lane == 0) {
            d = A[i + i * S];
            for (int k = 0; k < i; k++) d -= R[k + i * S] * R[k + i * S];
        }
        d = __shfl_sync(0xffffffffu, d, 0);
        if (!(d > 0.0)) return false;
        const double rii = sqrt(d);
        if (lane == 0) R[i + i * S] = rii;
        if (lane > i && lane < S) {
            double v = A[i + lane * S];
            for (int k = 0; k < i; k++) v -= R[k + i * S] * R[k + lane * S];
            R[i + lane * S] = v / rii;
        }
        __syncwarp();
    }
    if (lane < S) {
        const int j = lane;
        Rinv[j + j * S] = 1.0 / R[j + j * S];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int k = i + 1; k <= j; k++) v += R[i + k * S] * Rinv[k + j * S];
            Rinv[i + j * S] = -v / R[i + i * S];
        }
    }
    __syncwarp();
    return true;
}

// Small steps of the block orthogonalisation:
//   mode 0: C  = G (K1 x S, from G = Q^T W); Rinv = I  (projection coefficients)
//   mode 2: C2 = G (second projection sweep);  Rinv = I
//   mode 1: R1 = chol(G) (S x S Gram of the projected block); Rinv = R1^-1
//   mode 3: R2 = chol(G) (CholQR's second pass);             Rinv = R2^-1
__global__ void __launch_bounds__(256) chol_kernel(CycleState *cst, const double *G, int K1, int S, int mode) {
    const int tid = threadIdx.x;
    if (mode == 0 || mode == 2) {
        double *Cd = mode == 0 ? cst->C : cst->C2;
        for (int e = tid; e < K1 * S; e += blockDim.x) Cd[e] = G[e];
        for (int e = tid; e < S * S; e += blockDim.x) cst->Rinv[e] = (e % S == e / S) ? 1.0 : 0.0;
        return;
    }
    if (tid >= 32) return;
    __shared__ double sA[SMAX * SMAX], sR[SMAX * SMAX], sRi[SMAX * SMAX];
    for (int e = tid; e < S * S; e += 32) sA[e] = G[e];
    __syncwarp();
    if (!chol_inv_warp(sA, S, sR, sRi, tid)) {
        if (tid == 0) cst->status = 1;
        return;
    }
    double *R = mode == 1 ? cst->R1 : cst->R2;
    for (int e = tid; e < S * S; e += 32) {
        R[e] = sR[e];
        cst->Rinv[e] = sRi[e];
    }
}

// Hessenberg columns j..j+S-1 from R_full (C, R), shifts theta and the previous Arnoldi H;
// Givens rotations; convergence check against tol_abs.
// passes == 2: C_total = C1 + C2 R1, R_total = R2 R1 ; else C_total = C1, R_total = R2 R1.
__global__ void __launch_bounds__(256) hess_kernel(CycleState *cst, int j, int S, const double *theta,
                                                    double tol_abs, int m) {
    __shared__ int s_stop;
    if (cst->status) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int K1 = j + 1;
    const int ldh = MMAX + 1;
    const int NR = K1 + S;
    double *C = cst->Ct, *R = cst->Rt, *RF = cst->RF, *RHS = cst->RHS, *Hn = cst->Hn;
    const bool two = cst->nrm[3] > 0.5;
    if (tid == 0) s_stop = 0;
    // R = R2 R1 (upper triangular); C = C1 (+ C2: second projection sweep, when taken)
    for (int e = tid; e < S * S; e += nt) {
        const int a = e % S, c = e / S;
        double v = 0.0;
        if (a <= c)
            for (int k = a; k <= c; k++) v += cst->R2[a + k * S] * cst->R1[k + c * S];
        R[e] = v;
    }
    for (int e = tid; e < K1 * S; e += nt) {
        double v = cst->C[e];
        if (two) v += cst->C2[e];
        C[e] = v;
    }
    __syncthreads();
    // R_full: (K1 + S) x (S + 1), column 0 = e_j, columns 1..S = [C ; R]
    for (int e = tid; e < NR * (S + 1); e += nt) {
        const int a = e % NR, col = e / NR;
        double v;
        if (col == 0) v = a == j ? 1.0 : 0.0;
        else v = a < K1 ? C[a + (col - 1) * K1] : R[(a - K1) + (col - 1) * S];
        RF[e] = v;
    }
    __syncthreads();
    // rhs = R_full * Bm - H_prev[:, 0:j] * R_s[0:j, :],   Bm: (S+1) x S, theta on the
    // diagonal, ones below
    for (int e = tid; e < NR * S; e += nt) {
        const int a = e % NR, c = e / NR;
        double v = RF[a + c * NR] * theta[c] + RF[a + (c + 1) * NR];
        for (int q = 0; q < j; q++) v -= cst->H[a + q * ldh] * RF[q + c * NR];
        RHS[e] = v;
    }
    __syncthreads();
    // T = R_s[j:j+S, 0:S] upper triangular; H_new = RHS T^-1 (solve from the right, by columns)
    for (int c = 0; c < S; c++) {
        const double tcc = RF[(j + c) + c * NR];
        for (int a = tid; a < NR; a += nt) {
            double v = RHS[a + c * NR];
            for (int q = 0; q < c; q++) v -= Hn[a + q * NR] * RF[(j + q) + c * NR];
            Hn[a + c * NR] = a >= j + c + 2 ? 0.0 : v / tcc;   // Hessenberg structure
        }
        __syncthreads();
    }
    // store the new columns (unrotated and rotated copies), zero below the structure
    for (int e = tid; e < S * ldh; e += nt) {
        const int a = e % ldh, c = e / ldh;
        const double v = a < NR ? Hn[a + c * NR] : 0.0;
        cst->H[a + (j + c) * ldh] = v;
        cst->Hr[a + (j + c) * ldh] = v;
    }
    __syncthreads();
    // earlier rotations 0..j-1 on each new column (one thread per column)
    if (tid < S) {
        double *h = cst->Hr + (j + tid) * ldh;
        for (int i = 0; i < j; i++) {
            const double t = cst->cs[i] * h[i] + cst->sn[i] * h[i + 1];
            h[i + 1] = -cst->sn[i] * h[i] + cst->cs[i] * h[i + 1];
            h[i] = t;
        }
    }
    __syncthreads();
    // this block's rotations: rotation c from column c, then applied to the later columns
    for (int c = j; c < j + S; c++) {
        if (tid == 0) {
            double *h = cst->Hr + c * ldh;
            const double a = h[c], b = h[c + 1];
            double cs = 1.0, sn = 0.0;
            if (b != 0.0) {
                const double r = hypot(a, b);
                cs = a / r;
                sn = b / r;
            }
            cst->cs[c] = cs;
            cst->sn[c] = sn;
            h[c] = cs * a + sn * b;
            h[c + 1] = 0.0;
            cst->g[c + 1] = -sn * cst->g[c];
            cst->g[c] = cs * cst->g[c];
            cst->kdone = c + 1;
            cst->est = fabs(cst->g[c + 1]);
            cst->hist[c] = cst->est;
            if (fabs(cst->g[c + 1]) <= tol_abs) {
                cst->conv_k = c + 1;
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int cc = c + 1 + tid;
        if (cc < j + S) {
            double *h = cst->Hr + cc * ldh;
            const double t = cst->cs[c] * h[c] + cst->sn[c] * h[c + 1];
            h[c + 1] = -cst->sn[c] * h[c] + cst->cs[c] * h[c + 1];
            h[c] = t;
        }
        __syncthreads();
    }
    (void)m;
}

// y = Hr[0:k, 0:k]^-1 g[0:k]: back substitution by columns (y_i, then every row above it
// subtracts its multiple of y_i)
__global__ void __launch_bounds__(128) lsq_kernel(CycleState *cst, int k) {
    __shared__ double gg[MMAX + 1], yy[MMAX];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ldh = MMAX + 1;
    for (int i = tid; i < k; i += nt) gg[i] = cst->g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; i--) {
        if (tid == 0) yy[i] = gg[i] / cst->Hr[i + i * ldh];
        __syncthreads();
        const double yi = yy[i];
        for (int a = tid; a < i; a += nt) gg[a] -= cst->Hr[a + i * ldh] * yi;
        __syncthreads();
    }
    for (int i = tid; i < k; i += nt) cst->y[i] = yy[i];
}

__global__ void cycle_init_kernel(CycleState *cst, const double *beta) {
    const int tid = threadIdx.x;
    const double b = *beta;
    for (int i = tid; i <= MMAX; i += blockDim.x) cst->g[i] = i == 0 ? b : 0.0;
    if (tid == 0) {
        cst->status = 0;
        cst->conv_k = 0;
        cst->kdone = 0;
        cst->est = b;
        cst->nrm[3] = 0.0;
    }
}
__global__ void set_flag_kernel(CycleState *cst, double v) {
    if (threadIdx.x == 0) cst->nrm[3] = v;
}

// ------------------------------------------------------------------------------------------
// Host driver
// ------------------------------------------------------------------------------------------
struct Timer {
    // intervals are recorded without waiting; flush() adds them up once the stream is idle
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double total = 0.0;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {}
    ~Timer() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    void rec() {
        if (used == ev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            ev.push_back(e);
        }
        cudaEventRecord(ev[used++], s);
    }
    void start() { rec(); }
    void stop() { rec(); }
    void flush() {
        for (size_t i = 0; i + 1 < used; i += 2) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) total += ms;
            else cudaGetLastError();
        }
        used = 0;
    }
};

template <typename T>
struct Solver {
    mpk_plan_s *P;
    cudaStream_t st;
    mpk_gmres_opts o;
    int64_t n, ldv;
    DevBuf V, part, G, gpart2, cstate, vec;   // vec: b, x, r, norms (FP64)
    DevBuf serr;                               // latched by a staged kernel whose copy timed out
    DevBuf dth;                                // Newton shifts of the current cycle
    DevBuf ptmp;                               // polynomial preconditioner: 2 vectors of T
    DevBuf ptmp64;                             // and 2 FP64 vectors (FP64 polynomial)
    // polynomial preconditioner (Sec. 5.2): degree, Chebyshev interval and coefficients
    int poly_deg = 0;
    bool poly_on = false;
    double piv_lo = 0.0, piv_hi = 0.0;         // smallest and largest root
    std::vector<double> pgam, pa, pb, pc;
    double *bp, *xp, *rp, *nrm;
    CycleState *cst;
    int gram_grid, upd_grid;
    Timer t_mpk, t_ortho, t_other;
    std::vector<double> theta;
    int s_cur;
    mpk_gmres_info info{};
    bool trace_pending = false;   // the first Newton-basis cycle still has to be recorded
    double trace_scale = 1.0;     // norm of that cycle's right-hand side

    // the residual estimates |g_{c+1}| / ||r|| of the cycle's k columns and its Arnoldi H
    // ((m+1) x m, column-major, zeros past column k) into the caller's host buffers
    mpk_status record_trace(int k) {
        const int m = o.restart;
        std::vector<double> hist(k), Hh((size_t)(MMAX + 1) * m, 0.0);
        MPK_CUDA(cudaMemcpyAsync(hist.data(), cst->hist, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaMemcpyAsync(Hh.data(), cst->H, (size_t)(MMAX + 1) * k * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        const int cnt = std::min(k, std::max(0, o.trace_cap));
        if (o.trace_hist)
            for (int c = 0; c < cnt; c++) o.trace_hist[c] = trace_scale > 0 ? hist[c] / trace_scale : hist[c];
        if (o.trace_H)
            for (int c = 0; c < m; c++)
                for (int r = 0; r <= m; r++)
                    o.trace_H[(size_t)r + (size_t)c * (m + 1)] = c < k ? Hh[(size_t)r + (size_t)c * (MMAX + 1)] : 0.0;
        info.trace_len = cnt;
        trace_pending = false;
        return MPK_OK;
    }

    Solver(mpk_plan_s *p, cudaStream_t s_) : P(p), st(s_), t_mpk(s_), t_ortho(s_), t_other(s_) {}

    mpk_status alloc() {
        n = P->n;
        ldv = (n + 31) / 32 * 32;
        const int m = o.restart;
        MPK_TRY(V.alloc_on((size_t)(m + 1) * ldv * sizeof(T), st));
        gram_grid = 8 * P->n_sm;
        upd_grid = 4 * P->n_sm;
        const int maxK = m + 1 + SMAX;
        MPK_TRY(part.alloc_on((size_t)std::max(gram_grid, upd_grid) * maxK * SMAX * sizeof(double) + 4096, st));
        MPK_TRY(G.alloc_on((size_t)maxK * SMAX * sizeof(double) + 64, st));
        MPK_TRY(gpart2.alloc_on((size_t)upd_grid * SMAX * SMAX * sizeof(double) + 64, st));
        MPK_TRY(serr.alloc_on(64, st));
        MPK_CUDA(cudaMemsetAsync(serr.p, 0, 64, st));
        MPK_TRY(cstate.alloc_on(sizeof(CycleState), st));
        MPK_TRY(dth.alloc_on(SMAX * sizeof(double), st));
        if (uses_poly() || o.gs2) MPK_TRY(ptmp.alloc_on((size_t)2 * ldv * sizeof(T), st));
        if (o.gs2) MPK_TRY(ptmp64.alloc_on((size_t)3 * ldv * sizeof(double), st));
        else if (uses_poly() && poly64()) MPK_TRY(ptmp64.alloc_on((size_t)2 * ldv * sizeof(double), st));
        MPK_TRY(vec.alloc_on((size_t)3 * ldv * sizeof(double) + 64 * sizeof(double), st));
        bp = vec.as<double>();
        xp = bp + ldv;
        rp = xp + ldv;
        nrm = rp + ldv;
        cst = cstate.as<CycleState>();
        MPK_CUDA(cudaMemsetAsync(cstate.p, 0, sizeof(CycleState), st));
        return MPK_OK;
    }

    T *col(int a) { return V.as<T>() + (int64_t)a * ldv; }
    void flush_timers() {
        t_mpk.flush();
        t_ortho.flush();
        t_other.flush();
    }

    mpk_status norm2(const double *v, double *out) {
        const unsigned g = grid_rows(n);
        sumsq_partial_kernel<double><<<g, RED_BLOCK, 0, st>>>(v, n, part.as<double>());
        reduce_partials_kernel<<<redp_grid(1), 32 * REDP_WARPS, 0, st>>>(part.as<double>(), g, 1, 1, out, 1);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }

    // G (K x S) = X^T Y
    template <int SB> mpk_status gram_sb(const T *X, int K, const T *Y, int S, double *Gout) {
        if (K > MMAX + 1 + SMAX || S > SB) return MPK_ERR_ARG;
        // the basis columns are 128-byte aligned with ldv >= n rounded up to 32 rows, so the
        // staged kernel applies whenever its stages fit in shared memory
        int g = 0;
        const mpk_status sk = gram_stage_launch<T>(X, ldv, K, Y, ldv, S, n, P->n_sm, gram_grid, part.as<double>(),
                                                   serr.as<uint32_t>(), &g, st);
        if (sk == MPK_ERR_UNIMPLEMENTED) {
            g = (int)std::min<int64_t>(gram_grid, ceil_div(n, GRAM_RANGE));
            gram_kernel<T, SB><<<g, 256, 0, st>>>(X, ldv, K, Y, ldv, S, n, part.as<double>());
        } else {
            MPK_TRY(sk);
        }
        reduce_partials_kernel<<<redp_grid(K * S), 32 * REDP_WARPS, 0, st>>>(part.as<double>(), g, K * S, (int64_t)K * S, Gout, 0);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }
    mpk_status gram(const T *X, int K, const T *Y, int S, double *Gout) {
        if (S <= 4) return gram_sb<4>(X, K, Y, S, Gout);
        if (S <= 8) return gram_sb<8>(X, K, Y, S, Gout);
        return gram_sb<16>(X, K, Y, S, Gout);
    }
    // *grid: the CTAs whose Gram partials gp holds
    mpk_status update(const T *Q, int K1, T *W, int S, const double *C, const double *Ri, double *gp, int *grid = nullptr) {
        int ug = 0;
        const mpk_status sk = update_stage_launch<T>(Q, ldv, K1, W, ldv, S, C, Ri, n, P->n_sm, upd_grid, gp,
                                                     serr.as<uint32_t>(), &ug, st);
        if (sk == MPK_ERR_UNIMPLEMENTED) {
            ug = (int)std::min<int64_t>(upd_grid, ceil_div(n, 256));
            if (S <= 4) update_kernel<T, 4><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
            else if (S <= 8) update_kernel<T, 8><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
            else update_kernel<T, 16><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
        } else {
            MPK_TRY(sk);
        }
        if (grid) *grid = ug;
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }

    // one orthogonalisation of the block W = V[:, j+1 .. j+S] against Q = V[:, 0..j]:
    //   C = Q^T W, W <- W - Q C        (BOrtho, block classical Gram-Schmidt; optionally twice)
    //   R1 = chol(W^T W), W <- W R1^-1, R2 = chol(W^T W), W <- W R2^-1     (CholQR2)
    // The Gram of each step is fused into the update that produces W (s <= 8).
    mpk_status ortho(int j, int S) {
        const int K1 = j + 1;
        T *Q = col(0), *W = col(j + 1);
        double *Gd = G.as<double>();
        auto update_gram = [&](int k1, const double *C) -> mpk_status {
            if (S <= 8) {
                int ug = 0;
                MPK_TRY(update(Q, k1, W, S, C, cst->Rinv, gpart2.as<double>(), &ug));
                reduce_partials_kernel<<<redp_grid(S * S), 32 * REDP_WARPS, 0, st>>>(gpart2.as<double>(), ug, S * S, (int64_t)S * S, Gd, 0);
            } else {
                MPK_TRY(update(Q, k1, W, S, C, cst->Rinv, nullptr));
                MPK_TRY(gram(W, S, W, S, Gd));
            }
            return MPK_OK;
        };
        MPK_TRY(gram(Q, K1, W, S, Gd));
        chol_kernel<<<1, 256, 0, st>>>(cst, Gd, K1, S, 0);
        if (o.bcgs_passes >= 2) {
            MPK_TRY(update(Q, K1, W, S, cst->C, cst->Rinv, nullptr));
            MPK_TRY(gram(Q, K1, W, S, Gd));
            chol_kernel<<<1, 256, 0, st>>>(cst, Gd, K1, S, 2);
            MPK_TRY(update_gram(K1, cst->C2));
            set_flag_kernel<<<1, 32, 0, st>>>(cst, 1.0);
        } else {
            MPK_TRY(update_gram(K1, cst->C));
        }
        chol_kernel<<<1, 32, 0, st>>>(cst, Gd, 0, S, 1);
        MPK_TRY(update_gram(0, cst->C));      // W <- W R1^-1, Gram for the second pass
        chol_kernel<<<1, 32, 0, st>>>(cst, Gd, 0, S, 3);
        MPK_TRY(update(Q, 0, W, S, cst->C, cst->Rinv, nullptr));
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }

    // out = q(A) in, or out = A in (level order, precision U): one final-only MPK
    template <typename U> mpk_status apply_poly_u(const U *in, U *out) {
        mpk_coeffs co{poly_deg, pa.data(), pb.data(), pc.data(), pgam.data()};
        const uint32_t fl = MPK_PERMUTED_IO | MPK_FINAL_ONLY | (o.mpk_flags & MPK_UNBLOCKED) | jac_flag();
        return mpk_apply_internal(P, &co, sizeof(U) == 8 ? MPK_F64 : MPK_F32, in, ldv, out, ldv, 1, fl, st);
    }
    template <typename U> mpk_status apply_A_u(const U *in, U *out) {
        double one = 1.0, zero = 0.0;
        mpk_coeffs co{1, &one, &zero, &zero, nullptr};
        const uint32_t fl = MPK_PERMUTED_IO | MPK_FINAL_ONLY | (o.mpk_flags & MPK_UNBLOCKED) | jac_flag();
        return mpk_apply_internal(P, &co, sizeof(U) == 8 ? MPK_F64 : MPK_F32, in, ldv, out, ldv, 1, fl, st);
    }
    // a polynomial preconditioner: the GMRES polynomial, or k >= 2 Jacobi sweeps
    bool uses_poly() const { return o.poly_degree > 0 || o.jacobi >= 2; }
    // right Jacobi scaling: every operator application is one of A D^-1; GS2: of A P^-1 with
    // P^-1 one two-stage Gauss-Seidel iteration (sub-powers of the MPK)
    uint32_t jac_flag() const {
        if (o.gs2) return MPK_GS2 | MPK_GS2_GAMMA(o.gs2_gamma);
        return o.jacobi ? MPK_JACOBI : 0u;
    }
    const double *dinv() const { return (o.jacobi || o.gs2) ? P->dinv64.as<double>() : nullptr; }
    // the polynomial runs with the FP64 matrix values although the basis is FP32
    bool poly64() const { return sizeof(T) == 4 && o.poly_f64 != 0; }

    mpk_status mpk_block(int j, int S, bool newton) {
        if (poly_on) {
            // right-preconditioned column: v_{j+1} <- A q(A) v_j
            if (poly64()) {
                double *d0 = ptmp64.as<double>(), *d1 = d0 + ldv;
                cvt_kernel<T, double><<<grid_rows(n), 256, 0, st>>>(col(j), n, d0);
                MPK_CUDA(cudaGetLastError());
                MPK_TRY(apply_poly_u<double>(d0, d1));
                MPK_TRY(apply_A_u<double>(d1, d0));
                cvt_kernel<double, T><<<grid_rows(n), 256, 0, st>>>(d0, n, col(j + 1));
                MPK_CUDA(cudaGetLastError());
                return MPK_OK;
            }
            T *t0 = ptmp.as<T>();
            MPK_TRY(apply_poly_u<T>(col(j), t0));
            return apply_A_u<T>(t0, col(j + 1));
        }
        std::vector<double> a(S, 1.0), b(S, 0.0), c(S, 0.0);
        if (newton)
            for (int k = 0; k < S; k++) b[k] = -theta[k];
        mpk_coeffs co{S, a.data(), b.data(), c.data(), nullptr};
        const mpk_dtype dt = sizeof(T) == 8 ? MPK_F64 : MPK_F32;
        const uint32_t fl = MPK_PERMUTED_IO | MPK_Y0_IS_X | (o.mpk_flags & MPK_UNBLOCKED) | jac_flag();
        MPK_TRY(mpk_apply_internal(P, &co, dt, nullptr, ldv, col(j), ldv, 1, fl, st));
        return MPK_OK;
    }

    // one restart cycle on A d = r (r in rp, FP64); adds the correction to xp.  newton=false:
    // monomial s=1 with two BCGS sweeps (plain GMRES with classical Gram-Schmidt, reorthogonalised),
    // used to collect Ritz values.  Returns the number of columns used.
    mpk_status cycle(double tol_abs, bool newton, int s, int *k_used, bool *breakdown) {
        const int m = o.restart;
        norm2(rp, nrm);
        normalize_kernel<T><<<grid_rows(n), 256, 0, st>>>(rp, nrm, n, col(0));
        cycle_init_kernel<<<1, 128, 0, st>>>(cst, nrm);
        MPK_CUDA(cudaGetLastError());
        std::vector<double> th(s, 0.0);
        if (newton)
            for (int k = 0; k < s; k++) th[k] = theta[k];
        MPK_CUDA(cudaMemcpyAsync(dth.p, th.data(), s * sizeof(double), cudaMemcpyHostToDevice, st));
        int j = 0, k = 0;
        *breakdown = false;
        const int saved_passes = o.bcgs_passes;
        if (!newton) o.bcgs_passes = 2;
        while (j < m) {
            const int S = std::min(s, m - j);
            t_mpk.start();
            MPK_TRY(mpk_block(j, S, newton));
            t_mpk.stop();
            t_ortho.start();
            MPK_TRY(ortho(j, S));
            hess_kernel<<<1, 256, 0, st>>>(cst, j, S, dth.as<double>(), tol_abs, m);
            MPK_CUDA(cudaGetLastError());
            t_ortho.stop();
            int hs[3];
            MPK_CUDA(cudaMemcpyAsync(hs, &cst->status, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
            MPK_CUDA(cudaStreamSynchronize(st));
            flush_timers();
            if (hs[0]) {   // Cholesky breakdown: keep the columns before this block
                *breakdown = true;
                k = j;
                break;
            }
            k = hs[2];
            if (hs[1]) break;
            j += S;
        }
        o.bcgs_passes = saved_passes;
        if (k > 0) {
            t_other.start();
            lsq_kernel<<<1, 128, 0, st>>>(cst, k);
            if (poly_on) {
                // x += q(A) V y
                T *t0 = ptmp.as<T>(), *t1 = t0 + ldv;
                vy_kernel<T><<<grid_rows(n, 8), 256, 0, st>>>(V.as<T>(), ldv, k, cst->y, n, t0);
                MPK_CUDA(cudaGetLastError());
                if (poly64()) {
                    double *d0 = ptmp64.as<double>(), *d1 = d0 + ldv;
                    cvt_kernel<T, double><<<grid_rows(n), 256, 0, st>>>(t0, n, d0);
                    MPK_TRY(apply_poly_u<double>(d0, d1));
                    add_f64_kernel<double><<<grid_rows(n), 256, 0, st>>>(d1, n, dinv(), xp);
                } else {
                    MPK_TRY(apply_poly_u<T>(t0, t1));
                    add_f64_kernel<T><<<grid_rows(n), 256, 0, st>>>(t1, n, dinv(), xp);
                }
            } else if (o.gs2 && o.gs2_gamma >= 1) {
                // x += P^-1 V y = D~^-1 h_gamma(V y), the GS2 stages in FP64
                T *t0 = ptmp.as<T>();
                double *d0 = ptmp64.as<double>(), *d1 = d0 + ldv, *d2 = d1 + ldv;
                vy_kernel<T><<<grid_rows(n, 8), 256, 0, st>>>(V.as<T>(), ldv, k, cst->y, n, t0);
                cvt_kernel<T, double><<<grid_rows(n), 256, 0, st>>>(t0, n, d0);
                MPK_CUDA(cudaGetLastError());
                MPK_TRY(mpk_gs2_inner(P, MPK_F64, o.gs2_gamma, d0, d1, d2, st));
                add_f64_kernel<double><<<grid_rows(n), 256, 0, st>>>(d1, n, dinv(), xp);
            } else {
                xupdate_kernel<T><<<grid_rows(n, 8), 256, 0, st>>>(V.as<T>(), ldv, k, cst->y, n, dinv(), xp);
            }
            MPK_CUDA(cudaGetLastError());
            t_other.stop();
        }
        if (!newton && !poly_on && k > 0) {
            // Ritz values: eigenvalues of the leading k x k block of the cycle's Arnoldi H
            // (QR iteration on the host: k <= 128), real parts, Leja-ordered
            std::vector<double> Hh((size_t)(MMAX + 1) * k), wr(k), wi(k);
            MPK_CUDA(cudaMemcpyAsync(Hh.data(), cst->H, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            MPK_CUDA(cudaStreamSynchronize(st));
            MPK_TRY(mpk_hessenberg_eigvals(Hh.data(), MMAX + 1, k, wr.data(), wi.data()));
            theta.assign(o.s, 0.0);
            mpk_leja_order(wr.data(), k, o.s, theta.data());
        }
        if (newton && trace_pending && k > 0) MPK_TRY(record_trace(k));
        *k_used = k;
        return MPK_OK;
    }

    // The GMRES polynomial of the setup cycle's first d + 1 steps (Sec. 5.2), in root form: the
    // GMRES residual polynomial pi(t) = prod_i (1 - t / theta_i) has the harmonic Ritz values of
    // those steps as roots, and q(t) = (1 - pi(t)) / t gives
    //     q(A) x = sum_{k=0}^{d} (1 / theta_{k+1}) prod_{i<=k} (I - A / theta_i) x,
    // an MPK of d powers with a_k = -1 / theta_k, b_k = 1 and gamma_k = 1 / theta_{k+1}; the
    // roots are Leja-ordered, which keeps the partial products bounded.  For a symmetric A the
    // harmonic Ritz values are the eigenvalues of the pencil Hbar^T Hbar z = theta S z (Hbar the
    // leading (d+2) x (d+1) Arnoldi block, S the symmetric part of its square part), found by a
    // Cholesky S = L L^T and Jacobi rotations on L^-1 Hbar^T Hbar L^-T.  Host arithmetic on
    // O(d^2) numbers, like the Leja ordering of the shifts; no polynomial if S is not positive
    // definite.
    static bool jacobi_eigenvalues(std::vector<double> &Asym, int q, std::vector<double> &ev) {
        double fro = 0.0;
        for (double v : Asym) fro += v * v;
        for (int sweep = 0; sweep < 60; sweep++) {
            double off = 0.0;
            for (int c = 0; c < q; c++)
                for (int r = 0; r < q; r++)
                    if (r != c) off += Asym[r + c * q] * Asym[r + c * q];
            if (!(off > 1e-30 * fro)) break;
            for (int p = 0; p < q - 1; p++)
                for (int r = p + 1; r < q; r++) {
                    const double apq = Asym[p + r * q];
                    if (std::fabs(apq) < 1e-300) continue;
                    const double tau = (Asym[r + r * q] - Asym[p + p * q]) / (2.0 * apq);
                    const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                    const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
                    for (int i = 0; i < q; i++) {
                        const double aip = Asym[i + p * q], aiq = Asym[i + r * q];
                        Asym[i + p * q] = c * aip - sn * aiq;
                        Asym[i + r * q] = sn * aip + c * aiq;
                    }
                    for (int i = 0; i < q; i++) {
                        const double api = Asym[p + i * q], aqi = Asym[r + i * q];
                        Asym[p + i * q] = c * api - sn * aqi;
                        Asym[r + i * q] = sn * api + c * aqi;
                    }
                }
        }
        ev.resize(q);
        for (int i = 0; i < q; i++) ev[i] = Asym[i + i * q];
        return true;
    }

    // k Jacobi sweeps from zero (Sec. 5.1, Eq. (Jacobi)) as a right preconditioner: with
    // B = I - D^-1 A the sweeps give z_k = sum_{j<k} B^j D^-1 v, and since
    // B^j D^-1 = D^-1 (I - A D^-1)^j this is P^-1 = D^-1 p(A D^-1) with the Neumann polynomial
    // p(t) = sum_{j<k} (1 - t)^j: one final-only MPK on A D^-1 with a_j = -1, b_j = 1,
    // gamma_j = 1.  The Krylov operator is A D^-1 p(A D^-1) and the correction D^-1 p(A D^-1) V y.
    void setup_sweeps(int k) {
        const int dd = k - 1;
        pa.assign(dd, -1.0);
        pb.assign(dd, 1.0);
        pc.assign(dd, 0.0);
        pgam.assign(dd + 1, 1.0);
        poly_deg = dd;
        piv_lo = piv_hi = 0.0;
        poly_on = true;
    }

    mpk_status setup_poly(int k) {
        const int dd = std::min(std::min(o.poly_degree, k - 1), MPK_MAX_P);
        if (dd < 1) return MPK_OK;   // cycle too short: no polynomial
        const int ldh = MMAX + 1, q = dd + 1;
        std::vector<double> H((size_t)ldh * q);
        MPK_CUDA(cudaMemcpyAsync(H.data(), cst->H, H.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        // G = Hbar^T Hbar, S = sym(H[0:q, 0:q])
        std::vector<double> G((size_t)q * q, 0.0), L((size_t)q * q, 0.0), X((size_t)q * q, 0.0);
        for (int a = 0; a < q; a++)
            for (int b = 0; b < q; b++) {
                double v = 0.0;
                for (int r = 0; r <= q; r++) v += H[r + a * ldh] * H[r + b * ldh];
                G[a + b * q] = v;
            }
        // Cholesky of S (lower L)
        for (int c = 0; c < q; c++) {
            for (int r = c; r < q; r++) {
                double v = 0.5 * (H[r + c * ldh] + H[c + r * ldh]);
                for (int t = 0; t < c; t++) v -= L[r + t * q] * L[c + t * q];
                if (r == c) {
                    if (!(v > 0.0)) return MPK_OK;   // not positive definite: no polynomial
                    L[c + c * q] = std::sqrt(v);
                } else {
                    L[r + c * q] = v / L[c + c * q];
                }
            }
        }
        // X = L^-1 G, then C = L^-1 X^T (= L^-1 G L^-T for symmetric G)
        auto fwd = [&](const std::vector<double> &B, std::vector<double> &Out, bool transpose_in) {
            for (int c = 0; c < q; c++)
                for (int r = 0; r < q; r++) {
                    double v = transpose_in ? B[c + r * q] : B[r + c * q];
                    for (int t = 0; t < r; t++) v -= L[r + t * q] * Out[t + c * q];
                    Out[r + c * q] = v / L[r + r * q];
                }
        };
        fwd(G, X, false);
        std::vector<double> C((size_t)q * q, 0.0);
        fwd(X, C, true);
        for (int a = 0; a < q; a++)
            for (int b = a + 1; b < q; b++) {
                const double v = 0.5 * (C[a + b * q] + C[b + a * q]);
                C[a + b * q] = v;
                C[b + a * q] = v;
            }
        std::vector<double> ev, roots(q);
        jacobi_eigenvalues(C, q, ev);
        for (double v : ev)
            if (!(v > 0.0) || !std::isfinite(v)) return MPK_OK;
        MPK_TRY(mpk_leja_order(ev.data(), q, q, roots.data()));
        pa.assign(dd, 0.0);
        pb.assign(dd, 1.0);
        pc.assign(dd, 0.0);
        pgam.assign(dd + 1, 0.0);
        for (int kk = 0; kk < dd; kk++) pa[kk] = -1.0 / roots[kk];
        for (int kk = 0; kk <= dd; kk++) pgam[kk] = 1.0 / roots[kk];
        poly_deg = dd;
        piv_lo = *std::min_element(roots.begin(), roots.end());
        piv_hi = *std::max_element(roots.begin(), roots.end());
        poly_on = true;
        return MPK_OK;
    }

    mpk_status run(const double *b, double *x) {
        MPK_TRY(alloc());
        const unsigned g = grid_rows(n);
        const int32_t *perm = P->perm.as<int32_t>();
        gather_f64_kernel<<<g, 256, 0, st>>>(b, perm, n, bp);
        gather_f64_kernel<<<g, 256, 0, st>>>(x, perm, n, xp);
        MPK_CUDA(cudaGetLastError());
        norm2(bp, nrm + 1);
        double hb = 0.0;
        MPK_CUDA(cudaMemcpyAsync(&hb, nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        s_cur = o.s;
        if (o.shifts) theta.assign(o.shifts, o.shifts + o.s);
        bool need_shifts = !o.shifts || o.poly_degree > 0;
        if (o.jacobi >= 2) {   // Jacobi sweeps: fixed polynomial, single-column cycles from the start
            setup_sweeps(o.jacobi);
            need_shifts = false;
        }
        bool have_shifts = !need_shifts;
        trace_pending = o.trace_hist != nullptr || o.trace_H != nullptr;
        mpk_status result = MPK_ERR_NOT_CONVERGED;
        double relres = 1.0, best_rel = 1e300;
        int since_best = 0;
        for (int outer = 0; outer <= o.max_outer; outer++) {
            t_other.start();
            MPK_TRY(mpk_launch_residual(P, xp, bp, rp, st));
            norm2(rp, nrm + 2);
            double hr = 0.0;
            MPK_CUDA(cudaMemcpyAsync(&hr, nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            t_other.stop();
            MPK_CUDA(cudaStreamSynchronize(st));
            flush_timers();
            relres = hb > 0 ? hr / hb : 0.0;
            info.outer = outer;
            if (relres <= o.tol || hb == 0.0) {
                result = MPK_OK;
                break;
            }
            if (outer == o.max_outer || info.iters >= o.max_iters) break;
            if (!std::isfinite(hr)) break;
            // stagnation: no new best true residual (by 0.1 %) in 50 refinement steps
            if (relres < 0.999 * best_rel) {
                best_rel = relres;
                since_best = 0;
            } else if (++since_best >= 50) {
                break;
            }
            // one restart cycle on A d = r; target: inner_tol relative to ||r|| in the basis
            // precision, never tighter than the overall target
            double tol_abs = std::max(o.inner_tol * hr, 0.5 * o.tol * hb);
            if (sizeof(T) == 8) tol_abs = 0.5 * o.tol * hb;
            int k = 0;
            bool bd = false;
            if (!have_shifts) {
                MPK_TRY(cycle(tol_abs, false, 1, &k, &bd));
                have_shifts = true;
                if (o.poly_degree > 0) MPK_TRY(setup_poly(k));
            } else if (poly_on) {
                MPK_TRY(cycle(tol_abs, false, 1, &k, &bd));   // single columns on A q(A)
            } else {
                trace_scale = hr;
                MPK_TRY(cycle(tol_abs, true, s_cur, &k, &bd));
                if (bd) {
                    // CholQR breakdown: the following cycles run at s / 2.  (Stepping back up
                    // to s after clean cycles measured slower on the 256^3 log-normal matrix
                    // in FP32: 13,344 Krylov columns in 6.7 s, against 11,672 in 6.1 s - the
                    // FP32 basis of a smaller block keeps more digits per column.)
                    info.breakdowns++;
                    if (s_cur == 1) { result = MPK_ERR_BREAKDOWN; break; }
                    s_cur = std::max(1, s_cur / 2);
                }
            }
            info.iters += k;
            info.restarts++;
            if (k == 0 && !bd) break;
        }
        scatter_f64_kernel<<<g, 256, 0, st>>>(xp, perm, n, x);
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaStreamSynchronize(st));
        flush_timers();
        info.rel_residual = relres;
        info.status = result;
        for (size_t i = 0; i < theta.size() && i < 64; i++) info.shifts[i] = theta[i];
        info.poly_degree = poly_deg;
        info.poly_interval[0] = piv_lo;
        info.poly_interval[1] = piv_hi;
        info.ms_mpk = t_mpk.total;
        info.ms_ortho = t_ortho.total;
        info.ms_other = t_other.total;
        info.s_final = s_cur;
        return result;
    }
};

// ==========================================================================================
// s-step CG (the short-recurrence method the paper names for the MPK, Sec. 4 and Sec. 7): per
// outer iteration one MPK of s powers on p and one of s - 1 powers on r (Newton basis) give
// Y = [p, .., rho_s(A) p, r, .., rho_{s-1}(A) r] (M = 2s + 1 columns of ldv), the Gram matrix
// G = Y^T Y in FP64, s CG steps on coordinate vectors of length M, and the recovery
// x += Y x', p = Y p', r = Y r'.  The MPK dominates; the only tall-skinny product left is one
// Gram matrix per s steps (the reason the paper expects the MPK speedup to carry over).
// ==========================================================================================
constexpr int CG_SMAX = 15;                   // M = 2s + 1 <= 31: one warp owns the coordinates
constexpr int CG_MMAX = 2 * CG_SMAX + 1;
constexpr int CG_SETUP_MAX = 4 * CG_SMAX;     // setup-phase steps recorded for the Ritz values

struct CgState {                              // device memory, one per solve
    double xc[CG_MMAX], rc[CG_MMAX], pc[CG_MMAX];
    double rr;                                // r'^T G r' after the last step taken
    double alpha[CG_SETUP_MAX], beta[CG_SETUP_MAX];
    int32_t steps;                            // steps taken by the last outer iteration
    int32_t done;                             // the recurrence residual reached the target
    int32_t breakdown;                        // p'^T G B p' <= 0 met (steps counts good ones)
    int32_t n_setup;                          // setup-phase coefficients recorded
};

// The CG steps of one outer iteration on coordinate vectors; one warp, lane a owns component
// a < M.  With B the change of basis (theta_j on the diagonal and a one below it inside each
// block, nothing in the last column of a block):
//   alpha = r'G r' / p'G B p',  x' += alpha p',  r' -= alpha B p',
//   beta = r'G r' (new) / r'G r' (old),  p' = r' + beta p'.
// G B is formed once (column c is theta_c G e_c + G e_{c+1}), and G r' is carried along by
// G r' -= alpha (G B p'), so each step costs one FP64 matrix-vector product (G B p').
// Starts from p' = e_0, r' = e_{s+1}, x' = 0 (Y's first columns are p and r).  Dot products
// are FP64 shuffle trees in a fixed order.  Stops after s steps, at `max_steps`, when
// sqrt(r'G r') <= target, or at a non-positive p'G B p' (breakdown: that step is not taken).
// record: append alpha_j, beta_j to the setup-phase coefficients (Lanczos tridiagonal).
__global__ void __launch_bounds__(32) cg_coord_kernel(CgState *cs, const double *G, int M, int s,
                                                      const double *theta, double target,
                                                      int max_steps, int record, int bs) {
    __shared__ double sGB[CG_MMAX * CG_MMAX];
    __shared__ double sv[CG_MMAX];
    const int a = threadIdx.x;
    // diagonal of B in column c and whether B has a one below it (c not last in its block)
    auto bdiag = [&](int c) -> double {
        const int j = c <= s ? c : c - s - 1;
        const int len = c <= s ? s + 1 : s;
        return j < len - 1 ? theta[j] : 0.0;
    };
    auto bsub = [&](int c) -> bool {
        const int j = c <= s ? c : c - s - 1;
        const int len = c <= s ? s + 1 : s;
        return j < len - 1;
    };
    // G: the upper triangle over the basis storage's 2s + 2 columns in pair order (column
    // 2k + q: slot q of pair k), packed by bs x bs blocks (gram_sym_kernel); basis column a is
    // storage column a <= s ? 2a : 2(a - s - 1) + 1.  Read symmetrically.
    const int nbk = (2 * (s + 1) + bs - 1) / bs;
    auto g = [&](int r, int c) -> double {
        r = r <= s ? 2 * r : 2 * (r - s - 1) + 1;
        c = c <= s ? 2 * c : 2 * (c - s - 1) + 1;
        if (r > c) {
            const int t_ = r;
            r = c;
            c = t_;
        }
        const int ab = r / bs, bb = c / bs;
        const int pb = ab * nbk - ab * (ab - 1) / 2 + (bb - ab);
        return G[pb * bs * bs + (r - ab * bs) * bs + (c - bb * bs)];
    };
    double gr = 0.0;                               // (G r')_a, r' = e_{s+1}
    if (a < M) {
        for (int c = 0; c < M; c++) {
            double v = bdiag(c) * g(a, c);
            if (bsub(c)) v += g(a, c + 1);
            sGB[a + c * M] = v;
        }
        gr = g(a, s + 1);
    }
    const bool inP = a <= s;
    const int jl = inP ? a : a - s - 1;           // position inside the block
    const bool sub = a < M && jl >= 1;
    const double th = a < M ? bdiag(a) : 0.0;
    double pc = a == 0 ? 1.0 : 0.0, rc = a == s + 1 ? 1.0 : 0.0, xc = 0.0;
    __syncwarp();
    auto wsum = [&](double v) -> double {
        v = a < M ? v : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    auto bmul = [&](double v) -> double {         // (B v)_a
        const double up = __shfl_up_sync(0xffffffffu, v, 1);
        return sub ? fma(th, v, up) : th * v;
    };
    double rr = wsum(rc * gr);
    int steps = 0, done = 0, bd = 0;
    int nrec = cs->n_setup;
    for (int j = 0; j < s && steps < max_steps; j++) {
        // v1 = (G B p')_a, two partial sums to halve the dependent chain
        if (a < M) sv[a] = pc;
        __syncwarp();
        double v1 = 0.0, v2 = 0.0;
        if (a < M) {
            int c = 0;
            for (; c + 1 < M; c += 2) {
                v1 = fma(sGB[a + c * M], sv[c], v1);
                v2 = fma(sGB[a + (c + 1) * M], sv[c + 1], v2);
            }
            if (c < M) v1 = fma(sGB[a + c * M], sv[c], v1);
        }
        __syncwarp();
        v1 += v2;
        const double bp = bmul(pc);
        const double den = wsum(pc * v1);
        if (!(den > 0.0)) {
            bd = 1;
            break;
        }
        const double alpha = rr / den;
        xc = fma(alpha, pc, xc);
        rc = fma(-alpha, bp, rc);
        gr = fma(-alpha, v1, gr);
        const double rrn = wsum(rc * gr);
        const double beta = rrn / rr;
        pc = fma(beta, pc, rc);
        rr = rrn;
        steps++;
        if (record && nrec < CG_SETUP_MAX) {
            if (a == 0) {
                cs->alpha[nrec] = alpha;
                cs->beta[nrec] = beta;
            }
            nrec++;
        }
        if (sqrt(fmax(rr, 0.0)) <= target) {
            done = 1;
            break;
        }
    }
    if (a < M) {
        cs->xc[a] = xc;
        cs->rc[a] = rc;
        cs->pc[a] = pc;
    }
    __syncwarp();
    if (a == 0) {
        cs->rr = rr;
        cs->steps = steps;
        cs->done = done;
        cs->breakdown = bd;
        cs->n_setup = nrec;
    }
}

// Symmetric Gram of the CG basis storage: the upper triangle of G = Y^T Y over its 2s + 2
// columns in pair order (column 2k + q is slot q of pair k; P_s(A) r, column 2s + 1, is
// summed too and not used), stored packed by BS x BS blocks: block pair pb = (ab, bb),
// ab <= bb, enumerated row by row, entry (i, j) of the block at pb * BS^2 + i * BS + j.  A
// block of columns is then whole pairs (FP32: two, FP64: one), read from the staged tile by
// vector loads.  A CTA stages tiles of TR rows of Y in shared memory; thread t owns block
// pair t % NBP and the rows g, g + RG, ... of each tile (g = t / NBP, RG = 256 / NBP row
// groups).  Precision: a thread sums its products in the basis precision over at most 32 rows
// (F tiles), the RG row groups' block sums of each entry are then added by a fixed pairwise
// tree in shared memory (at most eight levels), and the result is added to the CTA's FP64
// total of the entry (in shared memory); the CTA writes one FP64 partial per entry, which
// reduce_partials_kernel sums over the CTAs in a fixed order.  For an FP32 basis
// |G^ - G| <= (40 u32 + m u64) |Y|^T |Y| entrywise.  FP32: BS = 6 (three pairs; loads of 12
// values per 36 FMAs; s = 8 gives 6 block pairs and 216 products per row for the 171 of the
// triangle, against 15 and 240 with BS = 4) and TR = 168, so that the 42 row groups of s = 8
// sum four rows each.  FP64: BS = 2 (fewer wasted products on the slow FP64 pipe), TR = 128.
// Tiles arrive by 16-byte asynchronous copies (cp.async) into a ring of GSYM_STAGES shared
// buffers, GSYM_STAGES - 1 tiles ahead of the one being summed: with one tile in flight per
// CTA the kernel was bound by memory latency (about 1 TB/s on the FP32 basis).
constexpr int GSYM_STAGES = 4;
constexpr int GSYM_MP = 32;                   // M padded (<= 32 columns)
template <typename T> __host__ __device__ constexpr int gsym_bs() { return sizeof(T) == 4 ? 6 : 2; }
template <typename T> __host__ __device__ constexpr int gsym_tr() { return sizeof(T) == 4 ? 168 : 128; }
static inline int gsym_nbp(int M, int bs) {
    const int nb = (M + bs - 1) / bs;
    return nb * (nb + 1) / 2;
}
// shared elements of one pair's tile: 2 TR values and padding that keeps every copy 16-byte
// aligned and starts the pairs of a stage in different banks (FP32: 356 = 4 mod 32 words, so
// the three column blocks of a stage start 12 banks apart)
template <typename T> __host__ __device__ constexpr int gsym_pstride() {
    return sizeof(T) == 4 ? 2 * gsym_tr<T>() + 20 : 2 * gsym_tr<T>() + 2;
}
// pairs of a stage for np stored pairs: whole column blocks of BS / 2 pairs (the padding
// pairs read zeros)
template <typename T> __host__ __device__ constexpr int gsym_pairs(int np) {
    return (np + gsym_bs<T>() / 2 - 1) / (gsym_bs<T>() / 2) * (gsym_bs<T>() / 2);
}
// dynamic shared memory of gram_sym_kernel for np pairs: the stage ring, then the row groups'
// block sums (256 BS^2 values of the basis type), then the CTA's FP64 totals (NBP BS^2)
template <typename T> __host__ __device__ size_t gsym_ring_bytes(int np) {
    return (size_t)GSYM_STAGES * gsym_pairs<T>(np) * gsym_pstride<T>() * sizeof(T);
}
template <typename T> __host__ __device__ size_t gsym_flush_bytes() {
    return (size_t)256 * gsym_bs<T>() * gsym_bs<T>() * sizeof(T);
}
template <typename T> size_t gsym_smem_bytes(int np) {
    constexpr int BS = gsym_bs<T>();
    return gsym_ring_bytes<T>(np) + gsym_flush_bytes<T>() + (size_t)gsym_nbp(2 * np, BS) * BS * BS * sizeof(double);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Basis storage of s-step CG: the two Krylov sequences P_k(A) p (k = 0..s) and P_k(A) r
// (k = 0..s-1) sit as interleaved pairs, pair k = (P_k(A) p, P_k(A) r) at Y + 2 k ldv with
// element i of the pair at offsets 2i and 2i + 1.  One two-rhs MPK call then builds both
// sequences and reads the matrix once per power for both (two single-rhs calls read it
// 2s - 1 times).  Basis column a (a <= s: P_a(A) p; a > s: P_{a-s-1}(A) r) has element i at
// Y[cg_col_ofs(a, s, ldv) + 2 i].  Pair s also holds P_s(A) r, which the method does not use.
__host__ __device__ __forceinline__ int64_t cg_col_ofs(int a, int s, int64_t ldv) {
    return a <= s ? (int64_t)a * 2 * ldv : (int64_t)(a - s - 1) * 2 * ldv + 1;
}

template <typename T>
__global__ void __launch_bounds__(256, 2) gram_sym_kernel(const T *Y, int64_t ldv, int s, int64_t n,
                                                          double *part) {
    constexpr int BS = gsym_bs<T>();
    constexpr int TR = gsym_tr<T>();
    constexpr int PS = gsym_pstride<T>();
    constexpr int CE = 16 / (int)sizeof(T);          // elements per 16-byte copy
    constexpr int CH = 2 * TR / CE;                  // copies per pair and tile
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T *sY = reinterpret_cast<T *>(sh_raw);
    const int np = s + 1;                            // stored pairs
    const int npad = gsym_pairs<T>(np);              // pairs of a stage
    const int stage = npad * PS;
    const int M = 2 * np;                            // storage columns
    const int nb = (M + BS - 1) / BS;
    const int NBP = nb * (nb + 1) / 2;
    const int RG = (int)blockDim.x / NBP;
    const int t = threadIdx.x;
    const bool act = t < NBP * RG;
    const int pb = t % NBP, g = t / NBP;
    int ab = 0, rem = pb;
    while (rem >= nb - ab) {
        rem -= nb - ab;
        ab++;
    }
    const int bb = ab + rem;
    // this thread's column blocks inside a stage: BS / 2 whole pairs each
    const int oa = ab * (BS / 2) * PS, ob = bb * (BS / 2) * PS;
    // padding pairs (never copied) read zeros
    for (int i = t; i < GSYM_STAGES * (npad - np) * PS; i += blockDim.x) {
        const int stg = i / ((npad - np) * PS), e = i % ((npad - np) * PS);
        sY[stg * stage + np * PS + e] = (T)0;
    }
    T tacc[BS * BS];
#pragma unroll
    for (int k = 0; k < BS * BS; k++) tacc[k] = (T)0;
    // block sums of the row groups: fl[(g * NBP + pb) * BS^2 + k], after the stage ring; then
    // the CTA's FP64 totals acc[pb * BS^2 + k] (read only after the first flush's barriers)
    T *fl = reinterpret_cast<T *>(sh_raw + gsym_ring_bytes<T>(np));
    double *acc = reinterpret_cast<double *>(sh_raw + gsym_ring_bytes<T>(np) + gsym_flush_bytes<T>());
    for (int i = t; i < NBP * BS * BS; i += blockDim.x) acc[i] = 0.0;
    const int rpt = (TR + RG - 1) / RG;               // rows of a tile per thread, at most
    const int F = rpt >= 32 ? 1 : 32 / rpt;           // tiles per block sum: <= 32 terms
    // every thread of the CTA (the barriers): the row groups' block sums of each entry by a
    // pairwise tree over g, added to the FP64 totals of the g = 0 threads
    auto flush = [&]() {
        if (act) {
#pragma unroll
            for (int k = 0; k < BS * BS; k++) {
                fl[(g * NBP + pb) * BS * BS + k] = tacc[k];
                tacc[k] = (T)0;
            }
        }
        __syncthreads();
        for (int step = 1; step < RG; step <<= 1) {
            if (act && (g % (2 * step)) == 0 && g + step < RG) {
#pragma unroll
                for (int k = 0; k < BS * BS; k++)
                    fl[(g * NBP + pb) * BS * BS + k] += fl[((g + step) * NBP + pb) * BS * BS + k];
            }
            __syncthreads();
        }
        if (act && g == 0) {
#pragma unroll
            for (int k = 0; k < BS * BS; k++) acc[pb * BS * BS + k] += (double)fl[pb * BS * BS + k];
        }
        __syncthreads();
    };
    int since = 0;
    const int64_t ntiles = (n + TR - 1) / TR;
    // copies of the rows of `tile` that exist (pair k: 2 rows' values per row, contiguous)
    // into ring buffer stg; one commit group per call, empty past the last tile
    auto issue = [&](int64_t tile, int stg) {
        if (tile < ntiles) {
            const int64_t r0 = tile * TR;
            const int vals = 2 * (int)(n - r0 < TR ? n - r0 : TR);
            T *dst = sY + stg * stage;
            for (int idx = t; idx < np * CH; idx += blockDim.x) {
                const int k = idx / CH, e = (idx % CH) * CE;
                if (e < vals) cp_async16(dst + k * PS + e, Y + (int64_t)k * 2 * ldv + 2 * r0 + e);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < GSYM_STAGES - 1; j++) issue((int64_t)blockIdx.x + (int64_t)j * gridDim.x, j);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
        // the buffer refilled here was summed in the previous iteration (barrier below)
        issue(tile + (int64_t)(GSYM_STAGES - 1) * gridDim.x, (it + GSYM_STAGES - 1) % GSYM_STAGES);
        cp_async_wait<GSYM_STAGES - 1>();
        __syncthreads();
        const T *sb = sY + (it % GSYM_STAGES) * stage;
        const int rows = (int)(n - tile * TR < TR ? n - tile * TR : TR);
        if (act) {
            for (int r = g; r < rows; r += RG) {
                T xa[BS], xb[BS];
#pragma unroll
                for (int h = 0; h < BS / 2; h++) {
                    const T2 va = *reinterpret_cast<const T2 *>(sb + oa + h * PS + 2 * r);
                    const T2 vb = *reinterpret_cast<const T2 *>(sb + ob + h * PS + 2 * r);
                    xa[2 * h] = va.x;
                    xa[2 * h + 1] = va.y;
                    xb[2 * h] = vb.x;
                    xb[2 * h + 1] = vb.y;
                }
#pragma unroll
                for (int i = 0; i < BS; i++)
#pragma unroll
                    for (int j = 0; j < BS; j++) tacc[i * BS + j] = fma(xa[i], xb[j], tacc[i * BS + j]);
            }
        }
        __syncthreads();
        if (++since == F) {   // the same count in every thread
            flush();
            since = 0;
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    flush();
    const int m = NBP * BS * BS;
    for (int i = t; i < m; i += blockDim.x) part[(int64_t)blockIdx.x * m + i] = acc[i];
}

// x += scale * Y x' (in the basis precision, added to the FP64 x); p = Y p' and r = Y r' in
// place (pair 0).  A thread reads a row of Y before it writes that row.
template <typename T>
__global__ void __launch_bounds__(256) cg_recover_kernel(T *Y, int64_t ldv, int M, int s, const CgState *cs,
                                                         int64_t n, double scale, double *x) {
    __shared__ T cx[CG_MMAX], cp[CG_MMAX], cr[CG_MMAX];
    if (threadIdx.x < M) {
        cx[threadIdx.x] = (T)cs->xc[threadIdx.x];
        cp[threadIdx.x] = (T)cs->pc[threadIdx.x];
        cr[threadIdx.x] = (T)cs->rc[threadIdx.x];
    }
    __syncthreads();
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T dx = 0, pn = 0, rn = 0;
        // pair k: basis columns k (from p) and s + 1 + k (from r, k < s)
        for (int k = 0; k <= s; k++) {
            const T2 y = *reinterpret_cast<const T2 *>(Y + (int64_t)k * 2 * ldv + 2 * i);
            dx = fma(cx[k], y.x, dx);
            pn = fma(cp[k], y.x, pn);
            rn = fma(cr[k], y.x, rn);
            if (k < s) {
                const int a = s + 1 + k;
                dx = fma(cx[a], y.y, dx);
                pn = fma(cp[a], y.y, pn);
                rn = fma(cr[a], y.y, rn);
            }
        }
        x[i] += scale * (double)dx;
        T2 o;
        o.x = pn;
        o.y = rn;
        *reinterpret_cast<T2 *>(Y + 2 * i) = o;
    }
}

// r column of pair 0 = (T)(r64 * inv): residual replacement
template <typename T>
__global__ void cg_replace_kernel(const double *r, int64_t n, double inv, T *Y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        Y[2 * i + 1] = (T)(r[i] * inv);
}

// p = r = (T)(r64 / scale): both columns of pair 0
template <typename T>
__global__ void cg_start_kernel(const double *r, int64_t n, double inv, T *Y) {
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = (T)(r[i] * inv);
        T2 o;
        o.x = v;
        o.y = v;
        *reinterpret_cast<T2 *>(Y + 2 * i) = o;
    }
}

template <typename T>
struct CgSolver {
    mpk_plan_s *P;
    cudaStream_t st;
    mpk_cg_opts o;
    int64_t n, ldv;
    int M;
    DevBuf Y, part, G, cstate, vec, dth;
    double *bp, *xp, *rp, *nrm;
    CgState *cs;
    int gram_grid;
    Timer t_mpk, t_gram, t_other;
    std::vector<double> theta;
    int s_cur;
    mpk_cg_info info{};

    CgSolver(mpk_plan_s *p, cudaStream_t s_) : P(p), st(s_), t_mpk(s_), t_gram(s_), t_other(s_) {}

    mpk_status alloc() {
        n = P->n;
        ldv = (n + 31) / 32 * 32;
        M = 2 * o.s + 1;
        MPK_TRY(Y.alloc_on((size_t)(o.s + 1) * 2 * ldv * sizeof(T), st));   // s + 1 pairs
        gram_grid = 8 * P->n_sm;
        // symmetric Gram partials: (CTA, row group) x packed entries <= CTAs x 256 threads x BS^2
        MPK_TRY(part.alloc_on((size_t)(2 * P->n_sm) * 256 * BS * BS * sizeof(double) + 4096, st));
        MPK_TRY(G.alloc_on((size_t)GSYM_MP * GSYM_MP * sizeof(double), st));
        // the attribute is per function and shared by every caller: always the same maximum,
        // never this solve's size, so that concurrent launches cannot race on it
        MPK_CUDA(cudaFuncSetAttribute(gram_sym_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)gsym_smem_bytes<T>(CG_SMAX + 1)));
        MPK_TRY(cstate.alloc_on(sizeof(CgState), st));
        MPK_TRY(dth.alloc_on(CG_SMAX * sizeof(double), st));
        MPK_TRY(vec.alloc_on((size_t)3 * ldv * sizeof(double) + 64 * sizeof(double), st));
        bp = vec.as<double>();
        xp = bp + ldv;
        rp = xp + ldv;
        nrm = rp + ldv;
        cs = cstate.as<CgState>();
        MPK_CUDA(cudaMemsetAsync(cstate.p, 0, sizeof(CgState), st));
        return MPK_OK;
    }
    void flush_timers() {
        t_mpk.flush();
        t_gram.flush();
        t_other.flush();
    }
    mpk_status norm2(const double *v, double *out) {
        const unsigned g = grid_rows(n);
        sumsq_partial_kernel<double><<<g, RED_BLOCK, 0, st>>>(v, n, part.as<double>());
        reduce_partials_kernel<<<redp_grid(1), 32 * REDP_WARPS, 0, st>>>(part.as<double>(), g, 1, 1, out, 1);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }
    // G = Y^T Y over the basis storage: upper triangle packed by blocks (gram_sym_kernel)
    static constexpr int BS = gsym_bs<T>();
    int gsym_grid() const { return (int)std::min<int64_t>(2 * P->n_sm, std::max<int64_t>(1, ceil_div(n, gsym_tr<T>()))); }
    // G over the basis storage's 2 sc + 2 columns (pair order)
    mpk_status gram(int sc) {
        const int g = gsym_grid();
        const int m = gsym_nbp(2 * sc + 2, BS) * BS * BS;
        gram_sym_kernel<T><<<g, 256, gsym_smem_bytes<T>(sc + 1), st>>>(Y.as<T>(), ldv, sc, n, part.as<double>());
        reduce_partials_kernel<<<redp_grid(m), 32 * REDP_WARPS, 0, st>>>(part.as<double>(), g, m, (int64_t)m,
                                                                       G.as<double>(), 0);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }
    // both Newton sequences, p powers each, as pairs 1..p (pair 0 holds p and r)
    mpk_status basis(int p) {
        std::vector<double> a(p, 1.0), b(p, 0.0), c(p, 0.0);
        for (int k = 0; k < p; k++) b[k] = -theta_use[k];
        mpk_coeffs co{p, a.data(), b.data(), c.data(), nullptr};
        const uint32_t fl = MPK_PERMUTED_IO | MPK_Y0_IS_X | MPK_RHS_INTERLEAVED | (o.mpk_flags & MPK_UNBLOCKED);
        return mpk_apply_internal(P, &co, sizeof(T) == 8 ? MPK_F64 : MPK_F32, nullptr, ldv, Y.p, ldv, 2, fl, st);
    }
    std::vector<double> theta_use;

    // One inner solve of A d = r (r in rp, norm hr) by s-step CG with sc steps per outer
    // iteration; the correction is added to xp as it goes.  Returns the steps taken.
    mpk_status inner(int sc, const std::vector<double> &th, double hr, double tol_abs, int max_steps,
                     bool record, int *steps_out, bool *bd_out) {
        const int Mc = 2 * sc + 1;
        theta_use = th;
        *bd_out = false;
        *steps_out = 0;
        cg_start_kernel<T><<<grid_rows(n), 256, 0, st>>>(rp, n, 1.0 / hr, Y.as<T>());
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaMemcpyAsync(dth.p, th.data(), sc * sizeof(double), cudaMemcpyHostToDevice, st));
        int steps = 0;
        for (int it = 0; steps < max_steps; it++) {
            if (o.replace > 0 && it > 0 && it % o.replace == 0) {
                // residual replacement: r = (b - A x) / hr in FP64 (x holds the start plus the
                // correction so far, so this is the inner residual), p kept
                t_other.start();
                MPK_TRY(mpk_launch_residual(P, xp, bp, rp, st));
                cg_replace_kernel<T><<<grid_rows(n), 256, 0, st>>>(rp, n, 1.0 / hr, Y.as<T>());
                MPK_CUDA(cudaGetLastError());
                t_other.stop();
            }
            t_mpk.start();
            MPK_TRY(basis(sc));
            t_mpk.stop();
            t_gram.start();
            MPK_TRY(gram(sc));
            t_gram.stop();
            t_other.start();
            cg_coord_kernel<<<1, 32, 0, st>>>(cs, G.as<double>(), Mc, sc, dth.as<double>(), tol_abs / hr,
                                              max_steps - steps, record ? 1 : 0, BS);
            cg_recover_kernel<T><<<grid_rows(n, 8), 256, 0, st>>>(Y.as<T>(), ldv, Mc, sc, cs, n, hr, xp);
            MPK_CUDA(cudaGetLastError());
            int hs[3];
            MPK_CUDA(cudaMemcpyAsync(hs, &cs->steps, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
            t_other.stop();
            MPK_CUDA(cudaStreamSynchronize(st));
            flush_timers();
            steps += hs[0];
            if (hs[2]) {
                *bd_out = true;
                break;
            }
            if (hs[1] || hs[0] == 0) break;
        }
        *steps_out = steps;
        return MPK_OK;
    }

    // Ritz values of the setup phase: eigenvalues of the Lanczos tridiagonal of its k steps
    mpk_status setup_shifts() {
        int k = 0;
        MPK_CUDA(cudaMemcpyAsync(&k, &cs->n_setup, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        k = std::min(k, CG_SETUP_MAX);
        if (k < 1) return MPK_ERR_BREAKDOWN;
        std::vector<double> al(k), be(k);
        MPK_CUDA(cudaMemcpyAsync(al.data(), cs->alpha, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaMemcpyAsync(be.data(), cs->beta, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        std::vector<double> T_((size_t)k * k, 0.0), ev;
        for (int j = 0; j < k; j++) {
            T_[j + j * k] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
            if (j + 1 < k) {
                const double e = std::sqrt(std::max(be[j], 0.0)) / al[j];
                T_[j + (j + 1) * k] = e;
                T_[(j + 1) + j * k] = e;
            }
        }
        Solver<double>::jacobi_eigenvalues(T_, k, ev);
        s_cur = std::min(s_cur, k);
        theta.assign(o.s, 0.0);
        MPK_TRY(mpk_leja_order(ev.data(), k, s_cur, theta.data()));
        return MPK_OK;
    }

    mpk_status run(const double *b, double *x) {
        MPK_TRY(alloc());
        const unsigned g = grid_rows(n);
        const int32_t *perm = P->perm.as<int32_t>();
        gather_f64_kernel<<<g, 256, 0, st>>>(b, perm, n, bp);
        gather_f64_kernel<<<g, 256, 0, st>>>(x, perm, n, xp);
        MPK_CUDA(cudaGetLastError());
        norm2(bp, nrm + 1);
        double hb = 0.0;
        MPK_CUDA(cudaMemcpyAsync(&hb, nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        s_cur = o.s;
        bool have_shifts = o.shifts != nullptr;
        if (have_shifts) theta.assign(o.shifts, o.shifts + o.s);
        mpk_status result = MPK_ERR_NOT_CONVERGED;
        double relres = 1.0, best_rel = 1e300;
        int since_best = 0;
        for (int outer = 0; outer <= o.max_outer; outer++) {
            t_other.start();
            MPK_TRY(mpk_launch_residual(P, xp, bp, rp, st));
            norm2(rp, nrm + 2);
            double hr = 0.0;
            MPK_CUDA(cudaMemcpyAsync(&hr, nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            t_other.stop();
            MPK_CUDA(cudaStreamSynchronize(st));
            flush_timers();
            relres = hb > 0 ? hr / hb : 0.0;
            info.outer = outer;
            if (relres <= o.tol || hb == 0.0) {
                result = MPK_OK;
                break;
            }
            if (outer == o.max_outer || info.iters >= o.max_iters || !std::isfinite(hr)) break;
            if (relres < 0.999 * best_rel) {
                best_rel = relres;
                since_best = 0;
            } else if (++since_best >= 50) {
                break;
            }
            double tol_abs = std::max(o.inner_tol * hr, 0.5 * o.tol * hb);
            if (sizeof(T) == 8 || o.replace > 0) tol_abs = 0.5 * o.tol * hb;
            const int left = o.max_iters - info.iters;
            int k = 0;
            bool bd = false;
            if (!have_shifts) {
                // setup phase: plain CG (s = 1, no shift), its coefficients recorded
                MPK_TRY(inner(1, std::vector<double>(1, 0.0), hr, tol_abs, std::min(4 * o.s, left), true, &k, &bd));
                if (bd) {
                    result = MPK_ERR_BREAKDOWN;
                    info.iters += k;
                    break;
                }
                MPK_TRY(setup_shifts());
                have_shifts = true;
            } else {
                std::vector<double> th(theta.begin(), theta.begin() + s_cur);
                MPK_TRY(inner(s_cur, th, hr, tol_abs, left, false, &k, &bd));
                if (bd) {
                    if (s_cur == 1) {
                        info.iters += k;
                        result = MPK_ERR_BREAKDOWN;
                        break;
                    }
                    s_cur = std::max(1, s_cur / 2);
                }
            }
            info.iters += k;
            if (k == 0 && !bd) break;
        }
        scatter_f64_kernel<<<g, 256, 0, st>>>(xp, perm, n, x);
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaStreamSynchronize(st));
        flush_timers();
        info.rel_residual = relres;
        info.status = result;
        info.s_used = s_cur;
        for (size_t i = 0; i < theta.size() && i < 16; i++) info.shifts[i] = theta[i];
        info.ms_mpk = t_mpk.total;
        info.ms_gram = t_gram.total;
        info.ms_other = t_other.total;
        return result;
    }
};

}  // namespace

extern "C" mpk_status mpk_gmres_opts_default(mpk_gmres_opts *o) {
    if (!o) return MPK_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->s = 8;
    o->restart = 48;
    o->tol = 1e-8;
    o->inner_tol = 1e-5;
    o->max_outer = 1000;
    o->inner_cycles = 1;
    o->max_iters = 100000;
    o->basis = MPK_F32;
    o->bcgs_passes = 1;
    o->shifts = nullptr;
    o->mpk_flags = 0;
    o->poly_degree = 0;
    o->poly_f64 = 1;
    o->jacobi = 0;
    o->gs2 = 0;
    o->gs2_gamma = 1;
    return MPK_OK;
}

extern "C" mpk_status sstep_gmres_solve(mpk_plan_t A, const double *b, double *x,
                                        const mpk_gmres_opts *opts, mpk_gmres_info *info,
                                        cudaStream_t stream) {
    if (!A || !b || !x) return MPK_ERR_ARG;
    mpk_gmres_opts o;
    if (opts) o = *opts;
    else mpk_gmres_opts_default(&o);
    if (o.s < 1 || o.s > SMAX || o.restart < o.s || o.restart > MMAX || !(o.tol > 0) ||
        o.bcgs_passes < 1 || o.bcgs_passes > 2 || o.max_outer < 0 || o.poly_degree < 0 ||
        o.poly_degree > MPK_MAX_P || o.jacobi < 0 || o.jacobi > MPK_MAX_P + 1 ||
        (o.jacobi >= 2 && o.poly_degree > 0) || o.gs2 < 0 || o.gs2 > 1 || o.gs2_gamma < 0 ||
        o.gs2_gamma > 15 || (o.gs2 && (o.jacobi || o.poly_degree > 0)))
        return MPK_ERR_ARG;
    if (!A->has64) return MPK_ERR_ARG;                       // FP64 residual needs FP64 values
    if (o.basis == MPK_F32 && !A->has32) return MPK_ERR_ARG;
    if ((o.poly_degree > 0 || o.jacobi >= 2) && o.basis == MPK_F32 && !o.poly_f64 && !A->has32)
        return MPK_ERR_ARG;
    if (o.s > A->p_max) return MPK_ERR_ARG;
    if ((o.jacobi || o.gs2) && !A->jacobi) return MPK_ERR_ARG;   // the plan keeps no A D^-1
    auto t0 = std::chrono::steady_clock::now();
    mpk_status st;
    mpk_gmres_info inf{};
    if (o.basis == MPK_F64) {
        Solver<double> S(A, stream);
        S.o = o;
        st = S.run(b, x);
        inf = S.info;
    } else {
        Solver<float> S(A, stream);
        S.o = o;
        st = S.run(b, x);
        inf = S.info;
    }
    auto t1 = std::chrono::steady_clock::now();
    inf.ms_total = std::chrono::duration<double, std::milli>(t1 - t0).count();
    inf.status = st;
    if (info) *info = inf;
    return st;
}

extern "C" mpk_status mpk_cg_opts_default(mpk_cg_opts *o) {
    if (!o) return MPK_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->s = 8;
    o->tol = 1e-8;
    o->inner_tol = 1e-5;
    o->max_outer = 1000;
    o->max_iters = 100000;
    o->basis = MPK_F32;
    o->shifts = nullptr;
    o->mpk_flags = 0;
    o->replace = 1;
    return MPK_OK;
}

extern "C" mpk_status sstep_cg_solve(mpk_plan_t A, const double *b, double *x, const mpk_cg_opts *opts,
                                     mpk_cg_info *info, cudaStream_t stream) {
    if (!A || !b || !x) return MPK_ERR_ARG;
    mpk_cg_opts o;
    if (opts) o = *opts;
    else mpk_cg_opts_default(&o);
    if (o.s < 1 || o.s > CG_SMAX || !(o.tol > 0) || !(o.inner_tol > 0) || o.max_outer < 0 ||
        o.max_iters < 0 || (o.basis != MPK_F32 && o.basis != MPK_F64) || o.replace < 0)
        return MPK_ERR_ARG;
    if (!A->has64) return MPK_ERR_ARG;                       // FP64 residual needs FP64 values
    if (o.basis == MPK_F32 && !A->has32) return MPK_ERR_ARG;
    if (o.s > A->p_max) return MPK_ERR_ARG;
    if (o.shifts)
        for (int i = 0; i < o.s; i++)
            if (!std::isfinite(o.shifts[i])) return MPK_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    mpk_status st;
    mpk_cg_info inf{};
    if (o.basis == MPK_F64) {
        CgSolver<double> S(A, stream);
        S.o = o;
        st = S.run(b, x);
        inf = S.info;
    } else {
        CgSolver<float> S(A, stream);
        S.o = o;
        st = S.run(b, x);
        inf = S.info;
    }
    inf.status = st;
    inf.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

// ==========================================================================================
// The orthogonalisation steps on their own (the kernels the solvers run, callable directly).
// ==========================================================================================
namespace {
mpk_status sm_count(int *nsm) {
    int dev = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev));
    return MPK_OK;
}

template <typename T>
mpk_status gram_launch(const T *X, int64_t ldx, int K, const T *Y, int64_t ldy, int S, int64_t n, double *G,
                       cudaStream_t s) {
    int nsm = 1;
    MPK_TRY(sm_count(&nsm));
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(8 * nsm, ceil_div(n, GRAM_RANGE)));
    DevBuf part, err;
    MPK_TRY(part.alloc_on((size_t)std::max(g, 2 * nsm) * K * S * sizeof(double), s));
    MPK_TRY(err.alloc_on(64, s));
    MPK_CUDA(cudaMemsetAsync(err.p, 0, 64, s));
    // staged (copy-engine ring) when the columns allow it, else register-streaming tiles
    const mpk_status sk = gram_stage_launch<T>(X, ldx, K, Y, ldy, S, n, nsm, 2 * nsm, part.as<double>(),
                                               err.as<uint32_t>(), &g, s);
    if (sk != MPK_ERR_UNIMPLEMENTED) {
        MPK_TRY(sk);
    } else if (S <= 4) gram_kernel<T, 4><<<g, 256, 0, s>>>(X, ldx, K, Y, ldy, S, n, part.as<double>());
    else if (S <= 8) gram_kernel<T, 8><<<g, 256, 0, s>>>(X, ldx, K, Y, ldy, S, n, part.as<double>());
    else gram_kernel<T, 16><<<g, 256, 0, s>>>(X, ldx, K, Y, ldy, S, n, part.as<double>());
    reduce_partials_kernel<<<redp_grid(K * S), 32 * REDP_WARPS, 0, s>>>(part.as<double>(), g, K * S, (int64_t)K * S, G, 0);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

template <typename T>
mpk_status update_launch(const T *Q, int64_t ldq, int K1, T *W, int64_t ldw, int S, const double *C,
                         const double *Rinv, int64_t n, double *G, cudaStream_t s) {
    int nsm = 1;
    MPK_TRY(sm_count(&nsm));
    int ug = (int)std::max<int64_t>(1, std::min<int64_t>(4 * nsm, ceil_div(n, 256)));
    const bool fused = G && S <= 8;
    DevBuf gp, err;
    if (fused) MPK_TRY(gp.alloc_on((size_t)std::max(ug, 2 * nsm) * S * S * sizeof(double), s));
    MPK_TRY(err.alloc_on(64, s));
    MPK_CUDA(cudaMemsetAsync(err.p, 0, 64, s));
    double *gpp = fused ? gp.as<double>() : nullptr;
    const mpk_status sk = update_stage_launch<T>(Q, ldq, K1, W, ldw, S, C, Rinv, n, nsm, 2 * nsm, gpp,
                                                 err.as<uint32_t>(), &ug, s);
    if (sk != MPK_ERR_UNIMPLEMENTED) {
        MPK_TRY(sk);
    } else if (S <= 4) update_kernel<T, 4><<<ug, 256, 0, s>>>(Q, ldq, K1, W, ldw, S, C, Rinv, n, gpp);
    else if (S <= 8) update_kernel<T, 8><<<ug, 256, 0, s>>>(Q, ldq, K1, W, ldw, S, C, Rinv, n, gpp);
    else update_kernel<T, 16><<<ug, 256, 0, s>>>(Q, ldq, K1, W, ldw, S, C, Rinv, n, nullptr);
    MPK_CUDA(cudaGetLastError());
    if (fused) {
        reduce_partials_kernel<<<redp_grid(S * S), 32 * REDP_WARPS, 0, s>>>(gp.as<double>(), ug, S * S, (int64_t)S * S, G, 0);
        MPK_CUDA(cudaGetLastError());
    } else if (G) {
        MPK_TRY(gram_launch<T>(W, ldw, S, W, ldw, S, n, G, s));
    }
    return MPK_OK;
}

// the packed block-pair layout of gram_sym_kernel -> the full M x M matrix (column-major)
__global__ void gsym_unpack_kernel(const double *packed, int M, int bs, double *G) {
    const int nb = (M + bs - 1) / bs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += gridDim.x * blockDim.x) {
        const int i = e % M, j = e / M;
        int a = i, b = j;
        if (a / bs > b / bs) {   // the lower block is the transpose of a stored upper one
            a = j;
            b = i;
        }
        const int ab = a / bs, bb = b / bs;
        const int pb = ab * nb - ab * (ab - 1) / 2 + (bb - ab);
        G[e] = packed[(int64_t)pb * bs * bs + (a % bs) * bs + (b % bs)];
    }
}

template <typename T>
mpk_status gram_pairs_launch(const T *Y, int64_t ldv, int s, int64_t n, double *G, cudaStream_t st) {
    int nsm = 1;
    MPK_TRY(sm_count(&nsm));
    constexpr int BS = gsym_bs<T>();
    const int g = (int)std::min<int64_t>(2 * nsm, std::max<int64_t>(1, ceil_div(n, gsym_tr<T>())));
    const int M = 2 * s + 2;
    const int m = gsym_nbp(M, BS) * BS * BS;
    DevBuf part, packed;
    MPK_TRY(part.alloc_on((size_t)g * m * sizeof(double), st));
    MPK_TRY(packed.alloc_on((size_t)m * sizeof(double), st));
    const size_t smem = gsym_smem_bytes<T>(s + 1);
    MPK_CUDA(cudaFuncSetAttribute(gram_sym_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gsym_smem_bytes<T>(CG_SMAX + 1)));
    gram_sym_kernel<T><<<g, 256, smem, st>>>(Y, ldv, s, n, part.as<double>());
    reduce_partials_kernel<<<redp_grid(m), 32 * REDP_WARPS, 0, st>>>(part.as<double>(), g, m, (int64_t)m, packed.as<double>(), 0);
    gsym_unpack_kernel<<<(M * M + 255) / 256, 256, 0, st>>>(packed.as<double>(), M, BS, G);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}
}  // namespace

extern "C" mpk_status mpk_gram(mpk_dtype dtype, const void *X, int64_t ldx, int32_t K, const void *Y,
                               int64_t ldy, int32_t S, int64_t n, double *G, cudaStream_t s) {
    if (dtype != MPK_F32 && dtype != MPK_F64) return MPK_ERR_ARG;
    if (K < 1 || K > MMAX + 1 + SMAX || S < 1 || S > SMAX || n < 0 || !G) return MPK_ERR_ARG;
    if (n > 0 && (!X || !Y || ldx < n || ldy < n)) return MPK_ERR_ARG;
    if (n == 0) {
        MPK_CUDA(cudaMemsetAsync(G, 0, (size_t)K * S * sizeof(double), s));
        return MPK_OK;
    }
    if (dtype == MPK_F32)
        return gram_launch<float>((const float *)X, ldx, K, (const float *)Y, ldy, S, n, G, s);
    return gram_launch<double>((const double *)X, ldx, K, (const double *)Y, ldy, S, n, G, s);
}

extern "C" mpk_status mpk_block_update(mpk_dtype dtype, const void *Q, int64_t ldq, int32_t K1, void *W,
                                       int64_t ldw, int32_t S, const double *C, const double *Rinv,
                                       int64_t n, double *G, cudaStream_t s) {
    if (dtype != MPK_F32 && dtype != MPK_F64) return MPK_ERR_ARG;
    if (K1 < 0 || K1 > MMAX + 1 || S < 1 || S > SMAX || n < 0 || !Rinv) return MPK_ERR_ARG;
    if (K1 > 0 && (!C || !Q || ldq < n)) return MPK_ERR_ARG;
    if (n > 0 && (!W || ldw < n)) return MPK_ERR_ARG;
    if (n == 0) {
        if (G) MPK_CUDA(cudaMemsetAsync(G, 0, (size_t)S * S * sizeof(double), s));
        return MPK_OK;
    }
    if (dtype == MPK_F32)
        return update_launch<float>((const float *)Q, ldq, K1, (float *)W, ldw, S, C, Rinv, n, G, s);
    return update_launch<double>((const double *)Q, ldq, K1, (double *)W, ldw, S, C, Rinv, n, G, s);
}

extern "C" mpk_status mpk_gram_pairs(mpk_dtype dtype, const void *Y, int64_t ldv, int32_t s, int64_t n,
                                     double *G, cudaStream_t st) {
    if (dtype != MPK_F32 && dtype != MPK_F64) return MPK_ERR_ARG;
    if (s < 1 || s > CG_SMAX || n < 0 || !G) return MPK_ERR_ARG;
    const int M = 2 * s + 2;
    if (n == 0) {
        MPK_CUDA(cudaMemsetAsync(G, 0, (size_t)M * M * sizeof(double), st));
        return MPK_OK;
    }
    // 16-byte copies: an aligned base, pairs 16-byte aligned, and room for the copy that
    // carries the last (odd) row of a pair
    if (!Y || (uintptr_t)Y % 16 != 0 || ldv < n + (n & 1) || (dtype == MPK_F32 && ldv % 2 != 0))
        return MPK_ERR_ARG;
    if (dtype == MPK_F32) return gram_pairs_launch<float>((const float *)Y, ldv, s, n, G, st);
    return gram_pairs_launch<double>((const double *)Y, ldv, s, n, G, st);
}
