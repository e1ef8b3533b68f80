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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
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
__global__ void reduce_partials_kernel(const double *part, int nb, int m, int64_t stride, double *out, int take_sqrt) {
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += part[(int64_t)b * stride + e];
        out[e] = take_sqrt ? sqrt(s) : s;
    }
}

// ------------------------------------------------------------------------------------------
// Tall-skinny Gram G = X^T Y (X: n x K, Y: n x S, column-major), G col-major K x S.
// CTA: rows in chunks of 64 staged in shared memory; thread (tile, group) accumulates a 4 x S
// micro-tile over the rows of its group in the basis precision; per-CTA partials in FP64.
// ------------------------------------------------------------------------------------------
constexpr int GR = 64;   // rows per chunk

template <typename T, int SB>
__global__ void __launch_bounds__(256) gram_kernel(const T *X, int64_t ldx, int K, const T *Y,
                                                   int64_t ldy, int S, int64_t n, double *part) {
    extern __shared__ __align__(16) unsigned char gsm[];
    T *xs = reinterpret_cast<T *>(gsm);                 // GR x K   (row-major)
    T *ys = xs + GR * K;                                // GR x S
    const int ntile = (K + 3) / 4;
    const int ngroup = max(1, (int)blockDim.x / ntile);
    const int tile = threadIdx.x % ntile, group = threadIdx.x / ntile;
    const bool active = group < ngroup && threadIdx.x < ngroup * ntile;
    T acc[4][SB];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < SB; b++) acc[a][b] = (T)0;
    for (int64_t r0 = (int64_t)blockIdx.x * GR; r0 < n; r0 += (int64_t)gridDim.x * GR) {
        const int rows = (int)((n - r0) < (int64_t)GR ? (n - r0) : (int64_t)GR);
        __syncthreads();
        for (int e = threadIdx.x; e < GR * K; e += blockDim.x) {
            const int c = e / GR, r = e % GR;
            xs[r * K + c] = r < rows ? X[(int64_t)c * ldx + r0 + r] : (T)0;
        }
        for (int e = threadIdx.x; e < GR * S; e += blockDim.x) {
            const int c = e / GR, r = e % GR;
            ys[r * S + c] = r < rows ? Y[(int64_t)c * ldy + r0 + r] : (T)0;
        }
        __syncthreads();
        if (active) {
            for (int r = group; r < rows; r += ngroup) {
                T xv[4];
#pragma unroll
                for (int a = 0; a < 4; a++) xv[a] = (tile * 4 + a < K) ? xs[r * K + tile * 4 + a] : (T)0;
#pragma unroll
                for (int b = 0; b < SB; b++) {
                    if (b < S) {
                        const T yv = ys[r * S + b];
#pragma unroll
                        for (int a = 0; a < 4; a++) acc[a][b] = fma(xv[a], yv, acc[a][b]);
                    }
                }
            }
        }
    }
    // combine the groups of the CTA in FP64 (fixed order), one partial per CTA
    __syncthreads();
    double *red = reinterpret_cast<double *>(gsm);      // K x S doubles
    const int KS = K * S;
    for (int e = threadIdx.x; e < KS; e += blockDim.x) red[e] = 0.0;
    __syncthreads();
    for (int g = 0; g < ngroup; g++) {
        if (active && group == g) {
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < SB; b++)
                    if (b < S && tile * 4 + a < K) red[b * K + tile * 4 + a] += (double)acc[a][b];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < KS; e += blockDim.x) part[(int64_t)blockIdx.x * KS + e] = red[e];
}

// ------------------------------------------------------------------------------------------
// W <- (W - Q C) Rinv, row by row, and (optionally) the Gram of the new W for the next step.
// Q: n x K1, W: n x S (in place), C: K1 x S, Rinv: S x S (FP64, converted to T).
// ------------------------------------------------------------------------------------------
template <typename T, int SB>
__global__ void __launch_bounds__(256) update_kernel(const T *Q, int64_t ldq, int K1, T *W, int64_t ldw,
                                                     int S, const double *C, const double *Rinv, int64_t n,
                                                     double *gpart) {
    __shared__ T cs[MMAX + 1][SB];
    __shared__ T ri[SB][SB];
    __shared__ double red[SB * SB];
    for (int e = threadIdx.x; e < K1 * S; e += blockDim.x) cs[e % K1][e / K1] = (T)C[e];
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) ri[e % S][e / S] = (T)Rinv[e];
    for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) red[e] = 0.0;
    __syncthreads();
    // fused Gram of the new block only up to s = 8 (register budget); larger blocks take a
    // separate Gram pass
    constexpr bool FUSE = SB <= 8;
    constexpr int NG = FUSE ? SB * (SB + 1) / 2 : 1;
    T g2[NG];
#pragma unroll
    for (int e = 0; e < NG; e++) g2[e] = (T)0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T w[SB];
#pragma unroll
        for (int b = 0; b < SB; b++) w[b] = b < S ? W[(int64_t)b * ldw + i] : (T)0;
        for (int a = 0; a < K1; a++) {
            const T q = Q[(int64_t)a * ldq + i];
#pragma unroll
            for (int b = 0; b < SB; b++)
                if (b < S) w[b] = fma(-q, cs[a][b], w[b]);
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
        if (FUSE && gpart) {
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
    if (!FUSE || !gpart) return;
    // per-CTA FP64 sum over threads: warp shuffles then shared memory, fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int w = 0; w < nw; w++) {
        int e = 0;
        for (int b = 0; b < S; b++)
            for (int c = 0; c <= b; c++, e++) {
                double v = (double)g2[e];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (warp == w && lane == 0) red[b * S + c] += v;
            }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        const int b = e / S, c = e % S;
        // symmetric S x S, column-major: G[b + c*S]
        gpart[(int64_t)blockIdx.x * S * S + b + c * S] = b >= c ? red[b * S + c] : red[c * S + b];
    }
}

// x[i] += sum_a V[i, a] y[a]  (correction in the basis precision, added to FP64 x)
template <typename T>
__global__ void xupdate_kernel(const T *V, int64_t ldv, int k, const double *y, int64_t n, double *x) {
    __shared__ T ys[MMAX + 1];
    for (int a = threadIdx.x; a < k; a += blockDim.x) ys[a] = (T)y[a];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T d = (T)0;
        for (int a = 0; a < k; a++) d = fma(V[(int64_t)a * ldv + i], ys[a], d);
        x[i] += (double)d;
    }
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
    double ritz[MMAX];
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

// Cholesky of an S x S SPD matrix A (col-major) into upper R with R^T R = A; Rinv = R^-1.
__device__ bool chol_inv(const double *A, int S, double *R, double *Rinv) {
    for (int e = 0; e < S * S; e++) { R[e] = 0.0; Rinv[e] = 0.0; }
    for (int i = 0; i < S; i++) {
        double d = A[i + i * S];
        for (int k = 0; k < i; k++) d -= R[k + i * S] * R[k + i * S];
        if (!(d > 0.0)) return false;
        const double rii = sqrt(d);
        R[i + i * S] = rii;
        for (int j = i + 1; j < S; j++) {
            double v = A[i + j * S];
            for (int k = 0; k < i; k++) v -= R[k + i * S] * R[k + j * S];
            R[i + j * S] = v / rii;
        }
    }
    // inverse of upper triangular R by columns
    for (int j = 0; j < S; j++) {
        Rinv[j + j * S] = 1.0 / R[j + j * S];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int k = i + 1; k <= j; k++) v += R[i + k * S] * Rinv[k + j * S];
            Rinv[i + j * S] = -v / R[i + i * S];
        }
    }
    return true;
}

// Small steps of the block orthogonalisation:
//   mode 0: C  = G (K1 x S, from G = Q^T W); Rinv = I  (projection coefficients)
//   mode 2: C2 = G (second projection sweep);  Rinv = I
//   mode 1: R1 = chol(G) (S x S Gram of the projected block); Rinv = R1^-1
//   mode 3: R2 = chol(G) (CholQR's second pass);             Rinv = R2^-1
__global__ void chol_kernel(CycleState *cst, const double *G, int K1, int S, int mode) {
    if (threadIdx.x != 0) return;
    if (mode == 0 || mode == 2) {
        double *Cd = mode == 0 ? cst->C : cst->C2;
        for (int e = 0; e < K1 * S; e++) Cd[e] = G[e];
        for (int e = 0; e < S * S; e++) cst->Rinv[e] = (e % S == e / S) ? 1.0 : 0.0;
        return;
    }
    double *R = mode == 1 ? cst->R1 : cst->R2;
    if (!chol_inv(G, S, R, cst->Rinv)) cst->status = 1;
}

// Hessenberg columns j..j+S-1 from R_full (C, R), shifts theta and the previous Arnoldi H;
// Givens rotations; convergence check against tol_abs.
// passes == 2: C_total = C1 + C2 R1, R_total = R2 R1 ; else C_total = C1, R_total = R2 R1.
__global__ void hess_kernel(CycleState *cst, int j, int S, const double *theta, double tol_abs, int m) {
    if (threadIdx.x != 0) return;
    if (cst->status) return;
    const int K1 = j + 1;
    const int ldh = MMAX + 1;
    double *C = cst->Ct, *R = cst->Rt;
    for (int e = 0; e < S * S; e++) R[e] = 0.0;
    for (int c = 0; c < S; c++)
        for (int a = 0; a <= c; a++) {
            double v = 0.0;
            for (int k = a; k <= c; k++) v += cst->R2[a + k * S] * cst->R1[k + c * S];
            R[a + c * S] = v;
        }
    // W = Q (C + C2) + Q_new R2 R1  (C2: second projection sweep, when taken)
    for (int b = 0; b < S; b++)
        for (int a = 0; a < K1; a++) {
            double v = cst->C[a + b * K1];
            if (cst->nrm[3] > 0.5) v += cst->C2[a + b * K1];
            C[a + b * K1] = v;
        }
    // R_full: (K1 + S) x (S + 1), column 0 = e_j, columns 1..S = [C ; R]
    const int NR = K1 + S;
    double *RF = cst->RF;
    for (int e = 0; e < NR * (S + 1); e++) RF[e] = 0.0;
    RF[j + 0 * NR] = 1.0;
    for (int b = 0; b < S; b++) {
        for (int a = 0; a < K1; a++) RF[a + (b + 1) * NR] = C[a + b * K1];
        for (int a = 0; a < S; a++) RF[K1 + a + (b + 1) * NR] = R[a + b * S];
    }
    // rhs = R_full * Bm - H_prev[:, 0:j] * R_s[0:j, :],   Bm: (S+1) x S, theta on the
    // diagonal, ones below
    double *RHS = cst->RHS;
    for (int c = 0; c < S; c++)
        for (int a = 0; a < NR; a++) {
            double v = RF[a + c * NR] * theta[c] + RF[a + (c + 1) * NR];
            for (int q = 0; q < j; q++) v -= cst->H[a + q * ldh] * RF[q + c * NR];
            RHS[a + c * NR] = v;
        }
    // T = R_s[j:j+S, 0:S] upper triangular; H_new = RHS T^-1 (solve from the right, by columns)
    double *Hn = cst->Hn;
    for (int c = 0; c < S; c++) {
        const double tcc = RF[(j + c) + c * NR];
        for (int a = 0; a < NR; a++) {
            double v = RHS[a + c * NR];
            for (int q = 0; q < c; q++) v -= Hn[a + q * NR] * RF[(j + q) + c * NR];
            Hn[a + c * NR] = v / tcc;
        }
        for (int a = j + c + 2; a < NR; a++) Hn[a + c * NR] = 0.0;   // Hessenberg structure
    }
    // store into H (unrotated) and Hr, then rotate the new columns
    for (int c = 0; c < S; c++)
        for (int a = 0; a < NR && a <= MMAX; a++) {
            cst->H[a + (j + c) * ldh] = Hn[a + c * NR];
            cst->Hr[a + (j + c) * ldh] = Hn[a + c * NR];
        }
    for (int c = j; c < j + S; c++) {
        double *h = cst->Hr + c * ldh;
        for (int i = 0; i < c; i++) {
            const double t = cst->cs[i] * h[i] + cst->sn[i] * h[i + 1];
            h[i + 1] = -cst->sn[i] * h[i] + cst->cs[i] * h[i + 1];
            h[i] = t;
        }
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
        if (fabs(cst->g[c + 1]) <= tol_abs) {
            cst->conv_k = c + 1;
            break;
        }
    }
    (void)m;
}

// y = Hr[0:k, 0:k]^-1 g[0:k] (back substitution)
__global__ void lsq_kernel(CycleState *cst, int k) {
    if (threadIdx.x != 0) return;
    const int ldh = MMAX + 1;
    for (int i = k - 1; i >= 0; i--) {
        double v = cst->g[i];
        for (int q = i + 1; q < k; q++) v -= cst->Hr[i + q * ldh] * cst->y[q];
        cst->y[i] = v / cst->Hr[i + i * ldh];
    }
}

// Ritz values: eigenvalues of the symmetric part of the leading k x k Arnoldi H by cyclic
// Jacobi rotations (for a symmetric A the Arnoldi H is symmetric tridiagonal up to rounding,
// so these are its Ritz values; for an unsymmetric A they are real values from its field of
// values).
__global__ void ritz_kernel(CycleState *cst, int k) {
    if (threadIdx.x != 0) return;
    const int ldh = MMAX + 1;
    double *A = cst->Hr;   // reuse as scratch after the cycle (ld ldh)
    for (int c = 0; c < k; c++)
        for (int r = 0; r < k; r++) A[r + c * ldh] = 0.5 * (cst->H[r + c * ldh] + cst->H[c + r * ldh]);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int c = 0; c < k; c++)
            for (int r = 0; r < c; r++) off += A[r + c * ldh] * A[r + c * ldh];
        if (off < 1e-30) break;
        for (int p = 0; p < k - 1; p++)
            for (int q = p + 1; q < k; q++) {
                const double apq = A[p + q * ldh];
                if (fabs(apq) < 1e-300) continue;
                const double app = A[p + p * ldh], aqq = A[q + q * ldh];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int r = 0; r < k; r++) {   // columns p, q
                    const double arp = A[r + p * ldh], arq = A[r + q * ldh];
                    A[r + p * ldh] = c * arp - s * arq;
                    A[r + q * ldh] = s * arp + c * arq;
                }
                for (int r = 0; r < k; r++) {   // rows p, q
                    const double apr = A[p + r * ldh], aqr = A[q + r * ldh];
                    A[p + r * ldh] = c * apr - s * aqr;
                    A[q + r * ldh] = s * apr + c * aqr;
                }
            }
    }
    for (int i = 0; i < k; i++) cst->ritz[i] = A[i + i * ldh];
}

__global__ void cycle_init_kernel(CycleState *cst, const double *beta) {
    if (threadIdx.x != 0) return;
    cst->status = 0;
    cst->conv_k = 0;
    cst->kdone = 0;
    cst->g[0] = *beta;
    cst->est = *beta;
    for (int i = 1; i <= MMAX; i++) cst->g[i] = 0.0;
    cst->nrm[3] = 0.0;
}
__global__ void set_flag_kernel(CycleState *cst, double v) {
    if (threadIdx.x == 0) cst->nrm[3] = v;
}

// ------------------------------------------------------------------------------------------
// Host driver
// ------------------------------------------------------------------------------------------
struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    double total = 0.0;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, s); }
    void stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        total += ms;
    }
};

template <typename T>
struct Solver {
    mpk_plan_s *P;
    cudaStream_t st;
    mpk_gmres_opts o;
    int64_t n, ldv;
    DevBuf V, part, G, gpart2, cstate, vec;   // vec: b, x, r, norms (FP64)
    double *bp, *xp, *rp, *nrm;
    CycleState *cst;
    int gram_grid, upd_grid;
    Timer t_mpk, t_ortho, t_other;
    std::vector<double> theta;
    int s_cur;
    mpk_gmres_info info{};

    Solver(mpk_plan_s *p, cudaStream_t s_) : P(p), st(s_), t_mpk(s_), t_ortho(s_), t_other(s_) {}

    mpk_status alloc() {
        n = P->n;
        ldv = (n + 31) / 32 * 32;
        const int m = o.restart;
        MPK_TRY(V.alloc((size_t)(m + 1) * ldv * sizeof(T)));
        gram_grid = 2 * P->n_sm;
        upd_grid = 4 * P->n_sm;
        const int maxK = m + 1 + SMAX;
        MPK_TRY(part.alloc((size_t)std::max(gram_grid, upd_grid) * maxK * SMAX * sizeof(double) + 4096));
        MPK_TRY(G.alloc((size_t)maxK * SMAX * sizeof(double) + 64));
        MPK_TRY(gpart2.alloc((size_t)upd_grid * SMAX * SMAX * sizeof(double) + 64));
        MPK_TRY(cstate.alloc(sizeof(CycleState)));
        MPK_TRY(vec.alloc((size_t)3 * ldv * sizeof(double) + 64 * sizeof(double)));
        bp = vec.as<double>();
        xp = bp + ldv;
        rp = xp + ldv;
        nrm = rp + ldv;
        cst = cstate.as<CycleState>();
        MPK_CUDA(cudaMemsetAsync(cstate.p, 0, sizeof(CycleState), st));
        return MPK_OK;
    }

    T *col(int a) { return V.as<T>() + (int64_t)a * ldv; }

    mpk_status norm2(const double *v, double *out) {
        const unsigned g = grid_rows(n);
        sumsq_partial_kernel<double><<<g, RED_BLOCK, 0, st>>>(v, n, part.as<double>());
        reduce_partials_kernel<<<1, 32, 0, st>>>(part.as<double>(), g, 1, 1, out, 1);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }

    // G (K x S) = X^T Y
    template <int SB> mpk_status gram_sb(const T *X, int K, const T *Y, int S, double *Gout) {
        const size_t sm = std::max((size_t)GR * (K + S) * sizeof(T), (size_t)K * S * sizeof(double));
        // one fixed maximum for every caller (the attribute is shared by all threads)
        constexpr int smax = (int)(GR * (MMAX + 1 + 2 * SMAX) * sizeof(T));
        if (sm > (size_t)smax) return MPK_ERR_ARG;
        MPK_CUDA(cudaFuncSetAttribute(gram_kernel<T, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        const int g = (int)std::min<int64_t>(gram_grid, ceil_div(n, GR));
        gram_kernel<T, SB><<<g, 256, sm, st>>>(X, ldv, K, Y, ldv, S, n, part.as<double>());
        reduce_partials_kernel<<<1, 256, 0, st>>>(part.as<double>(), g, K * S, (int64_t)K * S, Gout, 0);
        MPK_CUDA(cudaGetLastError());
        return MPK_OK;
    }
    mpk_status gram(const T *X, int K, const T *Y, int S, double *Gout) {
        if (S <= 4) return gram_sb<4>(X, K, Y, S, Gout);
        if (S <= 8) return gram_sb<8>(X, K, Y, S, Gout);
        return gram_sb<16>(X, K, Y, S, Gout);
    }
    mpk_status update(const T *Q, int K1, T *W, int S, const double *C, const double *Ri, double *gp) {
        const int ug = (int)std::min<int64_t>(upd_grid, ceil_div(n, 256));
        if (S <= 4) update_kernel<T, 4><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
        else if (S <= 8) update_kernel<T, 8><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
        else update_kernel<T, 16><<<ug, 256, 0, st>>>(Q, ldv, K1, W, ldv, S, C, Ri, n, gp);
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
        const int ug = (int)std::min<int64_t>(upd_grid, ceil_div(n, 256));
        auto update_gram = [&](int k1, const double *C) -> mpk_status {
            if (S <= 8) {
                MPK_TRY(update(Q, k1, W, S, C, cst->Rinv, gpart2.as<double>()));
                reduce_partials_kernel<<<1, 256, 0, st>>>(gpart2.as<double>(), ug, S * S, (int64_t)S * S, Gd, 0);
            } else {
                MPK_TRY(update(Q, k1, W, S, C, cst->Rinv, nullptr));
                MPK_TRY(gram(W, S, W, S, Gd));
            }
            return MPK_OK;
        };
        MPK_TRY(gram(Q, K1, W, S, Gd));
        chol_kernel<<<1, 32, 0, st>>>(cst, Gd, K1, S, 0);
        if (o.bcgs_passes >= 2) {
            MPK_TRY(update(Q, K1, W, S, cst->C, cst->Rinv, nullptr));
            MPK_TRY(gram(Q, K1, W, S, Gd));
            chol_kernel<<<1, 32, 0, st>>>(cst, Gd, K1, S, 2);
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

    mpk_status mpk_block(int j, int S, bool newton) {
        std::vector<double> a(S, 1.0), b(S, 0.0), c(S, 0.0);
        if (newton)
            for (int k = 0; k < S; k++) b[k] = -theta[k];
        mpk_coeffs co{S, a.data(), b.data(), c.data(), nullptr};
        const mpk_dtype dt = sizeof(T) == 8 ? MPK_F64 : MPK_F32;
        const uint32_t fl = MPK_PERMUTED_IO | MPK_Y0_IS_X | (o.mpk_flags & MPK_UNBLOCKED);
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
        cycle_init_kernel<<<1, 32, 0, st>>>(cst, nrm);
        MPK_CUDA(cudaGetLastError());
        std::vector<double> th(s, 0.0);
        if (newton)
            for (int k = 0; k < s; k++) th[k] = theta[k];
        DevBuf dth;
        MPK_TRY(dth.alloc(SMAX * sizeof(double)));
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
            hess_kernel<<<1, 32, 0, st>>>(cst, j, S, dth.as<double>(), tol_abs, m);
            MPK_CUDA(cudaGetLastError());
            t_ortho.stop();
            int hs[3];
            MPK_CUDA(cudaMemcpyAsync(hs, &cst->status, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
            MPK_CUDA(cudaStreamSynchronize(st));
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
            lsq_kernel<<<1, 32, 0, st>>>(cst, k);
            xupdate_kernel<T><<<grid_rows(n, 8), 256, 0, st>>>(V.as<T>(), ldv, k, cst->y, n, xp);
            MPK_CUDA(cudaGetLastError());
            t_other.stop();
        }
        if (!newton && k > 0) {
            ritz_kernel<<<1, 32, 0, st>>>(cst, k);
            std::vector<double> rz(k);
            MPK_CUDA(cudaMemcpyAsync(rz.data(), cst->ritz, k * sizeof(double), cudaMemcpyDeviceToHost, st));
            MPK_CUDA(cudaStreamSynchronize(st));
            theta.assign(o.s, 0.0);
            mpk_leja_order(rz.data(), k, o.s, theta.data());
        }
        *k_used = k;
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
        const bool need_shifts = !o.shifts;
        bool have_shifts = !need_shifts;
        mpk_status result = MPK_ERR_NOT_CONVERGED;
        double relres = 1.0;
        for (int outer = 0; outer <= o.max_outer; outer++) {
            t_other.start();
            MPK_TRY(mpk_launch_residual(P, xp, bp, rp, st));
            norm2(rp, nrm + 2);
            double hr = 0.0;
            MPK_CUDA(cudaMemcpyAsync(&hr, nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            MPK_CUDA(cudaStreamSynchronize(st));
            t_other.stop();
            relres = hb > 0 ? hr / hb : 0.0;
            info.outer = outer;
            if (relres <= o.tol || hb == 0.0) {
                result = MPK_OK;
                break;
            }
            if (outer == o.max_outer || info.iters >= o.max_iters) break;
            if (!std::isfinite(hr)) break;
            // one restart cycle on A d = r; target: inner_tol relative to ||r|| in the basis
            // precision, never tighter than the overall target
            double tol_abs = std::max(o.inner_tol * hr, 0.5 * o.tol * hb);
            if (sizeof(T) == 8) tol_abs = 0.5 * o.tol * hb;
            int k = 0;
            bool bd = false;
            if (!have_shifts) {
                MPK_TRY(cycle(tol_abs, false, 1, &k, &bd));
                have_shifts = true;
            } else {
                MPK_TRY(cycle(tol_abs, true, s_cur, &k, &bd));
                if (bd) {
                    if (s_cur == 1) { result = MPK_ERR_BREAKDOWN; break; }
                    s_cur = std::max(1, s_cur / 2);   // recorded in info via restarts
                }
            }
            info.iters += k;
            info.restarts++;
            if (k == 0 && !bd) break;
        }
        scatter_f64_kernel<<<g, 256, 0, st>>>(xp, perm, n, x);
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaStreamSynchronize(st));
        info.rel_residual = relres;
        info.status = result;
        for (size_t i = 0; i < theta.size() && i < 64; i++) info.shifts[i] = theta[i];
        info.ms_mpk = t_mpk.total;
        info.ms_ortho = t_ortho.total;
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
    o->max_outer = 50;
    o->inner_cycles = 1;
    o->max_iters = 100000;
    o->basis = MPK_F32;
    o->bcgs_passes = 1;
    o->shifts = nullptr;
    o->mpk_flags = 0;
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
        o.bcgs_passes < 1 || o.bcgs_passes > 2 || o.max_outer < 0)
        return MPK_ERR_ARG;
    if (!A->has64) return MPK_ERR_ARG;                       // FP64 residual needs FP64 values
    if (o.basis == MPK_F32 && !A->has32) return MPK_ERR_ARG;
    if (o.s > A->p_max) return MPK_ERR_ARG;
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
