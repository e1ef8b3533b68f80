// FMA-rate microbenchmark: the arithmetic roofline the measurement reports a kernel against
// when its bound is instruction issue, not memory.  The paper measures its CPUs' bandwidth
// with a copy benchmark and compares the MPK with the SpMV roofline (Sec. 6); on GB300 the
// FP64 MPK is bound by the FP64 FMA rate, which this measures on the device at run time.
#include <algorithm>

#include "mpk_internal.cuh"

namespace {

constexpr int FMA_CHAINS = 8;      // independent FMA chains per thread
constexpr int FMA_BLOCK = 256;

// Every thread runs FMA_CHAINS independent chains x <- x a + b for `iters` steps (a < 1, so the
// values stay bounded); the chains' sum is stored only if it takes an impossible value, which
// keeps the compiler from dropping the work without a store per thread.
template <typename T>
__global__ void __launch_bounds__(FMA_BLOCK) fma_rate_kernel(T *out, int iters, T a, T b) {
    T x[FMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; i++) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < FMA_CHAINS; i++) x[i] = fma(x[i], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; i++) s += x[i];
    if (s == (T)-1) out[blockIdx.x] = s;
}

template <typename T>
mpk_status fma_rate(double *tflops, cudaStream_t s) {
    int dev = 0, nsm = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fma_rate_kernel<T>, FMA_BLOCK, 0));
    const int grid = nsm * std::max(1, occ);
    // about 20 ms per launch at the nominal rates (FP32 128, FP64 2 FMA/clk/SM at 2 GHz)
    const int iters = sizeof(T) == 8 ? 8192 : 262144;
    DevBuf out;
    MPK_TRY(out.alloc_on((size_t)grid * sizeof(T), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MPK_CUDA(cudaEventCreate(&e0));
    MPK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    mpk_status st = MPK_OK;
    for (int rep = 0; rep < 4 && st == MPK_OK; rep++) {   // the first launch warms up
        if (cudaEventRecord(e0, s) != cudaSuccess) st = MPK_ERR_CUDA;
        fma_rate_kernel<T><<<grid, FMA_BLOCK, 0, s>>>(out.as<T>(), iters, (T)0.999999, (T)1e-7);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            st = MPK_ERR_CUDA;
        float ms = 0;
        if (st == MPK_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = MPK_ERR_CUDA;
        if (st == MPK_OK && rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MPK_TRY(st);
    const double fmas = (double)grid * FMA_BLOCK * FMA_CHAINS * (double)iters;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return MPK_OK;
}

}  // namespace

extern "C" mpk_status mpk_fma_peak(mpk_dtype dtype, double *tflops, cudaStream_t s) {
    if (!tflops) return MPK_ERR_ARG;
    if (dtype == MPK_F64) return fma_rate<double>(tflops, s);
    if (dtype == MPK_F32) return fma_rate<float>(tflops, s);
    return MPK_ERR_ARG;
}
