// Autotuner for one call shape: plan options (blocked or p x SpMV, blocked kernel, slack, lanes
// per row, task and chunk size, level-group budget) timed on the caller's matrix.  The paper picks its blocking depth p_opt
// and cache size C by hand per machine (Sec. 3, Sec. 4); on this part the best choice depends
// on precision and on the number of right-hand sides (FP64 is bound by FP64 FMA issue, FP32 by
// memory, wide blocks of right-hand sides by vector gathers), so it is measured.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mpk_internal.cuh"

namespace {

__global__ void fill_kernel(float *p32, double *p64, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (p32) p32[i] = (float)v;
        else p64[i] = v;
    }
}

// the candidate list: deterministic, the caller's base options first.  Axes: blocked or
// p x SpMV; the blocked kernel (lane tasks, warp tasks with a ticket dispenser); the lane
// tasks' slack (resident_warps: about one ticket per resident warp) and task size; the warp
// tasks' chunk size; the level-group budget.  Lanes per row stays the base's: it changes the
// summation order, and every candidate must give the base's values bit for bit.
std::vector<mpk_plan_opts> candidates(const mpk_plan_opts &base, int64_t l2, int64_t resident_warps) {
    std::vector<mpk_plan_opts> c;
    auto add = [&](int blocked, int kernel, int cs, int64_t budget, int64_t slack, int lanes, int units) {
        mpk_plan_opts o = base;
        o.blocked = blocked;
        o.kernel = kernel;
        if (cs > 0) o.chunk_slices = cs;
        if (budget > 0) o.l2_budget_bytes = budget;
        if (slack > 0) o.slack_tasks = (int32_t)slack;
        if (lanes > 0) o.lanes_per_row = lanes;
        if (units > 0) o.task_units = units;
        c.push_back(o);
    };
    c.push_back(base);
    add(0, base.kernel, 0, 0, 0, 0, 0);                        // p back-to-back SpMVs
    add(1, 4, 0, 0, 2 * resident_warps, 0, 0);                 // lane tasks, less slack
    add(1, 4, 0, 0, 4 * resident_warps, 0, 0);                 // lane tasks, more slack
    add(1, 4, 0, 0, 0, 0, 2);                                  // two slices per task
    add(1, 0, 4, 0, 0, 0, 0);                                  // warp tasks, 4-slice chunks
    add(1, 0, 8, 0, 0, 0, 0);                                  // warp tasks, 8-slice chunks
    add(1, 4, 0, l2 / 4, 0, 0, 0);                             // smaller level groups
    add(1, 4, 0, l2, 0, 0, 0);                                 // larger level groups
    return c;
}

}  // namespace

extern "C" mpk_status mpk_autotune(const mpk_csr *A, int32_t p, const mpk_coeffs *co, mpk_dtype dtype,
                                   int32_t n_rhs, uint32_t flags, const mpk_plan_opts *base,
                                   int32_t reps, mpk_plan_opts *best, mpk_tune_info *info,
                                   cudaStream_t s) {
    if (!A || !co || !best || co->p != p || p < 1 || p > MPK_MAX_P || n_rhs < 1 || n_rhs > 1024 ||
        reps < 1 || reps > 1000)
        return MPK_ERR_ARG;
    if (flags & (MPK_HOST_IO | MPK_Y0_IS_X | MPK_UNBLOCKED | MPK_DEBUG_DROP_FLAG)) return MPK_ERR_ARG;
    if (dtype != MPK_F32 && dtype != MPK_F64) return MPK_ERR_ARG;
    mpk_plan_opts b;
    if (base) b = *base;
    else mpk_plan_opts_default(&b);
    if (dtype == MPK_F32) b.keep_f32 = 1;
    if (dtype == MPK_F64) b.keep_f64 = 1;
    int dev = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    int l2 = 0;
    MPK_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const int64_t n = A->n;
    const size_t es = dtype == MPK_F64 ? 8 : 4;
    const int64_t nout = (flags & MPK_FINAL_ONLY) ? 1 : (int64_t)p + 1;
    DevBuf X, Y;
    MPK_TRY(X.alloc((size_t)std::max<int64_t>(n, 1) * n_rhs * es));
    MPK_TRY(Y.alloc((size_t)std::max<int64_t>(n, 1) * n_rhs * nout * es));
    int n_sm = 1;
    MPK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n * n_rhs, 256), (int64_t)n_sm * 8));
    fill_kernel<<<g, 256, 0, s>>>(dtype == MPK_F32 ? X.as<float>() : nullptr,
                                  dtype == MPK_F64 ? X.as<double>() : nullptr, n * n_rhs, 1.0);
    MPK_CUDA(cudaGetLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MPK_CUDA(cudaEventCreate(&e0));
    MPK_CUDA(cudaEventCreate(&e1));
    // the lane-task kernel keeps five CTAs of eight warps per SM resident
    const std::vector<mpk_plan_opts> cand = candidates(b, l2, (int64_t)n_sm * 40);
    double best_ms = 1e300, base_ms = 1e300;
    int best_i = -1, trials = 0;
    mpk_status st = MPK_OK;
    for (size_t i = 0; i < cand.size() && st == MPK_OK; i++) {
        mpk_plan_t plan = nullptr;
        st = mpk_plan_create(A, p, &cand[i], s, &plan);
        if (st != MPK_OK) break;
        std::vector<float> ts;
        // two untimed calls (schedule, automatic choice), then reps timed ones
        for (int r = 0; r < reps + 2 && st == MPK_OK; r++) {
            if (r >= 2 && cudaEventRecord(e0, s) != cudaSuccess) st = MPK_ERR_CUDA;
            if (st == MPK_OK)
                st = mpk_apply_internal(plan, co, dtype, X.p, n, Y.p, n, n_rhs, flags, s);
            if (st == MPK_OK && r >= 2) {
                float ms = 0;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    st = MPK_ERR_CUDA;
                ts.push_back(ms);
            }
        }
        if (st == MPK_OK) st = mpk_plan_sync(plan, s);
        mpk_plan_destroy(plan);
        if (st != MPK_OK) break;
        std::sort(ts.begin(), ts.end());
        const double med = ts[ts.size() / 2];
        trials++;
        if (i == 0) base_ms = med;
        if (med < best_ms) {
            best_ms = med;
            best_i = (int)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MPK_OK) {
        cudaGetLastError();
        return st;
    }
    *best = cand[best_i];
    if (info) {
        info->n_trials = trials;
        info->best_index = best_i;
        info->best_ms = best_ms;
        info->base_ms = base_ms;
    }
    return MPK_OK;
}
