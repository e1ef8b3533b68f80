// Serving: a continuously batched stream of s-step GMRES solves on one GPU.
//
// submit() copies a request (CSR + right-hand side) into host memory the server owns and
// queues it.  poll() drives the server: it collects finished requests, then admits queued
// ones in arrival order while a slot is free and the request's device-memory estimate fits
// the budget next to the requests already on the GPU.  Each slot owns a CUDA stream and a
// worker thread that uploads the matrix, builds the plan (or reuses an idle plan of the same
// sparsity pattern, replacing its values), runs sstep_gmres_solve, downloads x and frees what
// it allocated; solves in different slots overlap on the device.  Bases, Hessenbergs and all
// solver state stay on the device for the whole solve.
//
// Every kernel the solve uses reduces in a fixed order, so a request's result does not
// depend on what else runs at the same time.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mpk_internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    int64_t n = 0, nnz = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> val, b;
    double *x_out = nullptr;
    int64_t est_bytes = 0;
    uint64_t pattern = 0;
    mpk_server_result res{};
    std::vector<double> x;
};

struct CachedPlan {
    uint64_t pattern;
    int64_t n, nnz;
    mpk_plan_t plan;
    int64_t bytes;
    // the pattern itself (host): a matching hash is confirmed entry by entry before reuse
    std::shared_ptr<const std::vector<int32_t>> rp, ci;
};

uint64_t hash_pattern(const std::vector<int32_t> &rp, const std::vector<int32_t> &ci) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix(rp.size());
    for (int32_t v : rp) mix((uint32_t)v);
    for (int32_t v : ci) mix((uint32_t)v);
    return h;
}

}  // namespace

struct mpk_server_s {
    mpk_server_opts o{};
    int device = 0;
    clk::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Request>> queue;              // waiting for admission
    std::vector<std::unique_ptr<Request>> done;              // finished, not yet reported
    int64_t next_id = 1;
    int64_t used_bytes = 0;                                  // admitted requests + idle plans
    int64_t in_flight = 0;
    std::list<CachedPlan> idle_plans;                        // reusable plans (LRU order)
    int64_t idle_bytes = 0;
    struct Slot {
        std::thread th;
        cudaStream_t stream = nullptr;
        std::unique_ptr<Request> job;
        bool busy = false;
    };
    std::vector<Slot> slots;
    bool stop = false;

    double now_ms() const { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); }

    // device bytes a request needs: input CSR (FP64), plan (permuted CSR in FP64 and FP32,
    // SELL copies (with padding counted as a second copy), level arrays, a p_max-deep schedule) and the solver (basis of m+1 columns in
    // the basis precision, FP64 vectors and partial sums)
    int64_t estimate(int64_t n, int64_t nnz) const {
        const int64_t m = o.gmres.restart;
        const int64_t wb = o.gmres.basis == MPK_F64 ? 8 : 4;
        const int64_t csr_in = 12 * nnz + 4 * (n + 1);
        // Jacobi scaling adds a second SELL value copy per precision and D^-1; GS2 also the
        // lower-entry mask, two inner-iterate vectors and three FP64 correction vectors
        const bool scaled = o.gmres.jacobi || o.gmres.gs2;
        const int64_t jac = (scaled ? 2 * (8 + 4) * nnz + 8 * n : 0) + (o.gmres.gs2 ? nnz / 8 + 48 * n : 0);
        const int64_t plan = 2 * (12 * nnz) + 2 * 8 * nnz + 64 * n + (8 << 20) + jac;
        const int64_t solver = (m + 1) * wb * ((n + 31) / 32 * 32) + 24 * n + (16 << 20);
        return csr_in + plan + solver;
    }

    mpk_status acquire_plan(Request &r, cudaStream_t s, const int32_t *drp, const int32_t *dci,
                            const double *dval, mpk_plan_t *out, int64_t *plan_bytes) {
        // reuse an idle plan of the same pattern: only the values change
        {
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = idle_plans.begin(); it != idle_plans.end(); ++it) {
                if (it->pattern == r.pattern && it->n == r.n && it->nnz == r.nnz && *it->rp == r.rp &&
                    *it->ci == r.ci) {
                    *out = it->plan;
                    *plan_bytes = it->bytes;
                    idle_bytes -= it->bytes;
                    idle_plans.erase(it);
                    mpk_csr A{r.n, r.nnz, drp, dci, dval, MPK_F64};
                    return mpk_plan_update_values(*out, &A, s);
                }
            }
        }
        mpk_plan_opts po;
        mpk_plan_opts_default(&po);
        po.keep_f64 = 1;
        po.keep_f32 = o.gmres.basis == MPK_F32 ? 1 : 0;
        po.jacobi = (o.gmres.jacobi || o.gmres.gs2) ? 1 : 0;
        mpk_csr A{r.n, r.nnz, drp, dci, dval, MPK_F64};
        MPK_TRY(mpk_plan_create(&A, std::max(o.gmres.s, 1), &po, s, out));
        mpk_plan_info pi;
        mpk_plan_stats(*out, &pi);
        *plan_bytes = pi.device_bytes;
        return MPK_OK;
    }

    void run_job(Slot &sl) {
        Request &r = *sl.job;
        cudaSetDevice(device);
        cudaStream_t s = sl.stream;
        r.res.t_start_ms = now_ms();
        mpk_status st = MPK_OK;
        DevBuf rp, ci, val, b, x;
        mpk_plan_t plan = nullptr;
        int64_t plan_bytes = 0;
        do {
            if ((st = rp.alloc_on((r.n + 1) * 4, s)) != MPK_OK) break;
            if ((st = ci.alloc_on(std::max<int64_t>(r.nnz, 1) * 4, s)) != MPK_OK) break;
            if ((st = val.alloc_on(std::max<int64_t>(r.nnz, 1) * 8, s)) != MPK_OK) break;
            if ((st = b.alloc_on(std::max<int64_t>(r.n, 1) * 8, s)) != MPK_OK) break;
            if ((st = x.alloc_on(std::max<int64_t>(r.n, 1) * 8, s)) != MPK_OK) break;
            cudaMemcpyAsync(rp.p, r.rp.data(), (r.n + 1) * 4, cudaMemcpyHostToDevice, s);
            if (r.nnz) {
                cudaMemcpyAsync(ci.p, r.ci.data(), r.nnz * 4, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(val.p, r.val.data(), r.nnz * 8, cudaMemcpyHostToDevice, s);
            }
            if (r.n) {
                cudaMemcpyAsync(b.p, r.b.data(), r.n * 8, cudaMemcpyHostToDevice, s);
                cudaMemsetAsync(x.p, 0, r.n * 8, s);
            }
            if ((st = acquire_plan(r, s, rp.as<int32_t>(), ci.as<int32_t>(), val.as<double>(), &plan, &plan_bytes)) != MPK_OK)
                break;
            mpk_gmres_info info{};
            st = sstep_gmres_solve(plan, b.as<double>(), x.as<double>(), &o.gmres, &info, s);
            r.res.iters = info.iters;
            r.res.outer = info.outer;
            r.res.rel_residual = info.rel_residual;
            r.x.resize(r.n);
            if (r.n) cudaMemcpyAsync(r.x.data(), x.p, r.n * 8, cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) st = MPK_ERR_CUDA;
        } while (false);
        cudaStreamSynchronize(s);
        r.res.status = st;
        r.res.t_done_ms = now_ms();
        // keep the plan for a later request with the same pattern, within the budget
        std::lock_guard<std::mutex> lk(mu);
        used_bytes -= r.est_bytes;
        if (plan) {
            if (st == MPK_OK && used_bytes + idle_bytes + plan_bytes <= o.hbm_budget_bytes) {
                idle_plans.push_back(CachedPlan{r.pattern, r.n, r.nnz, plan, plan_bytes,
                                                std::make_shared<const std::vector<int32_t>>(r.rp),
                                                std::make_shared<const std::vector<int32_t>>(r.ci)});
                idle_bytes += plan_bytes;
            } else {
                mpk_plan_destroy(plan);
            }
        }
        in_flight--;
        done.push_back(std::move(sl.job));
        sl.busy = false;
    }

    void worker(int k) {
        cudaSetDevice(device);
        Slot &sl = slots[k];
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv.wait(lk, [&] { return stop || (sl.busy && sl.job); });
            if (stop) return;
            lk.unlock();
            run_job(sl);
            lk.lock();
        }
    }

    // admit queued requests in arrival order while a slot is free and the memory fits; idle
    // cached plans are released first when memory is short
    void admit() {
        std::lock_guard<std::mutex> lk(mu);
        while (!queue.empty()) {
            Request &r = *queue.front();
            int free_slot = -1;
            for (size_t k = 0; k < slots.size(); k++)
                if (!slots[k].busy) { free_slot = (int)k; break; }
            if (free_slot < 0) return;
            while (used_bytes + idle_bytes + r.est_bytes > o.hbm_budget_bytes && !idle_plans.empty()) {
                mpk_plan_destroy(idle_plans.front().plan);
                idle_bytes -= idle_plans.front().bytes;
                idle_plans.pop_front();
            }
            if (used_bytes + idle_bytes + r.est_bytes > o.hbm_budget_bytes) return;   // wait
            used_bytes += r.est_bytes;
            in_flight++;
            Slot &sl = slots[free_slot];
            sl.job = std::move(queue.front());
            queue.pop_front();
            sl.busy = true;
            cv.notify_all();
        }
    }
};

extern "C" mpk_status mpk_server_opts_default(mpk_server_opts *o) {
    if (!o) return MPK_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 120ll << 30;
    o->max_active = 4;
    o->n_streams = 4;
    return mpk_gmres_opts_default(&o->gmres);
}

extern "C" mpk_status mpk_server_create(const mpk_server_opts *o, mpk_server_t *out) {
    if (!out) return MPK_ERR_ARG;
    *out = nullptr;
    mpk_server_opts opts;
    if (o) opts = *o;
    else mpk_server_opts_default(&opts);
    if (opts.max_active < 1 || opts.max_active > 64 || opts.hbm_budget_bytes <= 0) return MPK_ERR_ARG;
    auto *S = new (std::nothrow) mpk_server_s();
    if (!S) return MPK_ERR_OOM;
    S->o = opts;
    S->t0 = clk::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return MPK_ERR_CUDA;
    }
    S->slots.resize(opts.max_active);
    for (int k = 0; k < opts.max_active; k++) {
        if (cudaStreamCreateWithFlags(&S->slots[k].stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (int q = 0; q < k; q++) cudaStreamDestroy(S->slots[q].stream);
            delete S;
            return MPK_ERR_CUDA;
        }
    }
    for (int k = 0; k < opts.max_active; k++) S->slots[k].th = std::thread(&mpk_server_s::worker, S, k);
    *out = S;
    return MPK_OK;
}

extern "C" mpk_status mpk_server_submit(mpk_server_t S, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                        const int32_t *col, const double *val, const double *b,
                                        double *x_out, int64_t *id) {
    if (!S || n < 0 || nnz < 0 || !row_ptr || (nnz && (!col || !val)) || (n && (!b || !x_out)) || !id)
        return MPK_ERR_ARG;
    if (row_ptr[0] != 0 || row_ptr[n] != nnz) return MPK_ERR_ARG;
    std::unique_ptr<Request> r(new Request());
    r->n = n;
    r->nnz = nnz;
    r->est_bytes = S->estimate(n, nnz);
    if (r->est_bytes > S->o.hbm_budget_bytes) return MPK_ERR_BUDGET;
    r->rp.assign(row_ptr, row_ptr + n + 1);
    r->ci.assign(col, col + nnz);
    r->val.assign(val, val + nnz);
    r->b.assign(b, b + n);
    r->x_out = x_out;
    r->pattern = hash_pattern(r->rp, r->ci);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->res.id = r->id;
        r->res.t_submit_ms = S->now_ms();
        *id = r->id;
        S->queue.push_back(std::move(r));
    }
    S->admit();
    return MPK_OK;
}

extern "C" mpk_status mpk_server_poll(mpk_server_t S, mpk_server_result *out, int32_t max_results,
                                      int32_t *n_out) {
    if (!S || !n_out || max_results < 0 || (max_results && !out)) return MPK_ERR_ARG;
    S->admit();
    std::vector<std::unique_ptr<Request>> fin;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const int32_t k = (int32_t)std::min<size_t>(max_results, S->done.size());
        for (int32_t i = 0; i < k; i++) fin.push_back(std::move(S->done[i]));
        S->done.erase(S->done.begin(), S->done.begin() + k);
    }
    for (size_t i = 0; i < fin.size(); i++) {
        Request &r = *fin[i];
        if (r.n && r.x.size() == (size_t)r.n) memcpy(r.x_out, r.x.data(), r.n * 8);
        out[i] = r.res;
    }
    *n_out = (int32_t)fin.size();
    S->admit();
    return MPK_OK;
}

extern "C" mpk_status mpk_server_pending(mpk_server_t S, int64_t *n_pending) {
    if (!S || !n_pending) return MPK_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *n_pending = (int64_t)S->queue.size() + S->in_flight + (int64_t)S->done.size();
    return MPK_OK;
}

extern "C" mpk_status mpk_server_destroy(mpk_server_t S) {
    if (!S) return MPK_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    // workers finish the job they are running (a solve is not interrupted), then exit
    for (auto &sl : S->slots)
        if (sl.th.joinable()) sl.th.join();
    for (auto &sl : S->slots) cudaStreamDestroy(sl.stream);
    for (auto &cp : S->idle_plans) mpk_plan_destroy(cp.plan);
    delete S;
    return MPK_OK;
}
