"""Benchmark: level-blocked MPK vs p back-to-back SpMVs on one GB300 (per GPU).

Workload (the 27-point benchmark matrix): 3-D 27-point stencil on a 160^3 grid, n = 4,096,000,
nnz = 109,215,352, diagonal 26, off-diagonals -1 - U[0,0.1) (seed 2, symmetric), CSR FP64;
MPK in the Newton basis, shifts = the first p Leja points of [0, 52] (10,001 candidates);
x ~ U[-1,1) (seed 0).  One step = one mpk_apply call with p = 4 (inputs in HBM, original row
order in and out, all p+1 vectors written).  GFLOP/s = 2 * nnz * p / t (the paper's formula).
The matrix (1.33 GB) is larger than L2, so every step streams it from HBM.

Also reported: p = 2 and 8, the unblocked p x SpMV on the same GPU, the same matrix in FP32,
kernel-only timings with the roofline of the dominant kernel, an end-to-end number through the
C ABI with pinned host buffers, the CPU oracle on the host cores, and GPU clocks sampled
during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs its own replica (no data-path exchange exists in this
path on one GPU); value = total GFLOP over all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mpk_inputs as mi  # noqa: E402

METRIC = "MPK GFLOP/s blocked vs p×SpMV; solves/s + p99 latency at rel. residual 1e-8"
N_GRID = 160
P_MAIN = 4
P_SWEEP = (2, 4, 8)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic of the dominant kernel: a committed ncu summary records, per kernel and call,
# dram__bytes_read.sum + dram__bytes_write.sum per launch and the SHA-256 of the kernel's
# source file when it was captured.  The bench reports the figure only while the source is
# unchanged, and null (with the reason) once the kernel has changed since the capture.
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "lane_kernel_f64_p4_27pt160_dram.md")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2309_02228_gb300", "csrc", "apply.cu")


def source_sha(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(path=TRAFFIC_PROFILE):
    """(bytes per launch, note) from the committed capture, or (None, why)."""
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_launch:"):
                    rec["bytes"] = float(line.split(":", 1)[1])
                elif line.startswith("source_sha256_16:"):
                    rec["sha"] = line.split(":", 1)[1].strip()
        if "bytes" not in rec or "sha" not in rec:
            return None, "no capture recorded in %s" % os.path.relpath(path, ROOT)
        now = source_sha(KERNEL_SOURCE)
        if now != rec["sha"]:
            return None, "stale: kernel source changed since the capture (%s, now %s)" % (rec["sha"], now)
        return rec["bytes"], ("ncu capture of one launch of the default plan on this matrix and call "
                              "(one slice per task), %s" % os.path.relpath(path, ROOT))
    except OSError as e:
        return None, "no capture: %s" % e


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thr.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def gen_workload():
    A = mi.stencil27(N_GRID, seed=2)
    x = mi.uniform_vectors(A.n, 0)[0]
    theta = mi.leja_points_interval(0.0, 52.0, max(P_SWEEP))
    return A, x, theta


def max_over_ranks(ms, world, device):
    """The slowest rank's time per step (every rank runs its own replica; no data-path
    exchange exists on one GPU's path): an all-reduce MAX over the process group, or ms
    itself on one rank."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flop_per_rank, world, ms_step):
    """Whole-job throughput: the GFLOP all ranks did in one step over the slowest rank's time."""
    return world * flop_per_rank / (ms_step * 1e-3) / 1e9


def cpu_baseline(A, x, theta, budget_s=8.0, budget_1core_s=6.0):
    """The oracle as it stands (plain FP64 CSR loops) on the host cores: full 27-point matrix,
    p = 4 Newton, repeated until about budget_s seconds with a static OpenMP row loop on all
    cores, and until about budget_1core_s seconds on one core."""
    import oracle
    from oracle import sstep
    oracle.build()
    cf = sstep.newton_coeffs(theta[:P_MAIN])

    def run(threads, budget):
        reps, t_total = 0, 0.0
        while t_total < budget or reps == 0:
            t0 = time.perf_counter()
            oracle.mpk(A, P_MAIN, cf, x, threads=threads)
            t_total += time.perf_counter() - t0
            reps += 1
            if reps >= 1000:
                break
        return 2.0 * A.nnz * P_MAIN * reps / t_total / 1e9, reps, t_total

    gf, reps, t_total = run(True, budget_s)
    gf1, reps1, t1 = run(False, budget_1core_s)
    return {"value": gf, "unit": "GFLOP/s", "cores": oracle.omp_threads(), "kind": "oracle",
            "sample": "full 160^3 27-point FP64 matrix, p=4 Newton, %d calls in %.1f s" % (reps, t_total),
            "seconds": t_total, "cpu_model": cpu_model(),
            "one_core": {"value": gf1, "unit": "GFLOP/s", "cores": 1,
                         "sample": "the same call, %d calls in %.1f s" % (reps1, t1)}}


def headline_config(n, nnz):
    """The headline workload, shared by both arms' JSON lines."""
    return {"workload": "27-point 160^3 CSR FP64 (diag 26, off-diag -1-U[0,0.1) seed 2), "
                        "Newton MPK p=4 with Leja shifts on [0,52], original-order I/O",
            "n": n, "nnz": nnz, "p": P_MAIN, "parallelism": "replica per GPU",
            "l2_policy": "inputs larger than L2 (1.33 GB matrix)"}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores for the same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, x, theta = gen_workload()
    import oracle
    from oracle import sstep
    oracle.build()
    cf = sstep.newton_coeffs(theta[:P_MAIN])
    for _ in range(args.warmup):
        oracle.mpk(A, P_MAIN, cf, x, threads=True)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.mpk(A, P_MAIN, cf, x, threads=True)
        ts.append(time.perf_counter() - t0)
    t = sum(ts)
    gf = 2.0 * A.nnz * P_MAIN * args.steps / t / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": gf, "unit": "GFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": dict(headline_config(A.n, A.nnz), plan="oracle: plain CSR rows, OpenMP static"),
           "cpu_baseline": {"value": gf, "unit": "GFLOP/s", "kind": "oracle",
                            "cores": oracle.omp_threads(),
                            "sample": "full matrix, %d timed calls of p=4" % args.steps},
           "e2e": {"value": gf, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def solver_leg(m, torch, dev, n_edge=64, solves=5, bases=("f32", "f64"), warm=True, poly_degree=0,
               jacobi=0, gs2=0, gs2_gamma=1):
    """s-step GMRES(s=8, restart 48) to rel. residual 1e-8 on the log-normal diffusion matrix
    (7-point, sigma = 1, rows randomly permuted) at n_edge^3, FP32 basis + FP64 refinement vs an
    FP64 basis: solves/s and per-solve latency (p50/p99) over `solves` solves each.  poly_degree:
    GMRES-polynomial preconditioning (Sec. 5.2); jacobi: right Jacobi scaling fused into the
    MPK (Sec. 5.1); gs2: two-stage Gauss-Seidel with gs2_gamma inner iterations as MPK
    sub-powers (Sec. 5.1, Alg. GS2)."""
    A = mi.diffusion7_lognormal(n_edge)
    b = mi.uniform_vectors(A.n, 4)[0]
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val).to(dev)
    plan = m.mpk_plan_create(rp, ci, vv, 8, m.mpk_plan_opts_default(keep_f64=1, keep_f32=1,
                                                                    jacobi=1 if (jacobi or gs2) else 0))
    B = torch.from_numpy(b).to(dev)
    out = {"workload": "7-point log-normal diffusion %d^3 (sigma 1, rows permuted seed 1), b ~ U[-1,1) "
                       "seed 4, s=8, restart 48, tol 1e-8" % n_edge, "n": A.n, "nnz": A.nnz}
    for basis in bases:
        lat, iters, rr, ok = [], [], [], True
        for _ in range(solves + (1 if warm else 0)):
            X = torch.zeros_like(B)
            o = m.mpk_gmres_opts_default(s=8, restart=48, tol=1e-8, poly_degree=poly_degree,
                                         jacobi=jacobi, gs2=gs2, gs2_gamma=gs2_gamma,
                                         basis=m.MPK_F32 if basis == "f32" else m.MPK_F64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = m.sstep_gmres_solve(plan, B, X, o, check=False)
            torch.cuda.synchronize()
            lat.append(1e3 * (time.perf_counter() - t0))
            iters.append(info["iters"])
            rr.append(info["rel_residual"])
            ok = ok and info["status_code"] == m.MPK_OK
        if warm and len(lat) > 1:
            lat = lat[1:]   # the first solve also loads the solver's kernels
        out[basis] = {"solves_per_s": 1e3 * len(lat) / sum(lat), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "iters": iters[-1],
                      "rel_residual": max(rr), "converged": ok}
    return out


def cg_leg(m, torch, dev, n_edge=64, solves=5, bases=("f32", "f64"), warm=True, s=8):
    """s-step CG (s = 8, Ritz shifts from a setup phase) to rel. residual 1e-8 on the same SPD
    log-normal diffusion matrix as the GMRES leg, FP32 basis + FP64 refinement vs an FP64 basis:
    solves/s, latency, CG steps and the time split (MPK / Gram / rest)."""
    A = mi.diffusion7_lognormal(n_edge)
    b = mi.uniform_vectors(A.n, 4)[0]
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val).to(dev)
    plan = m.mpk_plan_create(rp, ci, vv, s, m.mpk_plan_opts_default(keep_f64=1, keep_f32=1))
    B = torch.from_numpy(b).to(dev)
    out = {"workload": "7-point log-normal diffusion %d^3 (sigma 1, rows permuted seed 1), b ~ U[-1,1) "
                       "seed 4, s-step CG s=%d, tol 1e-8" % (n_edge, s), "n": A.n, "nnz": A.nnz}
    for basis in bases:
        lat, info = [], None
        ok = True
        for _ in range(solves + (1 if warm else 0)):
            X = torch.zeros_like(B)
            o = m.mpk_cg_opts_default(s=s, tol=1e-8, basis=m.MPK_F32 if basis == "f32" else m.MPK_F64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = m.sstep_cg_solve(plan, B, X, o, check=False)
            torch.cuda.synchronize()
            lat.append(1e3 * (time.perf_counter() - t0))
            ok = ok and info["status_code"] == m.MPK_OK
        if warm and len(lat) > 1:
            lat = lat[1:]
        out[basis] = {"solves_per_s": 1e3 * len(lat) / sum(lat), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "iters": info["iters"],
                      "rel_residual": info["rel_residual"], "converged": ok, "refinement_steps": info["outer"],
                      "s_used": info["s_used"],
                      "ms_mpk": info["ms_mpk"], "ms_gram": info["ms_gram"], "ms_other": info["ms_other"]}
    return out


def gs2_mpk_leg(m, torch, dev, A, rp, ci, vv, p=P_MAIN, gammas=(1, 2), reps=20):
    """MPK of the GS2-preconditioned operator (Sec. 5.1, Alg. GS2(b)) on the 27-point benchmark
    matrix, level-order I/O: each power is gamma inner stages on the strictly lower part plus
    the product with A, all blocked as sub-powers in one launch, against the same steps as
    separate launches.  Flops per power: 2 nnz (product) + gamma * 2 nnz_L (inner stages)."""
    n, nnz = A.n, A.nnz
    nnz_l = int(np.sum(A.col < np.repeat(np.arange(n, dtype=np.int64), np.diff(A.row_ptr))))
    out = {"workload": "27-point 160^3 (seed 2), GS2 from zero, Newton p=%d (Leja on [0,2]), "
                       "level-order I/O" % p, "nnz_lower": nnz_l}
    theta = mi.leja_points_interval(0.0, 2.0, p)
    cf = m.mpk_coeffs_newton(theta)
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        vals = vv if dt == torch.float64 else vv.float()
        # blocking depth in sub-powers: every stage of every power in one blocked launch
        plan = m.mpk_plan_create(rp, ci, vals, p * (max(gammas) + 1), m.mpk_plan_opts_default(
            assume_symmetric=1, blocked=1, jacobi=1))
        Y = torch.zeros((p + 1) * n, dtype=dt, device=dev)
        Y[:n] = 1.0
        res = {}
        for g in gammas:
            fl = m.MPK_GS2 | m.MPK_GS2_GAMMA(g) | m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X
            tb = time_stream(lambda: m.mpk_apply(plan, cf, None, Y, flags=fl), reps, torch)
            tu = time_stream(lambda: m.mpk_apply(plan, cf, None, Y, flags=fl | m.MPK_UNBLOCKED), reps, torch)
            flop = p * (2.0 * nnz + g * 2.0 * nnz_l)
            res["gamma%d" % g] = {"blocked_ms": tb, "unblocked_ms": tu, "speedup": tu / tb,
                                  "blocked_gflops": flop / tb / 1e6, "unblocked_gflops": flop / tu / 1e6,
                                  "matrix_passes": p * (g + 1)}
        assert m.mpk_plan_sync(plan) == m.MPK_OK
        out[name] = res
        del plan
    return out


def serving_leg(m, n_req=24, n_min=32, n_max=192, seed=7):
    """The solve stream (Poisson arrivals at 200/s, 7- or 27-point anisotropic diffusion,
    anisotropy log-uniform in [1, 100], grid edge uniform in [n_min, n_max], the c5
    distribution) through the server under a 120 GB budget, FP32 basis + FP64 refinement to
    1e-8, then the same stream with an FP64 basis.  A bounded sample of n_req requests: at
    200/s the stream offers far more work than one GPU completes (an average request of this
    size distribution is a solve of about half a second), so the server runs saturated, the
    reported solves/s is its saturation throughput and the latency percentiles are dominated
    by queueing."""
    stream = mi.solve_stream(n_req, seed=seed, n_min=n_min, n_max=n_max)
    mats = []
    for r in stream:
        A = mi.anisotropic(r["N"], r["stencil"], r["a"])
        mats.append((A, mi.uniform_vectors(A.n, r["b_seed"] % 100000)[0]))
    out = {"workload": "%d requests of the solve stream (seed %d, 200/s Poisson arrivals, grid edge "
                       "%d..%d, 7/27-point, anisotropy 1..100), tol 1e-8" % (n_req, seed, n_min, n_max)}
    for basis in ("f32", "f64"):
        o = m.mpk_server_opts_default(hbm_budget_bytes=120 << 30)
        o.gmres.basis = m.MPK_F32 if basis == "f32" else m.MPK_F64
        srv = m.Server(o)
        # warm-up: one request (kernels loaded before the timed stream)
        A0, b0 = mats[0]
        srv.submit(A0.row_ptr, A0.col, A0.val, b0)
        while srv.pending():
            srv.poll(64)
            time.sleep(0.0005)
        srv.poll(64)
        t_start = time.perf_counter()
        sub, done, ids = {}, {}, []
        i = 0
        while len(done) < n_req:
            now = time.perf_counter() - t_start
            while i < n_req and stream[i]["t_arrival"] <= now:
                A, b = mats[i]
                rid, _ = srv.submit(A.row_ptr, A.col, A.val, b)
                sub[rid] = time.perf_counter()
                ids.append(rid)
                i += 1
            for res in srv.poll(64):
                if res["id"] in sub:
                    done[res["id"]] = (time.perf_counter(), res)
            time.sleep(0.0002)
        t_end = time.perf_counter()
        srv.close()
        lat = [1e3 * (done[r][0] - sub[r]) for r in ids]
        statuses = [done[r][1]["status"] for r in ids]
        span = max(stream[-1]["t_arrival"], 1e-9)
        out[basis] = {"solves_per_s": n_req / (t_end - t_start), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)),
                      "offered_per_s": n_req / span,
                      "offered_over_served": (n_req / span) / (n_req / (t_end - t_start)),
                      "all_converged": all(st == m.MPK_OK for st in statuses),
                      "max_rel_residual": max(done[r][1]["rel_residual"] for r in ids)}
    return out


def _gen_request(r):
    """One request of the solve stream (runs in a worker process): CSR arrays and b."""
    A = mi.anisotropic(r["N"], r["stencil"], r["a"])
    return A.row_ptr, A.col, A.val, mi.uniform_vectors(A.n, r["b_seed"] % 100000)[0]


def serving_full_leg(m, n_req=2000, n_f64=300, seed=7, workers=15, window=30, max_pending=16):
    """The solve stream at its stated size: n_req requests (Poisson arrivals at 200/s, grid edge
    32..192, 7- or 27-point anisotropic diffusion, anisotropy 1..100) under a 120 GB budget,
    FP32 basis + FP64 refinement; the FP64 basis on the first n_f64 requests.  A request's
    matrix (up to 2.3 GB of CSR at 192^3, 27-point) is generated by a pool of worker
    processes a few requests ahead, and the client holds back submissions while max_pending
    requests wait in the server, so host memory stays bounded; latency is measured from the
    request's stated arrival time, so time spent waiting on the client counts.  At 200/s the
    stream offers far more than one GPU serves: solves/s is the saturation throughput over the
    steady window (completions 10 % .. 90 %), and the latencies grow with the queue.
    starved_s: time the server held no request while the next one was still being generated
    (the host generator, not the GPU, limited the stream then)."""
    import multiprocessing as mp
    stream = mi.solve_stream(n_req, seed=seed, n_min=32, n_max=192)
    ctx = mp.get_context("spawn")
    out = {"workload": "%d requests of the solve stream (seed %d, 200/s Poisson arrivals, grid edge 32..192, "
                       "7/27-point, anisotropy 1..100), tol 1e-8, 120 GB budget; FP64 basis on the first %d"
                       % (n_req, seed, n_f64)}
    with ctx.Pool(workers) as pool:
        for basis, count in (("f32", n_req), ("f64", min(n_f64, n_req))):
            o = m.mpk_server_opts_default(hbm_budget_bytes=120 << 30)
            o.gmres.basis = m.MPK_F32 if basis == "f32" else m.MPK_F64
            srv = m.Server(o)
            futs = {}
            nxt = 0
            t_start = time.perf_counter()
            sub, arr, done, ids = {}, {}, {}, []
            i = 0
            starved = 0.0
            t_last = time.perf_counter()
            while len(done) < count:
                t_now = time.perf_counter()
                if i < count and i in futs and srv.pending() == 0 and not futs[i].ready():
                    starved += t_now - t_last
                t_last = t_now
                while nxt < count and len(futs) < window:
                    futs[nxt] = pool.apply_async(_gen_request, (stream[nxt],))
                    nxt += 1
                now = time.perf_counter() - t_start
                if i < count and stream[i]["t_arrival"] <= now and srv.pending() < max_pending and futs[i].ready():
                    rp_, col_, val_, b_ = futs.pop(i).get()
                    rid, _ = srv.submit(rp_, col_, val_, b_)
                    arr[rid] = t_start + stream[i]["t_arrival"]
                    sub[rid] = time.perf_counter()
                    ids.append(rid)
                    i += 1
                    continue
                for res in srv.poll(64):
                    if res["id"] in sub:
                        done[res["id"]] = (time.perf_counter(), res)
                time.sleep(0.0005)
            srv.close()
            order = sorted(ids, key=lambda r: done[r][0])
            lo, hi = int(0.1 * count), max(int(0.9 * count), int(0.1 * count) + 1)
            win = order[lo:hi]
            t0w, t1w = done[order[lo - 1]][0] if lo > 0 else t_start, done[order[hi - 1]][0]
            lat = [1e3 * (done[r][0] - arr[r]) for r in win]
            out[basis] = {"requests": count, "steady_solves_per_s": len(win) / max(t1w - t0w, 1e-9),
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "total_s": max(d[0] for d in done.values()) - t_start, "starved_s": starved,
                          "all_converged": all(done[r][1]["status"] == m.MPK_OK for r in ids),
                          "max_rel_residual": max(done[r][1]["rel_residual"] for r in ids)}
    return out


def batch_leg(m, torch, dev, p=8, reps=10, cases=((256, 8, 32), (64, 16, 48)), seed=7):
    """Batched MPK (mpk_batch_apply): many uneven systems (7- or 27-point anisotropic
    diffusion, anisotropy log-uniform in [1, 100], grid edge uniform in [lo, hi]) in one
    persistent launch, against one mpk_apply per system (automatic blocked / unblocked
    choice) and p back-to-back SpMVs per system; Newton p = 8 with Leja shifts, level-order
    I/O, each variant graph-captured once and replayed.  GFLOP/s = sum_i 2 nnz_i p / t."""
    rng = np.random.default_rng(seed)
    out = {}
    for count, lo, hi in cases:
        for dt in ("f32", "f64"):
            tdt = torch.float32 if dt == "f32" else torch.float64
            plans, cfs, Ys, nnz = [], [], [], 0
            for i in range(count):
                N = int(rng.integers(lo, hi + 1))
                A = mi.anisotropic(N, 7 if i % 2 else 27, float(np.exp(rng.uniform(0.0, np.log(100.0)))))
                nnz += A.nnz
                plans.append(m.mpk_plan_create(torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col).to(dev),
                                               torch.from_numpy(A.val).to(dev, tdt), p))
                cfs.append(m.mpk_coeffs_newton(mi.leja_points_interval(0.0, 6.6 * float(np.abs(A.val).max()), p)))
                Y = torch.zeros(((p + 1) * A.n,), dtype=tdt, device=dev)
                Y[: A.n] = 1.0
                Ys.append(Y)
            B = m.Batch(plans, p, tdt)
            fl = m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X

            def batch():
                B.apply(cfs, None, Ys, flags=fl)

            def each(extra=0):
                for pl, c, y in zip(plans, cfs, Ys):
                    m.mpk_apply(pl, c, None, y, flags=fl | extra)
            res = {"systems": count, "grid_edges": [lo, hi], "nnz": nnz}
            for name, fn in (("batch", batch), ("each_auto", each),
                             ("each_pxspmv", lambda: each(m.MPK_UNBLOCKED))):
                fn()
                fn()
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    fn()
                g.replay()
                ms = time_stream(g.replay, reps, torch)
                res[name] = {"ms": ms, "gflops": 2.0 * nnz * p / ms / 1e6}
            assert B.sync() == m.MPK_OK
            res["speedup_vs_each"] = res["each_auto"]["ms"] / res["batch"]["ms"]
            out["%d_systems_%d_%d_%s" % (count, lo, hi, dt)] = res
            del B, plans, Ys
            torch.cuda.empty_cache()
    return out


def run_profile(args, m, torch, local):
    """Small profiling case (no timing printed): 27-point matrix on a --profile-n grid, default
    plan, --profile-reps repetitions of one blocked and one unblocked call with y_0 already in
    level order.  The blocked kernel's launches are the (2r)-th kernel launches of this family."""
    dev = torch.device("cuda", local)
    if args.profile_nrhs > 0:
        # block MPK: per repetition one blocked and one unblocked call, level-order interleaved
        A = mi.stencil27(args.profile_n, seed=5)
        p, nr = 6, args.profile_nrhs
        rp = torch.from_numpy(A.row_ptr).to(dev)
        ci = torch.from_numpy(A.col).to(dev)
        vv = torch.from_numpy(A.val.astype(np.float32)).to(dev)
        plan = m.mpk_plan_create(rp, ci, vv, p, m.mpk_plan_opts_default(assume_symmetric=1, p_blk=p, blocked=1))
        co = m.mpk_coeffs_chebyshev(0.1, 52.0, p)
        X = torch.from_numpy(mi.uniform_vectors(A.n, 6, nr).T.copy()).to(dev, torch.float32)
        Y = torch.empty((p + 1) * A.n * nr, dtype=torch.float32, device=dev)
        fl = m.MPK_PERMUTED_IO | m.MPK_RHS_INTERLEAVED
        for _ in range(args.profile_reps):
            m.mpk_apply(plan, co, X, Y, n_rhs=nr, flags=fl)
            m.mpk_apply(plan, co, X, Y, n_rhs=nr, flags=fl | m.MPK_UNBLOCKED)
        torch.cuda.synchronize()
        status = m.mpk_plan_sync(plan)
        print(json.dumps({"profile": "block", "status": status, "n": A.n, "nnz": A.nnz, "p": p, "n_rhs": nr}))
        return 0 if status == m.MPK_OK else 1
    A = mi.stencil27(args.profile_n, seed=2)
    x = mi.uniform_vectors(A.n, 0)[0]
    p = args.profile_p
    theta = mi.leja_points_interval(0.0, 52.0, p)
    dt = torch.float64 if args.profile_dtype == "f64" else torch.float32
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val).to(dev).to(dt)
    gs2 = args.profile_gs2 >= 0
    # GS2: every sub-power of every power in one blocked launch
    pmax = p * (args.profile_gs2 + 1) if gs2 else p
    opts = m.mpk_plan_opts_default(assume_symmetric=1, p_blk=pmax, blocked=1, jacobi=1 if gs2 else 0)
    if args.profile_cs > 0:
        opts.chunk_slices = args.profile_cs
    if args.profile_slack > 0:
        opts.slack_tasks = args.profile_slack
    if args.profile_kernel >= 0:
        opts.kernel = args.profile_kernel
    if args.profile_lag > 0:
        opts.owner_lag = args.profile_lag
    plan = m.mpk_plan_create(rp, ci, vv, pmax, opts)
    perm = m.mpk_plan_perm(plan)["perm"].long()
    Y = torch.empty((p + 1) * A.n, dtype=dt, device=dev)
    X = torch.from_numpy(x).to(dev).to(dt)
    Y[:A.n] = X[perm]
    co = m.mpk_coeffs_newton(theta)
    fl = m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X
    if gs2:
        fl |= m.MPK_GS2 | m.MPK_GS2_GAMMA(args.profile_gs2)
    for _ in range(args.profile_reps):
        if args.profile_orig:
            # the headline's call: original order in and out (gather, blocked kernel that also
            # stores every power in the original order)
            m.mpk_apply(plan, co, X, Y)
            m.mpk_apply(plan, co, X, Y, flags=m.MPK_UNBLOCKED)
        else:
            m.mpk_apply(plan, co, None, Y, flags=fl)
            m.mpk_apply(plan, co, None, Y, flags=fl | m.MPK_UNBLOCKED)
    torch.cuda.synchronize()
    status = m.mpk_plan_sync(plan)
    print(json.dumps({"profile": "done", "status": status, "n": A.n, "nnz": A.nnz, "p": p,
                      "dtype": args.profile_dtype, "plan": m.mpk_plan_stats(plan)}))
    return 0 if status == m.MPK_OK else 1


def block_mpk_leg(m, torch, dev, hbm_peak, reps=20):
    """Block MPK as an AMG polynomial smoother: 27-point 128^3 matrix (seed 5) in FP32,
    Chebyshev basis p = 6 on [0.1, 52], n_rhs = 8, 16, 32 right-hand sides interleaved in level
    order (X ~ U[-1,1), seed 6).  Each variant is captured once in a CUDA graph and replayed;
    modes: all p+1 powers out (basis) and the final polynomial sum_k y_k only (smoother); plans:
    blocked, unblocked, the automatic choice, and the autotuner's options for the call shape.
    GFLOP/s = 2 nnz p n_rhs / t; effective GB/s = the algorithmic minimum bytes / t."""
    A = mi.stencil27(128, seed=5)
    n, nnz, p = A.n, A.nnz, 6
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val.astype(np.float32)).to(dev)
    co = m.mpk_coeffs_chebyshev(0.1, 52.0, p)
    cog = m.Coeffs(co.a, co.b, co.c, gamma=np.ones(p + 1))
    M = 4 * (n + 1) + nnz * 8
    out = {"workload": "27-point 128^3 FP32 (seed 5), Chebyshev p=6 on [0.1,52], X ~ U[-1,1) seed 6, "
                       "interleaved level-order I/O, one graph-captured call per step",
           "n": n, "nnz": nnz, "p": p}
    plans = {}
    for mode in ("blocked", "unblocked", "auto"):
        opts = m.mpk_plan_opts_default(assume_symmetric=1, p_blk=p,
                                       blocked={"blocked": 1, "unblocked": 0, "auto": -1}[mode])
        plans[mode] = m.mpk_plan_create(rp, ci, vv, p, opts)
    for n_rhs in (8, 16, 32):
        X = torch.from_numpy(mi.uniform_vectors(n, 6, n_rhs).T.copy()).to(dev, torch.float32)   # n x n_rhs
        Y = torch.empty((p + 1) * n * n_rhs, dtype=torch.float32, device=dev)
        res = {}
        for final in (False, True):
            fl = m.MPK_PERMUTED_IO | m.MPK_RHS_INTERLEAVED | (m.MPK_FINAL_ONLY if final else 0)
            cc = cog if final else co
            bmin = M + 4 * n * n_rhs * (2 if final else p + 2)
            # the autotuner's choice for this call shape (plan options timed on this matrix)
            best, tinfo = m.mpk_autotune(rp, ci, vv, cc, n_rhs=n_rhs, flags=fl,
                                         base=m.mpk_plan_opts_default(assume_symmetric=1, p_blk=p), reps=3)
            tuned = m.mpk_plan_create(rp, ci, vv, p, best)
            modes = dict(plans)
            modes["tuned"] = tuned
            for mode, plan in modes.items():
                call = lambda: m.mpk_apply(plan, cc, X, Y, n_rhs=n_rhs, flags=fl)
                call()                                  # schedule, automatic choice
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    call()
                g.replay()
                torch.cuda.synchronize()
                ms = time_stream(g.replay, reps, torch)
                assert m.mpk_plan_sync(plan) == m.MPK_OK
                res["%s_%s" % ("final" if final else "basis", mode)] = {
                    "ms": ms, "gflops": 2.0 * nnz * p * n_rhs / ms / 1e6,
                    "eff_gbs": bmin / ms / 1e6, "eff_frac": bmin / ms / 1e6 / hbm_peak}
            res["%s_tuned" % ("final" if final else "basis")].update(
                {"candidate": tinfo["best_index"], "blocked": int(best.blocked), "kernel": int(best.kernel),
                 "chunk_slices": int(best.chunk_slices), "l2_budget_bytes": int(best.l2_budget_bytes)})
            del tuned
        out["n_rhs%d" % n_rhs] = res
        del X, Y
    del plans
    torch.cuda.empty_cache()
    return out


def time_stream(fn, reps, torch):
    """Average ms per call of fn() on the current stream, CUDA events on that stream."""
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-solver", action="store_true", help="skip the solver and serving legs")
    ap.add_argument("--no-block", action="store_true", help="skip the n_rhs block MPK leg")
    ap.add_argument("--serving-full", type=int, default=0,
                    help="only run the solve stream at this many requests (the stated size is 2000) and "
                         "print its result")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: plan, then per repetition one blocked and one unblocked "
                         "call (level-order I/O) on the 27-point matrix of --profile-n")
    ap.add_argument("--profile-n", type=int, default=N_GRID, help="grid edge of the profiling case")
    ap.add_argument("--profile-dtype", default="f64", choices=["f32", "f64"])
    ap.add_argument("--profile-p", type=int, default=P_MAIN)
    ap.add_argument("--profile-reps", type=int, default=3)
    ap.add_argument("--profile-kernel", type=int, default=-1,
                    help="blocked kernel of the profiling plan (plan option kernel; -1: default)")
    ap.add_argument("--profile-gs2", type=int, default=-1,
                    help="profiling run of the GS2-preconditioned MPK with this many inner stages "
                         "(-1: plain MPK)")
    ap.add_argument("--profile-orig", action="store_true",
                    help="profiling run with original-order I/O (the headline's call)")
    ap.add_argument("--profile-solver", action="store_true",
                    help="profiling run of the solver: two s-step GMRES solves (FP32 basis) on the "
                         "log-normal diffusion matrix at --profile-n")
    ap.add_argument("--profile-cg", action="store_true",
                    help="profiling run of s-step CG: --profile-reps solves (FP32 basis) on the "
                         "log-normal diffusion matrix at --profile-n")
    ap.add_argument("--profile-nrhs", type=int, default=0,
                    help="profiling run of the block MPK (c4: 27-point --profile-n grid, seed 5, FP32, "
                         "Chebyshev p = 6 on [0.1, 52]) with this many interleaved right-hand sides")
    ap.add_argument("--profile-cs", type=int, default=0, help="chunk_slices (0: plan default)")
    ap.add_argument("--profile-slack", type=int, default=0, help="slack_tasks (0: plan default)")
    ap.add_argument("--profile-lag", type=int, default=0, help="owner_lag of the owner kernel (0: plan default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2309_02228_gb300 import build as B
    B.build()
    import paper_2309_02228_gb300 as m

    if args.profile_solver:
        out = solver_leg(m, torch, torch.device("cuda", local), n_edge=args.profile_n,
                         solves=args.profile_reps, bases=("f32",))
        print(json.dumps({"profile": "solver", "result": out}))
        return 0 if out["f32"]["converged"] else 1
    if args.profile_cg:
        out = cg_leg(m, torch, torch.device("cuda", local), n_edge=args.profile_n,
                     solves=args.profile_reps, bases=("f32",), warm=False)
        print(json.dumps({"profile": "cg", "result": out}))
        return 0 if out["f32"]["converged"] else 1
    if args.profile:
        return run_profile(args, m, torch, local)
    if args.serving_full > 0:
        out = serving_full_leg(m, n_req=args.serving_full)
        print(json.dumps({"serving_full": out}))
        return 0 if out["f32"]["all_converged"] else 1
    A, x, theta = gen_workload()
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    vv = torch.from_numpy(A.val).to(dev)
    n, nnz = A.n, A.nnz
    cfs = {p: m.mpk_coeffs_newton(theta[:p]) for p in P_SWEEP}
    # the pattern is symmetric (a 27-point stencil): the plan skips building A^T.  The
    # autotuner picks the blocked plan's options (chunk size, kernel variant, group budget) for
    # the headline call; the headline is the blocked MPK, so blocking stays on.
    base = m.mpk_plan_opts_default(assume_symmetric=1, p_blk=P_MAIN, blocked=1)
    tuned, tinfo = m.mpk_autotune(rp, ci, vv, cfs[P_MAIN], base=base, reps=5)
    tuned.blocked = 1
    t0 = time.perf_counter()
    plan = m.mpk_plan_create(rp, ci, vv, max(P_SWEEP), tuned)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    pst = m.mpk_plan_stats(plan)
    X = torch.from_numpy(x).to(dev)
    Y = torch.empty((max(P_SWEEP) + 1) * n, dtype=torch.float64, device=dev)

    def step(p=P_MAIN, flags=0):
        m.mpk_apply(plan, cfs[p], X, Y, flags=flags)

    hbm_peak, peak_kind = measured_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # ---- headline: K steps of the full call (original order in/out), CUDA events
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    status = m.mpk_plan_sync(plan)
    assert status == m.MPK_OK, m.status_name(status)
    flop = 2.0 * nnz * P_MAIN
    value = whole_job_gflops(flop, world, ms_step)

    # ---- the p x SpMV baseline through the same call, and the p sweep
    reps = max(5, min(args.steps, 50))
    sweep = {}
    for p in P_SWEEP:
        tb = time_stream(lambda: step(p), reps, torch)
        tu = time_stream(lambda: step(p, m.MPK_UNBLOCKED), reps, torch)
        sweep["p%d" % p] = {"blocked_gflops": 2.0 * nnz * p / tb / 1e6,
                            "pxspmv_gflops": 2.0 * nnz * p / tu / 1e6,
                            "speedup": tu / tb, "blocked_ms": tb, "pxspmv_ms": tu}

    # ---- kernel only (level-order I/O, y_0 already in place): one launch of the blocked kernel
    perm = m.mpk_plan_perm(plan)["perm"].long()
    Yp = torch.empty((max(P_SWEEP) + 1) * n, dtype=torch.float64, device=dev)
    Yp[:n] = X[perm]
    kern = {}
    w = 8
    M_bytes = 4 * (n + 1) + nnz * (4 + w)
    v_bytes = w * n
    for p in P_SWEEP:
        kb = time_stream(lambda: m.mpk_apply(plan, cfs[p], None, Yp, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X), reps, torch)
        ku = time_stream(lambda: m.mpk_apply(plan, cfs[p], None, Yp, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X | m.MPK_UNBLOCKED), reps, torch)
        kern["p%d" % p] = {"blocked_ms": kb, "pxspmv_ms": ku,
                           "blocked_gflops": 2.0 * nnz * p / kb / 1e6,
                           "pxspmv_gflops": 2.0 * nnz * p / ku / 1e6,
                           "blocked_min_bytes": M_bytes + v_bytes * (p + 1),
                           "pxspmv_bytes": p * (M_bytes + 2 * v_bytes)}
    status = m.mpk_plan_sync(plan)
    assert status == m.MPK_OK, m.status_name(status)
    clk = clocks.stop()

    # ---- FP32 copy of the same matrix (the bandwidth-bound precision)
    fp32 = {}
    vv32 = vv.float()
    plan32 = m.mpk_plan_create(rp, ci, vv32, max(P_SWEEP), m.mpk_plan_opts_default(assume_symmetric=1, p_blk=P_MAIN,
                                                                                   blocked=1))
    X32 = X.float()
    Y32 = torch.empty((max(P_SWEEP) + 1) * n, dtype=torch.float32, device=dev)
    perm32 = m.mpk_plan_perm(plan32)["perm"].long()
    Y32[:n] = X32[perm32]
    M32 = 4 * (n + 1) + nnz * 8
    for p in P_SWEEP:
        kb = time_stream(lambda: m.mpk_apply(plan32, cfs[p], None, Y32, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X), reps, torch)
        ku = time_stream(lambda: m.mpk_apply(plan32, cfs[p], None, Y32, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X | m.MPK_UNBLOCKED), reps, torch)
        bmin = M32 + 4 * n * (p + 1)
        fp32["p%d" % p] = {"blocked_gflops": 2.0 * nnz * p / kb / 1e6,
                           "pxspmv_gflops": 2.0 * nnz * p / ku / 1e6, "speedup": ku / kb,
                           "blocked_eff_gbs": bmin / kb / 1e6,
                           "blocked_eff_frac": bmin / kb / 1e6 / hbm_peak,
                           "pxspmv_gbs": p * (M32 + 8 * n) / ku / 1e6}
    assert m.mpk_plan_sync(plan32) == m.MPK_OK
    del plan32
    # the owner-share kernel (one share of every level group per CTA, the paper's wavefront
    # schedule): DRAM traffic at the algorithmic minimum at lag 1 and two matrix passes at lag 2
    # (profiles/owner_kernel_f32_p4_27pt128_dram.md), timed here on the same FP32 call
    fp32["owner_p4"] = {}
    for lag in (1, 2):
        plano = m.mpk_plan_create(rp, ci, vv32, P_MAIN, m.mpk_plan_opts_default(
            assume_symmetric=1, p_blk=P_MAIN, blocked=1, kernel=6, owner_lag=lag))
        Yo = torch.empty((P_MAIN + 1) * n, dtype=torch.float32, device=dev)
        Yo[:n] = X32[m.mpk_plan_perm(plano)["perm"].long()]
        ko = time_stream(lambda: m.mpk_apply(plano, cfs[P_MAIN], None, Yo, flags=m.MPK_PERMUTED_IO | m.MPK_Y0_IS_X),
                         reps, torch)
        assert m.mpk_plan_sync(plano) == m.MPK_OK
        fp32["owner_p4"]["lag%d" % lag] = {"ms": ko, "gflops": 2.0 * nnz * P_MAIN / ko / 1e6,
                                           "vs_pxspmv": (2.0 * nnz * P_MAIN / ko / 1e6) / fp32["p4"]["pxspmv_gflops"]}
        del plano, Yo

    # ---- GS2-preconditioned MPK (sub-powers) blocked vs one launch per sub-power
    gs2_mpk = gs2_mpk_leg(m, torch, dev, A, rp, ci, vv, reps=reps)

    # ---- solver and serving legs (solves/s and latency at rel. residual 1e-8)
    solver = serving = None
    if not args.no_solver:
        solver = {"n64": solver_leg(m, torch, dev, n_edge=64, solves=5),
                  # the full-size workload (n = 16.8 M), one solve per basis (kernels already loaded)
                  "n256": solver_leg(m, torch, dev, n_edge=256, solves=1, warm=False),
                  # GMRES-polynomial preconditioning of degree 32 (Sec. 5.2) on the 64^3 matrix
                  "n64_poly32": solver_leg(m, torch, dev, n_edge=64, solves=5, poly_degree=32),
                  # right Jacobi scaling fused into the MPK (Sec. 5.1), 64^3 and full size
                  "n64_jacobi": solver_leg(m, torch, dev, n_edge=64, solves=5, jacobi=1),
                  "n256_jacobi": solver_leg(m, torch, dev, n_edge=256, solves=1, warm=False, jacobi=1),
                  # two-stage Gauss-Seidel (gamma = 1) as MPK sub-powers (Sec. 5.1, Alg. GS2)
                  "n64_gs2": solver_leg(m, torch, dev, n_edge=64, solves=5, gs2=1, gs2_gamma=1),
                  "n256_gs2": solver_leg(m, torch, dev, n_edge=256, solves=1, warm=False, gs2=1, gs2_gamma=1),
                  # s-step CG on the same SPD matrices (the short-recurrence method, Sec. 4 / Sec. 7)
                  "n64_cg": cg_leg(m, torch, dev, n_edge=64, solves=5),
                  "n256_cg": cg_leg(m, torch, dev, n_edge=256, solves=1, warm=False)}
        serving = serving_leg(m)
    block = None
    if not args.no_block:
        block = block_mpk_leg(m, torch, dev, hbm_peak)
    batch = None
    if not args.no_block:
        batch = batch_leg(m, torch, dev)

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timing)
    Xh = torch.from_numpy(x.copy()).pin_memory()
    Yh = torch.empty((P_MAIN + 1) * n, dtype=torch.float64).pin_memory()
    e2e_reps = max(3, min(args.steps, 20))
    m.mpk_apply(plan, cfs[P_MAIN], Xh, Yh, flags=m.MPK_HOST_IO)
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        m.mpk_apply(plan, cfs[P_MAIN], Xh, Yh, flags=m.MPK_HOST_IO)
    t_e2e = (time.perf_counter() - t0) / e2e_reps
    e2e = {"value": world * flop / t_e2e / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n * (P_MAIN + 1)}

    # ---- roofline of the dominant kernel (blocked, p = 4).  Its two bounds: FP64 FMA issue
    # (the FP64 FMA rate measured on this device by mpk_fma_peak) and HBM (the measured copy
    # bandwidth on the algorithmic minimum bytes); the binding one is reported, the other
    # beside it.
    kb = kern["p%d" % P_MAIN]["blocked_ms"]
    bytes_min = kern["p%d" % P_MAIN]["blocked_min_bytes"]
    fp64_peak = m.mpk_fma_peak(m.MPK_F64)
    fp32_peak = m.mpk_fma_peak(m.MPK_F32)
    lane = int(tuned.kernel) == 4 or int(tuned.lanes_per_row) > 1
    kname = "mpk_lane_kernel<double,%d,%d>" % (max(1, int(tuned.lanes_per_row)), int(tuned.task_dispatch)) \
        if lane else "mpk_wave_kernel<double,1>"
    traffic, traffic_note = recorded_traffic() if lane else (None, "no capture of this kernel")
    t_hbm = bytes_min / (hbm_peak * 1e9)
    t_alu = flop / (fp64_peak * 1e12)
    hbm_view = {"achieved_gbs": bytes_min / (kb * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                "frac": bytes_min / (kb * 1e-3) / 1e9 / hbm_peak, "peak_kind": peak_kind}
    if t_alu >= t_hbm:
        ach = flop / (kb * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": traffic,
                "traffic_note": traffic_note + "; algorithmic minimum %.4g bytes" % bytes_min,
                "peak_source": "measured: mpk_fma_peak(FP64) on this device (of measured)",
                "kernel": kname, "hbm_view": hbm_view}
    else:
        ach = bytes_min / (kb * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "traffic_note": traffic_note,
                "peak_kind": peak_kind, "kernel": kname,
                "alu_view": {"achieved_tflops": flop / (kb * 1e-3) / 1e12, "peak_tflops": fp64_peak}}
    roof["fma_peaks_tflops"] = {"f64": fp64_peak, "f32": fp32_peak}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(A, x, theta)

    # kernels launched per headline step: gather_in + blocked (p=4 <= p_blk: one launch, which
    # also stores every power in the original order); the y_0 copies are memcpys
    launches_per_step = 2
    out = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(headline_config(n, nnz),
                       plan=dict({k: pst[k] for k in ("n_levels", "n_groups", "n_chunks", "p_blk",
                                                      "l2_budget_bytes", "sell_nnz", "root")},
                                 autotuned={"candidate": tinfo["best_index"], "kernel": int(tuned.kernel),
                                            "chunk_slices": int(tuned.chunk_slices),
                                            "lanes_per_row": int(tuned.lanes_per_row),
                                            "task_units": int(tuned.task_units),
                                            "slack_tasks": int(tuned.slack_tasks),
                                            "best_ms": tinfo["best_ms"], "base_ms": tinfo["base_ms"]})),
        "pxspmv_gflops": sweep["p%d" % P_MAIN]["pxspmv_gflops"],
        "speedup_vs_pxspmv": sweep["p%d" % P_MAIN]["speedup"],
        "sweep": sweep, "kernel_only": kern, "fp32": fp32, "plan_ms": plan_ms,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "solver": solver, "serving": serving,
        "block_mpk": block, "batch_mpk": batch, "gs2_mpk": gs2_mpk,
        "gpu_launches": launches_per_step * args.steps, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main() or 0)
