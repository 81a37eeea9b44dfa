"""Benchmark of the curl-div solve loop on GB300 (one JSON line on stdout, rank 0).

Workload (one step): the 2D sweep -- p in {2, 3, 4}, n = 256 (m = n + p - 2 per axis,
2 m^2 unknowns per solve), alpha = 1, beta in {1e-6, 1e-3, 1, 1e3, 1e6}, 8 seeded
uniform[-1, 1] right-hand sides per (p, beta): 120 solves to relative residual 1e-10 of the
double-FP64 solution x + x_lo (cd_solve_ext), multigrid-preconditioned flexible CG with
FP32 inner solves (FP64 inner solves at parameter ratios >= 1e4) inside a refinement loop
whose residual is evaluated in double-FP64.  The 40 solves of one p form one batched call.
All right-hand sides are resident in HBM before timing; L2 is flushed (256 MB write)
before every timed step.  `value` counts the solves that reached the tolerance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the solves are independent, so N ranks run N replicas of the workload with
no collective on the data path ("weak" scaling, value = solves of all ranks / max time).
"""
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

METRIC = "solves/s + p50/p99 latency at 1e-10 residual; operator-apply GB/s vs HBM peak"
PS = (2, 3, 4)
N_INT = 256
BETAS = (1e-6, 1e-3, 1.0, 1e3, 1e6)
SEEDS = tuple(range(8))
RTOL = 1e-10
WORKLOAD = ("2D curl-div sweep: p in {2,3,4}, n=256 (~131k-133k DoF/solve), alpha=1, "
            "beta in {1e-6,1e-3,1,1e3,1e6}, 8 uniform[-1,1] RHS per case (120 solves), "
            "MG-preconditioned FCG, FP32 inner + double-FP64 refinement, rtol 1e-10")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(total_ms, solves_local, ws, device=None):
    """Whole-job throughput over ws ranks: every rank's solves over the slowest rank's time
    (all_reduce MAX of the timed milliseconds).  Returns (max_ms, solves per second)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, ws * solves_local / (total_ms / 1e3)


# ------------------------------------------------------------------ reference (oracle) arm
# The oracle's sparse direct solve takes minutes per n = 256 system and its Krylov solves need
# 10^3-10^4 iterations away from beta = 1, so the CPU legs time a bounded sample of the sweep:
# the oracle's P_MIM (Section 6.2, the paper's best strategy: CG preconditioned by two V-cycles
# with symmetric Gauss-Seidel and PGMRES-T post-smoothing) at beta = 1, p = 2, n = 256, one
# uniform right-hand side per solve, rtol 1e-10, one solve per host core in spawned processes.
REF_P = 2
REF_SAMPLE = ("oracle P_MIM (FP64, Section 6.2) to rtol 1e-10 at beta=1, p=2, n=256, one uniform RHS "
              "per solve, one solve per host core")


def host_cores():
    """CPUs this process may run on (at most 16 worker processes)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 16))


def oracle_job(args):
    """One oracle solve: returns (setup s, solve s, iterations, DoF).  Setup = assembly of A
    and of the multigrid hierarchy; solve = the preconditioned CG iterations."""
    p, seed, method = args
    from oracle import assemble, solvers
    from paper_1805_10058_gb300 import inputs
    t0 = time.perf_counter()
    b = inputs.uniform_rhs(2, p, N_INT, seed=seed)[0]
    A = assemble.galerkin_kron(2, p, N_INT, 1.0, 1.0)
    prec = solvers.mim_preconditioner(A, 2, p, N_INT + p - 2) if method == "pmim" else None
    t1 = time.perf_counter()
    x, k, _ = solvers.cg(A, b, RTOL, 100000, prec, flexible=prec is not None)
    t2 = time.perf_counter()
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert rel <= 1.01 * RTOL, rel
    return t1 - t0, t2 - t1, k, b.size


def _pool_rounds(nrounds, warmup, method, p=REF_P):
    """Times rounds of one oracle solve per host core (spawned single-threaded processes: the
    caller may have initialised CUDA).  Returns (cores, [round seconds], [job results]) or None
    when no process pool can run here."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = host_cores()
    if cores == 1:
        return None
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    ex = None
    try:
        ex = cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
        times, jobs_out = [], []
        for it in range(warmup + nrounds):
            jobs = [(p, 1000 * it + k, method) for k in range(cores)]
            t0 = time.perf_counter()
            res = list(ex.map(oracle_job, jobs, timeout=900))
            if it >= warmup:
                times.append(time.perf_counter() - t0)
                jobs_out.extend(res)
        ex.shutdown(wait=True)
        return cores, times, jobs_out
    except Exception:
        if ex is not None:  # stop this pool's own workers without waiting on them
            procs = list(getattr(ex, "_processes", {}).values())
            ex.shutdown(wait=False, cancel_futures=True)
            for pr in procs:
                pr.kill()
        return None
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    par = _pool_rounds(args.steps, args.warmup, "pmim")
    if par is not None:
        cores, times, jobs = par
        nsolves = cores * len(times)
        sample = f"{len(times)} steps of {cores} solves: {REF_SAMPLE}"
    else:  # one core, one solve per step
        cores, times, jobs = 1, [], []
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle_job((REF_P, it, "pmim"))
            if it >= args.warmup:
                times.append(time.perf_counter() - t0)
                jobs.append(r)
        nsolves = len(times)
        sample = f"{len(times)} solves on one core: {REF_SAMPLE}"
    tot = sum(times)
    val = nsolves / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "step": REF_SAMPLE},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample,
                             "setup_s_median": float(np.median([j[0] for j in jobs])),
                             "solve_s_median": float(np.median([j[1] for j in jobs]))},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample():
    """The oracle as it stands on a bounded sample (REF_SAMPLE): three rounds of one P_MIM solve
    per host core (median round reported), setup and solve timed separately, DoF/s; beside it one
    round of the oracle's plain CG on the same systems."""
    par = _pool_rounds(3, 0, "pmim")
    cg = _pool_rounds(1, 0, "cg")
    if par is None:  # no process pool here: one solve on one core
        t = oracle_job((REF_P, 1, "pmim"))
        return {"value": 1.0 / (t[0] + t[1]), "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": "1 solve on one core: " + REF_SAMPLE, "setup_s_median": t[0],
                "solve_s_median": t[1], "dof_per_s": t[3] / (t[0] + t[1])}
    cores, times, jobs = par
    med = float(np.median(times))
    out = {"value": cores / med, "unit": "solves/s", "cores": cores, "kind": "oracle",
           "sample": f"median of 3 rounds of {cores} solves: {REF_SAMPLE}",
           "round_s": times, "setup_s_median": float(np.median([j[0] for j in jobs])),
           "solve_s_median": float(np.median([j[1] for j in jobs])),
           "iters_median": float(np.median([j[2] for j in jobs])),
           "dof_per_s": cores * jobs[0][3] / med}
    if cg is not None:
        c_cores, c_times, c_jobs = cg
        out["plain_cg"] = {"value": c_cores / c_times[0], "unit": "solves/s",
                           "iters_median": float(np.median([j[2] for j in c_jobs])),
                           "sample": "one round, same systems, oracle plain CG (Section 6.2 CG column)"}
    return out


# ------------------------------------------------------------------ our arm
def alu_peak_tops(dev):
    """Nominal FP32 operation rate of this GPU: SMs x 128 FP32 lanes x the maximum SM clock, one
    FMA, add or multiply per lane per clock (a packed FFMA2 / FADD2 occupies two lanes)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, sms, mhz


def fp64_peak_tflops(dev):
    """Measured FP64 peak of this GPU: cuBLAS DGEMM (torch.matmul, 4096^3, best of 5)."""
    import torch
    a = torch.rand(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.rand(4096, 4096, dtype=torch.float64, device=dev)
    best = float("inf")
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2 * 4096 ** 3 / best / 1e12


def time_apply(s, stream, flush, B, dtype, alphas, betas, reps=20):
    """Mean CUDA-event time of one cd_apply(_f32) launch group on the library stream, L2 flushed
    before each; a sleep queued ahead of the first event keeps the host's enqueue out of it."""
    import torch
    w = torch.rand(B * s.N, dtype=dtype, device=flush.device)
    y = torch.empty_like(w)
    fn = s.cd_apply_f32 if dtype == torch.float32 else s.cd_apply
    for _ in range(3):
        fn(w, y, alphas, betas)
    times = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            torch.cuda._sleep(1_000_000)
        e0.record(stream)
        fn(w, y, alphas, betas)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return statistics.mean(times)


def measure_c3(dev, cdl, inputs, flush):
    """3D curl-div, p = 3, n = 64 (823875 DoF), beta in {1e-4, 1, 1e4} x 8 smooth sine right-hand
    sides (24 solves, one batched call), FD-D-preconditioned flexible CG with the FD transforms
    on the tensor cores (TF32, FP32 accumulation) inside double-FP64 refinement, rtol 1e-10.
    One timed pass after one untimed one, CUDA events."""
    import torch
    p, n, betas = 3, 64, (1e-4, 1.0, 1e4)
    B = len(betas) * len(SEEDS)
    s = cdl.Solver(3, p, n, max_batch=B, precond=cdl.CD_PC_FD_D, precision=cdl.CD_PREC_FP32_IR,
                   fd_tensor_cores=1, rtol=RTOL, maxit=20000)
    b = torch.as_tensor(np.concatenate([inputs.sine_rhs(3, p, n, seed=sd)[0] for _ in betas
                                        for sd in SEEDS]), device=dev)
    x, xl = torch.zeros_like(b), torch.zeros_like(b)
    al, be = np.ones(B), np.repeat(betas, len(SEEDS))
    s.cd_solve_ext(b, x, xl, al, be, check=False)  # untimed pass (set-up of the FD eigenbases)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st, res = s.cd_solve_ext(b, x, xl, al, be, check=False)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    ok = sum(1 for r in res if r["status"] == 0)
    out = {"workload": "3D p=3 n=64 (823875 DoF), beta in {1e-4,1,1e4} x 8 sine RHS, FD-D (tcgen05 "
                       "TF32 transforms) FCG in double-FP64 refinement, rtol 1e-10",
           "solves_per_s": ok / sec, "converged": ok, "total": B, "seconds": sec,
           "dof_per_s": ok * s.N / sec,
           "iters_median": {f"{bv:g}": float(np.median([r["iters_inner"] for r, x_ in zip(res, be) if x_ == bv]))
                            for bv in betas},
           "worst_relres": max(r["relres"] for r in res)}
    del s
    torch.cuda.synchronize()
    return out


def measure_c4(dev, cdl, inputs, flush, fp64_also):
    """3D curl-div, n = 128, p in {2,3,4,5} (6.3M-6.7M DoF), one uniform right-hand side per p,
    beta log-uniform in [1e-6, 1e6] (one draw per p from default_rng(p)), multigrid FCG, mixed
    precision in double-FP64 refinement (and all-FP64 when asked).  Also the operator apply at
    p = 3 against the HBM roofline (the autotuned FP32 3D apply, one right-hand side, L2
    flushed; 33 (2p+1) multiply-adds per grid point beside it as flops)."""
    import torch
    out = {"workload": "3D n=128, p in {2,3,4,5}, one RHS each, beta log-uniform (default_rng(p)), "
                       "MG FCG, mixed precision + double-FP64 refinement, rtol 1e-10", "solves": []}
    hbm, peak_kind = peaks()
    for p in (2, 3, 4, 5):
        beta = float(inputs.loguniform_params(p, 1)[0])
        b = torch.as_tensor(inputs.uniform_rhs(3, p, 128, seed=p)[0], device=dev)
        for prec, name in ((cdl.CD_PREC_FP32_IR, "mixed"), (cdl.CD_PREC_FP64, "fp64")):
            if name == "fp64" and not fp64_also:
                continue
            s = cdl.Solver(3, p, 128, max_batch=1, precond=cdl.CD_PC_MG, precision=prec, rtol=RTOL,
                           maxit=20000)
            x, xl = torch.zeros_like(b), torch.zeros_like(b)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, res = s.cd_solve_ext(b, x, xl, [1.0], [beta], check=False)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            out["solves"].append({"p": p, "beta": beta, "precision": name, "seconds": sec,
                                  "status": res[0]["status"], "relres": res[0]["relres"],
                                  "iters": res[0]["iters_inner"], "dof": s.N, "dof_per_s": s.N / sec})
            if p == 3 and name == "mixed":
                t = time_apply(s, torch.cuda.current_stream(dev), flush, 1, torch.float32, [1.0], [beta])
                ach = 2 * s.N * 4 / t / 1e9
                out["apply_roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                         "frac": ach / hbm, "peak_kind": peak_kind,
                                         "kernel": "3D FP32 apply, autotuned (tuned three passes "
                                                   "or streaming kernel; p=3, n=128, 1 RHS)",
                                         "flops_tflops": 66 * (2 * 3 + 1) * (s.N // 3) / t / 1e12,
                                         "launch_us": t * 1e6}
                t64 = time_apply(s, torch.cuda.current_stream(dev), flush, 1, torch.float64, [1.0], [beta])
                out["apply_fp64_us"] = t64 * 1e6
            del s
            torch.cuda.synchronize()
    ok = sum(1 for r in out["solves"] if r["status"] == 0)
    tot = sum(r["seconds"] for r in out["solves"])
    out["solves_per_s"] = ok / tot
    out["converged"] = ok
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1805_10058_gb300 import curldiv as cdl
    from paper_1805_10058_gb300 import inputs

    stream = torch.cuda.current_stream(dev)
    streams = [torch.cuda.Stream(dev) for _ in PS]  # one stream (and host thread) per shape
    prec = cdl.CD_PREC_FP64 if args.precision == "fp64" else cdl.CD_PREC_FP32_IR
    pcs = {"mg": cdl.CD_PC_MG, "mim": cdl.CD_PC_MIM, "fdd": cdl.CD_PC_FD_D, "none": cdl.CD_PC_NONE}
    B = len(BETAS) * len(SEEDS)
    solvers_, rhs, xs, xlos, alph, bet, rhs_host = [], [], [], [], [], [], []
    for p in PS:
        s = cdl.Solver(2, p, N_INT, max_batch=B, precond=pcs[args.precond], precision=prec,
                       rtol=RTOL, maxit=args.maxit, stream=streams[len(solvers_)].cuda_stream)
        solvers_.append(s)
        bh = np.concatenate([inputs.uniform_rhs(2, p, N_INT, seed=sd)[0] for _ in BETAS for sd in SEEDS])
        rhs_host.append(torch.from_numpy(bh).pin_memory())
        rhs.append(torch.as_tensor(bh, device=dev))
        xs.append(torch.zeros_like(rhs[-1]))
        xlos.append(torch.zeros_like(rhs[-1]))
        alph.append(np.ones(B))
        bet.append(np.repeat(BETAS, len(SEEDS)))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def concurrent(fn):
        """Runs fn(i) for the three shapes at once, one host thread each; returns the results
        and each call's completion time from the start."""
        out = [None] * len(solvers_)
        done = [None] * len(solvers_)
        t0 = time.perf_counter()

        def run(i):
            out[i] = fn(i)
            done[i] = time.perf_counter() - t0

        ths = [threading.Thread(target=run, args=(i,)) for i in range(len(solvers_))]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        return out, done

    def solve_dev(i):
        return solvers_[i].cd_solve_ext(rhs[i], xs[i], xlos[i], alph[i], bet[i], check=False)[1]

    for _ in range(args.warmup):
        flush.fill_(1.0)
        concurrent(solve_dev)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    lat_all, recs = [], []
    launches0 = cdl.cd_kernel_launches()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        # device time of the step: the solver streams start after ev0 and ev1 follows all of them
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for st in streams:
            st.wait_event(ev0)
        out, done = concurrent(solve_dev)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            stream.wait_event(e)
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        for i, res in enumerate(out):
            for k, r in enumerate(res):
                r["p"], r["beta"] = PS[i], float(bet[i][k])
            recs.append(res)
            lat_all.extend([done[i]] * len(res))
    launches = cdl.cd_kernel_launches() - launches0
    clk = clocks.stop()
    flat = [r for res in recs for r in res]
    ok = [r for r in flat if r["status"] == 0 and r["relres"] <= RTOL]
    n_conv_local = len(ok) / max(1, args.steps)
    total_ms_all, value = aggregate(total_ms, len(ok), ws, device=dev)
    _, value_all = aggregate(total_ms, len(flat), ws, device=dev)
    dofs_per_solve = {p: cdl.cd_dofs(2, p, N_INT) for p in PS}
    dof_s = sum(dofs_per_solve[r["p"]] for r in ok) * ws / (total_ms_all / 1e3)
    per_beta = {}
    for bv in BETAS:
        sel = [r for r in flat if r["beta"] == bv]
        per_beta[f"{bv:g}"] = {"converged": sum(1 for r in sel if r["status"] == 0),
                               "total": len(sel),
                               "iters_median": float(np.median([r["iters_inner"] for r in sel])),
                               "iters_max": int(max(r["iters_inner"] for r in sel)),
                               "worst_relres": max(r["relres"] for r in sel),
                               "worst_relres_fp64_part": max(r["relres_hi"] for r in sel)}

    # like-for-like with the CPU baseline: the beta = 1 solves of the sweep alone (8 per p)
    def solve_beta1(i):
        k = list(BETAS).index(1.0) * len(SEEDS)
        n1 = len(SEEDS)
        N = solvers_[i].N
        return solvers_[i].cd_solve_ext(rhs[i][k * N:(k + n1) * N], xs[i][:n1 * N],
                                        xlos[i][:n1 * N], alph[i][:n1], [1.0] * n1, check=False)[1]
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    out1, _ = concurrent(solve_beta1)
    torch.cuda.synchronize()
    beta1 = {"value": sum(1 for res in out1 for r in res if r["status"] == 0) / (time.perf_counter() - tb0),
             "unit": "solves/s", "sample": "the 24 beta = 1 solves of the sweep (8 per p), batched per p, "
                                           "wall time including the host calls"}

    # e2e through the public API with pinned host buffers: every step copies b in, solves, and
    # reads x and x_lo back; the copies run on each shape's stream
    xh = [torch.empty(B * sv.N, dtype=torch.float64).pin_memory() for sv in solvers_]
    xlh = [torch.empty(B * sv.N, dtype=torch.float64).pin_memory() for sv in solvers_]

    def solve_host(i):
        with torch.cuda.stream(streams[i]):
            rhs[i].copy_(rhs_host[i], non_blocking=True)
        res = solvers_[i].cd_solve_ext(rhs[i], xs[i], xlos[i], alph[i], bet[i], check=False)[1]
        with torch.cuda.stream(streams[i]):
            xh[i].copy_(xs[i], non_blocking=True)
            xlh[i].copy_(xlos[i], non_blocking=True)
        streams[i].synchronize()
        return res
    e2e_steps = max(1, min(args.steps, 2))
    e2e_ok = 0
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        out_h, _ = concurrent(solve_host)
        e2e_ok += sum(1 for res in out_h for r in res if r["status"] == 0 and r["relres"] <= RTOL)
    e2e_s = time.perf_counter() - te0
    h2d = sum(t.numel() * 8 for t in rhs_host)

    # rooflines of the two operator applies on the p = 3 batch (B = 40): FP32 (inner solves)
    # against the measured HBM copy bandwidth, FP64 (refinement residual products, FP64 inner
    # solves of the extreme ratios) against the measured FP64 DGEMM rate
    hbm, peak_kind = peaks()
    s3, st3 = solvers_[1], streams[1]
    t32 = time_apply(s3, st3, flush, B, torch.float32, alph[1], bet[1])
    t64 = time_apply(s3, st3, flush, B, torch.float64, alph[1], bet[1])
    p3 = PS[1]
    unknowns = B * s3.N
    fp64_tf = fp64_peak_tflops(dev)
    rl32 = {"bound": "hbm", "achieved": 2 * unknowns * 4 / t32 / 1e9, "peak": hbm, "unit": "GB/s",
            "traffic": None, "peak_kind": peak_kind,
            "kernel": "apply2d FP32 (autotuned v5/v3, p=3, n=256, batch 40)", "launch_us": t32 * 1e6}
    rl32["frac"] = rl32["achieved"] / hbm
    flops64 = 12 * (2 * p3 + 1) * unknowns
    rl64 = {"bound": "fp64", "achieved": flops64 / t64 / 1e12, "peak": fp64_tf, "unit": "TFLOP/s",
            "traffic": None, "peak_kind": "measured (cuBLAS DGEMM 4096^3 in this run)",
            "kernel": "apply2d_v2_kernel<double> (p=3, n=256, batch 40)", "launch_us": t64 * 1e6,
            "hbm_gbs": 2 * unknowns * 8 / t64 / 1e9}
    rl64["frac"] = rl64["achieved"] / fp64_tf
    # the step's dominant kernel (launch list of the tail: profiles/): the double-FP32 2D apply
    # of the FP64 inner solves at the extreme ratios, on the 16 right-hand sides that stay active
    # in a batch's tail.  Work = the plain double-FP32 form: 6 (2p+1) multiply-adds per unknown,
    # 12 FP32 operations each (two-product with cross terms 4, two-sum 6, low-part sums 2).
    Bff = 16
    os.environ["CURLDIV_APPLY_KERNEL_FP64"] = "ff"
    stff = torch.cuda.Stream(dev)
    sff = cdl.Solver(2, p3, N_INT, max_batch=Bff, precond=cdl.CD_PC_NONE, autotune=0,
                     stream=stff.cuda_stream)
    os.environ.pop("CURLDIV_APPLY_KERNEL_FP64", None)
    tff = time_apply(sff, stff, flush, Bff, torch.float64, np.ones(Bff), np.full(Bff, 1e6))
    sff.close()
    alu_tops, n_sm, sm_mhz = alu_peak_tops(dev)
    ops_ff = 72 * (2 * p3 + 1) * Bff * s3.N
    rlff = {"bound": "alu", "achieved": ops_ff / tff / 1e12, "peak": alu_tops, "unit": "TOP/s",
            "traffic": None,
            "peak_kind": f"nominal FP32 lanes x clock: {n_sm} SMs x 128 x {sm_mhz:.0f} MHz",
            "kernel": f"apply2d_ff2_kernel<3> (double-FP32 apply, p=3, n=256, batch {Bff})",
            "launch_us": tff * 1e6, "ops_per_launch": ops_ff,
            "ops_definition": "72 (2p+1) FP32 operations per unknown (the plain double-FP32 "
                              "sum-factorised form)",
            "fp64_equiv_tflops": 12 * (2 * p3 + 1) * Bff * s3.N / tff / 1e12,
            "hbm_gbs": 2 * Bff * s3.N * 8 / tff / 1e9}
    rlff["frac"] = rlff["achieved"] / alu_tops

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "solves_per_step": len(PS) * B, "batch": B,
                           "precond": args.precond, "precision": args.precision,
                           "solution": "double-FP64 (x + x_lo, cd_solve_ext); relres of x + x_lo",
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": f"replicas x{ws}"},
                "value_definition": "solves that reached relres <= 1e-10 (status OK) per second; "
                                    "value_all_solves counts every solve",
                "value_all_solves": value_all, "dof_per_s": dof_s,
                "latency_s": {"p50": float(np.percentile(lat_all, 50)), "p99": float(np.percentile(lat_all, 99)),
                              "definition": "per solve, from step start to the return of its batched call "
                                            "(three shape batches run concurrently on three streams)"},
                "solves": {"converged": len(ok), "total": len(flat),
                           "worst_relres": max(r["relres"] for r in flat),
                           "iters_median": float(np.median([r["iters_inner"] for r in flat])),
                           "iters_max": int(max(r["iters_inner"] for r in flat)),
                           "converged_per_step": n_conv_local},
                "per_beta": per_beta,
                "beta1_only": beta1,
                "e2e": {"value": e2e_ok / e2e_s, "unit": "solves/s", "steps": e2e_steps,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 2 * h2d,
                        "definition": "pinned host b -> device, cd_solve_ext, x and x_lo -> pinned host, "
                                      "wall time, converged solves counted"},
                "roofline": {"ff": rlff, "fp64": rl64, "fp32": rl32}[args.roofline_kernel],
                "roofline_other": [r for k, r in (("ff", rlff), ("fp32", rl32), ("fp64", rl64))
                                   if k != args.roofline_kernel],
                "roofline_choice": "kernel named by --roofline-kernel (default: the step's dominant "
                                   "kernel in its launch list, summarised under profiles/)",
                "gpu_launches": int(launches),
                "clocks": clk}
        cfgs = [c for c in args.configs.split(",") if c]
        if "c3" in cfgs:
            line["c3"] = measure_c3(dev, cdl, inputs, flush)
        if "c4" in cfgs:
            line["c4"] = measure_c4(dev, cdl, inputs, flush, args.c4_fp64)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_serving(args):
    """Serving-stream workload: the first K requests of the seeded Poisson stream (60% 2D with n
    in 32..256, 40% 3D with n in 16..96, p in 1..5, beta log-uniform in [1e-6, 1e6], 1-4 RHS),
    replayed at their arrival times (a) through the continuous-batching server (mixed precision,
    multigrid, iteration-level sessions, worker pool) and (b) through the plain solver: FP64, one request at a time (its
    right-hand sides in one call), a handle created per shape.  Same tolerance and iteration cap
    for both.  Host buffers in both arms; per-shape set-up is inside the timed region of both."""
    import torch
    from paper_1805_10058_gb300 import curldiv as cdl
    from paper_1805_10058_gb300 import inputs

    torch.cuda.init()
    reqs = inputs.serving_stream(seed=0, count=args.serving_requests)
    rhs = [inputs.uniform_rhs(r["d"], r["p"], r["n"], seed=r["seed"], nrhs=r["nrhs"]).ravel()
           for r in reqs]
    nsolves = sum(r["nrhs"] for r in reqs)
    solve_opts = dict(rtol=RTOL, maxit=args.maxit, precond=cdl.CD_PC_MG)

    def replay(submit, finish):
        t0 = time.perf_counter()
        pending = []
        for r, b in zip(reqs, rhs):
            dt = r["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            pending.append(submit(r, b))
        out = [finish(h) for h in pending]
        return time.perf_counter() - t0, out

    # (a) server
    srv = cdl.Server(workers=args.workers, max_batch=8,
                     solve=dict(solve_opts, precision=cdl.CD_PREC_FP32_IR))
    wall_a, out_a = replay(
        lambda r, b: srv.submit(r["d"], r["p"], r["n"], r["alpha"], r["beta"], b),
        lambda t: srv.wait(t))
    stats = srv.stats()
    srv.close()

    # (b) plain FP64, one request at a time
    lat_b = []

    def plain(r, b):
        t_arr = r["t"]
        s = cdl.Solver(r["d"], r["p"], r["n"], max_batch=r["nrhs"],
                       precision=cdl.CD_PREC_FP64, **solve_opts)
        x = np.zeros_like(b)
        st, res = s.cd_solve_host(b, x, [r["alpha"]] * r["nrhs"], [r["beta"]] * r["nrhs"])
        s.close()
        lat_b.append((time.perf_counter() - t_start[0]) - t_arr)
        return st, x, res

    t_start = [time.perf_counter()]
    wall_b, out_b = replay(plain, lambda h: h)

    def summary(out):
        rel = [rr["relres"] for o in out for rr in o[2]]
        return sum(1 for v in rel if v <= RTOL), max(rel)

    conv_a, worst_a = summary(out_a)
    conv_b, worst_b = summary(out_b)
    # agreement of the two arms on the solves both converged
    diffs = []
    for oa, ob, r in zip(out_a, out_b, reqs):
        N = cdl.cd_dofs(r["d"], r["p"], r["n"])
        for k in range(r["nrhs"]):
            if oa[2][k]["relres"] <= RTOL and ob[2][k]["relres"] <= RTOL:
                xa, xb = oa[1][k * N:(k + 1) * N], ob[1][k * N:(k + 1) * N]
                diffs.append(float(np.linalg.norm(xa - xb) / np.linalg.norm(xb)))
    lat_b.sort()
    line = {
        "metric": "serving solves/s + p50/p99 latency at 1e-10 residual",
        "value": conv_a / wall_a, "unit": "solves/s", "n_gpus": 1,
        "value_definition": "right-hand sides solved to relres <= 1e-10 by the server arm per "
                            "second of its wall time (arrivals replayed)",
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"serving stream, first {len(reqs)} requests of the seeded Poisson "
                               "stream (mean 200/s): 60% 2D n in 32..256, 40% 3D n in 16..96, "
                               "p in 1..5, beta log-uniform [1e-6, 1e6], 1-4 RHS, rtol 1e-10",
                   "requests": len(reqs), "solves": nsolves, "maxit": args.maxit,
                   "workers": args.workers, "distinct_shapes":
                       len({(r["d"], r["p"], r["n"]) for r in reqs})},
        "server": {"solves_per_s": conv_a / wall_a, "wall_s": wall_a, "p50_s": stats["p50_s"],
                   "p99_s": stats["p99_s"], "batches": stats["batches"],
                   "mean_batch": stats["mean_batch"], "converged": conv_a},
        "plain_fp64_one_at_a_time": {
            "solves_per_s": conv_b / wall_b, "wall_s": wall_b,
            "p50_s": lat_b[len(lat_b) // 2], "p99_s": lat_b[min(len(lat_b) - 1, int(0.99 * len(lat_b)))],
            "converged": conv_b},
        "speedup": (conv_a / wall_a) / (conv_b / wall_b) if conv_b else None,
        "agreement": {"max_rel_diff_x": max(diffs) if diffs else None, "compared": len(diffs)},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_kernel(args):
    """A few launches of one kernel on its profiling case, for ncu (no timing): `apply` = the
    FP32 2D apply at p = 3, n = 256, batch 40 (four calls); `fd` = two FP32 FD-D applications
    on the tensor cores at the same size (four passes each); `tail` = the kind of iteration that
    dominates a sweep step: 16 solves at beta/alpha = 1e-6 and 1e6 (p = 3, n = 256, mixed
    precision, which runs them in the FP64 inner group), multigrid FCG capped at 120 iterations;
    `ff` = the double-FP32 2D apply of those inner solves at p = 3, n = 256, batch 16; `ff3d` =
    the double-FP32 3D passes at p = 3, n = 64, batch 4."""
    import torch
    from paper_1805_10058_gb300 import curldiv as cdl
    B = 40
    if args.profile_kernel == "tail":
        from paper_1805_10058_gb300 import inputs
        B = 16
        s = cdl.Solver(2, 3, N_INT, max_batch=B, precond=cdl.CD_PC_MG, rtol=1e-10, maxit=120)
        b = torch.as_tensor(inputs.uniform_rhs(2, 3, N_INT, seed=0, nrhs=B).ravel(), device="cuda")
        x, xl = torch.zeros_like(b), torch.zeros_like(b)
        st, res = s.cd_solve_ext(b, x, xl, [1.0] * B, [1e-6] * 8 + [1e6] * 8, check=False)
        assert st in (cdl.CD_OK, cdl.CD_NOT_CONVERGED), st
        print("launches", cdl.cd_kernel_launches())
    elif args.profile_kernel == "ff":
        os.environ["CURLDIV_APPLY_KERNEL_FP64"] = "ff"
        B = 16
        s = cdl.Solver(2, 3, N_INT, max_batch=B, precond=cdl.CD_PC_NONE, autotune=0)
        w = torch.rand(B * s.N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(w)
        for _ in range(4):
            s.cd_apply(w, y, [1.0] * B, [1e6] * B)
    elif args.profile_kernel == "ff3d":
        os.environ["CURLDIV_APPLY_KERNEL_FP64"] = "ff"
        B = 4
        s = cdl.Solver(3, 3, 64, max_batch=B, precond=cdl.CD_PC_NONE, autotune=0)
        w = torch.rand(B * s.N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(w)
        for _ in range(3):
            s.cd_apply(w, y, [1.0] * B, [1e6] * B)
    elif args.profile_kernel == "apply":
        s = cdl.Solver(2, 3, N_INT, max_batch=B, precond=cdl.CD_PC_NONE, autotune=0)
        w = torch.rand(B * s.N, dtype=torch.float32, device="cuda")
        y = torch.empty_like(w)
        for _ in range(4):
            s.cd_apply_f32(w, y, [1.0] * B, [1e-3] * B)
    else:
        s = cdl.Solver(2, 3, N_INT, max_batch=B, precond=cdl.CD_PC_FD_D, fd_tensor_cores=1)
        r = torch.rand(B * s.N, dtype=torch.float32, device="cuda")
        z = torch.empty_like(r)
        for _ in range(2):
            s.cd_precond(cdl.CD_PC_FD_D, r, z, [1.0] * B, [1e-3] * B)
    torch.cuda.synchronize()
    print("ok")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--precond", default="mg", choices=["mg", "mim", "fdd", "none"])
    ap.add_argument("--roofline-kernel", default="ff", choices=["ff", "fp64", "fp32"],
                    help="which operator apply the roofline key reports (the step's dominant one)")
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs", default="c3,c4",
                    help="extra workloads measured after the timed sweep (comma list of c3, c4)")
    ap.add_argument("--c4-fp64", action="store_true", help="also run the C4 solves all-FP64")
    ap.add_argument("--serving", action="store_true", help="serving-stream workload instead")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--profile-kernel", choices=["apply", "fd", "tail", "ff", "ff3d"], default=None,
                    help="a few launches of one kernel for ncu, no timing")
    args = ap.parse_args()
    if args.profile_kernel:
        return run_profile_kernel(args)
    if args.serving:
        return run_serving(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
