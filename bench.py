#!/usr/bin/env python
"""Benchmark of Fourier-accelerated steepest-descent Landau gauge fixing.

Workload: a 32^4 SU(3) lattice built as U_mu(x) = h(x) exp(i eps sum_a c_a
lambda_a/2) h^dag(x+mu) (eps = 1.0, Haar h, seed = rank), alpha = 0.08.
One "step" is one body of Algorithm 1 (4D FFT of the divergence, filter,
inverse FFT, g = reunitarize(1 + Delta'), link update, measurement of Delta,
F and theta) in plain FP64 with 18-real links, run through the C-ABI.

Printed: one JSON line with iterations/s (the headline), site updates/s,
per-kernel times, the roofline of the dominant kernel, the FP32 12-real
rate, the wall time to theta < 1e-15 of plain FP64 and of the mixed
FP32 -> FP64 mode (with and without the learned multiplier), the 64-lattice
batch, overrelaxation sweeps/s and its time to theta < 1e-15 (the other
gauge-fixing method of Sec. 3.2), an end-to-end figure through host buffers,
the CPU oracle's rate on the host cores, and the SM clocks seen while timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lgf|reference]

With --impl reference the CPU oracle (plain FP64 numpy) is timed on the
same workload and metric instead.  Multi-GPU runs (torchrun) are replicas:
each rank fixes its own lattice, no data moves between GPUs.
"""

from __future__ import annotations

import argparse
import json
import os
import resource
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1206_0675_gb300 import accounting, fields  # noqa: E402

EXT = (32, 32, 32, 32)
EPS = 1.0
ALPHA = 0.08
TOL = 1e-15
OR_OMEGA = 1.7      # overrelaxation parameter of the overrelaxation measurements
OR_CHECK = 10       # their sweeps between measurements of theta
METRIC = "FA-SD iters/s at 32^4 (plain FP64, 18-real links)"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 pipe of a GB300: 152 SMs x 2 FP64 instructions per clock x 2070 MHz;
# counted as FMA-equivalents (2 flops per FP64 instruction).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# kernels of one step: the transform passes, g where it is not fused, update, measure
KERNELS_PER_STEP = {"2d2d": 5, "1d4": 10, "3d1d": 6}


# DRAM bytes (read + write) per launch of the FP64 update kernel at 32^4 from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only
# while the kernel's source text and the shared device header are unchanged
# (sha256 prefixes); reported as null otherwise.
NCU_TRAFFIC = {
    "update": {"bytes": 762.235904e6 + 548.043776e6, "kernel_sha": "6a87d4e0230e19cb",
               "common_sha": "51a6996aeb16a34c"},
}


def kernel_source_sha(name):
    """sha256 prefix of a kernel's definition text in lgf_site.cu and of lgf_common.cuh."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1206_0675_gb300/csrc/lgf_site.cu")).read()
    a = src.index(f"{name}_kernel(Geom")
    b = src.index("cudaError_t launch_", a)
    common = open(os.path.join(ROOT, "paper_1206_0675_gb300/csrc/lgf_common.cuh"), "rb").read()
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16], hashlib.sha256(common).hexdigest()[:16]


def ncu_traffic(kernel):
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None or rec["bytes"] is None:
        return None
    if kernel_source_sha(kernel) != (rec["kernel_sha"], rec["common_sha"]):
        return None
    return rec["bytes"]


def workload_desc():
    return (f"SU(3) {EXT[0]}^4 periodic lattice, U_mu(x)=h(x) exp(i eps sum_a c_a lambda_a/2) h^dag(x+mu), "
            f"eps={EPS}, c_a~N(0,1), Haar h, seed=rank; plain FA-SD alpha={ALPHA}")


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if exe is None:
            return
        self.proc = subprocess.Popen([exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                      "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                     stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def host_cores():
    """Cores this process may run on (the box's nproc unless an affinity mask is set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / 1e6
    except OSError:
        pass
    return None


# Resident memory of one oracle replica at 32^4 (links, divergence, FFTs and
# temporaries of numpy's whole-array operations), with a margin.
ORACLE_GB_PER_REPLICA_32X4 = 4.5


def _oracle_replica(ext, eps, seed, n, barrier, out):
    """One oracle replica in its own (spawned, single-threaded) process: build
    its field, wait for the others, then time n bodies of Algorithm 1."""
    from oracle import lgf_oracle as O
    U = fields.random_links(ext, eps, seed)
    K = O.fa_filter(O.extents_of(U), ALPHA)
    _, _, D = O.measure(U)
    barrier.wait()
    t0 = time.perf_counter()
    c0 = time.process_time()
    for _ in range(n):
        U, _ = O.fa_step(U, ALPHA, K, D)
        _, _, D = O.measure(U)
    out.put((seed, time.perf_counter() - t0, time.process_time() - c0))


def oracle_all_cores(ext, n, replicas=None):
    """The oracle as it stands on every host core: one single-threaded replica
    (its own seeded field, n bodies) per core, all started together after
    their fields are built.  Returns (iterations/s of all replicas together,
    replicas, wall seconds, per-replica seconds)."""
    import multiprocessing as mp
    P = replicas or host_cores()
    avail = mem_available_gb()
    if avail is not None:
        P = max(1, min(P, int(avail * 0.8 // ORACLE_GB_PER_REPLICA_32X4)))
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(P + 1), ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        procs = [ctx.Process(target=_oracle_replica, args=(ext, EPS, 100 + i, n, barrier, out)) for i in range(P)]
        for p in procs:
            p.start()
        barrier.wait()
        t0 = time.perf_counter()
        res = [out.get() for _ in range(P)]
        wall = time.perf_counter() - t0
        for p in procs:
            p.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return P * n / wall, P, wall, sorted(r[1] for r in res)


def oracle_iterations(U, n):
    """n bodies of Algorithm 1 with the CPU oracle; returns (seconds, cores used)."""
    from oracle import lgf_oracle as O
    K = O.fa_filter(O.extents_of(U), ALPHA)
    _, _, D = O.measure(U)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(n):
        U, _ = O.fa_step(U, ALPHA, K, D)
        _, _, D = O.measure(U)
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return dt, max(1, int(round(cpu / dt))), U


def run_reference(args, rank, world):
    if rank != 0:
        return
    U = fields.random_links(EXT, EPS, 0)
    # one warm-up body on one core sizes the run so that it ends within a few minutes
    t1, _, U = oracle_iterations(U, 1)
    budget = 120.0
    W = 1
    K = max(1, min(args.steps, int(budget / t1)))
    value, cores, wall, _ = oracle_all_cores(EXT, K)
    dt = wall
    sample = (f"{cores} single-threaded oracle replicas (one per host core, own seeded 32^4 field each), "
              f"{K} bodies of Algorithm 1 (FFT, filter, IFFT, g, update, measure) each, timed together after "
              f"one warm-up body on one core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(), "lattice": list(EXT), "precision": "fp64", "storage": "18-real",
                   "engine": "CPU oracle (numpy FP64)"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def max_over_ranks(ms, device):
    """The largest of the ranks' elapsed times (ms); the job is as slow as its slowest replica."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, world, max_ms):
    """Steps per second of all replicas together: world * steps in the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


def time_region(torch, lat, K, reps):
    """Median over reps timed regions of K steps each (ms), and all of them."""
    t = [time_steps(torch, lat, K) for _ in range(reps)]
    return float(np.median(t)), t


def time_steps(torch, lat, K):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(K):
        lat.step(ALPHA)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_lgf(args, rank, world, local_rank):
    import torch
    from paper_1206_0675_gb300 import lgf

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    V = int(np.prod(EXT))
    U = fields.random_links(EXT, EPS, rank)
    hbm_peak, peak_kind = peaks()

    # ---- plain FP64, 18-real: the headline --------------------------------
    lat = lgf.Lattice(EXT, "fp64")
    lat.set_links(U)
    tune = lat.autotune()["fp64"]
    chosen = tune["candidates"][tune["chosen"]]
    decomp = chosen["decomposition"]
    # the built-in 2D + 2D plan is the first candidate (a cached choice carries no timings)
    default_ms = None if tune["cached"] else tune["candidates"][0]["ms"]
    for _ in range(args.warmup):
        lat.step(ALPHA)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    # the headline: median of args.reps regions of K steps, no per-kernel events
    ms, ms_regions = time_region(torch, lat, args.steps, args.reps)
    # per-kernel split: one more region of K steps with CUDA events around every kernel
    lat.set_timing(True)
    ms_split = time_steps(torch, lat, args.steps)
    kms, nsteps = lat.get_timing()
    lat.set_timing(False)
    clocks = sampler.stop()
    if dist:
        ms = max_over_ranks(ms, "cuda")
    ms_step = ms / args.steps
    value = whole_job_rate(args.steps, world, ms)

    ops = accounting.fp64_ops_per_site(EXT, rows=3, decomposition=decomp)
    byt = accounting.bytes_per_site(8, 3, 3, k_bytes=8, decomposition=decomp)
    per_kernel = {}
    for name, t_ms in zip(accounting.KERNELS, kms):
        per_kernel[name] = {
            "ms": t_ms,
            "fp64_tflops": 2 * ops[name] * V / (t_ms * 1e-3) / 1e12 if t_ms > 0 else None,
            "gbs": byt[name] * V / (t_ms * 1e-3) / 1e9 if t_ms > 0 else None,
        }
    dom = max(accounting.KERNELS, key=lambda k: per_kernel[k]["ms"])
    achieved = per_kernel[dom]["fp64_tflops"]
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": ncu_traffic(dom),
                "note": "FP64 pipe: every FP64 instruction counted as one FMA (2 flops); peak = 152 SMs x 2 "
                        "FP64 inst/clk x 2070 MHz; per-launch time from CUDA events on the launching stream"}
    b_alg = accounting.b_alg_per_site(8, 3)
    step_hbm = {"b_alg_bytes_per_site": b_alg, "achieved_gbs": b_alg * V / (ms_step * 1e-3) / 1e9,
                "peak_gbs": hbm_peak, "peak_kind": peak_kind,
                "frac": b_alg * V / (ms_step * 1e-3) / 1e9 / hbm_peak,
                "schedule_bytes_per_site": sum(byt.values())}

    # ---- end to end through host buffers ----------------------------------
    pinned = torch.from_numpy(U).pin_memory()
    Ke = min(args.steps, 20)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        lat.set_links(pinned)
        lat.step(ALPHA)
        lat.measure()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = max_over_ranks(e2e_s * 1e3, "cuda") / 1e3
    e2e = {"value": world * Ke / e2e_s, "unit": "iters/s", "h2d_bytes_per_step": int(U.nbytes),
           "d2h_bytes_per_step": 16,
           "note": "per step: lgf_set_links from pinned host memory (H2D copy, SU(3) check, layout conversion, "
                   "measurement), lgf_step, lgf_measure (D2H of F and theta)"}
    lat.close()
    del pinned

    # ---- FP32 12-real rate --------------------------------------------------
    lat32 = lgf.Lattice(EXT, "fp32", store12=True)
    lat32.set_links(U)
    tune32 = lat32.autotune()["fp32"]
    decomp32 = tune32["candidates"][tune32["chosen"]]["decomposition"]
    for _ in range(args.warmup):
        lat32.step(ALPHA)
    ms32, _ = time_region(torch, lat32, args.steps, args.reps)
    lat32.set_timing(True)
    time_steps(torch, lat32, args.steps)
    kms32, _ = lat32.get_timing()
    lat32.set_timing(False)
    lat32.close()
    b32 = accounting.bytes_per_site(4, 2, 2, k_bytes=4, decomposition=decomp32)
    # FP32 lanes fuse the update with the measurement: "update" carries both
    b32["update"] = accounting.fused_update_measure_bytes(4, 2, 2)
    b32["measure"] = 0
    ops32 = accounting.fp32_path_fp64_ops_per_site()
    fp32 = {"iters_per_s": args.steps / (ms32 / 1e3), "ms_per_step": ms32 / args.steps,
            "fft_decomposition": decomp32, "autotune": tune32["candidates"][tune32["chosen"]],
            "fused_update_measure": True,
            "per_kernel": {k: {"ms": t, "gbs": b32[k] * V / (t * 1e-3) / 1e9 if t > 0 else None,
                               "fp64_tflops": 2 * ops32[k] * V / (t * 1e-3) / 1e12 if t > 0 else None}
                           for k, t in zip(accounting.KERNELS, kms32)},
            "hbm_frac_b_alg": accounting.b_alg_per_site(4, 2) * V / (ms32 / args.steps * 1e-3) / 1e9 / hbm_peak}

    # ---- time to theta < 1e-15: plain FP64 vs mixed -------------------------
    ttt = None
    if not args.no_tol:
        from paper_1206_0675_gb300.preconditioner import DEFAULT_WEIGHTS
        weights = np.load(DEFAULT_WEIGHTS)
        ttt = {"tol": TOL, "field": f"32^4 eps={EPS} seed={rank}"}
        modes = (("fp64_18", dict(precision="fp64"), None),
                 ("mixed_12", dict(precision="mixed", store12=True), None),
                 ("mixed_12_switch_1e-10", dict(precision="mixed", store12=True), 1e-10),
                 ("mixed_12_learned", dict(precision="mixed", store12=True, learned=True), None),
                 ("mixed_12_learned_switch_1e-10", dict(precision="mixed", store12=True, learned=True), 1e-10))
        for mode, kw, sw in modes:
            L2 = lgf.Lattice(EXT, **kw)
            if kw.get("learned"):
                L2.load_preconditioner(weights)
            if sw is not None:
                L2.set_switch_theta(sw)
            L2.set_links(U)
            L2.autotune()
            L2.fix(TOL, 1, ALPHA)           # builds the loop graph
            L2.set_links(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, F, th, conv = L2.fix(TOL, args.max_iter, ALPHA)
            torch.cuda.synchronize()
            ttt[mode] = {"seconds": time.perf_counter() - t0, "iters": it, "F": F, "theta": th, "converged": conv}
            if kw.get("learned"):
                ttt[mode]["fallbacks"] = L2.fallbacks()
            L2.close()
        ttt["speedup_mixed"] = ttt["fp64_18"]["seconds"] / ttt["mixed_12"]["seconds"]
        ttt["speedup_mixed_learned"] = ttt["fp64_18"]["seconds"] / ttt["mixed_12_learned"]["seconds"]
        ttt["speedup_mixed_switch_1e-10"] = ttt["fp64_18"]["seconds"] / ttt["mixed_12_switch_1e-10"]["seconds"]
        ttt["speedup_mixed_learned_switch_1e-10"] = (ttt["fp64_18"]["seconds"]
                                                     / ttt["mixed_12_learned_switch_1e-10"]["seconds"])

    # ---- 64 configurations of uneven shapes in one graph launch -------------
    batch = None
    if not args.no_batch:
        exts = fields.BATCH64_EXTENTS
        Ub = [fields.random_links(e, fields.batch_eps(i), 1000 * rank + i) for i, e in enumerate(exts)]
        with lgf.Batch(exts) as b:
            for i, u in enumerate(Ub):
                b.set_links(i, u)
            b.fix(1e-14, 1)            # builds the loop graph
            for i, u in enumerate(Ub):
                b.set_links(i, u)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it_b, F_b, th_b, conv_b = b.fix(1e-14, 30000)
            dt_b = time.perf_counter() - t0
            classes = b.describe()
        vols = np.array([int(np.prod(e)) for e in exts])
        batch = {"configs": len(exts), "tol": 1e-14, "seconds": dt_b, "converged": bool(conv_b),
                 "iters_total": int(it_b.sum()), "iters_max": int(it_b.max()),
                 "site_updates_per_s": float((vols * it_b).sum() / dt_b), "classes": classes,
                 "workload": "16x8^4, 16x12^4, 16x16^4, 8x16^3x32, 8x24^4; eps ~ U[0.3,1.0]; one graph launch"}

    # ---- overrelaxation (the lower-memory method of Sec. 3.2) ---------------
    orx = None
    if not args.no_or:
        orx = {"omega": OR_OMEGA, "field": f"32^4 eps={EPS} seed={rank}",
               "note": "checkerboard sweeps (even colour, then odd) of Cabibbo-Marinari hits with "
                       "Mandula-Ogilvie overrelaxation; each region is one lgf_or_sweep call of K sweeps "
                       "(2K colour kernels and one measurement)"}
        for mode, kw, real_bytes, rows in (("fp64_18", dict(precision="fp64"), 8, 3),
                                          ("fp32_12", dict(precision="fp32", store12=True), 4, 2)):
            Lo = lgf.Lattice(EXT, **kw)
            Lo.set_links(U)
            Lo.or_sweep(OR_OMEGA, args.warmup)
            torch.cuda.synchronize()
            t_or = []
            for _ in range(args.reps):
                st = torch.cuda.current_stream()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                Lo.or_sweep(OR_OMEGA, args.steps)
                e1.record(st)
                torch.cuda.synchronize()
                t_or.append(e0.elapsed_time(e1))
            Lo.close()
            ms_sw = float(np.median(t_or)) / args.steps
            byt_or = accounting.or_bytes_per_site_sweep(real_bytes, rows)
            ops_or = accounting.or_ops_per_site_sweep(rows)
            rec = {"sweeps_per_s": 1e3 / ms_sw, "ms_per_sweep": ms_sw, "site_updates_per_s": V * 1e3 / ms_sw,
                   "bytes_per_site_sweep": byt_or, "ops_per_site_sweep": ops_or,
                   "hbm_gbs": byt_or * V / (ms_sw * 1e-3) / 1e9,
                   "hbm_frac": byt_or * V / (ms_sw * 1e-3) / 1e9 / hbm_peak}
            if real_bytes == 8:
                rec["fp64_tflops"] = 2 * ops_or * V / (ms_sw * 1e-3) / 1e12
                rec["fp64_frac"] = rec["fp64_tflops"] / FP64_PEAK_TFLOPS
            orx[mode] = rec
        if not args.no_tol:
            for mode, kw in (("fix_fp64_18", dict(precision="fp64")),
                             ("fix_mixed_12", dict(precision="mixed", store12=True))):
                Lo = lgf.Lattice(EXT, **kw)
                Lo.set_links(U)
                Lo.or_fix(TOL, 1, OR_OMEGA, OR_CHECK)       # builds the loop graph
                Lo.set_links(U)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n, F, th, conv = Lo.or_fix(TOL, args.or_max_sweeps, OR_OMEGA, OR_CHECK)
                torch.cuda.synchronize()
                orx[mode] = {"seconds": time.perf_counter() - t0, "sweeps": n, "F": F, "theta": th,
                             "converged": conv, "tol": TOL, "check_every": OR_CHECK}
                Lo.close()

    # ---- CPU oracle on the host cores (rank 0, N = 1 only) ------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # every host core: one single-threaded oracle replica per core
        v_all, P, wall, per = oracle_all_cores(EXT, args.cpu_iters)
        # one core, on the bench's own field
        dt, cores1, _ = oracle_iterations(U, args.cpu_iters)
        cpu = {"value": v_all, "unit": "iters/s", "cores": P, "kind": "oracle", "nproc": host_cores(),
               "sample": f"{P} single-threaded replicas of the oracle (numpy FP64), one per host core, each "
                         f"{args.cpu_iters} bodies of Algorithm 1 on its own seeded 32^4 field (eps={EPS}), "
                         f"started together; value = {P * args.cpu_iters} bodies / {wall:.1f} s wall",
               "single_core": {"value": args.cpu_iters / dt, "unit": "iters/s", "cores": cores1,
                               "sample": f"{args.cpu_iters} oracle bodies on the bench's 32^4 field"},
               "seconds_per_iter": {"32^4": dt / args.cpu_iters, "32^4_all_cores_per_replica": float(np.median(per))
                                    / args.cpu_iters}}
        for L, n in ((8, 20), (16, 5)):     # the smaller lattices of the workload, a few seconds each
            dts, _, _ = oracle_iterations(fields.random_links((L,) * 4, EPS, rank), n)
            cpu["seconds_per_iter"][f"{L}^4"] = dts / n

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "timing": {"regions": args.reps, "steps_per_region": args.steps, "ms_per_region": ms_regions,
                       "statistic": "median of the regions (no per-kernel events inside them)",
                       "per_kernel_region_ms": ms_split,
                       "note": "per-kernel times come from one further region with CUDA events around every "
                               "kernel"},
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(), "lattice": list(EXT), "precision": "fp64",
                       "storage": "18-real", "alpha": ALPHA, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "no flush needed: each step streams 604 MB of links (> 129 MB L2)"},
            "site_updates_per_s": value * V,
            "per_kernel": per_kernel, "roofline": roofline, "step_hbm": step_hbm, "fp32_12": fp32,
            "time_to_tol": ttt, "batch64": batch, "overrelaxation": orx, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": KERNELS_PER_STEP[decomp] * args.steps * args.reps,
            "autotune": {"fft_decomposition": decomp, "fields_per_cta_xy": chosen["fields_per_cta_xy"],
                         "x_columns_zt": chosen["x_columns_zt"], "threads": chosen["threads"],
                         "lines_x": chosen["lines_x"], "x_columns_line": chosen["x_columns_line"],
                         "transform_ms": chosen["ms"], "default_plan_transform_ms": default_ms,
                         "candidates": len(tune["candidates"]), "cached": tune["cached"],
                         "note": "lgf_autotune before the warm-up: every tile plan of the 2D+2D passes and the "
                                 "1D x 4 / 3D + 1D decompositions timed on the device, fastest kept"},
            "paper_context": {"c2070_dp_ms_per_iter_12real_tex": 61.16, "c2070_dp_ms_per_iter_18real_tex": 100.65,
                              "note": "derived from the paper's Table 2 (real beta=5.8-6.2 configurations)"},
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lgf", choices=["lgf", "reference"])
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=5, help="timed regions of --steps steps (median reported)")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--no-tol", action="store_true", help="skip the time-to-threshold runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-configuration batch")
    ap.add_argument("--no-or", action="store_true", help="skip the overrelaxation measurements")
    ap.add_argument("--or-max-sweeps", type=int, default=20000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        # the CPU oracle runs on rank 0 only; other ranks exit without work
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        run_lgf(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
