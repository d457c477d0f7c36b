#!/usr/bin/env python
"""Benchmark of the ECS Helmholtz solver on the 512^2 + 64-layer workload.

Workload (one "step"): the 2D ECS Helmholtz problem with a 512 x 512 interior grid and a
64-node ECS layer on every side (640 x 640 = 409,600 unknowns), theta_gamma = 0.5, kh = 0.5
(k0 = 255.5), k(x) = k0 (1 + 0.3 exp(-|x - c|^2 / 0.02)), Gaussian source of width 2h at a
seeded position, solved to a relative residual of 1e-6 four times:
{Bi-CGSTAB, IDR(4)} x {CSG theta_beta = 0.3, CSL shift 1 + 0.5i}, one V(1,1) cycle with
omega-Jacobi (0.5) per preconditioned matvec.  Every solve is certified by the FP64 true
residual ||b - H x|| / ||b|| < 1e-6 recomputed on the device.  The four solves of a step run at
once through helm_solve_batch (one context and one stream each; a lone 640^2 solve leaves much of
the GPU idle in its small multigrid levels and reductions); the same solves one after another
give each solve's latency (`latency_ms`) and the `sequential` throughput.

`value` is the all-FP64 path (FP64 V-cycle and Krylov); the FP32-multigrid path (FP32 V-cycle,
FP64 Krylov and true residual) is measured on the same step and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU): every rank solves its own copy (replicas, no data
exchange); the barrier and the max over ranks time the job.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import helm_inputs as hi  # noqa: E402

METRIC = "solves/s at 1e-6 true rel. residual, FP32-MG vs FP64; p50/p99 latency; HBM %peak"
TOL = 1e-6
SOLVES = [("bicgstab", hi.BICGSTAB, "csg"), ("bicgstab", hi.BICGSTAB, "csl"),
          ("idr4", hi.IDR, "csg"), ("idr4", hi.IDR, "csl")]


def precond(name: str) -> hi.Precond:
    if name == "csg":
        return hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    return hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5)


def config(p, concurrent=True) -> dict:
    return {"workload": p.name, "grid": "512^2 interior + 64 ECS nodes per side (640^2 unknowns)",
            "n_unknowns": p.n, "solves_per_step": len(SOLVES),
            "solves": "{Bi-CGSTAB, IDR(4)} x {CSG theta_beta=0.3, CSL shift 1+0.5i}",
            "execution": ("the four solves at once through helm_solve_batch (one context and stream each)"
                          if concurrent else "the four solves one after another (host-driven loop)"),
            "multigrid": "V(1,1), omega-Jacobi 0.5, FW, bilinear, rediscretised levels, dense coarsest",
            "tol": TOL, "l2": "flushed (512 MiB device write) before every timed step"}


# ---- ranks -------------------------------------------------------------------------------

class Ranks:
    """Replica bookkeeping for N > 1: every rank solves its own copy of the workload (no data
    exchange); the only collectives are the timing barrier and the max over ranks."""

    def __init__(self, dist=None, device=None):
        self.dist = dist
        self.device = device
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v: float) -> float:
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: int, ms_per_rank: float) -> float:
        """Whole-job throughput: units all ranks processed / the slowest rank's time."""
        return units_per_rank * self.world / (self.max(ms_per_rank) / 1000.0)


# ---- clocks ------------------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle ---------------------------------------------------------------------------

def oracle_counts():
    path = os.path.join(ROOT, "oracle", "workload_counts.json")
    with open(path) as fh:
        d = json.load(fh)
    return {(s["method"], s["precond"]): s["matvecs"] for s in d["solves"]}


def oracle_sample(p, mv_per_method: int) -> dict:
    """Times the oracle (on the threads oracle.set_threads chose) on a bounded sample:
    mv_per_method preconditioned matvecs of Bi-CGSTAB and of IDR(4) on the workload (CSG);
    returns seconds per matvec."""
    import oracle
    o = oracle.Oracle(p, precond("csg"))
    sh = hi.shadow_space(p.n, 4)
    out = {}
    for name, method in (("bicgstab", hi.BICGSTAB), ("idr4", hi.IDR)):
        t = time.perf_counter()
        _, info = o.solve(p.b, hi.SolveOpts(method=method, s=4, tol=1e-30, maxmv=mv_per_method, max_restarts=0),
                          shadow=sh)
        out[name] = (time.perf_counter() - t) / max(info["matvecs"], 1)
    return out


def oracle_step_seconds(per_mv: dict, counts: dict) -> float:
    return sum(counts[(m, pc)] * per_mv[m] for (m, _, pc) in SOLVES)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_leg(p, gpu_solutions: dict) -> tuple:
    """The CPU baseline and the error reference, both from the oracle as it stands on this host's
    cores (its point-wise loops on every core, its inner products serial; the results do not depend
    on the thread count):
      - one complete solve of the step's first kind (Bi-CGSTAB, CSG, tol 1e-6), timed, on all cores;
      - a single-thread figure from a bounded sample (preconditioned matvecs of Bi-CGSTAB and IDR(4))
        scaled by the oracle's own matvec counts of the four solves;
      - the oracle's solution at tol 1e-12 (untimed), against which every GPU solution in
        `gpu_solutions` ({name: host complex128 vector}) gets its relative error."""
    import oracle
    cores = host_cores()
    oracle.set_threads(cores)
    o = oracle.Oracle(p, precond("csg"))
    t = time.perf_counter()
    _, info = o.solve(p.b, hi.SolveOpts(method=hi.BICGSTAB, tol=TOL, maxmv=4000))
    full_s = time.perf_counter() - t
    x_ref, iref = o.solve(p.b, hi.SolveOpts(method=hi.BICGSTAB, tol=1e-12, maxmv=8000))
    oracle.set_threads(1)
    mv = int(os.environ.get("HELM_CPU_SAMPLE_MV", "24"))
    per = oracle_sample(p, mv)
    single = len(SOLVES) / oracle_step_seconds(per, oracle_counts())
    oracle.set_threads(cores)
    nref = float(np.linalg.norm(x_ref))
    err = {"reference": "FP64 oracle, Bi-CGSTAB + CSG V(1,1), tol 1e-12 (the discrete solution of H x = b)",
           "reference_true_rel_res": iref["rel_res_true"],
           **{k: float(np.linalg.norm(v - x_ref) / nref) for k, v in gpu_solutions.items()}}
    cpu = {"value": 1.0 / full_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
           "sample": f"one complete solve of the workload (Bi-CGSTAB, CSG, tol 1e-6: {info['matvecs']} "
                     f"preconditioned matvecs, status {info['status']}) on all {cores} host cores, timed "
                     f"({full_s:.1f} s)",
           "single_thread": {"value": single, "unit": "solves/s", "cores": 1,
                             "sample": f"{mv} preconditioned matvecs each of Bi-CGSTAB and IDR(4) (CSG), one "
                                       f"thread; seconds per matvec x the oracle's own matvec counts of the "
                                       f"four solves (oracle/workload_counts.json)"}}
    return cpu, err


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    p = hi.workload_2d_512()
    counts = oracle_counts()
    cores = host_cores()
    oracle.set_threads(cores)
    mv = int(os.environ.get("HELM_REF_SAMPLE_MV", "24"))
    step_s = []
    for k in range(args.warmup + args.steps):
        per = oracle_sample(p, mv)
        if k >= args.warmup:
            step_s.append(oracle_step_seconds(per, counts))
    ms = 1000 * statistics.mean(step_s)
    value = len(SOLVES) / (ms / 1000)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": config(p),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: {mv} preconditioned matvecs each of Bi-CGSTAB and IDR(4) "
                                       f"(CSG) on the full 640^2 workload, on all {cores} host cores (point-wise "
                                       f"loops threaded, inner products serial); seconds per matvec x the "
                                       f"oracle's own matvec counts of the four solves "
                                       f"(oracle/workload_counts.json)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU ------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phase", default="all", choices=["all", "fp64", "fp32", "kernels"],
                    help="which timed paths to run: all (FP64 value, FP32-multigrid, e2e), only the "
                         "FP64 / FP32-multigrid device-timed path, or only the per-kernel rooflines "
                         "(for kernel profiling)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the Krylov loop from the host (one graph launch per iteration) so that "
                         "a kernel profiler sees every launch; slower, for profiling only")
    ap.add_argument("--workload", default="2d640", choices=["2d640", "c1", "3d160", "3d160g", "batch256", "serve", "mp2", "mp2s", "mp3", "mp3ilu", "mp2som", "mp3som", "mp3b", "mp3bsom", "mp1", "mp1som", "select", "gmres"],
                    help="2d640 (default): the 512^2 + 64-layer four-solve step; 3d160: 128^3 + 16-layer "
                         "k = 40 mixed-precision solve; batch256: 256 uneven 2D instances per step; "
                         "serve: a Poisson-arrival request stream through the solve server; mp2 / mp3: "
                         "the paper's model problems 2 and 3 with ECS layers on the north / east edges")
    ap.add_argument("--serve-requests", type=int, default=32, help="serve: requests in the stream")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serve: mean arrival rate (requests/s)")
    ap.add_argument("--serve-slots", type=int, default=8, help="serve: requests the server runs at once")
    ap.add_argument("--serve-sweep", default="", help="serve: comma-separated further offered rates (requests/s), "
                    "each run once on the FP32-multigrid path")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)
    if args.workload != "2d640":
        import bench_workloads
        bench_workloads.run(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if world > 1:
        dist.barrier()
    g.build()
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import Helm, solve_batch

    p = hi.workload_2d_512()
    sh = hi.shadow_space(p.n, 4)
    dev = torch.device("cuda", local)
    b_dev = torch.from_numpy(p.b).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ranks = Ranks(dist if world > 1 else None, dev)

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    # one context per solve of the step (a context holds one solve's workspace), per precision
    ctxs = {}
    for mg in ("c128", "c64"):
        for i, (_, _, pcn) in enumerate(SOLVES):
            ctxs[(mg, i)] = Helm(p, precond(pcn), mg_dtype=mg)
    methods = [m for (_, m, _) in SOLVES]
    shadows = [sh if m == hi.IDR else None for m in methods]
    xs_dev = {mg: [torch.empty(p.n, dtype=torch.complex128, device=dev) for _ in SOLVES] for mg in ("c128", "c64")}
    concurrent = not args.host_loop  # the host-driven loop (profiling) runs the solves one by one

    def one_step(mg: str, lat: list, infos: list, e2e_host=None, together=True):
        """The step: the four solves of the workload, at once through helm_solve_batch (one stream
        per solve) or one after another (then `lat` gets each solve's latency)."""
        b_in = e2e_host["b"].to(dev, non_blocking=True) if e2e_host is not None else b_dev
        if together:
            hs = [ctxs[(mg, i)] for i in range(len(SOLVES))]
            xs, inf = solve_batch(hs, [b_in] * len(SOLVES), method=methods, s=4, tol=TOL, maxmv=4000,
                                  shadows=shadows, xs=xs_dev[mg])
            infos.extend(inf)
        else:
            xs = []
            for i, method in enumerate(methods):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                x, info = ctxs[(mg, i)].solve(b_in, method=method, s=4, tol=TOL, maxmv=4000, shadow=sh,
                                              host_loop=args.host_loop)
                e1.record()
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
                infos.append(info)
                xs.append(x)
        if e2e_host is not None:
            for k, x in enumerate(xs):
                e2e_host["x"][k].copy_(x, non_blocking=True)

    def timed(mg: str, e2e=False, together=True):
        host = None
        if e2e:
            host = {"b": torch.from_numpy(p.b).pin_memory(),
                    "x": [torch.empty(p.n, dtype=torch.complex128).pin_memory() for _ in SOLVES]}
        for _ in range(args.warmup):
            one_step(mg, [], [], host, together)
        lat, infos, step_ms = [], [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record()
            one_step(mg, lat, infos, host, together)
            s1.record()
            barrier()
            step_ms.append(s0.elapsed_time(s1))
        return step_ms, lat, infos

    if args.phase == "kernels":
        kern = kernel_rooflines(torch, L, ctxs, p, dev, flush)
        line = {"metric": METRIC, "phase": "kernels", "config": config(p), "roofline": kern["dominant"],
                "roofline_fp32_mg": kern["fp32_mg"], "kernels": kern["table"]}
        for h in ctxs.values():
            h.close()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    run64 = args.phase in ("all", "fp64")
    run32 = args.phase in ("all", "fp32")
    ms64 = lat64 = inf64 = ms32 = lat32 = inf32 = None
    with ClockSampler(local) as clk:
        if run64:
            ms64, lat64, inf64 = timed("c128", together=concurrent)
        if run32:
            ms32, lat32, inf32 = timed("c64", together=concurrent)
        if args.phase == "all":
            # the same four solves one after another: each solve's latency on an otherwise idle GPU
            sq64, lat64, _ = timed("c128", together=False)
            sq32, lat32, _ = timed("c64", together=False)
    if args.phase != "all":
        ms, lat, inf = (ms64, lat64, inf64) if run64 else (ms32, lat32, inf32)
        step = ranks.max(statistics.mean(ms))
        line = {"metric": METRIC, "phase": args.phase, "value": ranks.job_rate(len(SOLVES), step),
                "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": step, "higher_is_better": True, "scaling": "weak",
                "dtype": "c128" if run64 else "c64 V-cycle, c128 Krylov", "data": "synthetic",
                "config": config(p, concurrent), "host_loop": bool(args.host_loop), "clocks": clk.summary(),
                "gpu_launches": int(sum(i.kernels for i in inf)),
                "matvecs": {f"{m}-{pc}": inf[i].matvecs for i, (m, _, pc) in enumerate(SOLVES)}}
        for h in ctxs.values():
            h.close()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    e2e_ms, _, _ = timed("c128", e2e=True)

    for info in inf64 + inf32:
        if info.status != 0 or not info.rel_res_true < TOL:
            raise SystemExit(f"a timed solve did not converge: {info}")

    step64 = ranks.max(statistics.mean(ms64))
    step32 = ranks.max(statistics.mean(ms32))
    stepe2e = ranks.max(statistics.mean(e2e_ms))
    nsol = len(SOLVES) * world
    value = ranks.job_rate(len(SOLVES), step64)

    # ---- per-kernel rooflines, measured with CUDA events on the launching stream ----
    kern = kernel_rooflines(torch, L, ctxs, p, dev, flush)
    # ---- the GPU solutions whose error the oracle's tight solution measures (untimed): the four
    # solves of the step at its tolerance in both precisions, and Bi-CGSTAB + CSG at 1e-7 ----
    gpu_x = {}
    for mg, tag in (("c128", "fp64"), ("c64", "fp32_mg")):
        for i, (mname, method, pcn) in enumerate(SOLVES):
            x, _ = ctxs[(mg, i)].solve(b_dev, method=method, s=4, tol=TOL, maxmv=4000, shadow=sh)
            gpu_x[f"{tag}_{mname}_{pcn}_tol1e-06"] = x.cpu().numpy()
        x, _ = ctxs[(mg, 0)].solve(b_dev, tol=1e-7, maxmv=4000)
        gpu_x[f"{tag}_bicgstab_csg_tol1e-07"] = x.cpu().numpy()
    err = {"reference": "skipped (--no-cpu-baseline)"}

    def pct(v, q):
        return float(np.percentile(np.asarray(v), q))

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": config(p, concurrent),
        "latency_ms": {"p50": pct(lat64, 50), "p99": pct(lat64, 99),
                       "what": "one solve alone on the GPU (the step's solves run one after another)"},
        "step_latency_ms": {"p50": pct(ms64, 50), "p99": pct(ms64, 99)},
        "sequential": {"value": nsol / (ranks.max(statistics.mean(sq64)) / 1000), "unit": "solves/s",
                       "fp32_mg": nsol / (ranks.max(statistics.mean(sq32)) / 1000),
                       "what": "the same four solves one after another"},
        "matvecs": {f"{m}-{pc}": inf64[i].matvecs for i, (m, _, pc) in enumerate(SOLVES)},
        "fp32_mg": {"value": nsol / (step32 / 1000), "unit": "solves/s", "ms_per_step": step32,
                    "dtype": "c64 V-cycle, c128 Krylov and true residual",
                    "latency_ms": {"p50": pct(lat32, 50), "p99": pct(lat32, 99)},
                    "step_latency_ms": {"p50": pct(ms32, 50), "p99": pct(ms32, 99)},
                    "matvecs": {f"{m}-{pc}": inf32[i].matvecs for i, (m, _, pc) in enumerate(SOLVES)},
                    "max_true_rel_res": max(i.rel_res_true for i in inf32)},
        "max_true_rel_res": max(i.rel_res_true for i in inf64),
        "error_vs_reference": err,
        "clocks": clk.summary(),
        "e2e": {"value": nsol / (stepe2e / 1000), "unit": "solves/s",
                "path": "FP64 path, helm_solve_batch with the right-hand side copied in from pinned host "
                        "memory and the four solutions copied out, every step",
                "h2d_bytes_per_step": p.n * 16, "d2h_bytes_per_step": len(SOLVES) * p.n * 16},
        "gpu_launches": int(sum(i.kernels for i in inf64[: len(SOLVES) * args.steps]) +
                            sum(i.kernels for i in inf32)),
        "roofline": kern["dominant"],
        "roofline_fp32_mg": kern["fp32_mg"],
        "kernels": kern["table"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"], line["error_vs_reference"] = oracle_leg(p, gpu_x)
        except Exception as e:  # the oracle is a reported baseline; never fail the GPU line on it
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": host_cores(), "kind": "oracle",
                                    "sample": f"unavailable: {e}"}
    for h in ctxs.values():
        h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Algorithmic cost of the fused first half of a V(1,1) level (smoothing sweep from the zero guess,
# residual, full weighting), per fine unknown: reads f and omega/D, writes u, writes a quarter of a
# coarse value; flops: u = f (omega/D) (complex multiply, 6), residual (1 - omega) f - a (sum of
# four neighbours) (3 complex adds, 1 complex multiply, 1 scale, 1 subtract: 16), full weighting
# (8 complex adds and a scale per coarse unknown: 18 / 4).
DOWN_FLOPS_PER_POINT = 6 + 16 + 18 / 4
# The same work in FP64-pipe operations (DADD, DMUL and DFMA each one issue slot of the FP64 pipe;
# interior point, complex CSG coefficients): u = f (omega/D) 4, residual 12 (neighbour pair sums 4,
# their sum 2, the complex coefficient 4, (1 - omega) f - a 2), full weighting 18 per coarse
# unknown = 4.5 per fine one.
DOWN_FP64_OPS_PER_POINT = 4 + 12 + 18 / 4

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one finest-level launch of the fused
# down kernel on this workload, from an ncu --set full capture of the current kernels (FP64, FP32);
# set back to None whenever k_down2d changes.
DOWN_TRAFFIC_BYTES = {"c128": 13133568, "c64": None}


def down_bytes_per_point(esz: int) -> float:
    return 3 * esz + esz / 4


def kernel_rooflines(torch, L, ctxs, p, dev, flush) -> dict:
    """Average duration of the hot kernels on the finest level, CUDA events on the launching
    stream with L2 flushed before every launch; achieved = algorithmic bytes (or FLOPs) per
    launch / duration."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # FP64 pipe peak: 152 SMs x 2 FP64 operations per clock per SM (ncu's peak_sustained) x 2.07 GHz
    fp64_ops_peak = 152 * 2 * 2.07e9 / 1e12  # T operations/s
    n = p.n
    st = torch.cuda.current_stream()
    table = {}

    def time_cold(fn, reps=20, name=None) -> float:
        # an NVTX range per kernel, so that a profiler can select exactly these launches
        if name:
            torch.cuda.nvtx.range_push(name)
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        if name:
            torch.cuda.nvtx.range_pop()
        return statistics.median(ts) / 1000.0  # seconds

    for mg, dt, esz in (("c128", torch.complex128, 16), ("c64", torch.complex64, 8)):
        h = ctxs[(mg, 0)]  # Bi-CGSTAB with CSG
        nc = h.level_shape(1)[0] * h.level_shape(1)[1]
        f = torch.randn(n, dtype=dt, device=dev)
        u = torch.empty(n, dtype=dt, device=dev)
        fc = torch.empty(nc, dtype=dt, device=dev)
        t = time_cold(lambda: h.level_op(L.HELM_OP_DOWN, 0, u, f, fc), name=f"k_down2d_{mg}")
        byt = n * down_bytes_per_point(esz)
        fl = n * DOWN_FLOPS_PER_POINT
        ops = n * DOWN_FP64_OPS_PER_POINT
        table[f"k_down2d_{mg}"] = {"us": t * 1e6, "bytes": byt, "GB/s": byt / t / 1e9, "flops": fl,
                                   "TFLOP/s": fl / t / 1e12, "fp64_ops": ops, "T_op/s": ops / t / 1e12}
        r = torch.randn(n, dtype=torch.complex128, device=dev)
        z = torch.empty(n, dtype=dt, device=dev)
        t = time_cold(lambda: h.vcycle(r, out=z), name=f"vcycle_{mg}")
        table[f"vcycle_{mg}"] = {"us": t * 1e6}
    h = ctxs[("c128", 0)]
    x = torch.randn(n, dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    t = time_cold(lambda: h.apply(x, out=y), name="k_h_apply_c128")
    byt = n * (16 + 16 + 8)
    table["k_h_apply_c128"] = {"us": t * 1e6, "bytes": byt, "GB/s": byt / t / 1e9}
    for v in table.values():
        if "GB/s" in v:
            v["frac_hbm"] = v["GB/s"] / hbm
    d64, d32 = table["k_down2d_c128"], table["k_down2d_c64"]
    dominant = {"kernel": "k_down2d<double> (fused smooth + residual + full weighting, finest level, FP64 path)",
                "bound": "alu", "achieved": d64["T_op/s"], "peak": fp64_ops_peak, "unit": "T FP64 op/s",
                "frac": d64["T_op/s"] / fp64_ops_peak, "traffic": DOWN_TRAFFIC_BYTES["c128"],
                "peak_source": "derived: 152 SMs x 2 FP64 operations/clk (ncu peak_sustained) x 2.07 GHz",
                "fp64_ops_per_launch": d64["fp64_ops"], "launch_us": d64["us"],
                "note": "DADD, DMUL and DFMA each take one FP64-pipe slot; ncu: the FP64 pipe is 76-80% busy over "
                        "active cycles, DRAM reads = the algorithmic reads (f and omega/D; writes stay in L2); "
                        "executed FP64 lane slots 22-33 per fine point against 20.5 algorithmic (halo, partial warps)"}
    fp32 = {"kernel": "k_down2d<float> (same kernel in the FP32 V-cycle)", "bound": "hbm",
            "achieved": d32["GB/s"], "peak": hbm, "unit": "GB/s", "frac": d32["GB/s"] / hbm,
            "traffic": DOWN_TRAFFIC_BYTES["c64"],
            "peak_source": hbm_src, "bytes_per_launch": d32["bytes"], "launch_us": d32["us"]}
    return {"dominant": dominant, "fp32_mg": fp32, "table": table}


if __name__ == "__main__":
    main()
