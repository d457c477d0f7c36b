"""The other workloads of bench.py (`--workload`): each prints one JSON line of its own.

  3d160     128^3 interior + 16-node ECS layers (160^3 = 4,096,000 unknowns), k = 40 constant,
            centre point source; one Bi-CGSTAB solve to 1e-6 per step, preconditioned by one CSG
            (theta_beta = 0.3) V(1,1) cycle with red-black Gauss-Seidel on 4 levels (coarsest
            20^3 = 8000 unknowns, dense inverse).  `value` is the all-FP64 path; `fp32_mg` is the
            complex-FP32 V-cycle under FP64 Bi-CGSTAB and FP64 true residual, with its solution's
            relative difference from the FP64 path's.
  3d160g    the same 3D solve with 27-point Galerkin coarse operators (omega-Jacobi V(1,1)).
  batch256  256 independent 2D instances (interior 63..511 per axis, 16..32-node layers, kh in
            [0.3, 0.6], constant or bump k, seeded point sources); one step solves all of them with
            helm_solve_batch (Bi-CGSTAB, CSG omega-Jacobi V(1,1), 1e-6).
  mp2, mp3  the paper's model problems 2 (nu = 7, k = 2, r = 50: 384^2 interior + 128 ECS nodes on
            the north / east edges, Dirichlet south / west; 512^2 unknowns) and 3 (r = 90, k = 2:
            1024^2 + 256; 1280^2 unknowns), theta_gamma = pi/6; one step solves them six times at
            once, {Bi-CGSTAB, IDR(4), IDR(8)} x {CSL, CSG} with the shift and angle of the paper's
            ECS rows and its Galerkin coarse operators (omega-Jacobi V(1,1) here, not the paper's
            ILU(0) V(0,1), so the paper's matvec counts, reported beside ours, are context).
  mp2som, mp3som  the same problems with the first-order Sommerfeld condition on the east / north
            edges instead of layers (the paper's Sommerfeld rows: shift 1 - 0.35i / 1 - 0.38i, angle
            -pi/20 / -pi/17).
  mp3ilu    mp3 with the paper's own multigrid: ILU(0) smoothing (lexicographic order), Galerkin
            coarse operators, V(0,1) cycles -- the configuration its matvec counts were measured with.
  mp2s      mp2 on the smooth ECS contour of the paper's Section 7 remark (the layer widths turn by
            theta_gamma / 128 per width over the whole 128-node layer).
  gmres     the paper's GMRES remark: MP2 (nu = 1, k = 4, ECS) to 1e-7 with GMRES(128), GMRES(30),
            Bi-CGSTAB and IDR(4) under the CSG (pi/26) Galerkin multigrid preconditioner.
  select    the automatic CSL shift / CSG angle choice of Section 7's remark on the 640^2 workload,
            then a solve with the default and with the chosen parameter each.
  serve     a Poisson-arrival stream (--serve-requests, default 32, at --serve-rate, default 200
            requests/s) of 2D (127^2 .. 1023^2 interior) and 3D (64^3 .. 160^3 interior) requests
            with 1..8 point-source right-hand sides each, submitted at their arrival times to the
            solve server (150 GB budget); reports right-hand-side solves/s and the server's
            submit-to-completion latencies.

  c1        64^2 interior + 16-node ECS layers, k = 20, centre point source, Bi-CGSTAB with the CSG
            red-black Gauss-Seidel V(1,1) preconditioner to 1e-8: one solve per step, its p50 / p99
            latency, the omega-Jacobi and FP32-multigrid variants, and the oracle's count and time.

Every timed solve is certified by the FP64 true residual; a step whose solves did not all reach
1e-6 aborts the run.
"""
from __future__ import annotations

import json
import os
import statistics
import time

import numpy as np

import helm_inputs as hi

TOL = 1e-6


def _pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q))


def _base(args, metric_value, ms_step, world, cfg, dtype):
    import bench
    return {"metric": bench.METRIC, "value": metric_value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg}


def _check(infos, what):
    for i in infos:
        if i.status != 0 or not i.rel_res_true < TOL:
            raise SystemExit(f"{what}: a timed solve did not converge: {i}")


def run(args):
    import torch
    import torch.distributed as dist

    import bench
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
    dev = torch.device("cuda", local)
    ranks = bench.Ranks(dist if world > 1 else None, dev)
    fn = {"c1": run_c1, "3d160": run_3d, "3d160g": run_3d, "batch256": run_batch, "serve": run_serve, "mp2": run_mp, "mp2s": run_mp, "mp3": run_mp,
          "mp3ilu": run_mp,
          "mp3b": run_mp, "mp3bsom": run_mp, "mp1": run_mp, "mp1som": run_mp,
          "mp2som": run_mp, "mp3som": run_mp,
          "select": run_select, "gmres": run_gmres}[args.workload]
    line = fn(args, torch, ranks, dev, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---- C1: the small single-solve latency case -------------------------------------------------

def run_c1(args, torch, ranks, dev, local):
    """64^2 interior + 16-node ECS layers (96^2 = 9216 unknowns), theta_gamma = 0.5, k = 20, unit
    point source at the centre; Bi-CGSTAB preconditioned by one CSG (theta_beta = 0.3) V(1,1) cycle
    with red-black Gauss-Seidel, to 1e-8, FP64 -- a single solve per step, latency-bound (its
    vectors live in L2), so the line reports the solve's latency rather than a roofline.  Beside it:
    the same solve with omega-Jacobi and with the FP32 V-cycle, the end-to-end time through pinned
    host buffers, and the oracle's matvec count, solution error and time on this host."""
    import bench
    import oracle
    from paper_0912_0180_gb300.helm import Helm
    p = hi.workload_small_2d()
    tol = 1e-8
    pcs = {"rbgs": hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS),
           "jacobi": hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)}
    b = torch.from_numpy(p.b).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    nlat = max(args.steps, 200)

    def latencies(h, count, host=None):
        for _ in range(args.warmup):
            h.solve(b, tol=tol, maxmv=2000)
        ms, infos = [], []
        for _ in range(count):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bi = host["b"].to(dev, non_blocking=True) if host else b
            x, info = h.solve(bi, tol=tol, maxmv=2000)
            if host:
                host["x"].copy_(x, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        _check_tol(infos, "c1", tol)
        return ms, infos

    ctx = {"rbgs64": Helm(p, pcs["rbgs"], mg_dtype="c128"), "rbgs32": Helm(p, pcs["rbgs"], mg_dtype="c64"),
           "jacobi64": Helm(p, pcs["jacobi"], mg_dtype="c128")}
    with bench.ClockSampler(local) as clk:
        ms, inf = latencies(ctx["rbgs64"], nlat)
        other = {k: latencies(ctx[k], nlat) for k in ("rbgs32", "jacobi64")}
    host = {"b": torch.from_numpy(p.b).pin_memory(), "x": torch.empty(p.n, dtype=torch.complex128).pin_memory()}
    e2e_ms, _ = latencies(ctx["rbgs64"], args.steps, host)
    # the oracle: same solve, its matvec count and solution, timed on this host's cores
    cores = bench.host_cores()
    oracle.set_threads(cores)
    o = oracle.Oracle(p, pcs["rbgs"])
    t = time.perf_counter()
    reps = 0
    while True:
        xo, io = o.solve(p.b, hi.SolveOpts(tol=tol, maxmv=2000))
        reps += 1
        if time.perf_counter() - t > 2.0:
            break
    cpu_s = (time.perf_counter() - t) / reps
    x12, _ = o.solve(p.b, hi.SolveOpts(tol=1e-12, maxmv=4000))
    nref = np.linalg.norm(x12)
    errs = {}
    for k, h in ctx.items():
        x, _ = h.solve(b, tol=tol, maxmv=2000)
        errs[k] = float(np.linalg.norm(x.cpu().numpy() - x12) / nref)
    step = ranks.max(statistics.mean(ms))
    cfg = {"workload": p.name, "grid": "64^2 interior + 16 ECS nodes per side (96^2 unknowns)", "n_unknowns": p.n,
           "solver": "Bi-CGSTAB, tol 1e-8 (FP64 true residual), one solve per step",
           "multigrid": "CSG theta_beta=0.3, V(1,1) red-black Gauss-Seidel, FW, bilinear, rediscretised levels",
           "l2": "flushed (256 MiB device write) before every timed solve"}
    line = _base(args, ranks.job_rate(1, step), step, ranks.world, cfg, "c128")
    line.update({
        "latency_ms": {"p50": _pct(ms, 50), "p99": _pct(ms, 99), "solves": len(ms)},
        "matvecs": inf[-1].matvecs, "oracle_matvecs": io["matvecs"],
        "variants": {k: {"latency_ms": {"p50": _pct(v[0], 50), "p99": _pct(v[0], 99)}, "matvecs": v[1][-1].matvecs}
                     for k, v in other.items()},
        "error_vs_reference": {"reference": "FP64 oracle at tol 1e-12", **errs},
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"the same solve, {reps} times, on all {cores} host cores"},
        "clocks": clk.summary(),
        "e2e": {"value": 1000.0 / statistics.mean(e2e_ms), "unit": "solves/s",
                "path": "helm_solve with b copied in from pinned host memory and x copied out, every solve",
                "h2d_bytes_per_step": p.n * 16, "d2h_bytes_per_step": p.n * 16},
        "gpu_launches": int(sum(i.kernels for i in inf[:args.steps])),
    })
    for h in ctx.values():
        h.close()
    return line


def _check_tol(infos, what, tol):
    for i in infos:
        if i.status != 0 or not i.rel_res_true < tol:
            raise SystemExit(f"{what}: a timed solve did not converge: {i}")


# ---- 3D ------------------------------------------------------------------------------------

def _pc3d(galerkin=False):
    if galerkin:  # Galerkin operators take the Jacobi smoother (red-black is no 2-colouring of 27 points)
        return hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5, max_levels=4,
                          galerkin=True)
    return hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS, max_levels=4)


def run_3d(args, torch, ranks, dev, local):
    import bench
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import Helm
    p = hi.workload_3d_128()
    galerkin = args.workload == "3d160g"
    b_dev = torch.from_numpy(p.b).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx, create_s = {}, {}
    for mg in ("c128", "c64"):
        t = time.perf_counter()
        ctx[mg] = Helm(p, _pc3d(galerkin), mg_dtype=mg)
        torch.cuda.synchronize()
        create_s[mg] = time.perf_counter() - t

    if args.phase == "kernels":  # only the per-kernel table (for kernel profiling)
        kern = _kernels_3d(torch, L, ctx, p, dev, flush)
        for h in ctx.values():
            h.close()
        return {"metric": bench.METRIC, "phase": "kernels", "config": {"workload": p.name},
                "roofline": kern["dominant"], "roofline_fp32_mg": kern["fp32_mg"], "kernels": kern["table"]}

    def step(mg, host=None):
        h = ctx[mg]
        if host is not None:
            x, info = h.solve(host["b"].to(dev, non_blocking=True), tol=TOL, maxmv=3000)
            host["x"].copy_(x, non_blocking=True)
        else:
            x, info = h.solve(b_dev, tol=TOL, maxmv=3000)
        return x, info

    def timed(mg, e2e=False):
        host = None
        if e2e:
            host = {"b": torch.from_numpy(p.b).pin_memory(),
                    "x": torch.empty(p.n, dtype=torch.complex128).pin_memory()}
        for _ in range(args.warmup):
            step(mg, host)
        ms, infos, x = [], [], None
        for _ in range(args.steps):
            flush.fill_(1.0)
            ranks.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            x, info = step(mg, host)
            e1.record()
            ranks.barrier()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos, x

    with bench.ClockSampler(local) as clk:
        ms64, inf64, x64 = timed("c128")
        ms32, inf32, x32 = timed("c64")
    e2e_ms, _, _ = timed("c64", e2e=True)
    _check(inf64 + inf32, "3d160")
    diff = float(torch.linalg.vector_norm(x32 - x64) / torch.linalg.vector_norm(x64))
    err = _errors_vs_reference(torch, ctx, b_dev)
    step64 = ranks.max(statistics.mean(ms64))
    step32 = ranks.max(statistics.mean(ms32))
    kern = None if galerkin else _kernels_3d(torch, L, ctx, p, dev, flush)
    cfg = {"workload": p.name + ("-galerkin" if galerkin else ""),
           "grid": "128^3 interior + 16 ECS nodes per side (160^3 unknowns)",
           "n_unknowns": p.n, "solves_per_step": 1, "solver": "Bi-CGSTAB, tol 1e-6 (FP64 true residual)",
           "multigrid": ("CSG theta_beta=0.3, V(1,1) omega-Jacobi 0.5 on 27-point Galerkin coarse operators R A P, "
                         if galerkin else "CSG theta_beta=0.3, V(1,1) red-black Gauss-Seidel, ") +
                        "4 levels, FW, trilinear, dense inverse of the 20^3 coarsest level",
           "l2": "flushed (512 MiB device write) before every timed step"}
    line = _base(args, ranks.job_rate(1, step64), step64, ranks.world, cfg, "c128")
    line.update({
        "latency_ms": {"p50": _pct(ms64, 50), "p99": _pct(ms64, 99)},
        "matvecs": inf64[-1].matvecs, "max_true_rel_res": max(i.rel_res_true for i in inf64),
        "fp32_mg": {"value": ranks.world / (step32 / 1000), "unit": "solves/s", "ms_per_step": step32,
                    "dtype": "c64 V-cycle, c128 Bi-CGSTAB and true residual",
                    "latency_ms": {"p50": _pct(ms32, 50), "p99": _pct(ms32, 99)},
                    "matvecs": inf32[-1].matvecs, "max_true_rel_res": max(i.rel_res_true for i in inf32),
                    "rel_diff_vs_fp64_solution": diff},
        "error_vs_reference": err,
        "create_s": create_s,
        "clocks": clk.summary(),
        "e2e": {"value": ranks.world / (ranks.max(statistics.mean(e2e_ms)) / 1000), "unit": "solves/s",
                "path": "fp32_mg through helm_solve with pinned host b and x",
                "h2d_bytes_per_step": p.n * 16, "d2h_bytes_per_step": p.n * 16},
        "gpu_launches": int(sum(i.kernels for i in inf64) + sum(i.kernels for i in inf32)),
    })
    if kern is not None:
        line.update({"roofline": kern["dominant"], "roofline_fp32_mg": kern["fp32_mg"], "kernels": kern["table"]})
    for h in ctx.values():
        h.close()
    return line


def _errors_vs_reference(torch, ctx, b, method=0, shadow=None):
    """Relative error of both paths' solutions at tol 1e-6 and 1e-7 against the FP64 path's
    solution at tol 1e-10 (untimed): two solutions that each meet a 1e-6 residual differ by up to
    cond(H) x 1e-6 whatever the V-cycle precision, so the error is reported per tolerance."""
    xr, ir = ctx["c128"].solve(b, method=method, s=4, tol=1e-10, maxmv=8000, shadow=shadow)
    nr = torch.linalg.vector_norm(xr)
    out = {"reference": "FP64 path at tol 1e-10", "reference_true_rel_res": ir.rel_res_true}
    for mg in ("c128", "c64"):
        for tol in (1e-6, 1e-7):
            x, info = ctx[mg].solve(b, method=method, s=4, tol=tol, maxmv=8000, shadow=shadow)
            key = ("fp64" if mg == "c128" else "fp32_mg") + f"_tol{tol:.0e}"
            out[key] = float(torch.linalg.vector_norm(x - xr) / nr)
    return out


def _time_cold(torch, flush, fn, reps=10, name=None):
    st = torch.cuda.current_stream()
    if name:  # an NVTX range per kernel, so that a profiler can select exactly these launches
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
    return statistics.median(ts) / 1000.0


# FP64 operations of one Helmholtz matvec point in the 3D uniform interior (k_h_apply): six
# neighbour additions (10), the scale (2), the diagonal 6/h^2 - k^2 (1) and its complex product
# with x added to the neighbour sum (4); counted as operations, not FMA-doubled flops.
H3D_FP64_OPS_PER_POINT = 17

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_h_apply<double, 3> launch on
# this workload, from an ncu --set full capture of the current kernel; None whenever it changes.
H3D_TRAFFIC_BYTES = 106760704 + 37031680


def _kernels_3d(torch, L, ctx, p, dev, flush):
    n = p.n
    fp64_ops_peak = 152 * 2 * 2.07e9 / 1e12  # FP64 operations per second (2 per clock per SM), in T/s
    table = {}
    x = torch.randn(n, dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    h = ctx["c128"]
    t = _time_cold(torch, flush, lambda: h.apply(x, out=y), name="k_h_apply_c128_3d")
    table["k_h_apply_c128"] = {"us": t * 1e6, "bytes": n * 40, "GB/s": n * 40 / t / 1e9,
                               "fp64_ops": n * H3D_FP64_OPS_PER_POINT}
    for mg, dt, esz in (("c128", torch.complex128, 16), ("c64", torch.complex64, 8)):
        hh = ctx[mg]
        f = torch.randn(n, dtype=dt, device=dev)
        u = torch.zeros(n, dtype=dt, device=dev)
        # u and f in the level's storage order (x-split rows on the FP32 levels), as inside the V-cycle
        t = _time_cold(torch, flush, lambda: hh.level_op(L.HELM_OP_SMOOTH | L.HELM_OP_STORED, 0, u, f, u),
                       name=f"rbgs_sweep_{mg}_3d")
        table[f"rbgs_sweep_{mg}"] = {"us": t * 1e6, "bytes": n * 4 * esz, "GB/s": n * 4 * esz / t / 1e9}
        r = torch.randn(n, dtype=torch.complex128, device=dev)
        z = torch.empty(n, dtype=dt, device=dev)
        t = _time_cold(torch, flush, lambda: hh.vcycle(r, out=z), name=f"vcycle_{mg}_3d")
        table[f"vcycle_{mg}"] = {"us": t * 1e6}
    # The FP32 sweep pair's bytes moved as contiguous streams, timed the same way (L2 flushed by a
    # write first): per colour three arrays of n/2 complex64 read and one written, the second pass
    # reading the first one's output as the black half-sweep reads the red values.  A library
    # elementwise kernel, used here only as the attainable rate for this many bytes in this regime.
    a1, b1, c1, o1, a2, b2, o2 = (torch.randn(n, dtype=torch.float32, device=dev) for _ in range(7))

    def streams():
        torch.addcmul(c1, a1, b1, out=o1)
        torch.addcmul(o1, a2, b2, out=o2)

    t = _time_cold(torch, flush, streams, name="stream_same_bytes_3d")
    table["stream_same_bytes_c64"] = {"us": t * 1e6, "bytes": n * 32, "GB/s": n * 32 / t / 1e9}
    del a1, b1, c1, o1, a2, b2, o2
    a = table["k_h_apply_c128"]
    achieved = a["fp64_ops"] / (a["us"] / 1e6) / 1e12
    dom = {"kernel": "k_h_apply<double, 3> (FP64 Helmholtz matvec; the stencil of the Krylov kernels)",
           "bound": "alu", "achieved": achieved, "peak": fp64_ops_peak, "unit": "T FP64 op/s",
           "frac": achieved / fp64_ops_peak, "traffic": H3D_TRAFFIC_BYTES,
           "peak_source": "derived: 152 SMs x 2 FP64 operations/clk (ncu peak_sustained) x 2.07 GHz",
           "launch_us": a["us"]}
    # the FP32 sweep against the measured copy bandwidth: per point and sweep, f, 1/D and the
    # other colour's u read and u written, 8 bytes each (x-split rows: no other sector comes along)
    hbm, hbm_src = _hbm_peak()
    rb = table["rbgs_sweep_c64"]
    fp32 = {"kernel": "k_rbgs3z2 (red and black half-sweeps of the finest level, x-split rows, two pairs of columns a thread, marching along z)",
            "bound": "hbm", "achieved": rb["GB/s"], "peak": hbm, "unit": "GB/s", "frac": rb["GB/s"] / hbm,
            "traffic": RBGS3Z_TRAFFIC_BYTES, "peak_source": hbm_src, "bytes_per_launch": rb["bytes"] / 2,
            "launch_us": rb["us"] / 2}
    sb = table["stream_same_bytes_c64"]
    fp32["stream_same_bytes"] = {"what": "torch.addcmul over contiguous FP32 arrays moving the pair's bytes, L2 flushed the same way",
                                 "us": sb["us"], "GB/s": sb["GB/s"], "frac_of_peak": sb["GB/s"] / hbm,
                                 "sweep_frac_of_stream": rb["GB/s"] / sb["GB/s"]}
    return {"dominant": dom, "fp32_mg": fp32, "table": table}


# DRAM bytes (read + write) of one k_rbgs3z2 half-sweep on the 160^3 level, from an ncu capture of
# the current kernel; None whenever it changes.
RBGS3Z_TRAFFIC_BYTES = 49200640 + 348672


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        peaks = {}
    return float(peaks.get("hbm_gbs", 6800.0)), ("measured" if "hbm_gbs" in peaks else "fallback")


# ---- batch ---------------------------------------------------------------------------------

def _pc2d():
    return hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)


def run_batch(args, torch, ranks, dev, local):
    import bench
    from paper_0912_0180_gb300.helm import Helm, solve_batch, solve_group
    inst = hi.workload_batch_2d(256)
    bs = [torch.from_numpy(p.b).to(dev) for p in inst]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    with bench.ClockSampler(local) as clk:
        for mg in ("c128", "c64"):
            hs = [Helm(p, _pc2d(), mg_dtype=mg) for p in inst]
            for _ in range(args.warmup):
                solve_batch(hs, bs, tol=TOL, maxmv=4000)
            ms, infos = [], []
            for _ in range(args.steps):
                flush.fill_(1.0)
                ranks.barrier()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                xs, inf = solve_batch(hs, bs, tol=TOL, maxmv=4000)
                e1.record()
                ranks.barrier()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                infos += inf
            _check(infos, "batch256")
            # the same step as ONE group (helm_solve_group): every kernel of an iteration is one launch
            # over all 256 instances
            for _ in range(args.warmup):
                solve_group(hs, bs, tol=TOL, maxmv=4000)
            gms, ginfos = [], []
            for _ in range(args.steps):
                flush.fill_(1.0)
                ranks.barrier()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                gxs, ginf = solve_group(hs, bs, tol=TOL, maxmv=4000)
                e1.record()
                ranks.barrier()
                torch.cuda.synchronize()
                gms.append(e0.elapsed_time(e1))
                ginfos += ginf
            _check(ginfos, "batch256 grouped")
            same = all(torch.equal(a, b_) for a, b_ in zip(gxs, xs))
            one = None
            if mg == "c64":  # the same instances one after another, for the batching gain
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for h, b in zip(hs, bs):
                    h.solve(b, tol=TOL, maxmv=4000)
                e1.record()
                torch.cuda.synchronize()
                one = e0.elapsed_time(e1)
                # e2e: host right-hand sides in, host solutions out, through the public calls
                hb = [torch.from_numpy(p.b).pin_memory() for p in inst]
                hx = [torch.empty(p.n, dtype=torch.complex128).pin_memory() for p in inst]
                e2e = []
                for _ in range(max(1, args.steps)):
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    bd = [b.to(dev, non_blocking=True) for b in hb]
                    xs2, _ = solve_batch(hs, bd, tol=TOL, maxmv=4000)
                    for xh, xd in zip(hx, xs2):
                        xh.copy_(xd, non_blocking=True)
                    e1.record()
                    torch.cuda.synchronize()
                    e2e.append(e0.elapsed_time(e1))
                res["e2e_ms"] = statistics.mean(e2e)
            res[mg] = {"ms": ranks.max(statistics.mean(ms)), "infos": infos, "one_by_one_ms": one,
                       "group_ms": ranks.max(statistics.mean(gms)), "group_infos": ginfos, "group_same": same}
            for h in hs:
                h.close()
    nb = len(inst)
    r64, r32 = res["c128"], res["c64"]
    cfg = {"workload": "batch-2d-256", "instances": nb, "n_unknowns_total": int(sum(p.n for p in inst)),
           "sizes": "interior {63,127,255,511}^2, 16..32-node layers, kh 0.3..0.6, const or bump k",
           "solver": "helm_solve_batch: Bi-CGSTAB, CSG theta_beta=0.3 omega-Jacobi V(1,1), tol 1e-6",
           "l2": "flushed (512 MiB device write) before every timed step"}
    line = _base(args, ranks.job_rate(nb, r64["ms"]), r64["ms"], ranks.world, cfg, "c128")
    lat64 = [i.matvecs for i in r64["infos"]]
    line.update({
        "matvecs_total_per_step": int(sum(lat64) / max(1, args.steps)),
        "fp32_mg": {"value": nb * ranks.world / (r32["ms"] / 1000), "unit": "solves/s", "ms_per_step": r32["ms"],
                    "dtype": "c64 V-cycle, c128 Krylov and true residual",
                    "one_by_one_solves_per_s": nb / (r32["one_by_one_ms"] / 1000),
                    "max_true_rel_res": max(i.rel_res_true for i in r32["infos"])},
        "max_true_rel_res": max(i.rel_res_true for i in r64["infos"]),
        "grouped": {mg: {"solves_per_s": nb * ranks.world / (res[mg]["group_ms"] / 1000),
                         "ms_per_step": res[mg]["group_ms"],
                         "launches_per_step": int(res[mg]["group_infos"][0].kernels),
                         "bitwise_equal_to_streams": bool(res[mg]["group_same"])}
                    for mg in ("c128", "c64")},
        "grouped_what": "helm_solve_group: the 256 instances as one group, each kernel of an iteration one launch "
                        "over all instances (per-instance descriptors), one captured loop graph",
        "clocks": clk.summary(),
        "e2e": {"value": nb / (res["e2e_ms"] / 1000), "unit": "solves/s",
                "path": "fp32_mg batch with pinned host right-hand sides and solutions",
                "h2d_bytes_per_step": int(sum(p.n for p in inst) * 16),
                "d2h_bytes_per_step": int(sum(p.n for p in inst) * 16)},
        "gpu_launches": int(sum(i.kernels for i in r64["infos"]) + sum(i.kernels for i in r32["infos"])),
    })
    return line


# ---- serve ---------------------------------------------------------------------------------

def _stream(torch, reqs, mg, budget, slots=8):
    """Submits every request at its arrival time; returns wall seconds, per-request results."""
    from paper_0912_0180_gb300.helm import Server
    srv = Server(budget, max_active=slots, smallest_first=True)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        wait = r.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(r.problem, _pc2d(), mg_dtype=mg, tol=TOL, maxmv=4000, rhs=r.rhs))
    out = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    srv.close()
    return wall, out


def run_serve(args, torch, ranks, dev, local):
    import bench
    reqs = hi.workload_serve(args.serve_requests, args.serve_rate)
    budget = 150 * 10**9
    nsol = int(sum(r.rhs.shape[0] for r in reqs))
    res = {}
    with bench.ClockSampler(local) as clk:
        for mg in ("c128", "c64"):
            _stream(torch, reqs[:4], mg, budget, args.serve_slots)  # warm-up: the first requests
            walls, outs = [], None
            for _ in range(args.steps):
                wall, outs = _stream(torch, reqs, mg, budget, args.serve_slots)
                walls.append(wall)
                for x, info, lat in outs:
                    if info.status != 0 or not info.rel_res_true < TOL:
                        raise SystemExit(f"serve: a request did not converge: {info}")
            res[mg] = (ranks.max(statistics.mean(walls)), outs)
    w64, o64 = res["c128"]
    w32, o32 = res["c64"]
    diff = max(float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])) for a, b in zip(o32, o64))
    lat64 = [o[2] * 1000 for o in o64]
    lat32 = [o[2] * 1000 for o in o32]
    cfg = {"workload": f"serve-stream-{len(reqs)}", "requests": len(reqs), "rhs_solves": nsol,
           "arrivals": f"Poisson, mean {args.serve_rate:g} requests/s (offered)",
           "mix": "1/2 2D (interior 127..1023), 1/2 3D (interior 64..160), 16..32-node layers, kh 0.3..0.6, "
                  "1..8 point-source right-hand sides each",
           "n_unknowns_total": int(sum(r.problem.n * r.rhs.shape[0] for r in reqs)),
           "server": f"150 GB budget, {args.serve_slots} slots, smallest work admitted first", "solver": "Bi-CGSTAB, CSG theta_beta=0.3 omega-Jacobi V(1,1), tol 1e-6",
           "timing": "wall clock from the first arrival to the last completion (host in, host out)"}
    line = _base(args, ranks.job_rate(nsol, w64 * 1000), w64 * 1000, ranks.world, cfg, "c128")
    line.update({
        "latency_ms": {"p50": _pct(lat64, 50), "p99": _pct(lat64, 99)},
        "requests_per_s": len(reqs) / w64,
        "offered_requests_per_s": args.serve_rate,
        "fp32_mg": {"value": nsol / w32, "unit": "solves/s", "ms_per_step": w32 * 1000,
                    "requests_per_s": len(reqs) / w32,
                    "latency_ms": {"p50": _pct(lat32, 50), "p99": _pct(lat32, 99)},
                    "max_rel_diff_vs_fp64_solution": diff,
                    "max_true_rel_res": max(o[1].rel_res_true for o in o32)},
        "max_true_rel_res": max(o[1].rel_res_true for o in o64),
        "clocks": clk.summary(),
        "e2e": {"value": nsol / w32, "unit": "solves/s",
                "path": "the served fp32_mg stream itself: host right-hand sides in, host solutions out",
                "h2d_bytes_per_step": int(sum(r.rhs.nbytes for r in reqs)),
                "d2h_bytes_per_step": int(sum(r.rhs.nbytes for r in reqs))},
        "gpu_launches": int(sum(o[1].kernels for o in o64) + sum(o[1].kernels for o in o32)),
    })
    if args.serve_sweep:
        # the same request mix at other offered rates (FP32-multigrid path, one stream each)
        sweep = []
        for rate in [float(v) for v in args.serve_sweep.split(",") if v]:
            rq = hi.workload_serve(args.serve_requests, rate)
            wall, outs = _stream(torch, rq, "c64", budget, args.serve_slots)
            for x, info, lat in outs:
                if info.status != 0 or not info.rel_res_true < TOL:
                    raise SystemExit(f"serve sweep: a request did not converge: {info}")
            lat = [o[2] * 1000 for o in outs]
            ns = int(sum(r.rhs.shape[0] for r in rq))
            sweep.append({"offered_requests_per_s": rate, "requests_per_s": len(rq) / wall,
                          "rhs_solves_per_s": ns / wall, "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99)}})
            line["gpu_launches"] += int(sum(o[1].kernels for o in outs))
        line["fp32_mg"]["rate_sweep"] = sweep
    return line


# ---- the paper's model problems 2 and 3 -------------------------------------------------------

# The paper's ECS rows (preconditioner parameters, and its matvec counts with ILU(0), Galerkin
# coarse operators and V(0,1), for context): shift = -beta^2 in its notation.
MP_CASES = {
    "mp2": {"problem": lambda: hi.workload_mp2(), "csl": 1 + 0.34j, "csg": np.pi / 20,
            "paper_matvecs": {"csl": {"bicgstab": 71, "idr4": 72, "idr8": 74},
                              "csg": {"bicgstab": 68, "idr4": 73, "idr8": 69}}},
    # MP2 on the smooth contour of the Section 7 remark, turning over the whole 128-node layer
    "mp2s": {"problem": lambda: hi.workload_mp2(ecs_ramp=128), "csl": 1 + 0.34j, "csg": np.pi / 20,
             "paper_matvecs": {"csl": {"bicgstab": 71, "idr4": 72, "idr8": 74},
                               "csg": {"bicgstab": 68, "idr4": 73, "idr8": 69}}},
    "mp3": {"problem": lambda: hi.workload_mp3(), "csl": 1 + 0.38j, "csg": np.pi / 17,
            "paper_matvecs": {"csl": {"bicgstab": 142, "idr4": 145, "idr8": 141},
                              "csg": {"bicgstab": 139, "idr4": 139, "idr8": 134}}},
    # the Sommerfeld rows: first-order condition on the east / north edges instead of layers; the
    # spectrum sits in the first quadrant, so the shift's imaginary part and the angle flip sign
    "mp2som": {"problem": lambda: hi.workload_mp2(n_l=-1), "csl": 1 - 0.35j, "csg": -np.pi / 20,
               "paper_matvecs": {"csl": {"bicgstab": 123, "idr4": 120, "idr8": 122},
                                 "csg": {"bicgstab": 113, "idr4": 115, "idr8": 115}}},
    "mp3som": {"problem": lambda: hi.workload_mp3(n_l=-1), "csl": 1 - 0.38j, "csg": -np.pi / 17,
               "paper_matvecs": {"csl": {"bicgstab": 207, "idr4": 214, "idr8": 232},
                                 "csg": {"bicgstab": 205, "idr4": 207, "idr8": 207}}},
    # MP3's second case of the paper's table: r = 150, k = 4 on 2048^2 interior nodes (+ 512 layer
    # nodes on the east / north edges), ECS and Sommerfeld rows
    "mp3b": {"problem": lambda: hi.workload_mp3(r=150.0, k=4.0, n_int=2049, n_l=512), "csl": 1 + 0.40j,
             "csg": np.pi / 17,
             "paper_matvecs": {"csl": {"bicgstab": 436, "idr4": 413, "idr8": 423},
                               "csg": {"bicgstab": 390, "idr4": 387, "idr8": 392}}},
    "mp3bsom": {"problem": lambda: hi.workload_mp3(r=150.0, k=4.0, n_int=2049, n_l=-1), "csl": 1 - 0.40j,
                "csg": -np.pi / 17,
                "paper_matvecs": {"csl": {"bicgstab": 681, "idr4": 682, "idr8": 669},
                                  "csg": {"bicgstab": 620, "idr4": 650, "idr8": 652}}},
    # MP1 (constant k = 160, centre point source, unit square), absorbing on all four edges: ECS
    # layers of 64 nodes, or the first-order Sommerfeld condition on every edge -- two of them low
    # sides, whose coarsening keeps node 0 and runs the per-component V-cycle with rediscretised
    # levels (no Galerkin operators there)
    "mp1": {"problem": lambda: hi.workload_mp1(), "csl": 1 + 0.2j, "csg": np.pi / 28,
            "paper_matvecs": {"csl": {"bicgstab": 59, "idr4": 62, "idr8": 60},
                              "csg": {"bicgstab": 58, "idr4": 62, "idr8": 56}}},
    # MP3 with the paper's own multigrid: ILU(0) smoothing, Galerkin coarse operators, V(0,1)
    "mp3ilu": {"problem": lambda: hi.workload_mp3(), "csl": 1 + 0.38j, "csg": np.pi / 17, "ilu": True,
               "paper_matvecs": {"csl": {"bicgstab": 142, "idr4": 145, "idr8": 141},
                                 "csg": {"bicgstab": 139, "idr4": 139, "idr8": 134}}},
    "mp1som": {"problem": lambda: hi.workload_mp1(n_l=-1), "csl": 1 - 0.2j, "csg": -np.pi / 28, "galerkin": False,
               "paper_matvecs": {"csl": {"bicgstab": 79, "idr4": 72, "idr8": 76},
                                 "csg": {"bicgstab": 74, "idr4": 70, "idr8": 72}}},
}


MP_MAXMV = 4000  # per solve; a solve that misses the tolerance is reported, not counted


def run_mp(args, torch, ranks, dev, local):
    import bench
    from paper_0912_0180_gb300.helm import Helm, solve_batch
    case = MP_CASES[args.workload]
    p = case["problem"]()
    b_dev = torch.from_numpy(p.b).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    solves = [(m, s, pcn) for pcn in ("csl", "csg") for (m, s) in (("bicgstab", 0), ("idr4", 4), ("idr8", 8))]
    gal = case.get("galerkin", True)
    ilu = case.get("ilu", False)
    sm = dict(smoother=hi.SM_ILU, nu1=0, nu2=1) if ilu else dict(smoother=hi.SM_JACOBI, omega=0.5)
    pcs = {"csl": hi.Precond(kind=hi.PC_CSL, shift=case["csl"], galerkin=gal, **sm),
           "csg": hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=case["csg"], galerkin=gal, **sm)}
    methods = [hi.BICGSTAB if s == 0 else hi.IDR for (_, s, _) in solves]
    svals = [max(s, 1) for (_, s, _) in solves]
    shadows = [hi.shadow_space(p.n, s) if s else None for (_, s, _) in solves]
    res = {}
    with bench.ClockSampler(local) as clk:
        for mg in ("c128", "c64"):
            hs = [Helm(p, pcs[pcn], mg_dtype=mg) for (_, _, pcn) in solves]
            for _ in range(args.warmup):
                solve_batch(hs, [b_dev] * len(hs), method=methods, s=svals, tol=TOL, maxmv=MP_MAXMV, shadows=shadows)
            ms, infos = [], None
            for _ in range(args.steps):
                flush.fill_(1.0)
                ranks.barrier()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                xs, infos = solve_batch(hs, [b_dev] * len(hs), method=methods, s=svals, tol=TOL, maxmv=MP_MAXMV,
                                        shadows=shadows)
                e1.record()
                ranks.barrier()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            res[mg] = (ranks.max(statistics.mean(ms)), infos)
            for h in hs:
                h.close()
    ns = len(solves)
    keyed = lambda infos: {f"{m}-{pcn}": infos[i].matvecs for i, (m, _, pcn) in enumerate(solves)}
    status = lambda infos: {f"{m}-{pcn}": infos[i].status for i, (m, _, pcn) in enumerate(solves)}
    # only solves that reached the tolerance (certified by the FP64 true residual) count
    done = lambda infos: sum(1 for i in infos if i.status == 0 and i.rel_res_true < TOL)
    cfg = {"workload": p.name, "n_unknowns": p.n, "solves_per_step": ns,
           "solves": "{Bi-CGSTAB, IDR(4), IDR(8)} x {CSL shift %s, CSG theta_beta %.4f}, run at once"
                     % (case["csl"], case["csg"]),
           "multigrid": ("V(0,1) ILU(0), FW, bilinear, " if ilu else "V(1,1) omega-Jacobi 0.5, FW, bilinear, ") +
                        ("Galerkin coarse operators R A P" if gal else "rediscretised coarse operators"),
           "boundaries": (("first-order Sommerfeld on all four edges" if args.workload.endswith("som") else
                           "ECS layers on all four edges (theta_gamma = pi/6)") if args.workload.startswith("mp1") else
                          "Dirichlet south / west, " + ("first-order Sommerfeld east / north"
                                                        if args.workload.endswith("som") else
                                                        "ECS layers east / north (theta_gamma = pi/6)")),
           "l2": "flushed (512 MiB device write) before every timed step"}
    line = _base(args, ranks.job_rate(done(res["c128"][1]), res["c128"][0]), res["c128"][0], ranks.world, cfg, "c128")
    line.update({
        "matvecs": keyed(res["c128"][1]),
        "status": status(res["c128"][1]),
        "converged_per_step": done(res["c128"][1]),
        "paper_matvecs_context": case["paper_matvecs"],
        "fp32_mg": {"value": done(res["c64"][1]) * ranks.world / (res["c64"][0] / 1000), "unit": "solves/s",
                    "ms_per_step": res["c64"][0], "matvecs": keyed(res["c64"][1]), "status": status(res["c64"][1]),
                    "converged_per_step": done(res["c64"][1]),
                    "max_true_rel_res": max(i.rel_res_true for i in res["c64"][1])},
        "max_true_rel_res": max(i.rel_res_true for i in res["c128"][1]),
        "clocks": clk.summary(),
        "e2e": {"value": None, "unit": "solves/s", "path": "not measured in this mode (see the default workload)",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": int(sum(i.kernels for i in res["c128"][1]) + sum(i.kernels for i in res["c64"][1])),
    })
    return line


def run_select(args, torch, ranks, dev, local):
    """The automatic parameter choice of Section 7's remark on the 640^2 workload: from a large
    start (CSL shift 1 + 4i, CSG angle 1.2), the parameter shrinks by 0.8 per trial while
    omega-Jacobi V(1,1) multigrid, run as a solver of M u = f, still reaches 1e-6 within 30 cycles
    (the paper's tables list multigrid factors up to 0.53 and 22 cycles; omega-Jacobi V(1,1) itself
    contracts by about 0.5 per cycle, so 20 cycles would admit nothing).  Then one Bi-CGSTAB solve
    (FP32 V-cycle, FP64 Krylov) with the default and with the chosen parameter each, for their
    matvecs and times."""
    import bench
    from paper_0912_0180_gb300.helm import Helm, select_precond
    p = hi.workload_2d_512()
    f = torch.from_numpy(hi.random_vector(p.n, 20091202)).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    starts = {"csl": (hi.Precond(kind=hi.PC_CSL, shift=1 + 4.0j, smoother=hi.SM_JACOBI, omega=0.5),
                      hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5)),
              "csg": (hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=1.2, smoother=hi.SM_JACOBI, omega=0.5),
                      hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5))}
    cycles_max, factor, trials_max = 30, 0.8, 16
    out, seconds, launches = {}, [], 0

    def timed_solve(pc):
        h = Helm(p, pc, mg_dtype="c64")
        for _ in range(args.warmup):
            h.solve(b, tol=TOL, maxmv=4000)
        ms, info = [], None
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x, info = h.solve(b, tol=TOL, maxmv=4000)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        h.close()
        return statistics.mean(ms), info

    with bench.ClockSampler(local) as clk:
        for name, (start, default) in starts.items():
            select_precond(p, start, f, cycles_max, 1e-6, factor, trials_max)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chosen, st, params, cycles = select_precond(p, start, f, cycles_max, 1e-6, factor, trials_max)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            seconds.append(sec)
            ms_def, info_def = timed_solve(default)
            ms_ch, info_ch = timed_solve(chosen)
            _check([info_def, info_ch], f"select-{name}")
            launches += info_def.kernels + info_ch.kernels
            par = (lambda pc: complex(pc.shift).imag) if name == "csl" else (lambda pc: pc.theta_beta)
            out[name] = {"start": par(start), "chosen": par(chosen), "status": int(st), "select_s": sec,
                         "trials": [{"param": float(a), "cycles": int(c)} for a, c in zip(params, cycles)],
                         "solve_default": {"param": par(default), "matvecs": info_def.matvecs, "ms": ms_def},
                         "solve_chosen": {"param": par(chosen), "matvecs": info_ch.matvecs, "ms": ms_ch}}
        # the CSL shift's sign (the paper's "1 - 0.5i" read literally, beta^2 = 1 - 0.5i, against the
        # sign matched to the fourth-quadrant ECS spectrum, 1 + 0.5i): the multigrid factor of
        # omega-Jacobi V(1,1) on M (30 cycles of the stationary iteration, FP64 hierarchy) and a
        # preconditioned Bi-CGSTAB solve (FP32 V-cycle) each
        sign = {}
        for tag, sh_ in (("1+0.5i", 1 + 0.5j), ("1-0.5i", 1 - 0.5j)):
            pc = hi.Precond(kind=hi.PC_CSL, shift=sh_, smoother=hi.SM_JACOBI, omega=0.5)
            hm = Helm(p, pc, mg_dtype="c128")
            k, _, hist = hm.mg_iterate(f, max_cycles=30, reduction=1e-12)
            hm.close()
            hs = Helm(p, pc, mg_dtype="c64")
            xs_, inf = hs.solve(b, tol=TOL, maxmv=4000)
            hs.close()
            launches += inf.kernels
            fac = float(hist[-1] ** (1.0 / len(hist))) if len(hist) else None
            sign[tag] = {"mg_factor": fac, "mg_cycles_run": int(len(hist)), "mg_residual_ratio_last": float(hist[-1]),
                         "bicgstab_status": int(inf.status), "bicgstab_matvecs": int(inf.matvecs),
                         "bicgstab_true_rel_res": float(inf.rel_res_true)}
        out["csl_shift_sign"] = sign
    total = sum(seconds)
    cfg = {"workload": "select-" + p.name, "n_unknowns": p.n,
           "rule": "parameter x 0.8 per trial (at most 16) while omega-Jacobi V(1,1) on M reaches 1e-6 in "
                   "<= 30 cycles (FP64 hierarchy, seeded random f)",
           "solves": "Bi-CGSTAB, FP32 V-cycle, FP64 Krylov, tol 1e-6, default vs chosen parameter"}
    line = {"metric": "automatic preconditioner-parameter selections per second", "value": len(seconds) / total,
            "unit": "selections/s", "n_gpus": ranks.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / len(seconds), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic", "config": cfg}
    line.update({"csl": out["csl"], "csg": out["csg"], "csl_shift_sign": out["csl_shift_sign"], "clocks": clk.summary(),
                 "e2e": {"value": None, "unit": "selections/s", "path": "not measured in this mode",
                         "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                 "gpu_launches": int(launches)})
    return line


def run_gmres(args, torch, ranks, dev, local):
    """The paper's GMRES remark (Section 7): multigrid-preconditioned GMRES on MP2 with nu = 1,
    k = 4 and ECS layers, the CSG preconditioner of Table MP2's row for that case (theta_beta =
    pi/26), residual reduced by seven orders of magnitude; beside it Bi-CGSTAB and IDR(4) on the
    same preconditioner.  GMRES(128) (restarted only past 128 steps) and GMRES(30) are timed one
    solve at a time, like the other two methods."""
    import bench
    from paper_0912_0180_gb300.helm import Helm
    p = hi.workload_mp2(nu=1.0, k=4.0)
    b = torch.from_numpy(p.b).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=np.pi / 26, smoother=hi.SM_JACOBI, omega=0.5, galerkin=True)
    tol = 1e-7
    methods = [("gmres128", hi.GMRES, 128), ("gmres30", hi.GMRES, 30), ("bicgstab", hi.BICGSTAB, 4),
               ("idr4", hi.IDR, 4)]
    shadow = hi.shadow_space(p.n, 4)
    res, launches = {}, 0
    with bench.ClockSampler(local) as clk:
        for mg in ("c128", "c64"):
            h = Helm(p, pc, mg_dtype=mg)
            for name, meth, s in methods:
                kw = dict(method=meth, s=s, tol=tol, maxmv=MP_MAXMV, shadow=shadow if meth == hi.IDR else None,
                          host_loop=args.host_loop)
                for _ in range(args.warmup):
                    h.solve(b, **kw)
                ms, info = [], None
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    x, info = h.solve(b, **kw)
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                if (mg, name) == ("c128", "gmres128") and (info.status != 0 or not info.rel_res_true < tol):
                    raise SystemExit(f"gmres workload: {name} ({mg}) did not converge: {info}")
                launches += info.kernels
                # a solve that misses tol within the matvec cap is reported, not hidden
                res[(mg, name)] = {"status": info.status, "matvecs": info.matvecs,
                                   "ms": ranks.max(statistics.mean(ms)), "restarts": info.restarts,
                                   "true_rel_res": info.rel_res_true}
            h.close()
    g = res[("c128", "gmres128")]
    cfg = {"workload": "gmres-" + p.name, "n_unknowns": p.n, "tol": tol,
           "preconditioner": "CSG theta_beta = pi/26, Galerkin omega-Jacobi V(1,1)",
           "solves": "one at a time: GMRES(128), GMRES(30), Bi-CGSTAB, IDR(4)",
           "l2": "flushed (512 MiB device write) before every timed solve"}
    line = _base(args, ranks.job_rate(1, g["ms"]), g["ms"], ranks.world, cfg, "c128")
    line.update({
        "methods": {mg: {name: res[(mg, name)] for name, _, _ in methods} for mg in ("c128", "c64")},
        "paper_context": {"gmres_iterations": 103, "bicgstab_matvecs": 115, "idr4_matvecs": 123,
                          "gmres_time_over_bicgstab": "about 5 (175 s against 36 s, MATLAB on a Xeon)"},
        "clocks": clk.summary(),
        "e2e": {"value": None, "unit": "solves/s", "path": "not measured in this mode",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": int(launches),
    })
    return line
