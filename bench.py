#!/usr/bin/env python
"""Throughput of the waveform-relaxation multigrid cycle on one GB300 (or N replicas).

A step is one V(2,2) waveform-Vanka cycle (Algorithm Vcycle) on the 64x64
Taylor-Hood Q3/Q2, DG(1), 64-slab, nu = 1e-3 Fourier-forced workload
(11,665,792 space-time DoFs, 6 levels), with the slab factors stored (step (b)
is timed once, separately, as ``factor_ms``).  Every step runs the whole hot
path: per-patch gathers and forward substitutions over slabs with the stored
factors (a, c), additive scatters (d), matrix-free residuals (e) and grid
transfers (f) on every level, plus the coarse direct solve.

value = space-time DoFs per second per cycle, summed over ranks (each rank runs
an independent replica; the method has no exchange step across GPUs on this
path).  The working set (~134 GB of stored factors streamed every cycle) is far
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import dataclasses
import hashlib
import json
import os
import resource
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time DoF/s per waveform-Vanka V(2,2) cycle"
UNIT = "DoF/s"
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--workload", default="q3q2", choices=["q3q2", "q2q1"],
                    help="cycle form: q3q2 = 64x64 Q3/Q2 DG(1) 64 slabs (default); "
                         "q2q1 = 128x128 Q2/Q1 DG(0) 128 slabs")
    ap.add_argument("--n", type=int, default=None, help="mesh (smaller only for profiling captures)")
    ap.add_argument("--slabs", type=int, default=None, help="time slabs (fewer only for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--members", type=int, default=None,
                    help="batch form: number of solves (256); serve form: number of requests (32)")
    ap.add_argument("--rates", default="10,20,50,100,200,500", help="serve form: Poisson arrival rates (requests/s)")
    ap.add_argument("--inflight", type=int, default=8, help="serve form: solves in flight at most (per-request mode)")
    ap.add_argument("--seq-members", type=int, default=0,
                    help="batch form: time the FP64 request-by-request arm on the first M members (0: all)")
    ap.add_argument("--serve-mode", default="both", choices=["stream", "batched", "both"],
                    help="serve form: one stream and context per request, cohorts batched per cycle, or both")
    ap.add_argument("--cohort", type=int, default=16, help="serve form, batched mode: members per cohort at most")
    ap.add_argument("--cohort-slots", type=int, default=2, help="serve form, batched mode: cohorts in flight at most")
    ap.add_argument("--budget-gb", type=float, default=96.0, help="serve form: device-memory budget")
    ap.add_argument("--tile", type=int, default=-1,
                    help="cycle and smoother forms: force a smoother-apply tile 0..4 (default: autotuned)")
    ap.add_argument("--time-parallel", type=int, default=None,
                    help="smoother form: also time the parallel-in-time patch solve (1 = auto, 2 = forced)")
    ap.add_argument("--grid", default=None,
                    help="serve form: comma-separated meshes and slab counts to draw from (overrides --full-mix)")
    ap.add_argument("--full-mix", action="store_true",
                    help="serve form: draw n and N from {16, 32, 64} (default {16, 32})")
    ap.add_argument("--form", default="cycle", choices=["cycle", "precision", "batch", "serve", "smoother", "timestepping", "lid", "heat",
                                                        "setup", "jacobian", "transfers"],
                    help="cycle: the V(2,2) throughput line (default); precision: the FP64/FP32/BF16 "
                         "solves of the 128x128 Q2/Q1 DG(0) 128-slab workload")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(args, seed=0):
    from paper_2407_13997_gb300 import inputs
    if args.workload == "q2q1":
        w = inputs.fourier_128x128_q2q1_dg0(seed)
        n, N = args.n or 128, args.slabs or 128
        if (n, N) != (128, 128):
            w.n_fine, w.N = n, N
            w.name = f"fourier_q2q1_dg0_n{n}_N{N}"
        return w
    w = inputs.fourier_64x64_q3q2_dg1(seed)
    n, N = args.n or 64, args.slabs or 64
    if (n, N) != (64, 64):
        w.n_fine, w.N = n, N
        w.name = f"fourier_q3q2_dg1_n{n}_N{N}"
    return w


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self, wait_first=True):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while wait_first and not self.lines and time.time() - t0 < 20:
            time.sleep(0.05)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _a10_pattern(w, patch, sp):
    """Sparsity pattern of the off-diagonal temporal block A10 of a DG(1) patch block
    among its real slots (spatial indices sp, in slot order), as a boolean matrix: two
    slots couple iff they share one of the patch's 2 x 2 cells and are not both pressure
    slots."""
    import numpy as np
    k, n = w.k, w.n_fine
    nv, npr = n * (k + 1) + 1, n * k + 1
    I, J = patch % (n + 1), patch // (n + 1)
    vel = sp < 2 * nv * nv
    t = np.where(vel, sp % (nv * nv), sp - 2 * nv * nv)
    gx = np.where(vel, t % nv, t % npr)
    gy = np.where(vel, t // nv, t // npr)
    ix = np.where(vel, gx - (I - 1) * (k + 1), gx - (I * k - (k - 1)))
    iy = np.where(vel, gy - (J - 1) * (k + 1), gy - (J * k - (k - 1)))

    def cells(c):
        lim = np.where(vel, k + 1, k - 1)
        return (c <= lim).astype(np.int64) | 2 * (c >= lim).astype(np.int64)

    cx, cy = cells(ix), cells(iy)
    return ((cx[:, None] & cx[None, :]) != 0) & ((cy[:, None] & cy[None, :]) != 0) & (vel[:, None] | vel[None, :])


def _a10_nonzeros(w, patch, sp):
    """Nonzeros of a DG(1) patch block's A10 among its real slots."""
    return int(_a10_pattern(w, patch, sp).sum())


def smoother_algorithmic(ctx, w, factor_bytes=8):
    """Algorithmic bytes and flops of one finest-level smoother-apply launch:
    every (patch, slab) streams its factor entries once (m = the patch's true
    size, padding excluded; factor_bytes per entry): (q+1)^2 m^2, except that FP64
    DG(1) blocks stream A10 by its nonzeros (3 m^2 + nnz(A10)); it reads its m (q+1)
    FP64 right-hand side values and writes as many FP64 outputs; 2 flops per
    factor entry."""
    L = ctx.fine
    n1 = w.n_fine + 1
    nt = w.q + 1
    sparse_a10 = factor_bytes == 8 and w.q == 1
    ent = vec = 0
    for p in range(n1 * n1):
        idx = ctx.patch_dofs(L, p, 0)  # (q+1) * m per slab, temporal index first
        m = len(idx) // nt
        vec += len(idx)
        ent += 3 * m * m + _a10_nonzeros(w, p, idx[:m]) if sparse_a10 else (nt * m) ** 2
    return factor_bytes * ent * w.N + 16.0 * vec * w.N, 2.0 * ent * w.N


def traffic_record(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu summary,
    valid only while the kernel source is unchanged (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    rec = d.get(f"{kernel}/{workload}")
    if not rec or not rec.get("source"):
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()
    return rec.get("dram_bytes_per_launch") if rec.get("source_sha256") == sha else None


def _oracle_sample(w):
    """The oracle's V(2,2) cycle on the 16x16, 8-slab instance of the workload's
    discretisation: (hierarchy, right-hand side)."""
    from oracle.fem import Problem
    from oracle.solver import Hierarchy, Options
    from paper_2407_13997_gb300 import inputs
    pb = Problem(kind="fourier", nu=w.nu, conv=w.conv, T=w.T, mx=w.mx, my=w.my, amp=w.amp)
    ws = inputs.fourier_64x64_q3q2_dg1(0)
    ws.n_fine, ws.N = 16, 8
    h = Hierarchy(ws.n_fine, ws.n_coarse, ws.k, ws.q, ws.N, pb, Options())
    W = inputs.forcing_shaped_iterate(ws)
    h.linearise(W)
    b = -h.fine.residual(W)
    h.vcycle(b)
    return h, b


def _oracle_replica(w, steps, barrier, out):
    """One process of the all-cores oracle run: set up, wait for every replica, time
    `steps` cycles."""
    h, b = _oracle_sample(w)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        h.vcycle(b)
    out.put((h.fine.ndofs * steps, time.perf_counter() - t0))


def cpu_baseline(w, steps=3, all_cores=True):
    """The oracle (FP64 CPU, test infrastructure) timed on this host: V(2,2) cycles
    on the 16x16, 8-slab instance of the same Q3/Q2 DG(1) Fourier problem, (1) in this
    process and (2) on every host core, one independent replica per core (processes
    started by spawn, one BLAS thread each), timed from a common barrier to the last
    replica's end.  The oracle's cost per DoF per cycle does not depend on the mesh
    (fixed patch size, fixed stencils), so DoF/s per cycle carries over to the 64x64
    workload."""
    h, b = _oracle_sample(w)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(steps):
        h.vcycle(b)
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    nd = h.fine.ndofs
    single = {"value": nd * steps / dt, "unit": UNIT, "cores": max(1, round(cpu / dt)), "kind": "oracle",
              "sample": f"{steps} oracle V(2,2) cycles on the 16x16, 8-slab instance ({nd} DoFs) of the same "
                        f"Q3/Q2 DG(1) Fourier problem, {dt / steps:.2f} s per cycle"}
    if not all_cores:
        return single, nd, dt / steps
    import multiprocessing as mp
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"  # inherited by the spawned replicas: one core each
    try:
        ctx = mp.get_context("spawn")
        barrier, out = ctx.Barrier(ncores + 1), ctx.Queue()
        procs = [ctx.Process(target=_oracle_replica, args=(w, steps, barrier, out)) for _ in range(ncores)]
        for p in procs:
            p.start()
        barrier.wait()
        t0 = time.perf_counter()
        res = [out.get() for _ in procs]
        wall = time.perf_counter() - t0
        for p in procs:
            p.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dofs = sum(r[0] for r in res)
    line = {"value": dofs / wall, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} independent replicas (one process and one BLAS thread per host core), each "
                      f"{steps} oracle V(2,2) cycles on the 16x16, 8-slab instance ({nd} DoFs) of the same "
                      f"Q3/Q2 DG(1) Fourier problem; {wall:.2f} s from a common start to the last replica's end",
            "single_thread": single}
    return line, nd, wall / steps


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    w = workload(args)
    base, nd, sec = cpu_baseline(w, steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "ndofs": w.ndofs(), "sample_ndofs": nd, "parallelism": "replicas"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    from paper_2407_13997_gb300.replicas import max_over_ranks

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = workload(args, seed=rank)
    prec = {"fp64": wrmg.WR_FP64, "fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16}[args.precision]
    ctx = wrmg.Context(w, wrmg.default_options(precision=prec, apply_tile=args.tile))
    stream = torch.cuda.current_stream()
    D = ctx.ndofs()
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    F = ctx.vector()
    ctx.residual(W, F)
    b = -F
    x = ctx.vector()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.linearise(W, eig=False)
    torch.cuda.synchronize()
    factor_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    ctx.linearise(W, eig=True)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    fp64_tflops = wrmg.measure_fp64_tflops(stream.cuda_stream)
    clocks = ClockSampler(local)
    clocks.start()  # returns after the first sample, before the warm-up
    ctx.profile(True)  # pre-creates the CUDA events
    for _ in range(args.warmup):
        ctx.vcycle(b, x)
    torch.cuda.synchronize()
    ctx.profile(True)  # drop the warm-up records
    clocks.lines.clear()
    launches0 = wrmg.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # ncu --nvtx --nvtx-include timed/ lists these launches only
    e0.record(stream)
    for _ in range(args.steps):
        ctx.vcycle(b, x)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = wrmg.launch_count() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    sm_ms, sm_n = ctx.profile_smoother(ctx.fine)
    jac_ms, jac_n, jac_flops = ctx.profile_jacobian(ctx.fine)
    ctx.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = D * world * args.steps / (ms * 1e-3)

    # end to end through the host-buffer ABI call: H2D of b, cycle, D2H of x every step
    hb = torch.empty(D, dtype=torch.float64).pin_memory()
    hx = torch.empty(D, dtype=torch.float64).pin_memory()
    hb.copy_(b.cpu())
    bn, xn = hb.numpy(), hx.numpy()
    ctx.vcycle_host(bn, xn)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.vcycle_host(bn, xn)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    assert np.isfinite(xn).all()

    alg_bytes, alg_flops = smoother_algorithmic(ctx, w, {wrmg.WR_FP64: 8, wrmg.WR_FP32: 4, wrmg.WR_BF16: 2}[prec])
    avg_s = sm_ms / max(sm_n, 1) * 1e-3
    hbm_peak, hbm_src = measured_peaks()
    achieved_tf = alg_flops / avg_s / 1e12
    achieved_gbs = alg_bytes / avg_s / 1e9
    if prec == wrmg.WR_FP64:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_tflops, "traffic": traffic_record("block_apply_kernel", w.name),
                "kernel": "block_apply_kernel (finest level)", "launches": sm_n, "avg_ms": avg_s * 1e3,
                "peak_source": "FP64 FMA rate measured live by wr_measure_fp64_tflops",
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src}}
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic_record(f"block_apply_kernel_{args.precision}", w.name),
                "kernel": f"block_apply_kernel (finest level, {args.precision} factors)", "launches": sm_n,
                "avg_ms": avg_s * 1e3, "peak_source": hbm_src}

    # the J(W) x element kernel of the finest level (step (e)): FP64-ALU bound; its
    # HBM figure is the method's bytes per apply, 8 (2 D + D_u)
    javg_s = jac_ms / max(jac_n, 1) * 1e-3
    nv = w.n_fine * (w.k + 1) + 1
    d_u = w.N * (w.q + 1) * 2 * nv * nv
    jac_tf = jac_flops / javg_s / 1e12 if jac_n else None
    jac_gbs = 8.0 * (2 * D + d_u) / javg_s / 1e9 if jac_n else None
    roof_jac = {"bound": "alu", "achieved": jac_tf, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": jac_tf / fp64_tflops if jac_n else None,
                "traffic": traffic_record("jac_kernel", w.name),
                "kernel": "jac_kernel (J(W) x element kernel, finest level)", "launches": jac_n,
                "avg_ms": javg_s * 1e3, "flops_per_launch": jac_flops,
                "peak_source": "FP64 FMA rate measured live by wr_measure_fp64_tflops",
                "hbm": {"achieved": jac_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": jac_gbs / hbm_peak if jac_n else None, "peak_source": hbm_src}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {wrmg.WR_FP64: "f64", wrmg.WR_FP32: "f32 factors+smoother / f64 residual+Krylov",
                      wrmg.WR_BF16: "bf16 factors, f32 smoother / f64 residual+Krylov"}[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "ndofs": D, "n": w.n_fine, "k": w.k, "q": w.q, "N": w.N,
                       "levels": ctx.num_levels, "factor_storage": args.precision,
                       "device_bytes": ctx.device_bytes(),
                       "apply_tiles": [ctx.apply_tile(l) for l in range(1, ctx.num_levels)],
                       "l2": f"no flush: {ctx.device_bytes() / 1e9:.0f} GB on the device, the stored factors "
                             "streamed every cycle >> 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "factor_ms": factor_ms, "setup_ms": setup_ms, "roofline": roof, "roofline_jacobian": roof_jac,
            "e2e": {"value": D * world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * D,
                    "d2h_bytes_per_step": 8 * D},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)[0]
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_precision_form(args):
    """Precision form on the 128x128 Q2/Q1 DG(0), 128-slab workload: the FP64 solve
    (run to 1e-11, the reference), then FP64, FP32 and BF16 smoother solves to 1e-8 and
    to 1e-10; each reports its final error against the FP64 reference, its FGMRES
    iterations, its V(2,2) cycle throughput and its solve time, and each reduced-
    precision solve its speed-up over the FP64 solve to the same tolerance."""
    import numpy as np
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    w = inputs.fourier_128x128_q2q1_dg0(0)
    if args.n or args.slabs:
        w.n_fine, w.N = args.n or w.n_fine, args.slabs or w.N
        w.name = f"fourier_q2q1_dg0_n{w.n_fine}_N{w.N}"
    out = {"form": "precision", "workload": w.name,
           "ndofs": w.ndofs(), "variants": {}}
    ref = None
    for name, prec, rtol in [("fp64", wrmg.WR_FP64, 1e-11), ("fp64", wrmg.WR_FP64, 1e-8), ("fp64", wrmg.WR_FP64, 1e-10),
                             ("fp32", wrmg.WR_FP32, 1e-8), ("fp32", wrmg.WR_FP32, 1e-10),
                             ("bf16", wrmg.WR_BF16, 1e-8), ("bf16", wrmg.WR_BF16, 1e-10)]:
        ctx = wrmg.Context(w, wrmg.default_options(precision=prec, newton_rtol=rtol))
        U = ctx.vector()
        ctx.initial_guess(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx.solve(U)
        torch.cuda.synchronize()
        solve_s = time.perf_counter() - t0
        # cycle throughput about the converged iterate
        F = ctx.vector()
        ctx.residual(U, F)
        x = ctx.vector()
        for _ in range(2):
            ctx.vcycle(-F, x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            ctx.vcycle(-F, x)
        e1.record()
        torch.cuda.synchronize()
        cyc_ms = e0.elapsed_time(e1) / 5
        u = U.cpu().numpy()
        rec = {"newton": st["newton_its"], "fgmres": st["gmres"], "fgmres_total": sum(st["gmres"]),
               "final_rel_residual": st["residuals"][-1] / st["residuals"][0], "solve_s": solve_s,
               "setup_s": st["setup_ms"] / 1e3, "cycle_ms": cyc_ms, "dof_per_s_per_cycle": w.ndofs() / cyc_ms * 1e3,
               "device_bytes": ctx.device_bytes(), "rtol": rtol}
        if ref is None:
            ref = u
        else:
            rec["rel_error_vs_fp64"] = float(np.abs(u - ref).max() / np.abs(ref).max())
        if name != "fp64" and f"fp64_rtol{rtol:g}" in out["variants"]:
            same = out["variants"][f"fp64_rtol{rtol:g}"]
            rec["speedup_vs_fp64_same_rtol"] = same["solve_s"] / solve_s
            rec["fp64_same_rtol_rel_error"] = same.get("rel_error_vs_fp64")
        out["variants"][f"{name}_rtol{rtol:g}"] = rec
        ctx.close()
        del U, F, x
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_batch_form(args):
    """Batching form: independent Q2/Q1 DG(0) solves of uneven sizes in one lock-step
    batch (FP32 smoother, FP64 residual and Krylov).  Reports the batched V(2,2)
    cycle throughput (DoFs of every member per second), the batched solve to 1e-8
    (solves/s), and the plain FP64 method run request by request on a sample."""
    import numpy as np
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    from paper_2407_13997_gb300.replicas import max_over_ranks, shard, sum_over_ranks
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:  # each rank runs its own shard of the members; no data-path collective
        import torch.distributed as dist
        dist.init_process_group("nccl")
    all_ws = inputs.batching_workloads(args.members or 256, seed=1)
    ws = [all_ws[i] for i in shard([w.ndofs() for w in all_ws], rank, world)]
    total = sum(w.ndofs() for w in ws)
    job_total = sum(w.ndofs() for w in all_ws)
    out = {"form": "batch", "members": len(all_ws), "total_ndofs": job_total, "n_gpus": world,
           "scaling": "strong (members sharded over GPUs)" if world > 1 else None,
           "mesh_mix": {str(n): sum(1 for w in all_ws if w.n_fine == n) for n in (8, 16, 24, 32, 48)}}
    t0 = time.perf_counter()
    batch = wrmg.Batch(ws, wrmg.default_options(precision=wrmg.WR_FP32))
    torch.cuda.synchronize()
    out["create_s"] = time.perf_counter() - t0
    out["device_bytes"] = batch.device_bytes()
    Ws = [torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda() for w in ws]
    t0 = time.perf_counter()
    batch.linearise(Ws)
    torch.cuda.synchronize()
    out["linearise_s"] = time.perf_counter() - t0
    rng = np.random.default_rng(2)
    bs = [torch.from_numpy(rng.standard_normal(w.ndofs())).cuda() for w in ws]
    xs = batch.vectors()
    batch.vcycle(bs, xs)
    for _ in range(2):
        batch.vcycle_resident()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = wrmg.launch_count()
    if dist:
        dist.barrier()
    e0.record()
    for _ in range(args.steps):
        batch.vcycle_resident()
    e1.record()
    torch.cuda.synchronize()
    cyc = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    out["cycle_ms"] = cyc
    out["dof_per_s_per_cycle"] = job_total / cyc * 1e3
    out["launches_per_cycle"] = (wrmg.launch_count() - launches0) / args.steps
    del Ws, bs, xs
    Us = batch.vectors()
    batch.initial_guess(Us)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    st = batch.solve(Us, check=False)
    torch.cuda.synchronize()
    solve_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    conv = [s["residuals"][-1] <= 1e-8 * s["residuals"][0] for s in st]
    nconv = int(sum_over_ranks(sum(conv), dist, "cuda"))
    out["batched_solve"] = {"seconds": solve_s, "solves_per_s": len(all_ws) / solve_s, "converged": nconv,
                            "newton_max": max(s["newton_its"] for s in st),
                            "fgmres_total_mean": float(np.mean([sum(s["gmres"]) for s in st]))}
    batch.close()
    del Us
    torch.cuda.empty_cache()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # the plain FP64 method, request by request, on every member (or the first
    # --seq-members of them), to the same rtol 1e-8
    sample = all_ws[:args.seq_members] if args.seq_members else all_ws
    t0 = time.perf_counter()
    seq_conv = 0
    for w in sample:
        ctx = wrmg.Context(w)
        U = ctx.vector()
        ctx.initial_guess(U)
        s64 = ctx.solve(U, check=False)
        seq_conv += s64["status"] == wrmg.WR_OK
        ctx.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    out["sequential_fp64"] = {"members": len(sample), "seconds": seq, "solves_per_s": len(sample) / seq,
                              "converged": seq_conv, "ndofs": sum(w.ndofs() for w in sample)}
    out["solves_per_s_ratio_batched_vs_sequential_fp64"] = out["batched_solve"]["solves_per_s"] / (len(sample) / seq)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serve_form(args):
    """Serving form: a seeded Poisson stream of solve requests (Q2/Q1 DG(0) or Q3/Q2
    DG(1), nu log-uniform in [1e-3, 1e-1]) served by the native request loop with
    FP32 factors and FP64 Newton/Krylov to rtol 1e-8, against the plain FP64 method
    run request by request.  The loop runs in per-request mode (a stream and context
    per request) and in batched mode (cohorts of queued requests solved as one
    lock-step batch per slot, per-cycle batching).  The FP64 arm is timed request by
    request (context set-up, solve and the host copy of the solution) and its
    latencies follow from those service times and the same arrivals through a single
    FIFO server."""
    import numpy as np
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    grid = tuple(int(v) for v in args.grid.split(",")) if args.grid else ((16, 32, 64) if args.full_mix else (16, 32))
    reqs = inputs.serving_workloads(args.members or 32, seed=2, ns=grid, slabs=grid)
    rates = [float(r) for r in args.rates.split(",")]
    o32 = wrmg.default_options(precision=wrmg.WR_FP32, newton_rtol=1e-8)
    o64 = wrmg.default_options(precision=wrmg.WR_FP64, newton_rtol=1e-8)
    out = {"form": "serve", "requests": len(reqs), "mesh_and_slab_grid": list(grid),
           "total_ndofs": sum(w.ndofs() for w in reqs), "inflight_cap": args.inflight,
           "budget_bytes": int(args.budget_gb * 2 ** 30), "options": "FP32 factors, FP64 Newton/FGMRES, rtol 1e-8",
           "cohort": args.cohort, "cohort_slots": args.cohort_slots}
    modes = ["stream", "batched"] if args.serve_mode == "both" else [args.serve_mode]
    warm = inputs.serving_workloads(2, seed=99, ns=(16,), slabs=(16,))
    for w in warm:                                    # module loading and first-launch set-up
        for o in (o32, o64):
            ctx = wrmg.Context(w, o)
            U = ctx.vector()
            ctx.initial_guess(U)
            ctx.solve(U, check=False)
            ctx.close()
    torch.cuda.synchronize()
    # plain FP64, request by request
    service, refs, seq_status = [], [], []
    for w in reqs:
        t0 = time.perf_counter()
        ctx = wrmg.Context(w, o64)
        U = ctx.vector()
        ctx.initial_guess(U)
        st = ctx.solve(U, check=False)
        refs.append(U.cpu().numpy())
        ctx.close()
        service.append(time.perf_counter() - t0)
        seq_status.append(st["status"])
        del U
    torch.cuda.empty_cache()
    out["sequential_fp64"] = {"converged": sum(1 for c in seq_status if c == wrmg.WR_OK),
                              "service_s_total": sum(service), "service_s_median": statistics.median(service),
                              "solves_per_s_saturated": len(reqs) / sum(service), "rates": {}}
    out["rates"] = {}
    errs = []
    for rate in rates:
        arr = inputs.poisson_arrivals(len(reqs), rate, seed=2)
        end, lat = 0.0, []
        for a, sv_t in zip(arr, service):             # the FIFO single server of the FP64 arm
            end = max(a, end) + sv_t
            lat.append(end - a)
        out["sequential_fp64"]["rates"][str(int(rate))] = {
            "solves_per_s": len(reqs) / (end - arr[0]), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99))}
        out["rates"][str(int(rate))] = {}
        for mode in modes:
            if mode == "batched":
                sv = wrmg.Server(out["budget_bytes"], args.cohort_slots, o32, batch_members=args.cohort)
            else:
                sv = wrmg.Server(out["budget_bytes"], args.inflight, o32)
            tickets = [None] * len(reqs)

            def feeder():
                t0 = time.perf_counter()
                for i, (a, w) in enumerate(zip(arr, reqs)):
                    dt = t0 + a - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    tickets[i] = sv.submit(w)

            t_start = time.perf_counter()
            th = threading.Thread(target=feeder)
            th.start()
            th.join()
            res = [sv.poll(t) for t in tickets]
            t_end = time.perf_counter()
            st = sv.stats()
            sv.close()
            lat = [r[3] for r in res]
            ok = sum(1 for r in res if r[0] == wrmg.WR_OK)
            for r, ref, c64 in zip(res, refs, seq_status):
                if r[1] is not None and r[0] == wrmg.WR_OK and c64 == wrmg.WR_OK:
                    errs.append(float(np.abs(r[1] - ref).max() / max(np.abs(ref).max(), 1e-300)))
            out.setdefault("per_request", [{"name": w.name, "nu": w.nu, "fp64_status": c, "fp64_s": t}
                                           for w, c, t in zip(reqs, seq_status, service)])
            for pr, r in zip(out["per_request"], res):
                pr[f"{mode}_status_{int(rate)}"] = r[0]
                pr[f"{mode}_latency_ms_{int(rate)}"] = r[3]
            out["rates"][str(int(rate))][mode] = {
                "solves_per_s": len(reqs) / (t_end - t_start - arr[0]), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "converged": ok, "peak_inflight": st["peak_inflight"],
                "peak_cohort": st["peak_cohort"], "peak_bytes": st["peak_bytes"],
                "newton_total": sum(r[2]["newton_its"] for r in res),
                "fgmres_total": sum(sum(r[2]["gmres"]) for r in res)}
    # over the requests both arms solved to 1e-8
    out["max_rel_diff_vs_fp64_solution"] = max(errs) if errs else None
    top = str(int(max(rates)))
    out["solves_per_s_ratio_vs_sequential_fp64"] = {
        mode: out["rates"][top][mode]["solves_per_s"] / out["sequential_fp64"]["rates"][top]["solves_per_s"]
        for mode in modes}
    print(json.dumps(out), flush=True)


def run_smoother_form(args):
    """The finest-level smoother apply alone (gather, forward substitution over slabs
    with the stored factors, scatter), K timed launches after W warm-ups: the burst
    roofline of the dominant kernel, and the command the ncu captures run."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    w = workload(args)
    prec = {"fp64": wrmg.WR_FP64, "fp32": wrmg.WR_FP32, "bf16": wrmg.WR_BF16}[args.precision]
    ctx = wrmg.Context(w, wrmg.default_options(precision=prec, apply_tile=args.tile))
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    ctx.linearise(W, eig=False)
    L = ctx.fine
    r = torch.from_numpy(inputs.seeded_vector(3, ctx.ndofs(L))).cuda()
    y = ctx.vector(L)
    stream = torch.cuda.current_stream()
    fp64_tflops = wrmg.measure_fp64_tflops(stream.cuda_stream)
    ctx.profile(True)
    for _ in range(args.warmup):
        ctx.patch_apply(L, r, y)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        ctx.patch_apply(L, r, y)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sm_ms, sm_n = ctx.profile_smoother(L)
    alg_bytes, alg_flops = smoother_algorithmic(ctx, w, {wrmg.WR_FP64: 8, wrmg.WR_FP32: 4, wrmg.WR_BF16: 2}[prec])
    avg_s = sm_ms / max(sm_n, 1) * 1e-3
    hbm_peak, hbm_src = measured_peaks()
    tp = None
    if args.time_parallel:
        # the same apply with the slabs split into chunks solved in parallel (all phases timed)
        ctx2 = wrmg.Context(w, wrmg.default_options(precision=prec, time_parallel=args.time_parallel))
        ctx2.linearise(W, eig=False)
        for _ in range(args.warmup):
            ctx2.patch_apply(L, r, y)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            ctx2.patch_apply(L, r, y)
        f1.record(stream)
        torch.cuda.synchronize()
        tp = {"apply_with_scatter_ms": f0.elapsed_time(f1) / args.steps, "mode": args.time_parallel}
        ctx2.close()
    out = {"form": "smoother", "workload": w.name, "precision": args.precision, "launches": sm_n,
           "apply_tile": ctx.apply_tile(L), "time_parallel": tp,
           "apply_kernel_ms": avg_s * 1e3, "apply_with_scatter_ms": e0.elapsed_time(e1) / args.steps,
           "algorithmic_bytes": alg_bytes, "algorithmic_flops": alg_flops,
           "achieved_gbs": alg_bytes / avg_s / 1e9, "hbm_frac": alg_bytes / avg_s / 1e9 / hbm_peak,
           "hbm_peak_source": hbm_src, "achieved_tflops": alg_flops / avg_s / 1e12,
           "fp64_peak_tflops": fp64_tflops, "fp64_frac": alg_flops / avg_s / 1e12 / fp64_tflops}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_jacobian_form(args):
    """The finest-level J(W) x apply alone (element kernel and assembly), K timed
    applications after W warm-ups, with the factors recomputed per window so that the
    context holds little besides the vectors and W at the Gauss points: the burst
    roofline of the element kernel, and the command its ncu captures run."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    w = workload(args)
    ctx = wrmg.Context(w, wrmg.default_options(store_factors=wrmg.WR_RECOMPUTE, recompute_slabs=1))
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    ctx.linearise(W, eig=False)
    L = ctx.fine
    x = torch.from_numpy(inputs.seeded_vector(3, ctx.ndofs(L))).cuda()
    y = ctx.vector(L)
    stream = torch.cuda.current_stream()
    fp64_tflops = wrmg.measure_fp64_tflops(stream.cuda_stream)
    ctx.profile(True)
    for _ in range(args.warmup):
        ctx.apply_jacobian(L, x, y)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        ctx.apply_jacobian(L, x, y)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    jms, jn, jflops = ctx.profile_jacobian(L)
    avg_s = jms / max(jn, 1) * 1e-3
    D = ctx.ndofs(L)
    nv = w.n_fine * (w.k + 1) + 1
    alg_bytes = 8.0 * (2 * D + w.N * (w.q + 1) * 2 * nv * nv)
    hbm_peak, hbm_src = measured_peaks()
    out = {"form": "jacobian", "workload": w.name, "launches": jn, "element_kernel_ms": avg_s * 1e3,
           "apply_ms": e0.elapsed_time(e1) / args.steps, "flops_per_launch": jflops,
           "achieved_tflops": jflops / avg_s / 1e12, "fp64_peak_tflops": fp64_tflops,
           "fp64_frac": jflops / avg_s / 1e12 / fp64_tflops, "algorithmic_bytes": alg_bytes,
           "achieved_gbs": alg_bytes / avg_s / 1e9, "hbm_frac": alg_bytes / avg_s / 1e9 / hbm_peak,
           "hbm_peak_source": hbm_src}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_transfers_form(args):
    """Restriction, prolongation and the smoother's scatter on the finest level alone,
    with the factors recomputed per one-slab window so that the context holds the
    full-size vectors (larger than L2) and little else: achieved GB/s of steps (d) and
    (f) against their algorithmic bytes, and the command their ncu captures run."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    w = workload(args)
    # no Krylov basis is needed here: the shortest restart keeps the context small
    ctx = wrmg.Context(w, wrmg.default_options(store_factors=wrmg.WR_RECOMPUTE, recompute_slabs=1,
                                               gmres_restart=2, eig_steps=1))
    W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
    ctx.linearise(W, eig=False)
    L = ctx.fine
    Df, Dc = ctx.ndofs(L), ctx.ndofs(L - 1)
    xf = torch.from_numpy(inputs.seeded_vector(3, Df)).cuda()
    xc = torch.from_numpy(inputs.seeded_vector(4, Dc)).cuda()
    yc, yf = ctx.vector(L - 1), ctx.vector(L)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps * 1e-3

    torch.cuda.nvtx.range_push("timed")
    t_r = timed(lambda: ctx.restrict(L, xf, yc))
    t_p = timed(lambda: ctx.prolong_add(L, xc, yf))
    torch.cuda.nvtx.range_pop()
    hbm_peak, hbm_src = measured_peaks()
    b_r, b_p = 8.0 * (Df + Dc), 8.0 * (Dc + 2 * Df)   # read fine + write coarse; read coarse + update fine
    out = {"form": "transfers", "workload": w.name, "fine_ndofs": Df, "coarse_ndofs": Dc,
           "restrict_ms": t_r * 1e3, "restrict_gbs": b_r / t_r / 1e9, "restrict_hbm_frac": b_r / t_r / 1e9 / hbm_peak,
           "prolong_add_ms": t_p * 1e3, "prolong_add_gbs": b_p / t_p / 1e9,
           "prolong_add_hbm_frac": b_p / t_p / 1e9 / hbm_peak, "hbm_peak_source": hbm_src,
           "algorithmic_bytes": {"restrict": b_r, "prolong_add": b_p}}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_timestepping_form(args):
    """Timestepping comparator on the Chorin problem (R = 10, t in [0, 0.1]): the
    all-at-once WRMG solve against N one-slab solves in sequence (the same
    Newton-FGMRES-multigrid machinery coupling one time element), for
    Q2/Q1 and Q3/Q2 with DG(0) and DG(1) and N = 10, 20, 40; solve times (context
    set-up excluded, every linearisation included), iterations, and the largest
    difference between the two discrete solutions."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    n = args.n or 32
    out = {"form": "timestepping", "problem": "chorin R=10, nu=1, t in [0, 0.1]", "n": n, "runs": []}
    warm = inputs.chorin(8, 1, 0, 2)
    for w in (warm, dataclasses.replace(warm, N=1, T=warm.T / warm.N)):
        ctx = wrmg.Context(w)
        U = ctx.vector()
        ctx.initial_guess(U)
        ctx.solve(U, check=False)
        ctx.close()
    for k, q in ((1, 0), (1, 1), (2, 0), (2, 1)):
        for N in (10, 20, 40):
            w = inputs.chorin(n, k, q, N)
            ctx = wrmg.Context(w)
            U = ctx.vector()
            ctx.initial_guess(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.solve(U, check=False)
            torch.cuda.synchronize()
            t_wrmg = time.perf_counter() - t0
            ctx.close()
            one = dataclasses.replace(w, N=1, T=w.T / N)
            c1 = wrmg.Context(one)
            Ut = torch.zeros(w.ndofs(), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = c1.solve_timestepping(Ut, N, check=False)
            torch.cuda.synchronize()
            t_ts = time.perf_counter() - t0
            c1.close()
            diff = float((Ut - U).abs().max() / U.abs().max())
            out["runs"].append({
                "space": f"Q{k + 1}/Q{k}", "time": f"DG({q})", "N": N, "ndofs": w.ndofs(),
                "wrmg": {"status": st["status"], "seconds": t_wrmg, "newton": st["newton_its"],
                         "fgmres_total": sum(st["gmres"])},
                "timestepping": {"status": sts["status"], "seconds": t_ts,
                                 "newton_per_step": sts["newton_its"] / N,
                                 "fgmres_per_step": sum(sts["gmres_per_step"][:N]) / min(N, 64)},
                "max_rel_diff": diff})
            del U, Ut
    print(json.dumps(out), flush=True)


def run_lid_form(args):
    """Lid-driven cavity (Sec. 4, Table lid): Q2/Q1 DG(0), t in [0, 0.02], N = 20,
    R = 1, 10, 100, on 16x16 and 32x32 meshes; whole WRMG solve times (context
    set-up excluded) and Newton (FGMRES) counts."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    out = {"form": "lid", "runs": []}
    warm = inputs.lid_cavity(8, 1, 0, 4, 10.0)
    ctx = wrmg.Context(warm)
    U = ctx.vector()
    ctx.initial_guess(U)
    ctx.solve(U, check=False)
    ctx.close()
    for n in (16, 32):
        for R in (1.0, 10.0, 100.0):
            w = inputs.lid_cavity(n, 1, 0, 20, R)
            ctx = wrmg.Context(w)
            U = ctx.vector()
            ctx.initial_guess(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.solve(U, check=False)
            torch.cuda.synchronize()
            out["runs"].append({"n": n, "R": R, "ndofs": w.ndofs(), "status": st["status"],
                                "seconds": time.perf_counter() - t0, "newton": st["newton_its"],
                                "fgmres_total": sum(st["gmres"])})
            ctx.close()
    print(json.dumps(out), flush=True)


def run_heat_form(args):
    """Heat equation (Sec. 5, Tables heat:time3/4): u_t - lap u = 0 with natural
    boundary conditions, u(0) = sin(pi x) + cos(2 pi y), t in [0, 0.02], N = 20;
    Q_k x DG(q) for k = 1, 2, 3 and q = 0..3 (the paper's grid of degrees) on the n x n
    mesh (--n, default 64; k = q = 3 coarsens to 1 x 1, every other case to 2 x 2);
    FGMRES-WRMG to a residual of max(1e-6 ||b||, 1e-6) (the paper's criterion),
    against the timestepping comparator with the same criterion per step.  Times
    exclude context set-up and include the factorisation and eigen-estimates."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    n = args.n or 64
    out = {"form": "heat", "n": n, "N": 20, "t": [0.0, 0.02], "runs": []}

    def options_for(w):
        ctx = wrmg.Context(w)
        U0, F = ctx.vector(), ctx.vector()
        ctx.residual(U0, F)           # F(0) = -b
        bn = float(F.norm())
        ctx.close()
        eta = max(1e-6, 1e-6 / bn) if bn > 0 else 1e-6
        return wrmg.default_options(newton_maxit=1, ew=0, eta_fixed=eta, newton_rtol=eta)

    warm = inputs.heat(8, 1, 0, 4)
    ctx = wrmg.Context(warm, options_for(warm))
    U = ctx.vector()
    ctx.solve(U, check=False)
    ctx.close()
    for k in (1, 2, 3):
        for q in (0, 1, 2, 3):
            w = inputs.heat(n, k, q, 20)
            o = options_for(w)
            ctx = wrmg.Context(w, o)
            U = ctx.vector()
            ctx.initial_guess(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.solve(U, check=False)
            torch.cuda.synchronize()
            t_wrmg = time.perf_counter() - t0
            # one V(2,2) cycle with the operators ready
            b = ctx.vector()
            ctx.residual(ctx.vector(), b)
            x = ctx.vector()
            for _ in range(2):
                ctx.vcycle(b, x)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                ctx.vcycle(b, x)
            e1.record()
            torch.cuda.synchronize()
            cyc = e0.elapsed_time(e1) / 5
            ctx.close()
            one = dataclasses.replace(w, N=1, T=w.T / 20)
            c1 = wrmg.Context(one, options_for(one))
            Ut = torch.zeros(w.ndofs(), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sts = c1.solve_timestepping(Ut, 20, check=False)
            torch.cuda.synchronize()
            t_ts = time.perf_counter() - t0
            c1.close()
            out["runs"].append({"space": f"Q{k}", "time": f"DG({q})", "ndofs": w.ndofs(), "n_coarse": w.n_coarse,
                                "wrmg": {"status": st["status"], "seconds": t_wrmg, "fgmres": sum(st["gmres"]),
                                         "vcycle_ms": cyc, "dof_per_s_per_cycle": w.ndofs() / cyc * 1e3},
                                "timestepping": {"status": sts["status"], "seconds": t_ts,
                                                 "fgmres_per_step": sum(sts["gmres_per_step"][:20]) / 20},
                                "max_rel_diff": float((Ut - U).abs().max() / U.abs().max())})
            del U, Ut, b, x
    print(json.dumps(out), flush=True)


def run_setup_form(args):
    """Linearisation (step (b) and the eigen-estimates) in FP64 and FP32 on the
    --workload (q2q1: 128x128 Q2/Q1 DG(0), 128 slabs; q3q2: 64x64 Q3/Q2 DG(1), 64
    slabs; --n/--slabs resize it): the first call (with
    the apply-tile tuning), the factorisation alone (convection matrices and the
    block inversions of every level) and factorisation + eigen-estimates.  The FP32
    factorisation + eigen-estimates call sits in the NVTX range `timed` (the ncu
    launch-list command).  FLOP rate: the inversions' algorithmic FMAs (m^3 per
    DG(0) block; 4 m^3 per DG(1) block: two inversions and two products) x 2 over
    the factorisation-alone time."""
    import torch
    from paper_2407_13997_gb300 import inputs, wrmg
    torch.cuda.set_device(0)
    w = workload(args)
    ms = 51 if w.k == 1 else 107
    blocks = sum((n + 1) ** 2 for n in [w.n_fine >> l for l in range(20)] if n > w.n_coarse) * w.N
    flops = 2.0 * blocks * ms ** 3 * (1 if w.q == 0 else 4)
    out = {"form": "setup", "workload": w.name, "ndofs": w.ndofs(), "blocks": blocks, "block_size": ms * (w.q + 1),
           "algorithmic_flops": flops}
    for name, prec in (("fp64", wrmg.WR_FP64), ("fp32", wrmg.WR_FP32)):
        ctx = wrmg.Context(w, wrmg.default_options(precision=prec))
        W = torch.from_numpy(inputs.forcing_shaped_iterate(w)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter(); ctx.linearise(W, eig=False); torch.cuda.synchronize()
        first = time.perf_counter() - t0
        t0 = time.perf_counter(); ctx.linearise(W, eig=False); torch.cuda.synchronize()
        fac = time.perf_counter() - t0
        if name == "fp32":
            torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter(); ctx.linearise(W, eig=True); torch.cuda.synchronize()
        full = time.perf_counter() - t0
        if name == "fp32":
            torch.cuda.nvtx.range_pop()
        out[name] = {"first_s": first, "factor_s": fac, "factor_eig_s": full, "factor_tflops": flops / fac / 1e12}
        ctx.close()
        del W
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "precision":
        run_precision_form(args)
    elif args.form == "batch":
        run_batch_form(args)
    elif args.form == "serve":
        run_serve_form(args)
    elif args.form == "jacobian":
        run_jacobian_form(args)
    elif args.form == "transfers":
        run_transfers_form(args)
    elif args.form == "smoother":
        run_smoother_form(args)
    elif args.form == "timestepping":
        run_timestepping_form(args)
    elif args.form == "lid":
        run_lid_form(args)
    elif args.form == "heat":
        run_heat_form(args)
    elif args.form == "setup":
        run_setup_form(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
