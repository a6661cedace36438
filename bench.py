#!/usr/bin/env python
"""Throughput of the pressure-correction sub-step on one GB300 (or N replicas under torchrun).

Workload: the 2D channel [0,20]x[0,10] with a cylinder (D=1 at (5,5)), 1024x512 pressure cells,
Neumann inflow / Dirichlet outflow in x, walls in y, ~4e5 meshless nodes refined radially around
the cylinder (seeded synthetic inputs; the paper publishes no dataset). One step = one full
projection: WLS transfer, divergence source, transform Poisson solve with FP64-residual
refinement, WLS gradient and correction with the IB force. Mixed precision by default.

Prints one JSON line. value = pressure cells projected per second over all ranks, device-timed
with CUDA events around each step, a 256 MB buffer written between steps to flush L2.
  --impl reference   the plain FP64 CPU oracle on the same workload (rank 0 only)
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("projected grid-points/s and HBM % of peak at 1e-10 rel-L2 vs plain FP64 GPU; "
          "p50/p99 ms")
UNIT = "grid-points/s"
WORKLOAD = "channel_cylinder 1024x512 cells, ~4.0e5 nodes, inflow/outflow x, walls y, cylinder D=1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--refine", type=int, default=4,
                    help="largest number of refinement sweeps (mixed precision)")
    ap.add_argument("--refine-tol", type=float, default=1e-13,
                    help="stopping rule ||r|| <= tol ||s|| (or the residual's rounding floor); <= 0: fixed sweeps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-problem batch measurement")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--batch-problems", type=int, default=512,
                    help="problems in the batch measurement (fewer: the same mix, for profiling)")
    ap.add_argument("--no-3d", action="store_true", help="skip the 256x128x128 box-with-sphere measurement")
    ap.add_argument("--steps-3d", type=int, default=20)
    ap.add_argument("--serve", action="store_true",
                    help="serving measurement: Poisson-arrival request stream with continuous batching")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-cold", action="store_true",
                    help="start with no resident plans (default: build every pool plan before the trace)")
    ap.add_argument("--serve-max-queue", type=int, default=512,
                    help="waiting requests beyond which arrivals are refused (backpressure)")
    ap.add_argument("--serve-deadline", type=float, default=0.5,
                    help="seconds a request may wait before it is dropped (load shedding)")
    ap.add_argument("--no-serve-leg", action="store_true",
                    help="skip the bounded serving leg of the default run")
    ap.add_argument("--serve-leg-pool", type=int, default=16)
    ap.add_argument("--serve-leg-requests", type=int, default=2000)
    ap.add_argument("--serve-fp64-requests", type=int, default=2000,
                    help="prefix of the trace also served one at a time by plain FP64 projections")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the accuracy, plain-FP64 and end-to-end measurements that follow the "
                         "timed region (shorter profiler launch lists); the timed step is unchanged")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def workload():
    from paper_2304_14690_gb300 import workloads as wl
    return wl.channel_cylinder()


# ----------------------------------------------------------------------------- oracle timing

def oracle_timing(steps, warmup, seconds=None, max_steps=None):
    """Time the CPU oracle's projection (plan built first, untimed). Returns (cells/s, info)."""
    from oracle import grid as G, projection as PR
    prob = workload()
    g = G.Grid(prob.dim, prob.n, prob.lo, prob.h, prob.bc_lo, prob.bc_hi)
    t0 = time.perf_counter()
    plan = PR.build_plan(g, prob.nodes, prob.node_type, K=prob.knn)
    plan_s = time.perf_counter() - t0
    for _ in range(warmup):
        PR.project(plan, prob.dt, prob.u_star)
    times = []
    t_start = time.perf_counter()
    while True:
        t = time.perf_counter()
        PR.project(plan, prob.dt, prob.u_star)
        times.append(time.perf_counter() - t)
        if seconds is None and len(times) >= steps:
            break
        if max_steps is not None and len(times) >= max_steps:
            break
        if seconds is not None and time.perf_counter() - t_start >= seconds and len(times) >= 2:
            break
    total = sum(times)
    cells = prob.num_cells
    return cells * len(times) / total, dict(projections=len(times), seconds=total,
                                            plan_seconds=plan_s, ms_per_projection=1e3 * total / len(times),
                                            times=times)


def cpu_baseline_subprocess(seconds):
    """Run the oracle timing single-threaded in a fresh interpreter (BLAS pinned to 1 thread)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-baseline-only",
           "--cpu-seconds", str(seconds)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-500:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, device_index):
        self.proc = None
        self.path = None
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50"]
            if device_index is not None:
                cmd += ["-i", str(device_index)]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "power_w_max": max(r["power"] for r in rows),
                "reasons": sorted(reasons)}


def _smi_id(dev, local_rank):
    """nvidia-smi -i selector of this rank's GPU (UUID when torch exposes it)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return None if os.environ.get("CUDA_VISIBLE_DEVICES") else local_rank


# ----------------------------------------------------------------------------- roofline

def phase_bytes(prob, precision, refine, sweeps_done=None, adaptive=False):
    """Algorithmic DRAM bytes per call of each phase, from the data each kernel must read and
    write once: WLS rows (index + weights), gathered node/cell values, outputs. The transform
    phase takes the scope table's figure for a multi-pass solve: (2 dim - 1) axis passes, each
    reading and writing 4 B per cell (24 B per cell per solve in 2D, 40 B in 3D), times the
    solves run (the first and one per refinement sweep)."""
    d, N, K, Kg = prob.dim, prob.num_nodes, prob.knn, 3 ** prob.dim
    nc = prob.num_cells
    faces = 0
    for a in range(d):
        nf = prob.n[a] if prob.bc_lo[a] == "P" else prob.n[a] + 1
        faces += nf * nc // prob.n[a]
    vb = prob.u_star.dtype.itemsize
    mixed = precision != "fp64"
    wbytes = 8                                   # FP64 weight, or FP32 hi + lo
    singular = all(b in ("P", "W", "I") for b in list(prob.bc_lo[:d]) + list(prob.bc_hi[:d]))
    tr = faces * (K * (4 + wbytes) + 8) + d * N * 8
    prep = d * N * (vb + 8)
    div = faces * 8 + nc * (8 + (4 if mixed else 0))
    sweeps = (refine if sweeps_done is None else sweeps_done) if precision == "mixed" else 0
    npass = 2 * d - 1
    xf = nc * npass * 8 * (1 + sweeps) * (1 if mixed else 2)
    # residuals: one per sweep, and with the stopping rule one more (the deciding one)
    res = (sweeps + (1 if adaptive and sweeps_done is not None else 0)) * nc * (8 + 8 + 4) if mixed else 0
    gauge = nc * ((8 + 16 + 8) if singular else 16) if mixed else (nc * 24 if singular else 0)
    grad = N * (Kg * (4 + d * wbytes) + d * vb * 3 + 1) + nc * 8
    return {"prep": prep, "transfer": tr, "divergence": div, "transform": xf, "residual": res,
            "gauge": gauge, "gradient": grad}


def transform_design_bytes(prob, precision, refine):
    """Bytes the transform passes of this design move per projection: FP32 passes read and write
    4 B per cell, the first reads the FP32 source, and the last pass of each solve writes the
    iterate as an FP32 pair (8 B; read and written, 16 B, when it accumulates in a sweep) and,
    in the last solve, p in FP64 (8 B). Reported beside the roofline, not used for it."""
    d, nc = prob.dim, prob.num_cells
    npass = 2 * d - 1
    if precision != "mixed" and precision != "fp32":
        return nc * (8 * (npass * 2 - 1) + 8)
    sweeps = refine if precision == "mixed" else 0
    first = 4 * (npass * 2 - 1) + 8
    return nc * (first + sweeps * (first + 8) + 8)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def transform_kernel_hash():
    """Hash of the transform kernels' device code (fft.cuh, axis_pass.cuh, lean_pass.cuh) with
    whole-line comments and blank lines left out, so host-only edits and comment edits keep a
    capture valid."""
    csrc = os.path.join(ROOT, "paper_2304_14690_gb300", "csrc")
    h = hashlib.sha1()
    for f in ("fft.cuh", "axis_pass.cuh", "lean_pass.cuh"):
        for line in open(os.path.join(csrc, f), encoding="utf-8"):
            t = line.strip()
            if t and not t.startswith("//"):
                h.update(t.encode())
                h.update(b"\n")
    return h.hexdigest()[:12]


def ncu_traffic(phase):
    """DRAM bytes per call of a phase from the committed ncu summary, or None when the summary
    is absent or was taken on other kernel sources (the transform sources are hashed)."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(phase)
        if not d:
            return None
        if transform_kernel_hash() != d.get("sources_sha1"):
            return None
        return d["dram_bytes_per_call"]
    except Exception:
        return None


# ----------------------------------------------------------------------------- ranks

def max_over_ranks(x, world, device=None):
    """The maximum of x over all ranks (x itself with one rank). Under NCCL the tensor lives on
    the rank's GPU; under gloo on the host."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, steps, total_ms, world):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


# ----------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    prob = workload()
    plan = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=local_rank)
    tune_ms = plan.autotune()          # transform schedule, chosen once per plan (untimed)
    u_dev = torch.as_tensor(prob.u_star, device=dev)
    outs = plan.alloc_outputs()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        plan.project(u_dev, out=outs)
    torch.cuda.synchronize(dev)

    # ---- device-timed region (the profiler is off: its event nodes would cut the programmatic
    # overlap at the phase boundaries; phases and the roofline come from a second timed region)
    steps = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(_smi_id(dev, local_rank))
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")   # the timed projections (ncu --nvtx-include timed/)
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        plan.project(u_dev, out=outs)
        evs[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    # ---- second timed region, same workload and L2 flush, with the per-phase CUDA events
    nprof = max(20, min(steps, 200))
    plan.profile(True)
    for _ in range(3):
        plan.project(u_dev, out=outs)
    plan.profile_read()
    torch.cuda.synchronize(dev)
    for k in range(nprof):
        flush.fill_(k & 0xFF)
        plan.project(u_dev, out=outs)
    torch.cuda.synchronize(dev)
    prof = plan.profile_read()
    plan.profile(False)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    cells = prob.num_cells
    value = job_value(cells, steps, total_ms, world)
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(0.99 * len(srt)))]

    # ---- roofline of the dominant phase (live CUDA events on the launching stream)
    calls = max(prof["calls"], 1)
    _, _, _, st0 = plan.project(u_dev, out=outs, stats=True)   # sweeps the stopping rule ran
    sweeps_done = st0["refine_iters_done"]
    adaptive = args.precision == "mixed" and args.refine_tol > 0 and args.refine > 0
    pb = phase_bytes(prob, args.precision, args.refine, sweeps_done, adaptive)
    phases = {k: v / calls for k, v in prof["phase_ms"].items() if v > 0}
    dom = max((k for k in phases if k in pb), key=lambda k: phases[k])
    peak, peak_src = measured_peaks()

    def roof(name):
        ms = phases[name]
        ach = pb[name] / (ms * 1e-3) / 1e9
        r = {"bound": "hbm", "phase": name, "achieved": round(ach, 1), "peak": peak,
             "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": ncu_traffic(name),
             "algorithmic_bytes": pb[name], "ms": round(ms, 5), "peak_source": peak_src}
        if name == "transform":
            r["bytes_rule"] = "(2 dim - 1) passes x 8 B per cell per solve, solves = 1 + sweeps"
            r["design_bytes"] = transform_design_bytes(prob, args.precision, sweeps_done)
            r["solves"] = 1 + (sweeps_done if args.precision == "mixed" else 0)
        return r

    roofline = roof(dom)
    roofline_transform = roof("transform") if "transform" in phases else None

    # ---- accuracy against the plain FP64 GPU path, and that path's own throughput
    acc = {}
    fp64 = None
    if rank == 0 and not args.no_extras:
        ref = pc.Plan(prob, precision="fp64", device=local_rank)
        ro = ref.alloc_outputs()
        ref.project(u_dev, out=ro)
        torch.cuda.synchronize(dev)

        def rel(a, b):
            return float(torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(b.double()))

        acc["rel_l2_p_vs_fp64_gpu"] = rel(outs[0], ro[0])
        acc["rel_l2_u_vs_fp64_gpu"] = rel(outs[1], ro[1])
        _, _, _, st = plan.project(u_dev, out=outs, stats=True)
        acc["max_div_after_rel"] = st["max_div_after"] * min(prob.h) / st["max_abs_u_star"]
        acc["residual_norms"] = st["residual_norm"]
        acc["refine_iters_done"] = st["refine_iters_done"]
        acc["refine_converged"] = st["refine_converged"]
        if args.precision == "mixed":
            p32 = pc.Plan(prob, precision="fp32", device=local_rank)
            o32 = p32.alloc_outputs()
            p32.project(u_dev, out=o32)
            acc["fp32_unrefined_rel_l2_p"] = rel(o32[0], ro[0])
            p32.close()
        # plain FP64 GPU path timed the same way
        n64 = max(20, min(200, steps // 5))
        e64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n64)]
        for _ in range(3):
            ref.project(u_dev, out=ro)
        for k in range(n64):
            flush.fill_(k & 0xFF)
            e64[k][0].record(stream)
            ref.project(u_dev, out=ro)
            e64[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ms64 = sum(a.elapsed_time(b) for a, b in e64) / n64
        fp64 = {"ms_per_step": round(ms64, 5), "value": cells / (ms64 * 1e-3),
                "speedup_of_this_path": round(ms64 / (total_ms / steps), 3)}
        ref.close()

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None if args.no_extras else run_e2e(plan, prob, stream, dev, steps, world)
    ib = None if args.no_extras else run_ib(plan, prob, u_dev, stream, dev, flush)
    variants = None if args.no_extras else run_variants(args, prob, u_dev, stream, dev, flush, ms_step=total_ms / steps)
    cufft = None if args.no_extras else {"shape": list(prob.n[:prob.dim]),
                                         "rfft_irfft_ms": round(cufft_reference(prob.n[:prob.dim], stream, dev, flush), 5),
                                         "this_fp32_solve_ms": round(tune_ms, 5)}

    batch = None
    if not args.no_batch:
        batch = run_batch(args, dev, stream, flush, world)
    box3d = None
    if not args.no_3d:
        box3d = run_3d(args, dev, stream, flush, world, rank)
    serve = None
    if rank == 0 and world == 1 and not args.no_serve_leg:
        serve = serving_leg(args, dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_subprocess(args.cpu_seconds)

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(total_ms / steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(prob.n), "nodes": prob.num_nodes,
                   "precision": args.precision, "refine_iters": args.refine, "refine_tol": args.refine_tol,
                   "knn": prob.knn, "l2": "256 MB buffer written between timed steps",
                   "headline": "the 1024x512 channel (the workload the metric is quoted on); the 512-problem "
                               "batch, where the scope table puts the transform-pass HBM target, is reported "
                               "with its own rooflines in batch_2d_512",
                   "transform_slots": plan.slots(), "transform_ctas_per_sm": plan.ctas(),
                   "tuned_solve_ms": round(tune_ms, 5),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "latency_ms": {"p50": round(p50, 5), "p99": round(p99, 5)},
        "roofline": roofline, "roofline_transform": roofline_transform,
        "phase_ms": {k: round(v, 5) for k, v in phases.items()},
        "accuracy": acc, "fp64_path": fp64, "e2e": e2e,
        "gpu_launches": int(prof["kernel_launches"] * steps / calls),
        "profiled_steps": {"steps": nprof, "ms_per_step": round(sum(prof["phase_ms"].values()) / calls, 5),
                           "note": "phase_ms and roofline come from this second timed region (per-phase events on)"},
        "clocks": clocks, "cpu_baseline": cpu, "wall_s": round(wall, 3),
        "ib_iteration": ib,
        "variants": variants,
        "cufft_reference": cufft,
        "batch_2d_512": batch,
        "box_sphere_3d": box3d,
        "serving": serve,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.close()


def run_e2e(plan, prob, stream, dev, steps, world):
    """The same projection through the public call with pinned HOST buffers: the H2D copy of u*
    and the D2H copies of p, u and f are inside the timed region."""
    import torch
    hu = torch.as_tensor(prob.u_star).pin_memory()
    ho = (torch.empty(plan.shape, dtype=torch.float64).pin_memory(),
          torch.empty((prob.dim, prob.num_nodes), dtype=plan.vdtype).pin_memory(),
          torch.empty((prob.dim, prob.num_nodes), dtype=plan.vdtype).pin_memory())
    ne = max(10, min(200, steps // 5))
    for _ in range(3):
        plan.project(hu, out=ho)
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ne)]
    torch.cuda.synchronize(dev)
    for k in range(ne):
        ee[k][0].record(stream)
        plan.project(hu, out=ho)          # H2D of u*, kernels, D2H of p, u, f inside the call
        ee[k][1].record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ee) / ne, world, dev)
    e2e = {"value": job_value(prob.num_cells, 1, e2e_ms, world), "unit": UNIT,
           "h2d_bytes_per_step": int(hu.numel() * hu.element_size()),
           "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in ho)),
           "ms_per_step": round(e2e_ms, 5)}
    return e2e


def run_ib(plan, prob, u_dev, stream, dev, flush, tol=1e-3, max_iters=50, reps=10):
    """One time step of the IB-force iteration (§2.3) at the paper's tolerance 1e-3, from zero
    force, through pc_project_ib: as one CUDA graph (while node, device-side stopping rule; the
    default) and driven from the host (graphs off; per-pass phases from the profiler), against
    the same number of full pc_project passes fed with the previous force."""
    import torch
    outs = plan.alloc_outputs()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for k in range(reps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev) / reps

    info = {}

    def step():
        info.update(plan.project_ib(u_dev, tol=tol, max_iters=max_iters, out=outs)[3])

    ms_graph = timed(step)
    its = info["iterations"]
    plan.graphs(False)
    plan.profile(True)
    ms_host = timed(step)
    prof = plan.profile_read()
    plan.profile(False)
    plan.graphs(True)
    fb = [plan.alloc_outputs() for _ in range(2)]

    def full():
        f = None
        for i in range(its):
            plan.project(u_dev, f, out=fb[i & 1])
            f = fb[i & 1][2]

    ms_full = timed(full)
    passes = max(prof["calls"], 1)
    return {"tol": tol, "iterations": its, "converged": info["converged"],
            "ib_nodes": int((prob.node_type != 0).sum()),
            "ms_per_time_step": round(ms_graph, 4), "ms_per_pass": round(ms_graph / its, 5),
            "host_loop_ms_per_time_step": round(ms_host, 4),
            "host_loop_pass_phase_ms": {k: round(v / passes, 5) for k, v in prof["phase_ms"].items() if v > 0},
            "full_passes_ms": round(ms_full, 4), "speedup_vs_full_passes": round(ms_full / ms_graph, 3),
            "cells_per_s_per_time_step": round(prob.num_cells / (ms_graph * 1e-3), 1),
            "history_last": info["history"][-1]}


def cufft_reference(shape, stream, dev, flush, reps=50):
    """cuFFT (through torch.fft) on the pressure grid's shape: one forward real-to-complex and one
    inverse transform of an FP32 array, the transform work of one FP32 solve (reference point
    only; the library does not use it)."""
    import torch
    x = torch.randn(tuple(int(v) for v in shape), dtype=torch.float32, device=dev)
    for _ in range(3):
        torch.fft.irfftn(torch.fft.rfftn(x), s=x.shape)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        torch.fft.irfftn(torch.fft.rfftn(x), s=x.shape)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    return sum(a.elapsed_time(b) for a, b in ev) / reps


def run_variants(args, prob, u_dev, stream, dev, flush, ms_step, reps=50):
    """The solve variants of the paper on the same workload, each timed per projection like the
    main step: pseudo-spectral eigenvalues (FP64 plan, against the FD FP64 plan), the direct WLS
    divergence at the cell centres (mixed; with the roofline of its gather kernel), and the RHS
    mask (mixed; the cells inside the cylinder masked out)."""
    import numpy as np
    import torch
    from paper_2304_14690_gb300 import pc

    def timed(plan, tag=None):
        outs = plan.alloc_outputs()
        for _ in range(3):
            plan.project(u_dev, out=outs)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        if tag:
            torch.cuda.nvtx.range_push(tag)   # ncu --nvtx-include <tag>/
        for k in range(reps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            plan.project(u_dev, out=outs)
            ev[k][1].record(stream)
        if tag:
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        plan.profile(True)                  # phases from a second run, per-phase events on
        for k in range(reps):
            flush.fill_(k & 0xFF)
            plan.project(u_dev, out=outs)
        torch.cuda.synchronize(dev)
        prof = plan.profile_read()
        plan.profile(False)
        calls = max(prof["calls"], 1)
        return (sum(a.elapsed_time(b) for a, b in ev) / reps,
                {k: v / calls for k, v in prof["phase_ms"].items() if v > 0})

    out = {}
    fd = pc.Plan(prob, precision="fp64", device=dev.index)
    ms_fd, _ = timed(fd)
    fd.close()
    sp = pc.Plan(prob, precision="fp64", device=dev.index, eigenvalues="spectral")
    ms_sp, _ = timed(sp)
    sp.close()
    out["spectral_fp64"] = {"ms_per_step": round(ms_sp, 5), "fd_fp64_ms_per_step": round(ms_fd, 5)}
    di = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index, div_mode="wls_direct")
    di.autotune()
    ms_di, ph = timed(di)
    di.close()
    d, N, K, nc = prob.dim, prob.num_nodes, prob.knn, prob.num_cells
    div_bytes = nc * K * (4 + d * 8) + d * N * 8 + nc * (8 + 4)
    peak, peak_src = measured_peaks()
    ach = div_bytes / (ph["divergence"] * 1e-3) / 1e9
    out["wls_direct_divergence"] = {
        "ms_per_step": round(ms_di, 5), "faces_ms_per_step": round(ms_step, 5),
        "value": round(nc / (ms_di * 1e-3), 1), "unit": UNIT,
        "phase_ms": {k: round(v, 5) for k, v in ph.items()},
        "roofline_divergence": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                                "frac": round(ach / peak, 4), "algorithmic_bytes": div_bytes,
                                "peak_source": peak_src}}
    mk = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index)
    mk.autotune()
    g = prob.n
    xc = prob.lo[0] + (np.arange(g[0]) + 0.5) * prob.h[0]
    yc = prob.lo[1] + (np.arange(g[1]) + 0.5) * prob.h[1]
    X, Y = np.meshgrid(xc, yc, indexing="ij")
    inside = np.zeros(X.shape, dtype=bool)
    for o in getattr(prob, "obstacles", None) or []:
        inside |= (X - o[1][0]) ** 2 + (Y - o[1][1]) ** 2 < o[2] ** 2
    mk.set_rhs_mask((~inside).astype(np.uint8))
    ms_mk, _ = timed(mk)
    mk.close()
    out["rhs_mask"] = {"ms_per_step": round(ms_mk, 5), "masked_cells": int(inside.sum())}

    def timed_solve(plan):
        gen = torch.Generator(device=dev).manual_seed(5)
        src = torch.randn(plan.shape, dtype=torch.float64, device=dev, generator=gen)
        dst = torch.empty_like(src)
        for _ in range(3):
            plan.solve_poisson(src, dst)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for k in range(reps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            plan.solve_poisson(src, dst, stream=stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev) / reps

    # the regular (vertex) grid: the 400x400 periodic grid of the cylinder results, and an all-wall
    # 512x512 vertex grid (513^2 unknowns, DCT-I along both axes), each against the cell-centred
    # solve of the same cells
    vert = {}
    for tag, n, lo, hi in (("periodic_400x400", (400, 400), ("P", "P"), ("P", "P")),
                           ("walls_512x512", (512, 512), ("W", "W"), ("W", "W"))):
        hh = (1.0 / n[0], 1.0 / n[1])
        row = {}
        for gt in ("vertices", "cells"):
            gp = pc.GridPlan(2, n, hh, lo, hi, grid_type=gt, precision=args.precision,
                             refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index)
            gp.autotune()
            row[gt + "_ms"] = round(timed_solve(gp), 5)
            if gt == "vertices":
                row["unknowns"] = int(np.prod(gp.shape))
            gp.close()
        vert[tag] = row
    out["vertex_grid_solve"] = vert
    # the whole pass on the vertex grid of the same workload (direct divergence at the vertex
    # unknowns; quarter-wave transforms along the I-D axis, DCT-I along the wall pair)
    vp = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index,
                 div_mode="wls_direct", grid_type="vertices")
    vp.autotune()
    ms_vp, ph_vp = timed(vp, "vertex")
    out["vertex_grid_project"] = {"ms_per_step": round(ms_vp, 5), "unknowns": int(np.prod(vp.shape)),
                                  "phase_ms": {k: round(v, 5) for k, v in ph_vp.items()}}
    vp.close()
    out["time_step"] = run_time_step(args, prob, u_dev, stream, dev, flush, reps)
    return out


def run_time_step(args, prob, u_dev, stream, dev, flush, reps):
    """Full time steps on the same workload: the AB2 predictor of Eq. 3 on the nodes (nu = 0.01,
    K = 12) followed by one pressure correction, both on the device; the predictor alone with
    its roofline (algorithmic bytes per node 4K + 8(d+1)K + 48d: columns, weights, own velocity,
    the stored R and u* read and written, u* written)."""
    import torch
    from paper_2304_14690_gb300 import pc
    plan = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index)
    plan.autotune()
    mom = pc.Momentum(plan, nu=0.01)
    outs = [plan.alloc_outputs() for _ in range(2)]
    us = torch.empty_like(u_dev)
    # a stable step for the explicit predictor: advective CFL 0.2 and diffusion number 0.1 on
    # the smallest node spacing (the rings around the cylinder are finer than the grid)
    try:
        from scipy.spatial import cKDTree
        sp = float(cKDTree(prob.nodes.T).query(prob.nodes.T, k=2)[0][:, 1].min())
    except ImportError:
        sp = 0.25 * min(prob.h[: prob.dim])
    umax = max(float(torch.abs(u_dev).max()), 1e-30)
    dt = min(0.2 * sp / umax, 0.1 * sp * sp / 0.01)
    u = u_dev.clone()
    for k in range(3):
        mom.predict(u, dt, out=us)
        plan.project(us, dt=dt, out=outs[k % 2])
        u = outs[k % 2][1]
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        mom.predict(u, dt, out=us, stream=stream)
        ev[k][1].record(stream)
        plan.project(us, dt=dt, out=outs[k % 2], stream=stream)
        ev[k][2].record(stream)
        u = outs[k % 2][1]
    torch.cuda.synchronize(dev)
    ms_pred = sum(a.elapsed_time(b) for a, b, _ in ev) / reps
    ms_step = sum(a.elapsed_time(c) for a, _, c in ev) / reps
    d, N, K = prob.dim, prob.num_nodes, 12
    nbytes = N * (4 * K + 8 * (d + 1) * K + 48 * d)
    peak, peak_src = measured_peaks()
    ach = nbytes / (ms_pred * 1e-3) / 1e9
    finite = bool(torch.isfinite(u).all())
    mom.close()
    plan.close()
    return {"ms_per_step": round(ms_step, 5), "predictor_ms": round(ms_pred, 5), "nu": 0.01, "dt": dt,
            "min_node_spacing": sp, "finite": finite,
            "roofline_predictor": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                                   "frac": round(ach / peak, 4), "algorithmic_bytes": nbytes,
                                   "peak_source": peak_src}}


def run_3d(args, dev, stream, flush, world, rank):
    """The 3D box with a sphere, 256x128x128 cells, ~4.3e6 nodes, K = 27, FP32 u*: mixed
    precision (autotuned schedule) against the plain FP64 path, both timed per projection."""
    import torch
    from paper_2304_14690_gb300 import pc, workloads as wl
    t0 = time.perf_counter()
    prob = wl.box_sphere()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    plan = pc.Plan(prob, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index)
    tune_ms = plan.autotune()
    setup_s = time.perf_counter() - t0
    u = torch.as_tensor(prob.u_star, device=dev)
    outs = plan.alloc_outputs()

    def timed(pl, out, k):
        for _ in range(3):
            pl.project(u, out=out)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            pl.project(u, out=out)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        t = sorted(a.elapsed_time(b) for a, b in ev)
        return sum(t) / k, t[len(t) // 2], t[min(k - 1, int(0.99 * k))]

    k = args.steps_3d
    ms, p50, p99 = timed(plan, outs, k)
    ms = max_over_ranks(ms, world, dev)
    plan.profile(True)                      # phases from a second run, per-phase events on
    timed(plan, outs, max(5, k // 2))
    prof = plan.profile_read()
    plan.profile(False)
    calls = max(prof["calls"], 1)
    out = {"workload": "box_sphere 256x128x128 cells, walls on all faces (DCT-II x3, zero mode), sphere D=1, "
                       "K=27, FP32 u*", "cells": prob.num_cells, "nodes": prob.num_nodes,
           "steps": k, "ms_per_step": round(ms, 4), "value": round(job_value(prob.num_cells, 1, ms, world), 1),
           "unit": UNIT, "latency_ms": {"p50": round(p50, 4), "p99": round(p99, 4)},
           "phase_ms": {kk: round(v / calls, 5) for kk, v in prof["phase_ms"].items() if v > 0},
           "transform_slots": plan.slots(), "tuned_solve_ms": round(tune_ms, 4),
           "generate_s": round(gen_s, 1), "plan_and_tune_s": round(setup_s, 1),
           "cufft_rfft_irfft_ms": round(cufft_reference(prob.n[:3], stream, dev, flush), 4)}
    # roofline of the transform phase by the scope table's bytes (40 B per cell per solve in 3D)
    _, _, _, st0 = plan.project(u, out=outs, stats=True)
    sweeps_done = st0["refine_iters_done"]
    adaptive = args.precision == "mixed" and args.refine_tol > 0 and args.refine > 0
    pb = phase_bytes(prob, args.precision, args.refine, sweeps_done, adaptive)
    peak, peak_src = measured_peaks()
    xf_ms = out["phase_ms"].get("transform", 0.0)
    if xf_ms > 0:
        ach = pb["transform"] / (xf_ms * 1e-3) / 1e9
        out["roofline_transform"] = {
            "bound": "hbm", "phase": "transform", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "algorithmic_bytes": pb["transform"], "ms": xf_ms,
            "solves": 1 + sweeps_done, "bytes_rule": "(2 dim - 1) passes x 8 B per cell per solve, solves = 1 + sweeps",
            "peak_source": peak_src}
    if rank == 0 and not args.no_extras:
        ref = pc.Plan(prob, precision="fp64", device=dev.index)
        ro = ref.alloc_outputs()
        ms64, _, _ = timed(ref, ro, max(5, k // 2))
        plan.project(u, out=outs)
        _, _, _, st = plan.project(u, out=outs, stats=True)
        torch.cuda.synchronize(dev)

        def rel(a, b):
            return float(torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(b.double()))

        out["accuracy"] = {"rel_l2_p_vs_fp64_gpu": rel(outs[0], ro[0]), "rel_l2_u_vs_fp64_gpu": rel(outs[1], ro[1]),
                           "max_div_after_rel": st["max_div_after"] * min(prob.h) / st["max_abs_u_star"],
                           "residual_norms": st["residual_norm"], "refine_iters_done": st["refine_iters_done"],
                           "refine_converged": st["refine_converged"]}
        out["fp64_path"] = {"ms_per_step": round(ms64, 4), "speedup_of_this_path": round(ms64 / ms, 3)}
        ref.close()
    plan.close()
    return out


def run_batch(args, dev, stream, flush, world):
    """512 independent 2D projections of mixed sizes (64..512 cells per side), boundary pairs and
    obstacles through pc_project_batch: one launch per pipeline stage for the whole batch."""
    import torch
    from paper_2304_14690_gb300 import pc, workloads as wl
    t0 = time.perf_counter()
    probs = wl.batch_2d(count=args.batch_problems)
    plans, bargs = [], []
    for pr in probs:
        plan = pc.Plan(pr, precision=args.precision, refine_iters=args.refine, refine_tol=args.refine_tol, device=dev.index)
        u = torch.as_tensor(pr.u_star, device=dev)
        p, uo, fo = plan.alloc_outputs()
        plans.append(plan)
        bargs.append(dict(dt=pr.dt, u_star=u, p=p, u=uo, f=fo))
    setup_s = time.perf_counter() - t0
    for _ in range(3):
        pc.project_batch(plans, bargs)
    torch.cuda.synchronize(dev)
    k = args.batch_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    torch.cuda.nvtx.range_push("batch")   # the timed batches (ncu --nvtx-include batch/)
    for i in range(k):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        pc.project_batch(plans, bargs)
        evs[i][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / k, world, dev)
    cells = sum(pr.num_cells for pr in probs)
    out = {"problems": len(probs), "cells": cells, "nodes": sum(pr.num_nodes for pr in probs),
           "ms_per_batch": round(ms, 4), "value": round(job_value(cells, 1, ms, world), 1), "unit": UNIT,
           "steps": k, "setup_s": round(setup_s, 1),
           "workload": "512 2D problems, n0,n1 in {64..512}, h=1/64, P-P / P-wall / wall-wall, 0-2 circles"}
    # phases of the batch: a second timed region whose stages record their boundaries into the
    # first plan's profiler (direct launches, same kernels); roofline of the transform passes by
    # the scope table's bytes, and of the whole batch by every phase's algorithmic bytes
    plans[0].profile(True)
    pc.project_batch(plans, bargs)
    plans[0].profile_read()
    for i in range(k):
        flush.fill_(i & 0xFF)
        pc.project_batch(plans, bargs)
    torch.cuda.synchronize(dev)
    prof = plans[0].profile_read()
    plans[0].profile(False)
    calls = max(prof["calls"], 1)
    phases = {kk: v / calls for kk, v in prof["phase_ms"].items() if v > 0}
    adaptive = args.precision == "mixed" and args.refine_tol > 0 and args.refine > 0
    done = []
    for pl, pr in zip(plans, probs):   # sweeps each problem's stopping rule ran (one stats call each)
        _, _, _, st = pl.project(torch.as_tensor(pr.u_star, device=dev), stats=True)
        done.append(st["refine_iters_done"])
    out["sweeps_done"] = {str(k): done.count(k) for k in sorted(set(done))}
    pbs = [phase_bytes(pr, args.precision, args.refine, d, adaptive) for pr, d in zip(probs, done)]
    tot = {kk: sum(b[kk] for b in pbs) for kk in pbs[0]}
    peak, peak_src = measured_peaks()
    xf_ms = phases.get("transform", 0.0)
    if xf_ms > 0:
        ach = tot["transform"] / (xf_ms * 1e-3) / 1e9
        out["roofline_transform"] = {
            "bound": "hbm", "phase": "transform", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "algorithmic_bytes": tot["transform"], "ms": round(xf_ms, 4),
            "bytes_rule": "(2 dim - 1) passes x 8 B per cell per solve, solves = 1 + sweeps",
            "design_bytes": sum(transform_design_bytes(pr, args.precision, d) for pr, d in zip(probs, done)),
            "peak_source": peak_src}
    step_bytes = sum(tot.values())
    ach = step_bytes / (ms * 1e-3) / 1e9
    out["roofline_step"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(ach / peak, 4), "algorithmic_bytes": step_bytes, "ms": round(ms, 4),
                            "peak_source": peak_src}
    out["phase_ms"] = {kk: round(v, 4) for kk, v in phases.items()}
    out["profiled_ms_per_batch"] = round(sum(phases.values()), 4)
    for pl in plans:
        pl.close()
    return out


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank):
    """The oracle as it stands, on this arm's workload and metric. A step is one full projection;
    the run is bounded to about 90 s of projections after the (untimed) plan build, so it takes
    min(steps, what fits) steps and says how many in cpu_baseline.sample."""
    if rank != 0:
        return
    val, info = oracle_timing(args.steps, min(args.warmup, 1), seconds=90.0, max_steps=args.steps)
    out = {
        "impl": "reference", "metric": METRIC, "value": round(val, 1), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(info["ms_per_projection"], 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "knn": 12},
        "cpu_baseline": {"value": round(val, 1), "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                         "sample": f"{info['projections']} full projections of the workload "
                                   f"(plan built first, {info['plan_seconds']:.1f} s, untimed)"},
        "e2e": {"value": round(val, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def serving_leg(args, dev):
    """A bounded serving run inside the default bench: the first serve_leg_pool geometries of
    the config-5 pool, serve_leg_requests Poisson arrivals at the configured 2000/s and at two
    lower rates, continuous batching with backpressure (bounded queue) and a deadline. Reports
    p50/p99 per rate, the highest rate served without shedding, and the accuracy of a sample of
    served results against plain FP64 projections of the same requests."""
    import torch
    from paper_2304_14690_gb300 import pc, serving, workloads as wl
    t0 = time.perf_counter()
    pool = wl.serving_pool(count=args.serve_pool)[: args.serve_leg_pool]
    gen_s = time.perf_counter() - t0
    budget = int(args.serve_budget_gb * (1 << 30))
    rates = [args.serve_rate, 0.75 * args.serve_rate, 0.5 * args.serve_rate]
    k = args.serve_leg_requests
    sample = set(range(0, k, max(1, k // 8)))
    srv = serving.Server(pool, budget_bytes=budget, precision=args.precision, refine=args.refine,
                         refine_tol=args.refine_tol, max_queue=args.serve_max_queue, deadline_s=args.serve_deadline,
                         keep_outputs=sample, device=dev.index)
    t1 = time.perf_counter()
    srv.warm(range(len(pool)))
    warm_s = time.perf_counter() - t1
    legs = []
    acc = None
    for ri, rate in enumerate(rates):
        trace = wl.serving_trace(count=k, rate=rate, pool_size=len(pool), seed=14696 + ri)
        srv.outputs = {}
        reqs = srv.run(trace)
        summ = serving.summarize(reqs, pool)
        summ.update(rate=rate, batches=srv.batches, mean_batch=round(summ["served"] / max(srv.batches, 1), 2))
        legs.append(summ)
        if acc is None:
            # sampled served requests against the plain FP64 projection of the same u*
            errs_p, errs_u = [], []
            for r in reqs:
                if r.shed or r.rid not in srv.outputs:
                    continue
                prob = pool[r.geometry]
                ref = pc.Plan(prob, precision="fp64", device=dev.index)
                u = torch.mul(torch.as_tensor(prob.u_star, device=dev), r.scale)
                p64, u64, _, _ = ref.project(u)
                got = srv.outputs[r.rid]
                errs_p.append(float(torch.linalg.vector_norm(got[0].to(dev) - p64) / torch.linalg.vector_norm(p64)))
                errs_u.append(float(torch.linalg.vector_norm(got[1].to(dev) - u64) / torch.linalg.vector_norm(u64)))
                ref.close()
            acc = {"sampled": len(errs_p), "max_rel_l2_p_vs_fp64_gpu": max(errs_p) if errs_p else None,
                   "max_rel_l2_u_vs_fp64_gpu": max(errs_u) if errs_u else None}
    srv.close()
    unshed = [lg["rate"] for lg in legs if lg["shed"]["queue"] + lg["shed"]["deadline"] == 0]
    n2 = sum(1 for p in pool if p.dim == 2)
    return {"workload": f"Poisson arrivals, {k} requests per rate, pool of the first {len(pool)} config-5 "
                        f"geometries ({n2} 2D, {len(pool) - n2} 3D), continuous batching, queue bound "
                        f"{args.serve_max_queue}, deadline {args.serve_deadline} s",
            "legs": legs, "highest_rate_without_shedding": max(unshed) if unshed else None,
            "accuracy": acc, "pool_generate_s": round(gen_s, 1), "warm_s": round(warm_s, 1)}


def run_serve(args, rank):
    """Config 5: a seeded Poisson-arrival stream of projection requests over a pool of 2D and 3D
    geometries, served with continuous batching under an HBM budget (mixed precision), and a
    prefix of the same trace served one request at a time by plain FP64 projections."""
    import torch
    from paper_2304_14690_gb300 import serving, workloads as wl
    if rank != 0:
        return
    t0 = time.perf_counter()
    pool = wl.serving_pool(count=args.serve_pool)
    gen_s = time.perf_counter() - t0
    trace = wl.serving_trace(count=args.serve_requests, rate=args.serve_rate, pool_size=len(pool))
    budget = int(args.serve_budget_gb * (1 << 30))

    def serve(tr, **kw):
        srv = serving.Server(pool, budget_bytes=budget, **kw)
        t = time.perf_counter()
        warm = srv.warm(range(len(pool))) if not args.serve_cold else 0
        warm_s = time.perf_counter() - t
        builds0 = srv.cache.builds
        reqs = srv.run(tr)
        out = serving.summarize(reqs, pool)
        out.update(batches=srv.batches, mean_batch=round(len(reqs) / max(srv.batches, 1), 2),
                   plan_builds=srv.cache.builds - builds0, evictions=srv.cache.evictions,
                   warm_plans=warm, warm_s=round(warm_s, 1), host_launch_s=round(srv.host_s, 3),
                   gpu_batch_s=round(srv.gpu_s, 3))
        srv.close()
        torch.cuda.synchronize()
        return out

    main = serve(trace, precision=args.precision, refine=args.refine, refine_tol=args.refine_tol)
    k = min(args.serve_fp64_requests, len(trace))
    prefix_mixed = serve(trace[:k], precision=args.precision, refine=args.refine, refine_tol=args.refine_tol)
    prefix_fp64 = serve(trace[:k], precision="fp64", batched=False, max_inflight=1)
    n2 = sum(1 for p in pool if p.dim == 2)
    out = {"metric": "served grid-points/s and p50/p99 latency (continuous batching)",
           "value": round(main["value"], 1), "unit": UNIT, "n_gpus": 1, "mode": "serve",
           "higher_is_better": True, "dtype": "f32" if args.precision != "fp64" else "f64",
           "data": "synthetic",
           "config": {"workload": f"Poisson arrivals {args.serve_rate:g}/s, {len(trace)} requests, pool of "
                                  f"{len(pool)} geometries ({n2} 2D n^2, n in 128..1024; {len(pool) - n2} 3D n^3, "
                                  f"n in 64..192), one obstacle each", "budget_gb": args.serve_budget_gb,
                      "precision": args.precision, "refine_iters": args.refine, "pool_generate_s": round(gen_s, 1)},
           "served": main, "prefix": {"requests": k, "mixed_batched": prefix_mixed,
                                      "fp64_one_at_a_time": prefix_fp64}}
    print(json.dumps(out), flush=True)


def _blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(k):
            try:
                return int(os.environ[k])
            except ValueError:
                pass
    return os.cpu_count()


def main():
    args = parse()
    if args.cpu_baseline_only:
        val, info = oracle_timing(0, 1, seconds=args.cpu_seconds)
        print(json.dumps({"value": round(val, 1), "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                          "sample": f"{info['projections']} full projections of the 1024x512 channel workload "
                                    f"({info['seconds']:.1f} s; plan built first in {info['plan_seconds']:.1f} s, "
                                    f"untimed), single thread"}))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.serve:
        import __graft_entry__
        __graft_entry__.build()
        run_serve(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
