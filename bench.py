#!/usr/bin/env python
"""Benchmark of the GMRES(3)-smoothed CSG multigrid preconditioner inside the FP64
flexible GMRES solve (arXiv:1012.5379), on GB300.

Metric: V-cycle Mpts/s = fine-grid unknowns x V-cycles / second over whole solves to
relative residual 1e-6 (one V-cycle per outer iteration).  A step is one pass of the
whole hot path over one batch of synthetic input: the full FGMRES(40) solve of the 3D
255^3 heterogeneous problem (unit cube, k(x) = 80 (1 + 0.3 g(x)) with 8 seeded Gaussian
bumps, point source, theta_beta 0.4, ECS layers 1/8 at 0.5 rad; complex64 V(1,1)
GMRES(3) V-cycle, outer FGMRES with the library's default arithmetic: double-float Krylov
basis, binary64 least squares and true residual), the largest single-GPU workload.  Extra keys of the same
line: the 2D 1023^2 theta_beta sweep (four solves batched), the 64-problem batch in
solves/s, and a short Poisson serving run with p50/p99 latency.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (each rank solves its own copy of the step; the only
collectives are a barrier and the max-over-ranks time).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import platform  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1012_5379_gb300 import inputs as I  # noqa: E402

METRIC = "V-cycle Mpts/s"
UNIT = "Mpts/s"
TOL = 1e-6
CUBE_N = 255
N = 1023          # the 2D theta_beta sweep (extra key)
K = 160.0
BETAS = I.LARGE_2D_BETAS
# FP64 peak: ncu's sustained DFMA peak on GB300 is 2 per SM per cycle (304 per cycle on 152
# SMs), x 2 flop x 2.07 GHz = 1.26 TFLOP/s, the recipe's nominal 1.25 TFLOP/s
FP64_PEAK_TFLOPS = 1.25
FP64_CLASSES = ("out.dots", "out.vnew", "out.apply_h")


def workload_config():
    return {"workload": "3D Helmholtz 255^3 interior on the unit cube, heterogeneous k(x)=80(1+0.3 g(x)) with g a "
                        "seeded sum of 8 Gaussian bumps (sigma 0.1, seed 1002) clipped to [-1,1], unit point source "
                        "at the centre, ECS layers 1/8 per face at 0.5 rad, CSG theta_beta 0.4; V(1,1) GMRES(3) "
                        "multigrid in complex64 down to 3^3, FGMRES(40) to rel. residual 1e-6 (the library's default "
                        "outer arithmetic on this grid: double-float Krylov basis and orthogonalisation, binary64 "
                        "Hessenberg, solution and true residual); one step = one full solve",
            "n": CUBE_N, "dim": 3, "k": "80(1+0.3g(x))", "theta_beta": 0.4, "tol": TOL, "restart": 40, "levels": 7,
            "l2": "inputs larger than L2: every level-0 vector is 134 MB and the FGMRES(40) basis 10.6 GB, "
                  "so no step reuses the previous step's data from the 126 MB L2"}


# Arm cores name themselves by implementer and part number in /proc/cpuinfo
ARM_PARTS = {("0x41", "0xd4f"): "Arm Neoverse V2", ("0x41", "0xd40"): "Arm Neoverse V1",
             ("0x41", "0xd0c"): "Arm Neoverse N1", ("0x41", "0xd49"): "Arm Neoverse N2"}


def host_info():
    cpu = platform.processor() or platform.machine()
    impl = part = None
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith(("model name", "cpu model")):
                cpu = line.split(":", 1)[1].strip()
                break
            if low.startswith("cpu implementer") and impl is None:
                impl = line.split(":", 1)[1].strip().lower()
            if low.startswith("cpu part") and part is None:
                part = line.split(":", 1)[1].strip().lower()
    except OSError:
        pass
    if impl and part:
        cpu = ARM_PARTS.get((impl, part), f"Arm implementer {impl} part {part}")
    return {"nproc": os.cpu_count(), "cpu": cpu, "machine": platform.machine()}


# ------------------------------------------------------------------ helpers
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        loaded = [v for v in sm if v > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel_class: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch: the ratio of ncu-measured DRAM bytes to algorithmic bytes
    of a captured launch of this kernel class (profiles/traffic.json), applied to the
    live launch's algorithmic bytes.  Null when the kernel sources changed since the
    capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_class)
    except Exception:
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec["dram_bytes"] / rec["algorithmic_bytes"] * alg_bytes_per_launch


def reduce_over_ranks(seconds, work, device):
    """Whole-job figures of a multi-rank run: the slowest rank's time and the work of
    all ranks (weak scaling: every rank solves its own replica of the step)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds, 0.0], dtype=torch.float64, device=device)
    w = torch.tensor([work, 0.0], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(w[0].item())


def vcycle_hbm(classes, peak_gbs):
    """Algorithmic bandwidth of the V-cycle kernel classes (vc.*): the library's
    algorithmic bytes of each class over its CUDA-event time, and their total, as a
    fraction of the measured HBM copy bandwidth.  Levels whose vectors fit in L2
    (129 MB; every level of a 1023^2 problem) can read above it."""
    out, tb, tms = {}, 0.0, 0.0
    for c, v in sorted(classes.items()):
        if not c.startswith("vc.") or v["ms"] <= 0 or v["bytes"] <= 0:
            continue
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        out[c] = {"GB/s": round(gbs, 1), "frac": round(gbs / peak_gbs, 3)}
        tb += v["bytes"]
        tms += v["ms"]
    if tms <= 0:
        return None
    gbs = tb / (tms * 1e-3) / 1e9
    return {"achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs, "classes": out}


# ------------------------------------------------------------------ our arm
def roofline_of(dominant, d, pk, fp64_outer=True):
    """Roofline object of one kernel class: the outer classes in binary64 against the
    DFMA pipe (their bound on GB300), the rest, and the outer classes of a double-float
    basis (FP32 pipe, bound by HBM), against the measured HBM copy bandwidth."""
    nl = max(d["launches"], 1)
    if fp64_outer and dominant in FP64_CLASSES and d["flops"] > 0:
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_for(dominant, d["bytes"] / nl),
                "kernel": dominant,
                "peak_source": "FP64 DFMA pipe: 2 DFMA/SM/cycle (ncu peak_sustained) x 152 SMs x 2.07 GHz "
                               "(= recipe nominal 1.25 TFLOP/s; MEASURED_PEAKS.json has no FP64 figure)",
                "launches": d["launches"], "avg_launch_us": 1e3 * d["ms"] / nl,
                "algorithmic_flops_per_launch": d["flops"] / nl, "algorithmic_bytes_per_launch": d["bytes"] / nl}
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    peak = pk.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_for(dominant, d["bytes"] / nl), "kernel": dominant,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in pk else "recipe fallback",
            "launches": d["launches"], "avg_launch_us": 1e3 * d["ms"] / nl,
            "algorithmic_bytes_per_launch": d["bytes"] / nl}


def class_shares(classes):
    tot = sum(v["ms"] for v in classes.values()) or 1.0
    return {c: round(v["ms"] / tot, 4) for c, v in sorted(classes.items(), key=lambda kv: -kv[1]["ms"])}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1012_5379_gb300 import helm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    w = I.cube_3d(CUBE_N)
    pts = float(w.n) ** 3
    b = torch.from_numpy(w.b).to(dev)
    phi = torch.from_numpy(w.phi).to(dev)
    h = helm.Handle(3, w.n, w.theta_beta, phi=phi, precision="c64", restart=w.restart, maxit=400)
    x = torch.zeros_like(b)

    basis = []

    def step():
        x.zero_()
        info = h.solve(b, x, w.tol)
        if info.status != 0:
            raise RuntimeError(f"solve did not converge: {info}")
        basis.append(info.basis)
        return info.iters

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up; the second warm-up step times every kernel class with CUDA events around
    # each launch: one problem on one stream, so the classes' times are serialised (in
    # the first solve of the process the level-0 V-cycle passes took about 1.5 times
    # their steady time)
    classes = {}
    prof_step = min(1, args.warmup - 1)
    for i in range(args.warmup):
        if i == prof_step:
            helm.profile_begin("")
        step()
        if i == prof_step:
            classes = helm.profile_end()
    dominant = max(classes, key=lambda c: classes[c]["ms"]) if classes else "out.dots"

    # timed region: per-step CUDA events on the solve's stream; events bracket only the
    # dominant class's launches (a few dozen per solve) for its live roofline
    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = helm.launch_count()
    helm.profile_begin(dominant)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    all_iters = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        all_iters.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    prof = helm.profile_end()
    launches = helm.launch_count() - launches0
    clocks = sampler.stop()
    ms_steps = [a.elapsed_time(c) for a, c in ev]
    ms_total = float(sum(ms_steps))
    work = pts * sum(all_iters)
    if world > 1:
        ms_total, work = reduce_over_ranks(ms_total, work, dev)
    value = work / (ms_total * 1e-3) / 1e6
    pk = peaks()
    roof = roofline_of(dominant, prof.get(dominant, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}), pk,
                       fp64_outer=basis[-1] == "f64")
    roof["selected_by"] = ("largest serialised class time in the second warm-up solve (CUDA events around every "
                           "launch, one stream); achieved from events around this class's launches in the timed "
                           "steps")

    # end to end through the public API with host buffers: helm_solve_host copies b to
    # the device, solves and copies x back (pinned host memory)
    e2e = None
    if args.e2e_steps > 0:
        bh = torch.empty(b.shape, dtype=torch.complex128, pin_memory=True)
        bh.copy_(torch.from_numpy(w.b))
        xh = torch.empty_like(bh, pin_memory=True)
        bh_np, xh_np = bh.numpy(), xh.numpy()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ework = 0.0
        for _ in range(args.e2e_steps):
            info = h.solve_host(bh_np, xh_np, w.tol)
            ework += pts * info.iters
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        if world > 1:
            et, ework = reduce_over_ranks(et, ework, dev)
        e2e = {"value": ework / et / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(pts * 16),
               "d2h_bytes_per_step": int(pts * 16), "steps": args.e2e_steps, "api": "helm_solve_host"}
    iters = all_iters[-1]
    h.close()
    del h, b, x, phi
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+df+f64" if basis[-1] == "df" else "c64+f64",
            "data": "synthetic", "outer_basis": basis[-1],
            "config": workload_config(), "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "iters": iters, "solves_per_s": args.steps * world / (ms_total * 1e-3),
            "ms_steps": ms_steps,
            "kernel_classes_warmup": classes, "kernel_class_shares_warmup": class_shares(classes),
            "vcycle_hbm": vcycle_hbm(classes, pk.get("hbm_gbs", 6800.0))}
    if line["vcycle_hbm"]:
        line["vcycle_hbm"]["note"] = ("V-cycle classes of the second warm-up solve (serialised, one stream), "
                                      "algorithmic bytes over CUDA-event time")
    if world == 1 and not args.no_extras:
        line["sweep_2d"] = sweep_2d(args, dev)
        line["batch_64"] = batch_extra(args)
        line["serving"] = serving_extra(args)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    else:
        line["cpu_baseline"] = None
    return line


def sweep_2d(args, dev):
    """The 2D 1023^2 workload (k = 160, unit-variance complex normal source, theta_beta
    0.1 / 0.2 / 0.3 / 0.5 solved together with helm_batch_solve, complex64 V-cycle, FP64
    FGMRES without restart to 1e-6): V-cycle Mpts/s over whole solves."""
    import torch

    from paper_1012_5379_gb300 import helm
    b = torch.from_numpy(I.random_source(2, N, 1001)).to(dev)
    handles = [helm.Handle(2, N, tb, k=K, precision="c64", maxit=300) for tb in BETAS]
    xs = [torch.zeros_like(b) for _ in BETAS]

    def step():
        for x in xs:
            x.zero_()
        infos = helm.batch_solve(handles, [b] * len(handles), xs, TOL)
        if any(i.status != 0 for i in infos):
            raise RuntimeError("2D sweep solve did not converge")
        return [i.iters for i in infos]

    for _ in range(2):
        step()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ms, iters = 0.0, None
    for i in range(3):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        iters = step()
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    for h in handles:
        h.close()
    del handles, xs, b, flush
    torch.cuda.empty_cache()
    return {"value": float(N * N) * sum(iters) * 3 / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / 3,
            "iters_per_beta": dict(zip([str(t) for t in BETAS], iters)), "steps": 3,
            "workload": "2D 1023^2, k=160, random source (seed 1001), theta_beta {0.1,0.2,0.3,0.5} batched, "
                        "complex64 V(1,1)-GMRES(3) / FGMRES to 1e-6 (double-float basis, binary64 least squares and "
                        "residual); L2 flushed between steps"}


def batch_extra(args):
    """The 64-problem batch (--mode batch) in solves/s, as a sub-object."""
    return _capture_mode(run_batch, args, batch=args.batch, steps=1, warmup=1)


def serving_extra(args):
    """A short Poisson serving run (--mode serve) with p50/p99 latency, as a sub-object."""
    return _capture_mode(run_serve, args, requests=args.serve_requests, rate=args.serve_rate, seq_sample=1,
                         seq_run=True)


def _capture_mode(fn, args, **over):
    import contextlib
    import io
    a = argparse.Namespace(**vars(args))
    for k, v in over.items():
        setattr(a, k, v)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        fn(a)
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    out = json.loads(lines[-1]) if lines else None
    if out:
        out.pop("ms_steps", None)
    return out


# ------------------------------------------------------------------ oracle (CPU)
_ORACLE = {}


def _oracle_setup():
    """Build the oracle's hierarchy of the 255^3 problem (once per process)."""
    if "levels" not in _ORACLE:
        import oracle as O
        w = I.cube_3d(CUBE_N)
        _ORACLE["w"] = w
        _ORACLE["levels"] = O.build_hierarchy(3, w.n, w.theta_beta, I.THETA_GAMMA, I.ECS_FRAC,
                                              phi=w.phi.astype(np.float64))
    return _ORACLE["w"], _ORACLE["levels"]


def oracle_sample(_=None):
    """The oracle's FGMRES(40) on the 3D 255^3 problem stopped after one outer iteration
    (one V-cycle and one H apply; the hierarchy set-up is outside the time).  Returns
    (wall-clock start, wall-clock end, V-cycles)."""
    import oracle as O
    w, levels = _oracle_setup()
    t0 = time.time()
    _, info = O.fgmres(levels[0].apply_h, lambda v: O.vcycle(levels, v), w.b, None, w.tol, w.restart, 1)
    return t0, time.time(), info.iters


def oracle_pool(samples, workers, warmup=0):
    """`samples` one-iteration oracle samples on `workers` spawned processes (each
    process builds the hierarchy once; `warmup` untimed samples first).  Returns
    (seconds from the first sample's start to the last one's end, V-cycles)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_oracle_setup) as pool:
        if warmup:
            pool.map(oracle_sample, range(warmup), chunksize=1)
        res = pool.map(oracle_sample, range(samples), chunksize=1)
    return max(r[1] for r in res) - min(r[0] for r in res), sum(r[2] for r in res)


def cpu_workers(cap):
    return max(1, min(os.cpu_count() or 1, 16, cap))


def cpu_baseline():
    """The oracle timed on the host: one core, then every core (one sample per spawned
    worker process, running together); the reported value is the faster of the two."""
    pts = float(CUBE_N) ** 3
    t0, t1, its1 = oracle_sample()
    sec1 = t1 - t0
    one = pts * its1 / sec1 / 1e6
    workers = cpu_workers(16)
    wall, its = oracle_pool(workers, workers)
    allc = pts * its / wall / 1e6
    best_all = allc >= one
    return {"value": allc if best_all else one, "unit": UNIT, "cores": workers if best_all else 1, "kind": "oracle",
            "single_core": {"value": one, "seconds": sec1},
            "all_cores": {"value": allc, "workers": workers, "wall_s": wall},
            "host": host_info(),
            "sample": f"NumPy FP64 oracle FGMRES(40) on the same 255^3 problem stopped after one outer iteration "
                      f"(one V-cycle, one H apply; hierarchy set-up excluded): {sec1:.1f} s on one core; "
                      f"{workers} such samples on {workers} spawned processes together in {wall:.1f} s"}


def run_reference(args, rank):
    """The oracle as the reference arm: each step is one one-iteration sample of the
    255^3 solve; the steps run on spawned processes over the host cores (the warm-up
    steps first, untimed), and the value is fine points x V-cycles over the time from
    the first timed sample's start to the last one's end."""
    if rank != 0:
        return None
    workers = cpu_workers(max(args.steps, 1))
    wall, its = oracle_pool(args.steps, workers, warmup=args.warmup) if args.steps > 0 else (1.0, 0)
    value = float(CUBE_N) ** 3 * its / wall / 1e6
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "host": host_info(),
                             "sample": f"each step: the NumPy FP64 oracle FGMRES(40) on the 255^3 problem stopped "
                                       f"after one outer iteration (hierarchy set-up excluded); steps on "
                                       f"{workers} spawned processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_precond(args):
    """V-cycles only (helm_precond_apply), for profiler captures of the V-cycle
    kernels on a chosen grid: --dim D --n N --reps R."""
    import torch

    from paper_1012_5379_gb300 import helm
    dev = torch.device("cuda", 0)
    n, dim = args.n, args.dim
    k = 0.156 * (n + 1)
    # maxit = 1: no FGMRES basis is allocated, the device holds the hierarchy only.  The
    # polynomial smoother needs a larger CSG angle than the workload's 0.3 rad on its
    # coarse levels (Sec. 4.5): it runs at theta_beta = 10 degrees.
    tb = 0.3 if args.smoother == "gmres" else np.radians(10.0)
    h = helm.Handle(dim, n, tb, k=k, precision="c64", maxit=1, smoother=args.smoother)
    r = torch.from_numpy(I.random_source(dim, n, 1001)).to(dev).to(torch.complex64)
    z = torch.empty_like(r)
    for _ in range(args.reps):
        h.precond_apply(r, z)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.reps):
        h.precond_apply(r, z)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.reps
    helm.profile_begin("")
    for _ in range(args.reps):
        h.precond_apply(r, z)
    classes = helm.profile_end()
    print(json.dumps({"mode": "precond", "dim": dim, "n": n, "smoother": args.smoother, "ms_per_vcycle": 1e3 * dt,
                      "mpts_per_s": n ** dim / dt / 1e6,
                      "vcycle_hbm": vcycle_hbm(classes, peaks().get("hbm_gbs", 6800.0)),
                      "classes_us_per_vcycle": {c: round(1e3 * v["ms"] / args.reps, 1) for c, v in classes.items()},
                      "launches_per_vcycle": {c: v["launches"] // args.reps for c, v in classes.items()}}),
          flush=True)


def run_single(args):
    """One complex64-preconditioned solve (--dim, --n, --maxit, --restart; kh = 0.156,
    theta_beta 0.3, random source), for profiler captures of the outer kernels on a
    bounded FGMRES basis.  Stopping at maxit is not an error here."""
    import torch

    from paper_1012_5379_gb300 import helm
    dev = torch.device("cuda", 0)
    n, dim = args.n, args.dim
    h = helm.Handle(dim, n, 0.3, k=0.156 * (n + 1), precision="c64", restart=args.restart, maxit=args.maxit)
    b = torch.from_numpy(I.random_source(dim, n, 1001)).to(dev)
    x = torch.zeros_like(b)
    t0 = time.perf_counter()
    info = h.solve(b, x, TOL)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "single", "dim": dim, "n": n, "iters": info.iters, "status": info.status,
                      "rel_res_true": info.rel_res_true, "s": time.perf_counter() - t0}), flush=True)


def run_cube(args):
    """The 3D workload: 255^3 unit cube, heterogeneous k(x) = 80 (1 + 0.3 g(x)) with
    8 seeded Gaussian bumps, point source, theta_beta 0.4, FGMRES(40) to 1e-6.  One
    solve with the complex64 and one with the complex128 preconditioner (each timed
    with CUDA events after an untimed solve)."""
    import torch

    from paper_1012_5379_gb300 import helm
    dev = torch.device("cuda", 0)
    w = I.cube_3d(args.n if args.n in (63, 127, 255) else 255)
    b = torch.from_numpy(w.b).to(dev)
    phi = torch.from_numpy(w.phi).to(dev)
    out = {"mode": "cube", "config": {"workload": f"3D {w.n}^3 unit cube, k(x)=80(1+0.3 g(x)), 8 seeded bumps "
                                                  "(seed 1002, sigma 0.1), point source, theta_beta 0.4, ECS 1/8 at "
                                                  "0.5 rad, V(1,1) GMRES(3), FGMRES(40) to 1e-6"}}
    for prec in ("c64", "c128"):
        h = helm.Handle(3, w.n, w.theta_beta, phi=phi, precision=prec, restart=w.restart, maxit=400)
        x = torch.zeros_like(b)
        h.solve(b, x, w.tol)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = h.solve(b, x, w.tol)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        out[prec] = {"iters": info.iters, "restarts": info.restarts, "rel_res_true": info.rel_res_true,
                     "status": info.status, "s": sec, "vcycle_mpts_per_s": float(w.n) ** 3 * info.iters / sec / 1e6,
                     "device_bytes": h.workspace_bytes()}
        h.close()
        del h
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


TUNE_WORKLOADS = (  # (dim, n, precision, field) whose levels the committed table covers
    (3, 255, "c64", True), (3, 127, "c64", True), (2, 4095, "c64", False), (2, 1023, "c64", False),
    (2, 511, "c64", False), (2, 255, "c64", False), (2, 127, "c128", False), (2, 1023, "c128", False))


def run_tune(args):
    """Tune the V-cycle's launch choices (helm_autotune) for the levels of the benchmark
    workloads, one after the other, and write the whole table to --tune-out."""
    import torch

    from paper_1012_5379_gb300 import helm
    out = {"mode": "tune", "path": args.tune_out, "runs": []}
    for dim, n, prec, field in TUNE_WORKLOADS:
        phi = None
        if field:
            phi = torch.from_numpy(I.cube_3d(n).phi).cuda()
        t0 = time.perf_counter()
        d0, d1 = helm.autotune(dim, n, 0.4 if dim == 3 else 0.3, k=None if field else 0.156 * (n + 1), phi=phi,
                               precision=prec, reps=args.reps, path=args.tune_out)
        out["runs"].append({"dim": dim, "n": n, "prec": prec, "default_ms": d0, "tuned_ms": d1,
                            "s": time.perf_counter() - t0})
        print(json.dumps(out["runs"][-1]), flush=True)
        del phi
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def gauss_key(nu, k, nint, cycle):
    """Key of one Gaussian-model solve in tests/golden/oracle_iters_gauss.json."""
    return f"nu={nu:g} k={k:g} nint={nint} V({cycle})"


def gauss_oracle_iters(path):
    """The FP64 oracle's iteration counts of the Gaussian-model solves (a stored file
    written from the oracle alone), or {} if the file is absent."""
    if not os.path.exists(path):
        return {}
    return {key: v["iters"] for key, v in json.load(open(path))["iters"].items()}


def run_gauss(args):
    """Benchmark 3 of Sec. 5, the Gaussian model: the five (k, grid) columns of
    Tables 4 and 5 for nu = 1 and nu = 7, V(1,0) and V(1,1) preconditioners (GMRES(3)
    smoothing, complex64), FGMRES without restart to 1e-7.  Each solve is timed with
    CUDA events after an untimed one; the paper's counts are printed beside ours."""
    import torch

    from paper_1012_5379_gb300 import helm
    dev = torch.device("cuda", 0)
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden")
    gold = json.load(open(os.path.join(golden, "paper_tables.json")))
    oracle_iters = gauss_oracle_iters(os.path.join(golden, "oracle_iters_gauss.json"))
    rows = []
    for table, nu in (("table4", 1.0), ("table5", 7.0)):
        for col, (k, nint) in enumerate(I.GAUSS_COLUMNS):
            w = I.gaussian_model(nint, k, nu)
            b = torch.from_numpy(w.b).to(dev)
            phi = torch.from_numpy(w.phi).to(dev)
            for cyc in ("1,0", "1,1"):
                nu1, nu2 = map(int, cyc.split(","))
                h = helm.Handle(2, w.n, w.theta_beta, phi=phi, precision=w.precision, theta_gamma=w.theta_gamma,
                                ecs_frac=w.ecs_frac, ecs_sides="high", nu1=nu1, nu2=nu2,
                                maxit=max(args.maxit, 600))
                x = torch.zeros_like(b)
                h.solve(b, x, w.tol)
                x.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                info = h.solve(b, x, w.tol)
                e1.record()
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) * 1e-3
                rows.append({"nu": nu, "k": k, "nint": nint, "n": w.n, "cycle": cyc, "iters": info.iters,
                             "oracle_iters": oracle_iters.get(gauss_key(nu, k, nint, cyc)),
                             "paper_iters": gold[table]["iters"][cyc][col], "status": info.status,
                             "rel_res_true": info.rel_res_true, "s": sec,
                             "vcycle_mpts_per_s": float(w.n) ** 2 * info.iters / sec / 1e6})
                h.close()
                del h
    out = {"mode": "gauss", "config": {"workload": "Gaussian model (Sec. 5, Benchmark 3): (0,50)^2, phi = nu (e^-x^2 + "
                                                   "e^-y^2) + k^2, Dirichlet S/W, ECS layer nint/4 N/E at pi/6, "
                                                   "theta_beta 10.3132 deg, FGMRES to 1e-7, the library's automatic "
                                                   "preconditioner precision and basis (complex128 and binary64 on "
                                                   "the 64^2 column's 79^2 grid, complex64 and double-float above)"},
           "rows": rows}
    print(json.dumps(out), flush=True)


def _seq_solves(helm, works, precision, bs, xs):
    """Solve `works` one at a time on fresh handles of `precision` (each timed with CUDA
    events after one untimed solve of the same handle); returns per-problem seconds and
    infos."""
    import torch
    times, infos = [], []
    for w, b, x in zip(works, bs, xs):
        h = helm.Handle(w.dim, w.n, w.theta_beta, k=w.k, precision=precision, restart=w.restart, maxit=400)
        x.zero_()
        h.solve(b, x, w.tol)   # graph capture, first touch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x.zero_()
        torch.cuda.synchronize()
        e0.record()
        info = h.solve(b, x, w.tol)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        infos.append(info)
        h.close()
    return times, infos


def run_batch(args):
    """64 independent 2D problems (n in {255, 511, 1023}, kh ~ U[0.1, 0.3], theta_beta
    0.3, random sources, FGMRES(40) to 1e-6): one step = all 64 solved together with
    helm_batch_solve (every V-cycle level and outer kernel is one launch for all
    problems of that size).  Compared with the same problems solved one at a time with
    the complex128 (FP64) preconditioner and with the complex64 one."""
    import torch

    from paper_1012_5379_gb300 import helm
    dev = torch.device("cuda", 0)
    works = I.batch_2d(args.batch)
    bs = [torch.from_numpy(w.b).to(dev) for w in works]
    xs = [torch.zeros_like(b) for b in bs]
    handles = [helm.Handle(w.dim, w.n, w.theta_beta, k=w.k, precision="c64", restart=w.restart, maxit=400)
               for w in works]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        for x in xs:
            x.zero_()
        infos = helm.batch_solve(handles, bs, xs, TOL)
        bad = [i for i in infos if i.status != 0]
        if bad:
            raise RuntimeError(f"{len(bad)} solves did not converge: {bad[0]}")
        return infos

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = helm.launch_count()
    ms, all_infos = [], []
    for s in range(args.steps):
        flush.fill_(float(s))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        all_infos.append(step())
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = helm.launch_count() - launches0
    clocks = sampler.stop()
    t = sum(ms) * 1e-3
    work = sum(float(w.n) ** 2 * i.iters for infos in all_infos for w, i in zip(works, infos))
    for h in handles:
        h.close()
    del handles
    torch.cuda.empty_cache()
    seq = {}
    for prec in ("c128", "c64"):
        times, infos = _seq_solves(helm, works, prec, bs, xs)
        seq[prec] = {"solves_per_s": len(works) / sum(times), "s_total": sum(times),
                     "iters_total": sum(i.iters for i in infos),
                     "max_rel_res_true": max(i.rel_res_true for i in infos)}
    infos = all_infos[-1]
    sizes = {}
    for w in works:
        sizes[w.n] = sizes.get(w.n, 0) + 1
    line = {"mode": "batch", "metric": "solves/s", "value": len(works) * args.steps / t, "unit": "solves/s",
            "higher_is_better": True, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "vcycle_mpts_per_s": work / t / 1e6, "gpu_launches": int(launches), "clocks": clocks,
            "config": {"workload": f"{len(works)} independent 2D problems, sizes {sizes}, kh ~ U[0.1,0.3], "
                                   "theta_beta 0.3, unit-variance complex normal sources (seed 1003), "
                                   "FGMRES(40) to 1e-6, complex64 V(1,1)-GMRES(3) / default outer arithmetic "
                                   "(double-float basis above 16384 unknowns, binary64 below)",
                       "l2": "flushed between steps"},
            "iters_total": sum(i.iters for i in infos), "max_rel_res_true": max(i.rel_res_true for i in infos),
            "sequential": seq,
            "speedup_vs_sequential_c128": (len(works) * args.steps / t) / seq["c128"]["solves_per_s"],
            "ms_steps": ms}
    print(json.dumps(line), flush=True)


def _sequential_server(helm, stream, srcs, xbuf, precision):
    """The same arrivals served for real by a plain single-solve server: one request at
    a time, first come first served, each on a fresh handle of `precision`
    (helm_setup), one helm_solve_host from the request's pinned source into its pinned
    solution buffer, then helm_destroy.  One untimed request per shape first (module
    loading, first graph capture).  Latency = completion - arrival."""
    import torch
    for sh in sorted({(r.work.dim, r.work.n) for r in stream}):
        w = next(r.work for r in stream if (r.work.dim, r.work.n) == sh)
        h = helm.Handle(sh[0], sh[1], w.theta_beta, k=w.k, precision=precision, restart=w.restart, maxit=400)
        h.solve_host(srcs[sh][0].numpy(), xbuf[sh][0].numpy(), w.tol)
        h.close()
        torch.cuda.empty_cache()
    lat, its, res = [], [], []
    t0 = time.perf_counter()
    for i, r in enumerate(stream):
        dt = t0 + r.arrival - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        sh = (r.work.dim, r.work.n)
        h = helm.Handle(sh[0], sh[1], r.work.theta_beta, k=r.work.k, precision=precision, restart=r.work.restart,
                        maxit=400)
        info = h.solve_host(srcs[sh][i % 2].numpy(), xbuf[sh][i % 2].numpy(), r.work.tol)
        h.close()
        lat.append(time.perf_counter() - t0 - r.arrival)
        its.append(info.iters)
        res.append(info.rel_res_true)
    t_total = max(r.arrival + l for r, l in zip(stream, lat))
    torch.cuda.empty_cache()
    return {"solves_per_s": len(stream) / t_total, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "iters_total": int(sum(its)),
            "max_rel_res_true": float(max(res)),
            "how": "measured: one request at a time, fresh handle per request, helm_solve_host from pinned memory"}


def run_serve(args):
    """Poisson stream of solve requests through helm_serve_* (continuous batching under
    a device-memory budget): solves/s over the stream and p50/p99 latency (submission to
    completion).  The same stream served one request at a time by the complex128
    (FP64) solver is simulated from measured per-request solve times of a sample and,
    with --seq-run (the default bench's serving extra), also served for real."""
    import threading

    import torch

    from paper_1012_5379_gb300 import helm
    stream = I.request_stream(count=args.requests, rate=args.rate)
    shapes = sorted({(r.work.dim, r.work.n) for r in stream})
    # sources: two seeded arrays per shape, page-locked, shared by that shape's requests
    srcs, xbuf = {}, {}
    for sh in shapes:
        srcs[sh] = [torch.from_numpy(I.request_source(j, *sh)).pin_memory() for j in range(2)]
        xbuf[sh] = [torch.empty_like(srcs[sh][0]).pin_memory() for _ in range(2)]
    budget = int(args.budget_gb * 1e9)
    srv = helm.Server(budget_bytes=budget, precision="c64", restart=40, maxit=400)
    # warm-up: one request per shape creates that shape's first slot
    for sh in shapes:
        t = srv.submit(sh[0], sh[1], 0.2 * (sh[1] + 1), 0.3, srcs[sh][0], xbuf[sh][0], TOL)
        srv.wait(t)
    st0 = srv.stats()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = helm.launch_count()
    results = [None] * len(stream)
    tickets = [None] * len(stream)
    submit_t = [0.0] * len(stream)
    ready = threading.Semaphore(0)

    def collector():
        for i in range(len(stream)):
            ready.acquire()
            info, lat, rc = srv.wait(tickets[i], timeout=3600.0)
            results[i] = (info, lat, rc)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(stream):
        dt = t0 + r.arrival - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        sh = (r.work.dim, r.work.n)
        submit_t[i] = time.perf_counter() - t0
        tickets[i] = srv.submit(sh[0], sh[1], r.work.k, r.work.theta_beta, srcs[sh][i % 2], xbuf[sh][i % 2],
                                r.work.tol)
        ready.release()
    th.join()
    launches = helm.launch_count() - launches0
    clocks = sampler.stop()
    stats = srv.stats()
    srv.stop()
    lat = np.array([x[1] for x in results])
    done = np.array(submit_t) + lat
    t_total = float(done.max())
    ok = sum(1 for x in results if x[2] == 0)
    work = sum(float(r.work.n) ** r.work.dim * x[0].iters for r, x in zip(stream, results))
    torch.cuda.empty_cache()
    # sequential baselines (complex128 and complex64 preconditioner): the solve time per
    # outer iteration of each shape, from a sample of the stream's requests solved one at
    # a time, times the iterations each request took when served (a problem's iterations
    # do not depend on what it was batched with)
    seq = {}
    served_iters = np.array([x[0].iters for x in results], dtype=float)
    for prec in ("c128", "c64"):
        per_shape, per_iter = {}, {}
        for sh in shapes:
            sample = [r for r in stream if (r.work.dim, r.work.n) == sh][:args.seq_sample]
            bs = [srcs[sh][0].to("cuda") for _ in sample]
            xs = [torch.zeros_like(b) for b in bs]
            times, infos = _seq_solves(helm, [r.work for r in sample], prec, bs, xs)
            per_shape[sh] = float(np.mean(times))
            per_iter[sh] = float(np.sum(times)) / max(1, sum(i.iters for i in infos))
            del bs, xs
            torch.cuda.empty_cache()
        svc = np.array([per_iter[(r.work.dim, r.work.n)] for r in stream]) * served_iters
        arr = np.array([r.arrival for r in stream])
        fin = np.empty_like(arr)
        prev = 0.0
        for i in range(len(arr)):           # one server, first come first served
            prev = max(arr[i], prev) + svc[i]
            fin[i] = prev
        slat = fin - arr
        seq[prec] = {"solves_per_s": len(stream) / float(fin.max()), "p50_s": float(np.percentile(slat, 50)),
                     "p99_s": float(np.percentile(slat, 99)),
                     "solve_s_per_shape": {f"{d}D {n}": v for (d, n), v in per_shape.items()},
                     "solve_s_per_iteration": {f"{d}D {n}": v for (d, n), v in per_iter.items()}}
    line = {"mode": "serve", "metric": "solves/s", "value": len(stream) / t_total, "unit": "solves/s",
            "higher_is_better": True, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "requests": len(stream), "ok": ok, "rate_per_s": args.rate,
            "vcycle_mpts_per_s": work / t_total / 1e6, "gpu_launches": int(launches), "clocks": clocks,
            "max_rel_res_true": max(x[0].rel_res_true for x in results),
            "server": {k: stats[k] - st0.get(k, 0) if k in ("completed", "submitted", "handles_created",
                                                           "handles_reused") else stats[k]
                       for k in stats},
            "config": {"workload": f"Poisson arrivals, mean {args.rate}/s, {len(stream)} requests, shapes uniform "
                                   f"over {shapes}, kh ~ U[0.1,0.3], theta_beta 0.3, FGMRES(40) to 1e-6, "
                                   "complex64 V(1,1)-GMRES(3) / default outer arithmetic",
                       "budget_bytes": budget,
                       "sources": "two seeded unit-variance complex normal sources per shape (pinned), "
                                  "request i uses source i mod 2; solutions land in pinned buffers"},
            "sequential_simulated": seq}
    if args.seq_run:
        run = _sequential_server(helm, stream, srcs, xbuf, "c128")
        line["sequential_run"] = {"c128": run}
        line["speedup_vs_sequential_c128"] = line["value"] / run["solves_per_s"]
        line["speedup_vs_sequential_c128_basis"] = "sequential_run (measured)"
    else:
        line["speedup_vs_sequential_c128"] = line["value"] / seq["c128"]["solves_per_s"]
        line["speedup_vs_sequential_c128_basis"] = "sequential_simulated"
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 2D sweep, 64-problem batch and serving keys of the default line")
    ap.add_argument("--serve-requests", type=int, default=120, help="requests of the default line's serving run")
    ap.add_argument("--serve-rate", type=float, default=8.0, help="arrivals/s of the default line's serving run")
    ap.add_argument("--mode", choices=["solve", "precond", "batch", "serve", "single", "cube", "gauss", "sweep2d",
                                       "tune"], default="solve")
    ap.add_argument("--tune-out", default=os.path.join(ROOT, "paper_1012_5379_gb300", "tuning.json"),
                    help="tune mode: where the table is written")
    ap.add_argument("--restart", type=int, default=0)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--seq-sample", type=int, default=2)
    ap.add_argument("--seq-run", action="store_true",
                    help="serve mode: also serve the stream for real one request at a time with complex128 handles")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=4095)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--smoother", choices=["gmres", "poly"], default="gmres",
                    help="precond mode: GMRES(3) sweeps or the Sec. 4 polynomial smoother (theta_beta 10 deg)")
    args = ap.parse_args()
    if args.mode != "solve":
        from paper_1012_5379_gb300 import build
        build.build()
        if args.mode == "sweep2d":
            print(json.dumps(sweep_2d(args, "cuda")), flush=True)
            return
        {"precond": run_precond, "batch": run_batch, "serve": run_serve, "single": run_single,
         "cube": run_cube, "gauss": run_gauss, "tune": run_tune}[args.mode](args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        from paper_1012_5379_gb300 import build
        build.build()
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
