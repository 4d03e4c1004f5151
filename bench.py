"""Throughput of the projected-CG homogenization solver on one GB300 (or N replicas).

A step is one converged effective-tangent solve of one RVE: all load cases
(the unit Mandel strains) to the accuracy target, then the homogenised
effective stiffness.  Default workload: 2D 1024x1024 two-phase thresholded
Gaussian field, contrast 100, nu = 0.3, 3 load cases, FP32-FFT inner solve
with FP64 refinement.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead (bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per projected-CG iteration and solves/s at 1e-9 rel. err; % HBM roofline"

WORKLOADS = {
    # name: (microstructures config, precision, relative residual tolerance)
    "gauss1024": ("gauss1024", "mixed", 1e-11),
    "gauss1024_fp64": ("gauss1024", "fp64", 1e-11),
    "lognormal64": ("lognormal64", "mixed", 1e-11),
    "spheres128": ("spheres128", "mixed", 1e-11),
    "lognormal128": ("lognormal128", "mixed", 1e-10),
    "batch64": ("batch64", "mixed", 1e-10),
    "lognormal256": ("lognormal256", "mixed", 1e-10),
    "lognormal256_fp64": ("lognormal256", "fp64", 1e-10),
}


# Workloads of the widened rows: zero-stiffness voxels, a derivative plug-in,
# finite strain and the adjoint gradient.  Same timing rules as the headline
# workloads; each reports its own unit of work.
EXTENSIONS = {
    "porous1024": "zero-stiffness voxels: 1024^2 log-normal moduli with 25% void voxels, mixed, 3 load cases",
    "fourier1024_fp64": "Fourier-derivative projection: the 1024^2 two-phase field, FP64, 3 load cases",
    "finite1024_fp64": "finite strain (St. Venant-Kirchhoff): 1024^2 log-normal moduli, FP64, one F_macro",
    "adjoint64": "adjoint gradient of C_1111: 64^3 log-normal moduli, mixed, 6 load cases + 1 adjoint solve",
}


def extension_inputs(name):
    """Seeded inputs of an extension workload (grid, moduli, loads, precision)."""
    import microstructures as ms
    if name == "porous1024":
        n = (1024, 1024)
        return dict(n=n, E=ms.porous_lognormal(n, 0.25, seed=1009), nu=0.3, prec="mixed", tol=1e-10,
                    Em=np.eye(3), unit="solves/s")
    if name == "fourier1024_fp64":
        cfg = ms.config_inputs("gauss1024")
        return dict(n=cfg["n"], E=cfg["E"], nu=cfg["nu"], prec="fp64", tol=1e-10, Em=np.eye(3),
                    derivative="fourier", unit="solves/s")
    if name == "finite1024_fp64":
        n = (1024, 1024)
        return dict(n=n, E=ms.lognormal_field(n, 0.0, 1.0, seed=1010), nu=0.3, prec="fp64", tol=1e-10,
                    Fm=np.array([[[1.05, 0.02], [0.0, 0.97]]]), unit="solves/s")
    if name == "adjoint64":
        cfg = ms.config_inputs("lognormal64")
        W = np.zeros((6, 6))
        W[0, 0] = 1.0
        return dict(n=cfg["n"], E=cfg["E"], nu=cfg["nu"], prec="mixed", tol=1e-10, Em=np.eye(6), W=W,
                    unit="gradients/s")
    raise KeyError(name)


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (the slowest rank sets the job time)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world):
    """Whole-job rate: every rank processes its own units (replicas, weak scaling)."""
    return world * units_per_rank / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Short hash of the CUDA sources (csrc/): ties a stored ncu traffic
    figure to the kernels it was measured on."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2105_03297_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))
                   + glob.glob(os.path.join(csrc, "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, form, kernel, dim):
    """DRAM bytes per launch of `kernel` from profiles/traffic.md, or None.

    The table rows are `| workload | form | kernel | bytes per launch | source hash | note |`; a row
    counts only if its hash is the hash of the kernels being run (otherwise the
    kernels changed since the counters were taken)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    name = f"{kernel}_{dim}d"
    with open(path) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 5 and cells[0] == workload and cells[1] == form and cells[2] == name:
                try:
                    return float(cells[3]) if cells[4] == want else None
                except ValueError:
                    return None
    return None


def model_bytes(dim, n, s, L_iters, form="stress"):
    """Algorithmic bytes of the CG-iteration passes, per load-case iteration.

    s: bytes per real scalar of the inner precision.  Returns dict pass -> bytes.
    Stress form: pass A reads r, p_old, x and E and writes p, x (the deferred
    x += alpha p) and the x-spectrum; pass C (2D) reads and writes the spectrum
    once; pass E reads the spectrum and r and writes r.  In 3D passes B, C, D
    each read and write the spectrum.
    Factored form: the force stencil reads r, p_old, x, E and writes p, x and
    the D nodal forces; the FFT passes move D-component spectra (pass A reads
    the forces, pass E writes w); the strain update reads w and r, writes r.
    """
    nq, ns = (2, 3) if dim == 2 else (6, 6)
    m = nq * ns
    N = int(np.prod(n))
    kx = n[0] // 2 + 1
    if form == "nodal":
        # force kernel: reads rho, pi_old, xi, E; writes pi, xi, f.  FFT passes on
        # D components.  Update: reads rho_old, w; writes rho.
        D = dim
        specd = D * kx * (N // n[0]) * 2 * s
        out = {
            "force_stencil": (6 * D + 1) * N * s,
            "pass_a": D * N * s + specd,
            "pass_c": 2 * specd,
            "pass_e": specd + D * N * s,
            "strain_update": 3 * D * N * s,
        }
        if dim == 3:
            out["pass_b"] = 2 * specd
            out["pass_d"] = 2 * specd
        return out
    if form == "factored":
        D = dim
        specd = D * kx * (N // n[0]) * 2 * s
        out = {
            "force_stencil": (5 * m + 1 + D) * N * s,
            "pass_a": D * N * s + specd,
            "pass_c": 2 * specd,
            "pass_e": specd + D * N * s,
            "strain_update": (D + 2 * m) * N * s,
        }
        if dim == 3:
            out["pass_b"] = 2 * specd
            out["pass_d"] = 2 * specd
        return out
    spec = m * kx * (N // n[0]) * 2 * s
    out = {
        "pass_a": 5 * m * N * s + N * s + spec,
        "pass_c": 2 * spec,
        "pass_e": spec + 2 * m * N * s,
    }
    if dim == 3:
        out["pass_b"] = 2 * spec
        out["pass_d"] = 2 * spec
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_fractions(mb, kt, lc_iters, steps, peak):
    """Achieved HBM fraction of every timed CG-iteration kernel: its model bytes
    per load-case iteration x the load-case iterations it served / its summed
    CUDA-event time, over the peak (GB/s).  Kernels without time are left out."""
    out = {}
    for k, (ms, launches) in kt.items():
        if k in mb and launches > 0 and ms > 0:
            out[k] = mb[k] * lc_iters * steps / (ms * 1e-3) / 1e9 / peak
    return out


def host_cpu(cpuinfo=None):
    """CPU model and logical core count of this host (for the CPU baseline).

    x86 lists a "model name"; Arm lists "CPU part" codes (and sometimes "Model")."""
    model = None
    try:
        if cpuinfo is None:
            with open("/proc/cpuinfo") as f:
                cpuinfo = f.read()
        info = cpuinfo
        for key in ("model name", "Model", "CPU part"):
            for ln in info.splitlines():
                if ln.split(":")[0].strip() == key:
                    model = ln.split(":", 1)[1].strip()
                    break
            if model:
                model = model if key != "CPU part" else f"{platform.machine()} CPU part {model}"
                break
    except OSError:
        pass
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def oracle_sample(cfg_name, seconds_budget=20.0):
    """Time the FP64 oracle's CG iterations on this host (bounded sample).

    Returns (seconds per CG iteration per load case, iterations timed, cores).
    """
    import microstructures as ms
    from oracle.fe_projection import Problem
    cfg = ms.config_inputs(cfg_name)
    P = Problem(cfg["n"], cfg["E"], cfg["nu"])
    Ef = P.broadcast_macro(cfg["E_macro"][0])
    r = -P.operator(Ef)
    p = r.copy()
    x = np.zeros_like(r)
    rr = float(np.sum(r * r))
    its = 0
    t0 = time.perf_counter()
    while True:
        q = P.operator(p)
        alpha = rr / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        its += 1
        if time.perf_counter() - t0 > seconds_budget and its >= 2:
            break
    dt = time.perf_counter() - t0
    return dt / its, its, 1


def golden_iterations(cfg_name):
    try:
        with open(os.path.join(ROOT, "tests", "golden", cfg_name + ".json")) as f:
            d = json.load(f)
        return d.get("iterations"), d.get("C_eff")
    except Exception:
        return None, None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg_name, prec, tol = WORKLOADS[args.workload]
    import microstructures as ms
    cfg = ms.config_inputs(cfg_name)
    its_gold, _ = golden_iterations(cfg_name)
    total_its = sum(its_gold) if its_gold else None
    per_step = []
    sample_its = 0
    budget = max(3.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for k in range(args.warmup + args.steps):
        sec_it, its, cores = oracle_sample(cfg_name, seconds_budget=budget)
        if k >= args.warmup:
            per_step.append(sec_it)
            sample_its += its
    sec_it = float(np.mean(per_step))
    ms_it = sec_it * 1e3
    solve_s = sec_it * total_its if total_its else None
    value = (1.0 / solve_s) if solve_s else None
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_s * 1e3 if solve_s else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg_name, "grid": list(cfg["n"]), "load_cases": len(cfg["E_macro"]),
                   "precision": "fp64 (CPU oracle)", "rel_tol": tol, "parallelism": "one CPU thread"},
        "ms_per_cg_iteration": ms_it,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample_its} FP64 CG iterations of one load case of {cfg_name} "
                                   f"(numpy oracle), scaled by the {total_its} iterations of the full solve",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_batch(args, world, rank, local, dist):
    """64 uneven 2D RVEs (sides 64..512), 3 load cases each, one batch solve per step."""
    import torch
    import microstructures as ms
    from paper_2105_03297_gb300 import RVEBatch

    cfg_name, prec, tol = WORKLOADS[args.workload]
    rves = ms.uneven_batch_2d(64, seed=1004 + rank)
    sizes = [n for n, _ in rves]
    Em = ms.unit_load_cases(2)
    b = RVEBatch(sizes, precision=prec, nu=0.3)
    for i, (_, E) in enumerate(rves):
        b.set_material(i, E)
    for _ in range(args.warmup):
        b.solve(Em, rel_tol=tol, max_iter=20000)
    stream = torch.cuda.current_stream()
    iters = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            code, info = b.solve(Em, rel_tol=tol, max_iter=20000)
            Cs = [b.effective_tangent(i) for i in range(len(sizes))]
            iters.append(max(v["iterations"] for rv in info for v in rv))
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
    dt = max_over_ranks(dt, dist if world > 1 else None, "cuda")
    # model bytes of every slot's CG iterations in this step (7 vector + 4 spectrum streams, FP32)
    total_bytes = 0.0
    for (n, _), rv in zip(rves, info):
        mb = model_bytes(2, n, 4, None)
        total_bytes += sum(v["iterations"] for v in rv) * (mb["pass_a"] + mb["pass_c"] + mb["pass_e"])
    peak, peak_kind = peaks()
    achieved = total_bytes / dt / 1e9
    out = {
        "metric": METRIC, "value": job_throughput(len(sizes), dt, world), "unit": "RVE solves/s (3 load cases each)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": cfg_name, "rves": len(sizes), "voxels": int(sum(np.prod(n) for n in sizes)),
                   "load_cases": 3, "precision": prec, "rel_tol": tol, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2"},
        "max_cg_iterations_per_solve": float(np.mean(iters)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole batch step (all passes, all groups)",
                     "peak_source": peak_kind},
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    b.close()
    if world > 1:
        dist.destroy_process_group()


def run_extension(args):
    """One GPU, one handle: time whole solves (or solve + adjoint) of an
    extension workload through the public API, inputs resident on the device."""
    import torch
    from paper_2105_03297_gb300 import RVE
    from paper_2105_03297_gb300.build import build_library
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build_library()
    x = extension_inputs(args.workload)
    n, dim = x["n"], len(x["n"])
    stream = torch.cuda.current_stream()
    r = RVE(n, precision=x["prec"], stream=stream.cuda_stream)
    if "derivative" in x:
        r.set_derivative(x["derivative"])
    if "Fm" in x:
        r.set_kinematics("finite")
    elif args.form != "stress":
        r.set_operator_form(args.form)
    E_dev = torch.from_numpy(np.ascontiguousarray(x["E"].reshape(-1))).cuda()
    r.set_material(E_dev, x["nu"])

    def step():
        if "Fm" in x:
            code, info = r.solve_finite(x["Fm"], rel_tol=x["tol"])
            r.mean_piola()
        else:
            code, info = r.solve(x["Em"], rel_tol=x["tol"], max_iter=20000)
            r.effective_tangent()
            if "W" in x:
                r.adjoint(x["W"], rel_tol=x["tol"], max_iter=20000)
        return code, info

    for _ in range(args.warmup):
        step()
    r.timing(True)
    r.timing_read()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    codes, lc_iters = [], 0.0
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            code, info = step()
            codes.append(code)
            lc_iters += sum(i["iterations"] for i in info)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    kt = r.timing_read()
    r.timing(False)
    r.close()
    peak, peak_kind = peaks()
    s = 4 if x["prec"] == "mixed" else 8
    out = {
        "metric": METRIC, "value": 1e3 * args.steps / ms_total, "unit": x["unit"], "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if x["prec"] == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": EXTENSIONS[args.workload], "grid": list(n),
                   "precision": x["prec"], "rel_tol": x["tol"], "operator_form": args.form,
                   "l2": "inputs larger than L2 (working set > 129 MB)"},
        "status_codes": codes,
        "cg_iterations_per_step": lc_iters / args.steps,
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "gpu_launches": int(sum(v[1] for v in kt.values())),
        "clocks": clk.summary(),
        "roofline": None,
    }
    if "Fm" not in x and "W" not in x and "derivative" not in x and args.form == "stress":
        # small-strain FE stress form: the byte model of the headline workloads applies
        mb = model_bytes(dim, n, s, 1)
        fr = hbm_fractions(mb, kt, lc_iters, 1, peak)
        out["kernels_hbm_frac"] = fr
        if fr:
            dom = max(fr, key=lambda k: kt[k][0])
            out["roofline"] = {"bound": "hbm", "achieved": fr[dom] * peak, "peak": peak, "unit": "GB/s",
                               "frac": fr[dom], "traffic": None, "kernel": dom, "peak_source": peak_kind}
    print(json.dumps(out), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2105_03297_gb300.build import build_library
    if rank == 0 or world == 1:
        build_library()
    if world > 1:
        dist.barrier()
    import microstructures as ms
    from paper_2105_03297_gb300 import RVE

    if args.workload.startswith("batch"):
        return run_batch(args, world, rank, local, dist)
    cfg_name, prec, tol = WORKLOADS[args.workload]
    cfg = ms.config_inputs(cfg_name)
    n, E, nu, Em = cfg["n"], cfg["E"], cfg["nu"], cfg["E_macro"]
    dim = len(n)
    L = len(Em)
    stream = torch.cuda.current_stream()
    r = RVE(n, precision=prec, stream=stream.cuda_stream)
    if args.schedule:
        r.set_schedule(*[int(v) for v in args.schedule.split(",")])
    r.set_operator_form(args.form)
    E_dev = torch.from_numpy(E.reshape(-1)).cuda()
    r.set_material(E_dev, nu)
    max_iter = 20000
    ns = 3 if dim == 2 else 6

    def homogenised():
        # the full tangent when all n_s load cases are solved, else the mean stresses
        return r.effective_tangent() if L == ns else r.mean_stress()

    for _ in range(args.warmup):
        code, info = r.solve(Em, rel_tol=tol, max_iter=max_iter)
        C = homogenised()
    _, C_gold = golden_iterations(cfg_name)
    acc = (float(np.abs(C - np.array(C_gold)).max() / np.abs(np.array(C_gold)).max())
           if C_gold is not None and L == ns else None)
    r.timing(True)
    r.timing_read()
    iters = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            code, info = r.solve(Em, rel_tol=tol, max_iter=max_iter)
            C = homogenised()
            iters.append([i["iterations"] for i in info])
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist if world > 1 else None, "cuda")
    if world > 1:
        dist.barrier()
    kt = r.timing_read()
    r.timing(False)
    ms_step = ms_total / args.steps
    lc_iters = float(np.sum(iters)) / args.steps          # load-case iterations per solve
    cg_iters = float(np.mean([max(v) for v in iters]))   # batched iterations per solve
    s = 4 if prec == "mixed" else 8
    mb = model_bytes(dim, n, s, lc_iters, args.form)
    # dominant kernel: the CG-iteration pass with the most device time
    cand = {k: v for k, v in kt.items() if k in mb and v[1] > 0}
    dom = max(cand, key=lambda k: cand[k][0])
    dom_ms, dom_launches = cand[dom]
    bytes_total = mb[dom] * lc_iters * args.steps
    achieved = bytes_total / (dom_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    cg_ms = sum(v[0] for k, v in kt.items() if k in mb) / (cg_iters * args.steps)

    # end to end through the C ABI with host buffers: E host->device, C_eff device->host
    E_host = np.ascontiguousarray(E.reshape(-1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.set_material(E_host, nu)
        r.solve(Em, rel_tol=tol, max_iter=max_iter)
        C_h = homogenised()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist if world > 1 else None, "cuda")

    value = job_throughput(1.0, ms_step / 1000.0, world)
    launches = int(sum(v[1] for v in kt.values()))

    extras = {}
    if rank == 0 and not args.no_comparisons:
        # the plain FP64 GPU solve of the same workload, to the same tolerance
        if prec == "mixed":
            with RVE(n, precision="fp64", stream=stream.cuda_stream) as r64:
                r64.set_material(E_dev, nu)
                r64.solve(Em, rel_tol=tol, max_iter=max_iter)      # warm-up (and autotune)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                code64, info64 = r64.solve(Em, rel_tol=tol, max_iter=max_iter)
                C64 = r64.effective_tangent() if L == ns else r64.mean_stress()
                torch.cuda.synchronize()
                t64 = time.perf_counter() - t0
            d64 = float(np.abs(C - C64).max() / np.abs(C64).max())
            extras["fp64_gpu_solve"] = {"ms_per_solve": t64 * 1e3, "speedup_of_mixed": t64 * 1e3 / ms_step,
                                        "iterations": [i["iterations"] for i in info64],
                                        "mixed_vs_fp64_rel_diff": d64}
        # the other orders of the same operator, same workload and tolerance
        for other in [f for f in ("stress", "factored", "nodal") if f != args.form]:
            with RVE(n, precision=prec, stream=stream.cuda_stream) as ro:
                ro.set_operator_form(other)
                ro.set_material(E_dev, nu)
                ro.solve(Em, rel_tol=tol, max_iter=max_iter)          # warm-up (and autotune)
                torch.cuda.synchronize()
                eo0, eo1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                eo0.record(stream)
                codeo, infoo = ro.solve(Em, rel_tol=tol, max_iter=max_iter)
                Co = ro.effective_tangent() if L == ns else ro.mean_stress()
                eo1.record(stream)
                torch.cuda.synchronize()
                t_o = eo0.elapsed_time(eo1)
            its_o = [i["iterations"] for i in infoo]
            extras[f"{other}_form_solve"] = {
                "ms_per_solve": t_o, "ratio_to_headline": t_o / ms_step, "iterations": its_o,
                "ms_per_cg_iteration": t_o / max(its_o), "status": codeo,
                "rel_diff_to_headline": float(np.abs(C - Co).max() / np.abs(Co).max())}
        # cuFFT (through torch.fft) on the same fields: context only, not part of the product
        m = (2 if dim == 2 else 6) * ns
        shape = (L * m,) + tuple(reversed(n))
        f = torch.randn(shape, device="cuda", dtype=torch.float32 if prec == "mixed" else torch.float64)
        dims = tuple(range(1, dim + 1))
        for _ in range(3):
            g = torch.fft.irfftn(torch.fft.rfftn(f, dim=dims), s=shape[1:], dim=dims)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            g = torch.fft.irfftn(torch.fft.rfftn(f, dim=dims), s=shape[1:], dim=dims)
        e1.record(stream)
        torch.cuda.synchronize()
        ours = sum(v[0] for k, v in kt.items() if k in mb) / (cg_iters * args.steps)
        extras["cufft_r2c_c2r_same_fields"] = {"ms": e0.elapsed_time(e1) / 5,
                                               "our_full_cg_iteration_ms": ours,
                                               "note": "cuFFT forward+inverse only (no material, projection "
                                                       "or CG update); context, not used by the solver"}
        del f, g
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": cfg_name, "grid": list(n), "load_cases": L, "precision": prec,
                   "rel_tol": tol, "operator_form": args.form, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (working set > 129 MB)"},
        "ms_per_cg_iteration": cg_ms,
        "cg_iterations_per_solve": cg_iters,
        "c_eff_rel_err_vs_oracle": acc,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(cfg_name, args.form, dom, dim), "kernel": dom,
                     "peak_source": peak_kind},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "kernels_hbm_frac": hbm_fractions(mb, kt, lc_iters, args.steps, peak),
        "schedule": dict(zip(("pass_a_tile_variant", "pass_e_tile_variant"), r.schedule()[0])),
        "e2e": {"value": job_throughput(1.0, e2e_s, world), "unit": "solves/s", "h2d_bytes_per_step": int(E_host.nbytes + Em.nbytes),
                "d2h_bytes_per_step": int(C_h.nbytes)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    out.update(extras)
    if rank == 0 and not args.no_cpu_baseline:
        its_gold, _ = golden_iterations(cfg_name)
        total_its = sum(its_gold) if its_gold else lc_iters
        sec_it, its, cores = oracle_sample(cfg_name, seconds_budget=15.0)
        v = 1.0 / (sec_it * total_its)
        out["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                               "sample": f"{its} FP64 CG iterations of one load case (numpy oracle, "
                                         f"{sec_it * 1e3:.0f} ms each), scaled by {total_its} iterations per solve",
                               "host": host_cpu()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    r.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="gauss1024", choices=sorted(WORKLOADS) + sorted(EXTENSIONS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="",
                    help="force the tile variants of passes A and E, e.g. 0,0 (default: autotune)")
    ap.add_argument("--form", default="stress", choices=["stress", "factored", "nodal"],
                    help="order of the operator inside CG (same operator; see include/rve.h)")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the FP64 GPU solve and cuFFT timings (context figures)")
    args = ap.parse_args()
    if args.workload in EXTENSIONS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle baseline is timed on the "
                              "headline workloads only"}), flush=True)
        elif int(os.environ.get("RANK", "0")) == 0:
            run_extension(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
