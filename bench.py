#!/usr/bin/env python
"""Throughput benchmark of the colloidal Shan-Chen lattice-Boltzmann step.

One step = one pass of the whole coupled update (remap, densities, wetting,
fused collide/stream with bounce-back, link forces, pair forces, integrator)
over the confined sheared bijel workload: 512x512x256 sites, walls normal to z
moving at +-0.05, radius-5.5 spheres at volume fraction 0.15 (14,444), 50/50
mixture with +-1 % seeded noise, G = 0.65, tau = 1, FP32 storage.

Prints one JSON line (rank 0).  ``value`` is MLUPS = sites x steps / time
(Eqs. 36-37, all sites), summed over ranks; every rank runs an independent
replica (the method is not sharded here).  ``--impl reference`` times the
plain FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline, FP32 vs FP16-store vs FP64 at stated error; adjoint/fwd time"
STORE = {"fp64": 8, "fp32": 4, "fp16": 2}   # bytes per stored population
COMPUTE = {"fp64": 8, "fp32": 4, "fp16": 4}  # bytes per psi value


def alg_bytes(prec):
    """Algorithmic bytes of one site update (the method's own traffic): one
    read and one write of the 2 x 19 populations and the 1-byte node mask,
    76 s + 1 for s bytes per stored population (FP64 609, FP32 305, FP16 153)."""
    return 76 * STORE[prec] + 1


def kernel_bytes(kname, prec):
    """Bytes per site that a lattice kernel itself must move (arrays touched
    once): the density pass reads the populations and the mask and writes
    rho^k and j^A + j^B; the lean momentum kernel reads j^A + j^B, psi^k and
    the 4-byte link classes and writes the populations; the two-pass kernel
    reads both; the plain kernel reads and writes the populations."""
    pops = 38 * STORE[prec]
    if kname == "k_density":
        return pops + 1 + 5 * COMPUTE[prec]
    if kname == "k_lean":
        return pops + 5 * COMPUTE[prec] + 4
    if kname == "k_fused_async":
        return 2 * pops + 2 * COMPUTE[prec] + 4
    return 2 * pops + 1


DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32-math"}
# stated parity bounds against the FP64 oracle (relative, fields after 100 steps), as tested
STATED_ERROR = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3}
# source of the lattice kernels (density pass, fused kernels) whose ncu DRAM
# record profiles/ keeps: the record applies while this file is unchanged
LATTICE_KERNEL_SRC = [os.path.join(ROOT, "paper_2004_04080_gb300", "csrc", f)
                      for f in ("lbgb_fluid.cu", "lbgb_colloid.cu")]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for p in LATTICE_KERNEL_SRC:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(prec):
    """ncu DRAM bytes per time step of the lattice kernels (density pass and
    fused kernel) at the full workload, if the committed record was taken on
    the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "lattice_traffic_shear512_fp32.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(prec)
        if e and e.get("kernel_sha") == kernel_hash():
            return float(e["bytes_per_launch_full_workload"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.uuid, "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model():
    """The host CPU as the OS names it."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_mlups(w, target_seconds, max_steps=50):
    """Steps the FP64 oracle on workload ``w`` for about target_seconds after
    one untimed step; returns (MLUPS, steps, seconds)."""
    from oracle import Oracle

    a, b = w.densities()
    c = w.colloids()
    o = Oracle(*w.shape, max(w.n_colloids, 1))
    o.set_params(**w.params)
    o.init_fields(a, b)
    if c is not None:
        o.add_colloids(c["pos"], c["radius"], c["mass"])
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > target_seconds or steps >= max_steps:
            break
    return w.n_sites * steps / el / 1e6, steps, el


# The paper's two-component Shan-Chen throughput per core without particles
# (1024^3, G = 0.65, 128 cores of 2x Xeon Gold 6148 nodes; Sec. 5.1 table of
# the two-component runs, case 0).
PAPER_MLUPS_PER_CORE_2COMP = 1.41


def cpu_baseline(name, target_seconds=20.0, extras=True):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample
    of the workload: a 128x128x64 sub-box with the same physics and particle
    volume fraction.  ``value`` uses every core (OpenMP over the site loops;
    the particle-link sums stay single-threaded).  With ``extras``: the same
    sample on one thread, and the 128^3 two-component mixture without
    particles (G = 0.65) on all cores and on one, per core beside the
    paper's figure for that case."""
    from oracle import set_threads
    from paper_2004_04080_gb300.workloads import workload

    sub = (128, 128, 64)
    w = workload(name, scale=sub)
    cores = set_threads(0)
    mlups, steps, el = oracle_mlups(w, target_seconds)
    out = {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": "%s sub-box %dx%dx%d, %d particles, %d steps, %.1f s, FP64, %d OpenMP threads" % (
               name, *sub, w.n_colloids, steps, el, cores),
           "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    if extras:
        try:
            set_threads(1)
            m1, s1, e1 = oracle_mlups(w, target_seconds / 3)
            out["one_thread"] = {"value": round(m1, 3), "steps": s1, "seconds": round(e1, 1)}
            # the paper's two-component case: G = 0.65 with density 1 per component
            w0 = dataclasses.replace(workload("bijel_demix"), n_colloids=0)
            two = {}
            for th in (0, 1):
                n = set_threads(th)
                m, s_, e_ = oracle_mlups(w0, target_seconds / 4, max_steps=20)
                two["all_cores" if th == 0 else "one_thread"] = {
                    "threads": n, "mlups": round(m, 3), "mlups_per_core": round(m / n, 3),
                    "steps": s_, "seconds": round(e_, 1)}
            two["case"] = "128^3 two-component Shan-Chen, G = 0.65, rho = 1 + 1, tau = 1, no particles, FP64"
            two["paper_mlups_per_core"] = PAPER_MLUPS_PER_CORE_2COMP
            two["paper_case"] = "1024^3 case 0, 128 cores (2x Xeon Gold 6148 per node), FP64 Fortran"
            out["two_component_no_particles"] = two
        finally:
            set_threads(0)
    return out


def workload_desc(name, w):
    """The workload as the bench line names it (both arms)."""
    return "%s: %dx%dx%d sites, %s, R=%g (%d particles), G=%g, tau=%g" % (
        name, *w.shape, "walls z +-%g" % w.params["wall_u_hi"][0] if w.params["bc"][2] == 0 else "periodic",
        w.radius, w.n_colloids, w.params["G"], w.params["tau"][0])


def run_reference(args, world, rank):
    from paper_2004_04080_gb300.workloads import workload

    if rank != 0:
        return 0
    base = cpu_baseline(args.workload, target_seconds=max(5.0, min(60.0, 2.0 * (args.steps + args.warmup))),
                        extras=False)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, workload(args.workload, tuple(args.shape) if args.shape else None)),
                       "prec": "fp64 oracle", "parallelism": "%d host threads (OpenMP)" % base["cores"]},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_timing(dev, torch, steps=500):
    """Adjoint / forward wall time on the 64^3 workload (8 immobile R=4.5
    spheres, FP32): forward = the checkpointed forward run (sqrt(N)
    checkpoints), adjoint = the reverse sweep (segment recomputation plus the
    adjoint steps); the objective is J_drag + A."""
    from paper_2004_04080_gb300.adjoint import AdjointRunner
    from paper_2004_04080_gb300.lbgb import LBLattice
    from paper_2004_04080_gb300.workloads import workload

    w = workload("adjoint64")
    a, b = w.densities()
    col = w.colloids()
    lat = LBLattice(w.shape, "fp32", max_colloids=w.n_colloids, device=dev)
    run = AdjointRunner(lat, steps)
    run.forward(w.params, a, b, col)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run.forward(w.params, a, b, col)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    grads, _ = run.backward(1.0, 1.0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del run, lat
    torch.cuda.empty_cache()
    return {"workload": "adjoint64: 64^3 periodic, 8 immobile R=4.5 spheres, FP32, %d steps, %d checkpoints"
                        % (steps, int(math.ceil(math.sqrt(steps)))),
            "forward_s": round(t1 - t0, 4), "adjoint_s": round(t2 - t1, 4),
            "adjoint_over_forward": round((t2 - t1) / (t1 - t0), 3),
            "grad_finite": bool(np.all(np.isfinite(grads)))}


def max_over_ranks(v, world, device=None):
    """Largest value over the ranks of the default process group (every rank
    runs an independent replica; the slowest one sets the job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(ms_local, n_sites, steps, world, device=None):
    """Whole-job MLUPS of `world` replicas of n_sites sites each: all sites
    updated `steps` times in the slowest replica's time."""
    ms = max_over_ranks(ms_local, world, device)
    return world * n_sites * steps / (ms / 1e3) / 1e6, ms


def case0_throughput(dev, torch, n=1024, steps=10):
    """The paper's two-component benchmark without particles (Sec. 5.1,
    two-component table, case 0): n^3 periodic sites, G = 0.65, density 1.0
    per component with standard deviation 0.004 (uniform noise of the same
    deviation, drawn per plane from PCG64), tau = 1, FP16 deviation storage
    (the FP32 form of 1024^3 needs 326 GB).  GLUPS over `steps` timed steps
    after 2 untimed ones, beside the paper's 1.37 GLUPS on 1024 cores."""
    from paper_2004_04080_gb300.lbgb import LBLattice

    N = n ** 3
    amp = 0.004 * math.sqrt(3.0)
    rhoA = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    rhoB = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    rng = np.random.Generator(np.random.PCG64(20040408))
    plane = n * n
    for z in range(n):
        eta = rng.random(plane) * 2.0 - 1.0
        rhoA[z * plane:(z + 1) * plane] = 1.0 + amp * eta
        rhoB[z * plane:(z + 1) * plane] = 1.0 - amp * eta
    lat = LBLattice((n, n, n), "fp16", max_colloids=0, device=dev)
    lat.set_params(G=0.65, tau=(1.0, 1.0), rho0=(1.0, 1.0))
    lat.init_fields(rhoA, rhoB)
    del rhoA, rhoB
    lat.step(2)
    ms = time_steps(lat, steps, torch)
    out = {"workload": "%d^3 periodic, two components, G = 0.65, rho = 1.0 + 1.0 (std 0.004), tau = 1, "
                       "no particles, FP16 storage (stochastic rounding)" % n,
           "steps": steps, "ms_per_step": round(ms / steps, 3), "glups": round(N * steps / (ms / 1e3) / 1e9, 3),
           "kernel": lat.fused_kernel(), "bytes_per_site": alg_bytes("fp16"),
           "hbm_frac": round(N * steps / (ms / 1e3) * alg_bytes("fp16") / 1e9 / peaks()[0], 4),
           "paper_glups": 1.37, "paper_case": "1024^3 case 0 on 1024 cores (Sec. 5.1 two-component table)"}
    del lat
    torch.cuda.empty_cache()
    return out


def single_throughput(dev, torch, n=1024, steps=10):
    """The paper's single-component benchmark (Sec. 5.1, first benchmark
    table; App. D benchmark test 1): n^3 periodic sites, one fluid component,
    Gaussian density of mean 1.0 and standard deviation 1e-4 (drawn per plane
    from PCG64), zero velocity, tau = 1, FP32 storage (163 GB at 1024^3).
    GLUPS over `steps` timed steps after 2 untimed ones, beside the paper's
    6.51 GLUPS (1024^3) and 5.37 GLUPS (512^3) on 2048 cores."""
    from paper_2004_04080_gb300.lbgb import LBLattice

    N = n ** 3
    rho = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    rng = np.random.Generator(np.random.PCG64(20040409))
    plane = n * n
    for z in range(n):
        rho[z * plane:(z + 1) * plane] = rng.normal(1.0, 1e-4, plane)
    lat = LBLattice((n, n, n), "fp32", max_colloids=0, device=dev, components=1)
    lat.set_params(tau=(1.0, 1.0), rho0=(1.0, 0.0))
    lat.init_fields(rho)
    del rho
    lat.step(2)
    ms = time_steps(lat, steps, torch)
    out = {"workload": "%d^3 periodic, one component, rho = 1.0 (Gaussian, std 1e-4), tau = 1, FP32 storage" % n,
           "steps": steps, "ms_per_step": round(ms / steps, 3), "glups": round(N * steps / (ms / 1e3) / 1e9, 3),
           "kernel": lat.fused_kernel(), "bytes_per_site": 152,
           "hbm_frac": round(152 * N * steps / (ms / 1e3) / 1e9 / peaks()[0], 4),
           "paper_glups": 6.51, "paper_case": "1024^3 single component on 2048 cores (Sec. 5.1 first table)"}
    del lat
    torch.cuda.empty_cache()
    return out


def time_steps(lat, steps, torch):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shear512")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--shape", type=int, nargs=3, default=None,
                    help="rescale the workload box (same physics and particle volume fraction)")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/FP64 side measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint / forward timing")
    ap.add_argument("--no-case0", action="store_true",
                    help="skip the paper-size runs without particles: 1024^3 two components in FP16 and one "
                         "component in FP32 (about 165 GB of device memory each)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist

    from paper_2004_04080_gb300.lbgb import LB_KERNEL_DENSITY, LBLattice
    from paper_2004_04080_gb300.workloads import workload

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w = workload(args.workload, tuple(args.shape) if args.shape else None)
    a, b = w.densities()
    col = w.colloids()
    lat = LBLattice(w.shape, args.prec, max_colloids=w.n_colloids, device=dev)
    lat.set_params(**w.params)
    lat.init_fields(a, b)
    lat.add_colloids(col["pos"], col["radius"], col["mass"])
    lat.step(args.warmup)
    barrier()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    launches0 = lat.launch_count()
    lat.profile(True)
    with ClockSampler(uuid) as clk:
        barrier()
        ms = time_steps(lat, args.steps, torch)
        barrier()
    launches = lat.launch_count() - launches0
    kern_ms, kern_n = lat.profile_read()
    dens_ms, dens_n = lat.profile_read(LB_KERNEL_DENSITY)
    lat.profile(False)
    value, ms = replica_mlups(ms, w.n_sites, args.steps, world, dev)
    ms_step = ms / args.steps
    peak, peak_kind = peaks()
    kname = lat.fused_kernel()
    abytes = alg_bytes(args.prec)
    alg = abytes * w.n_sites
    kavg = kern_ms / max(kern_n, 1)
    davg = dens_ms / dens_n if dens_n else 0.0
    traffic = recorded_traffic(args.prec)
    # The lattice update of a time step (one read and one write of every
    # population: the method's algorithmic bytes) is done by the density pass
    # and the lean kernel (with its small wall kernel) together when
    # particles are present, by the fused kernel alone otherwise; frac is
    # their rate against the measured copy bandwidth, step_frac the same
    # bytes over the whole step.
    lattice_ms = kavg + davg
    achieved = alg / (lattice_ms / 1e3) / 1e9
    kernels = [{"kernel": kname, "ms": round(kavg, 4), "own_bytes_per_site": kernel_bytes(kname, args.prec),
                "own_frac": round(kernel_bytes(kname, args.prec) * w.n_sites / (kavg / 1e3) / 1e9 / peak, 4)}]
    if dens_n:
        kernels.insert(0, {"kernel": "k_density", "ms": round(davg, 4),
                           "own_bytes_per_site": kernel_bytes("k_density", args.prec),
                           "own_frac": round(kernel_bytes("k_density", args.prec) * w.n_sites / (davg / 1e3) / 1e9
                                             / peak, 4)})
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": " + ".join(k["kernel"] for k in kernels), "kernel_ms": round(lattice_ms, 4),
                "alg_bytes_per_site": abytes, "alg_bytes_per_launch": alg, "peak_kind": peak_kind,
                "step_frac": round(alg / (ms_step / 1e3) / 1e9 / peak, 4),
                "traffic_ratio": round(traffic / alg, 3) if traffic else None,
                "kernels": kernels}

    # end to end through the public API with pinned host buffers
    N = w.n_sites
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    ha, hb = pin(N), pin(N)
    ha[:] = a
    hb[:] = b
    oa, ob, ou = pin(N), pin(N), pin(3 * N)
    n = w.n_colloids
    hp = pin(3 * n)
    hp[:] = col["pos"].ravel()
    hr, hm = pin(n), pin(n)
    hr[:] = col["radius"]
    hm[:] = col["mass"]
    cpos, cvel = pin(3 * n), pin(3 * n)
    # the caller's buffers exist before the run: first touches of fresh host
    # pages stay outside the timed region
    for buf in (oa, ob, ou, cpos, cvel):
        buf.fill(0.0)
    barrier()
    t0 = time.perf_counter()
    from paper_2004_04080_gb300 import lbgb as api

    api.lb_init_fields(lat.h, ha, hb)
    api.lb_add_colloids(lat.h, hp, hr, hm)
    api.lb_step(lat.h, args.steps)
    api.lb_get_fields(lat.h, oa, ob, ou)
    api.lb_get_colloids(lat.h, cpos, cvel, None, None, None, None)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": round(world * N * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int((2 * N * 8 + n * 5 * 8) / args.steps),
           "d2h_bytes_per_step": int((5 * N * 8 + n * 6 * 8) / args.steps)}
    del lat
    torch.cuda.empty_cache()

    forms = {}
    if not args.no_forms:
        for prec, steps in (("fp16", max(20, min(args.steps, 200))), ("fp64", 10)):
            if prec == args.prec:
                continue
            L2 = LBLattice(w.shape, prec, max_colloids=n, device=dev)
            L2.set_params(**w.params)
            L2.init_fields(a, b)
            L2.add_colloids(col["pos"], col["radius"], col["mass"])
            L2.step(3)
            L2.profile(True)
            barrier()
            m2 = max_over_ranks(time_steps(L2, steps, torch), world, dev)
            km, kn = L2.profile_read()
            dm, dn = L2.profile_read(LB_KERNEL_DENSITY)
            kk = km / max(kn, 1) + (dm / dn if dn else 0.0)
            forms[prec] = {"mlups": round(world * N * steps / (m2 / 1e3) / 1e6, 1), "steps": steps,
                           "kernel": L2.fused_kernel(),
                           "kernel_frac": round(alg_bytes(prec) * N / (kk / 1e3) / 1e9 / peak, 4),
                           "stated_rel_error_vs_fp64_oracle": STATED_ERROR[prec]}
            if prec == "fp16":
                forms[prec]["rounding"] = "stochastic (cvt.rs.f16x2.f32, the FP16 default)"
            del L2
            torch.cuda.empty_cache()
        forms[args.prec] = {"mlups": round(value, 1), "stated_rel_error_vs_fp64_oracle": STATED_ERROR[args.prec]}
        if "fp16" in forms and args.prec == "fp32":
            forms["fp16_speedup_over_fp32"] = round(forms["fp16"]["mlups"] / value, 3)

    case0 = case1 = None
    if not args.no_case0 and world == 1:
        case0 = case0_throughput(dev, torch)
        case1 = single_throughput(dev, torch)

    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_timing(dev, torch)

    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec],
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, w),
                       "prec": args.prec, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (%.1f GB of populations)" % (
                           2 * 38 * N * {"fp64": 8, "fp32": 4, "fp16": 2}[args.prec] / 1e9)},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
            "forms": forms, "adjoint": adjoint, "paper_case0": case0, "paper_single": case1}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
