#!/usr/bin/env python
"""Throughput of the colour-gradient LB step on B300: MLUPS and HBM roofline fraction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl native|reference]

One "step" is one lattice time step of the whole hot path (streaming, colour
field, wetting, curvature, collision, recolouring, reaction, reactant
transport) over the whole lattice.  The default workload is the 128 x 128 x 256
reactive flow-through column on a seeded Gaussian-random-field mask (synthetic
stand-in for the paper's bijel geometry).  Under torchrun each rank runs its
own replica (weak scaling, no collective on the data path).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores on bounded samples of the same workload instead.
"""
import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline at 1 B300 (plain vs FP16-storage/batched/adjoint)"
UNIT = "MLUPS"
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2608_15781_b300", "csrc", f)
                  for f in ("lattice.cuh", "kernels.cuh", "compact.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_main_dram_traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="column128x128x256")
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--storage", choices=("fp32", "fp16"), default="fp32",
                    help="population storage of the headline run (the other is reported under variants)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--launch", default=None, metavar="M,D,N,P,F",
                    help="fixed launch configuration (main, density and normal block sizes, programmatic launch "
                         "0/1, fields 0-3) instead of the tuner; for profiling runs, whose serialised timing "
                         "would mislead the tuner")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="T",
                    help="only time the adjoint variant over T steps and print its JSON (for profiling)")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_distributed(world, backend):
    """One process per GPU (replicas): the process group serves the barrier and the
    max-over-ranks of the timing only; no collective touches the lattice data."""
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend)


def max_over_ranks(v, world, device):
    """The slowest rank's value (timings are taken as the max over ranks)."""
    if world > 1:
        import torch

        tt = torch.tensor([float(v)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        v = float(tt.item())
    return v


def whole_job_mlups(world, nodes, steps, ms):
    """Lattice-node updates of all ranks (each advances its own replica) per second, in millions."""
    return world * nodes * steps / (ms * 1e-3) / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the device sources of the step kernels."""
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_fluid_node():
    """DRAM bytes per fluid node of k_main from the committed ncu summary, if the kernel is unchanged."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    with open(TRAFFIC_FILE) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_sources_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_fluid_node"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "power_w_max": float(max(power)), "reasons": sorted(reasons)}


def bytes_per_fluid_node(params):
    """Algorithmic bytes of one fluid-node update: populations read + written, plus 1 B of flags.

    FP32 storage: 361 B with the reactant populations (45 values each way), 305 B
    in the paper's reaction mode (38); FP16 storage: 181 B / 153 B.  Solid nodes
    carry no populations (the library
    stores the fluid nodes only), so a launch's algorithmic traffic is this
    figure times the number of fluid nodes.
    """
    npop = 45 if params.reaction_mode == 0 else 38
    width = 2 if params.storage == 1 else 4
    return 2 * width * npop + 1


def density_pass_bytes_per_fluid_node(params):
    """Bytes of the separate density pass (an implementation overhead, not part of the
    node update): the f^r and f^p of the 19 pulled directions read again, rho^N written."""
    width = 2 if params.storage == 1 else 4
    return 2 * 19 * width + 4


# --------------------------------------------------------------------------- CPU oracle legs
def _oracle_params(wl):
    from oracle import cglbm as O
    p = wl.params
    return O.Params(tau=p.tau, sigma=p.sigma, beta=p.beta, theta_deg=p.theta_deg, accel=tuple(p.accel),
                    diffusivity=p.diffusivity, k_rate=p.k_rate, c_init=p.c_init, c_in=p.c_in, u_in=p.u_in,
                    rho_out=p.rho_out, xi=p.xi, reaction_mode=p.reaction_mode, bc_z=wl.bc_z)


def _oracle_worker(job):
    """One process: the FP64 oracle on one z-slab crop of the workload's mask, single-threaded.

    Returns (seconds of the timed steps, lattice nodes of the crop)."""
    name, z0, crop, warmup, steps = job
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:            # NumPy's elementwise work is single-threaded anyway
        import contextlib

        def threadpool_limits(_n):
            return contextlib.nullcontext()
    from oracle import cglbm as O
    from paper_2608_15781_b300.configs import WORKLOADS
    wl = WORKLOADS[name]
    full = wl.mask()
    zz = (np.arange(crop[0]) + z0) % full.shape[0]
    solid = full[zz][:, : crop[1], : crop[2]]
    with threadpool_limits(1):
        g = O.Geometry(solid=solid, bc_z=wl.bc_z)
        op = _oracle_params(wl)
        st = O.init_state(g, op)
        for _ in range(warmup):
            st = O.step(st, g, op)
        t0 = time.perf_counter()
        for _ in range(steps):
            st = O.step(st, g, op)
        dt = time.perf_counter() - t0
    return dt, int(np.prod(solid.shape))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(wl, crop, warmup, steps, workers):
    """The oracle on `workers` host cores at once: one spawned process per core, each on its own
    z-slab crop of the mask.  Returns (whole-job MLUPS, slowest worker's seconds, nodes per worker)."""
    import multiprocessing as mp

    nz = wl.shape[0]
    jobs = [(wl.name, (w * crop[0]) % nz, crop, warmup, steps) for w in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_oracle_worker, jobs)
    t = max(r[0] for r in res)
    nodes = sum(r[1] for r in res)
    return nodes * steps / t / 1e6, t, res[0][1]


def baseline_workers():
    """Host cores used by the oracle legs: every core, at most 32 processes (each holds ~1 GB)."""
    return max(1, min(host_cores(), 32))


def cpu_baseline(wl):
    nz, ny, nx = wl.shape
    crop = (min(nz, 16), ny, nx)
    workers = baseline_workers()
    steps = 3
    mlups, dt, n = oracle_parallel(wl, crop, 0, steps, workers)
    return {"value": round(mlups, 4), "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{steps} steps on each of {workers} processes (one per host core of {host_cores()}), each on "
                      f"its own {crop[2]}x{crop[1]}x{crop[0]} (x,y,z) z-slab crop of the same mask and boundaries, "
                      f"FP64 NumPy, one thread per process; slowest process {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2608_15781_b300.configs import WORKLOADS
    wl = WORKLOADS[args.workload]
    nz, ny, nx = wl.shape
    workers = baseline_workers()
    # the largest crop whose whole run stays within ~150 s (calibrated on 1 step on every core)
    crops = [(min(nz, 16), ny, nx), (min(nz, 8), ny, nx), (min(nz, 4), min(ny, 64), min(nx, 64)),
             (min(nz, 2), min(ny, 32), min(nx, 32)), (1, min(ny, 16), min(nx, 16))]
    total = args.steps + args.warmup
    chosen = crops[-1]
    for crop in crops:
        _, dt, _ = oracle_parallel(wl, crop, 0, 1, workers)
        if dt * total <= 150.0:
            chosen = crop
            break
    mlups, dt, n = oracle_parallel(wl, chosen, args.warmup, args.steps, workers)
    sample = (f"each step: the FP64 NumPy oracle on {workers} processes (one per host core of {host_cores()}), "
              f"each on its own {chosen[2]}x{chosen[1]}x{chosen[0]} (x,y,z) z-slab crop of the workload's mask and "
              f"boundaries, one thread per process")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 5), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "nodes_per_step": n * workers, "crop_xyz": [chosen[2], chosen[1], chosen[0]],
                   "processes": workers},
        "cpu_baseline": {"value": round(mlups, 5), "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(mlups, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- native (GPU) leg
def run_native(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_distributed(world, "nccl")
    from paper_2608_15781_b300 import build, lbm
    from paper_2608_15781_b300.configs import WORKLOADS

    build.build()
    stream = torch.cuda.current_stream()
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps(measure_adjoint(lbm, torch, stream, world, args.adjoint_only)), flush=True)
        return 0
    wl = WORKLOADS[args.workload]
    solid = wl.mask()
    N = wl.nodes

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def measure(params, steps, warmup, clocks=None):
        """K timed steps, per-kernel CUDA events on the launching stream; time = max over ranks."""
        L = lbm.Lattice(solid, params, bc_z=wl.bc_z, stream=stream.cuda_stream)
        info = L.info()
        L.step(warmup)
        if args.launch:
            m, d, n, p, f = (int(v) for v in args.launch.split(","))
            info["launch"] = dict(main=m, density=d, normal=n, pdl=p, fields=f)
            L.set_launch(info["launch"])
        else:
            info["launch"] = L.tune()     # the library's launch-shape tuner, on the warmed-up state
        L.step(warmup)
        barrier()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        L.step(steps)                 # the production path: one CUDA graph replay per step
        e1.record(stream)
        barrier()
        clk = clocks.stop() if clocks else None
        t = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        ob = L.observables()
        # per-kernel split: a separate run with CUDA events around every launch (no graphs)
        psteps = steps
        L.profile(psteps * 6 + 16)
        L.step(psteps)
        prof = L.profile_read()
        L.profile(0)
        L.close()
        return t, prof, info, ob, clk

    def roofline(params, prof, nf):
        kname = max(prof, key=lambda k: prof[k][0])
        k_ms, k_n = prof[kname]
        per_node = bytes_per_fluid_node(params)
        alg = nf * per_node
        return kname, per_node, alg, alg / (k_ms / k_n * 1e-3) / 1e9

    peak, peak_kind = measured_peaks()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_idx = int(vis.split(",")[local]) if vis and vis.split(",")[local].strip().isdigit() else local
    head = dataclasses.replace(wl.params, storage={"fp32": 0, "fp16": 1}[args.storage])
    # end to end through the C ABI with host buffers: create from the host mask,
    # K x (step + copy of the step's reaction sums into pinned host memory), observables,
    # destroy.  Measured before the clock-sampled timed region: a run of nvidia-smi from
    # this process slows its later CUDA API calls (lattice creation +1.5 ms, destroy
    # +3.8 ms on the 128x128x256 column, measured), which a user's run does not pay.  An
    # untimed lattice, created and stepped first and destroyed after the timed leg, loads
    # the kernels (the process's first creation pays the lazy loading of the library's
    # modules, about 1 ms; a creation right after a destroy pays about as much for the
    # memory the destroy released).
    e2e = None
    if not args.no_e2e:
        # the host mask in page-locked memory, as the step results are
        pinned_mask = torch.empty(solid.shape, dtype=torch.uint8, pin_memory=True)
        solid_h = pinned_mask.numpy()
        solid_h[...] = solid
        ring = torch.empty(2 * args.steps, dtype=torch.float64, pin_memory=True)
        base = ring.data_ptr()
        Lw = lbm.Lattice(solid_h, head, bc_z=wl.bc_z, stream=stream.cuda_stream)
        Lw.step(2)
        Lw.reaction_async(base)
        Lw.observables()
        barrier()
        t0 = time.perf_counter()
        L2 = lbm.Lattice(solid_h, head, bc_z=wl.bc_z, stream=stream.cuda_stream)
        t_create = time.perf_counter() - t0
        for k in range(args.steps):
            L2.step(1)
            L2.reaction_async(base + 16 * k)
        ob2 = L2.observables()                      # synchronises the stream
        L2.close()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        Lw.close()
        rates = ring.numpy().reshape(-1, 2)
        assert abs(rates[-1, 1] - ob2["consumed"]) <= 1e-9 * max(1.0, abs(ob2["consumed"]))
        h2d = N * 1                                  # the mask
        d2h = 16 * args.steps + 8 * 8 * 2 + 3 * 8    # reaction sums per step, observables, layout totals
        e2e = {"value": round(whole_job_mlups(world, N, args.steps, te * 1e3), 2), "unit": UNIT,
               "h2d_bytes_per_step": round(h2d / args.steps, 2), "d2h_bytes_per_step": round(d2h / args.steps, 2),
               "create_ms": round(t_create * 1e3, 1),
               "includes": "lbm_create from the host mask in pinned memory (geometry precompute and slot layout on the GPU), "
                           "per step lbm_step(1) + lbm_reaction_async (D2H of the step's reaction sums into "
                           "pinned memory), lbm_observables (synchronises), lbm_destroy"}

    t_ms, prof, info, ob, clk = measure(head, args.steps, args.warmup, ClockSampler(gpu_idx))
    Nf = info["n_fluid"]
    value = whole_job_mlups(world, N, args.steps, t_ms)
    kname, per_node, alg_bytes, achieved = roofline(head, prof, Nf)
    traf = ncu_traffic_per_fluid_node() if (kname == "main" and head.storage == 0) else None
    psteps = args.steps
    # the timed region replays one graph per step holding the same launches as a profiled step
    launches = int(round(sum(n for _, n in prof.values()) / psteps * args.steps))

    variants = {}
    if not args.no_variants:
        vsteps = max(args.steps // 2, 1)
        names = {0: ("fp32_storage", "f32"), 1: ("fp16_storage", "f16 storage, f32 math")}
        for st in (0, 1):
            if st == head.storage:
                continue
            other = dataclasses.replace(head, storage=st)
            tv, pv, _, obv, _ = measure(other, vsteps, args.warmup)
            kv, pnv, _, achv = roofline(other, pv, Nf)
            variants[names[st][0]] = {
                "value": round(whole_job_mlups(world, N, vsteps, tv), 2), "unit": UNIT, "steps": vsteps,
                "ms_per_step": round(tv / vsteps, 5), "dtype": names[st][1],
                "roofline": {"kernel": f"k_{kv}", "achieved": round(achv, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achv / peak, 4), "bytes_model": f"{pnv} B per fluid-node update"},
                "conversion": obv["conversion"], "gas_saturation": obv["gas_saturation"]}

    if not args.no_variants:
        variants["batched"] = measure_batched(lbm, torch, stream, world, max(args.steps // 10, 20), args.warmup)
        variants["adjoint"] = measure_adjoint(lbm, torch, stream, world, 3000 if args.steps >= 1000 else 300)
        variants["precision_periodic256"] = measure_precision(lbm, torch, stream, world,
                                                              5000 if args.steps >= 1000 else 200)
        variants["precision_crop64_vs_fp64"] = measure_precision_crop(lbm, torch, stream)
        variants["paper_mode_analysis"] = measure_paper_mode(lbm, torch, stream)
        variants["column_series"] = measure_series(lbm, torch, stream, wl, head, 20000, 100)

    if rank != 0:
        return 0
    tot = max(sum(x[0] for x in prof.values()), 1e-9)
    kern = {k: {"ms_total": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot, 4)} for k, v in prof.items()}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ["f32", "f16 storage, f32 math"][head.storage],
        "data": "synthetic",
        "config": {"workload": wl.name, "lattice_xyz": [wl.shape[2], wl.shape[1], wl.shape[0]],
                   "mask": f"GRF shell |k|={wl.shell_k0}+-1, porosity {wl.porosity}, seed {wl.seed}",
                   "fluid_nodes": Nf, "porosity": round(Nf / N, 4),
                   "wall_nodes": info["n_wall"], "wall_fraction_of_fluid": round(info["n_wall"] / Nf, 4),
                   "boundary_solid_nodes": info["n_solid_bnd"],
                   "boundaries": "inlet/outlet in z" if wl.bc_z else "periodic",
                   "storage": ["fp32", "fp16 deviations"][head.storage],
                   "fluid_mlups": round(world * Nf * args.steps / (t_ms * 1e-3) / 1e6, 2),
                   "launch_shapes": info["launch"],
                   "l2": "state (2 x 45 x fluid nodes x 4 B) far above the 126 MB L2; no flush",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": f"k_{kname}", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": round(traf * Nf) if traf else None,
                     "algorithmic_bytes": int(alg_bytes),
                     "bytes_model": f"{per_node} B per fluid-node update (populations read+write + 1 B flags) "
                                    f"x {Nf} fluid nodes",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.4 TB/s",
                     "step_effective_gbs": round(alg_bytes / (t_ms / args.steps * 1e-3) / 1e9, 1),
                     "step_frac": round(alg_bytes / (t_ms / args.steps * 1e-3) / 1e9 / peak, 4),
                     "density_pass_bytes_per_fluid_node": density_pass_bytes_per_fluid_node(head),
                     "step_effective_gbs_incl_density_pass": round(
                         Nf * (per_node + density_pass_bytes_per_fluid_node(head)) / (t_ms / args.steps * 1e-3) / 1e9,
                         1),
                     "step_frac_incl_density_pass": round(
                         Nf * (per_node + density_pass_bytes_per_fluid_node(head)) / (t_ms / args.steps * 1e-3) / 1e9
                         / peak, 4)},
        "kernels": {"source": f"CUDA events around every launch of a separate {psteps}-step run (no graphs)",
                    **kern},
        "variants": variants,
        "gpu_launches": launches,
        "clocks": clk,
        "observables": {k: ob[k] for k in ("mass_r", "mass_p", "conversion", "gas_saturation", "n_bad")},
    }
    if e2e:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_batched(lbm, torch, stream, world, steps, warmup, seq_steps=20):
    """64 uneven columns (48^3 - 96^3) in one batch against the same 64 lattices run one after another."""
    from paper_2608_15781_b300.configs import batched_workload

    masks, params, bcs, edges = batched_workload()
    nodes = sum(int(np.prod(m.shape)) for m in masks)
    B = lbm.Batch(masks, params, bc_z=bcs, stream=stream.cuda_stream)
    B.step(warmup)
    blocks = B.tune()
    B.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_b = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    B.profile(steps * 6 + 16)
    B.step(steps)
    prof = B.profile_read()
    B.profile(0)
    obs = B.observables()
    nf = sum(o["n_fluid"] for o in obs)
    B.close()
    # the same lattices one after another, each through its own context (graph replay too)
    t_s = 0.0
    for m, p, bc in zip(masks, params, bcs):
        L = lbm.Lattice(m, p, bc_z=bc, stream=stream.cuda_stream)
        L.step(warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        L.step(seq_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_s += e0.elapsed_time(e1)
        L.close()
    k_ms, k_n = prof["main"]
    peak, _ = measured_peaks()
    alg = nf * bytes_per_fluid_node(params[0])
    achieved = alg / (k_ms / k_n * 1e-3) / 1e9
    t_s = max_over_ranks(t_s, world, "cuda")
    v_b = whole_job_mlups(world, nodes, steps, t_b)
    v_s = whole_job_mlups(world, nodes, seq_steps, t_s)
    return {"value": round(v_b, 2), "unit": UNIT, "steps": steps, "ms_per_step": round(t_b / steps, 5),
            "workload": f"64 columns, edges {min(edges)}-{max(edges)}, {nodes} nodes, {nf} fluid",
            "blocks": blocks, "sequential_value": round(v_s, 2), "speedup_vs_sequential": round(v_b / v_s, 3),
            "roofline": {"kernel": "k_main", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4)}}


_C19 = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0], [1, -1, 0],
                 [1, 0, 1], [1, 0, -1], [-1, 1, 0], [-1, -1, 0], [-1, 0, 1], [-1, 0, -1], [0, 1, 1], [0, 1, -1],
                 [0, -1, 1], [0, -1, -1], [0, 0, 0]], dtype=np.float64)


def velocity_difference(fa, fb, solid, chunk=16):
    """(max |u_a - u_b|, max |u_b|) over the fluid nodes of two (45, nz, ny, nx) states, in z chunks."""
    fl_all = ~solid.astype(bool)
    dmax = umax = 0.0
    for z0 in range(0, solid.shape[0], chunk):
        sl = slice(z0, z0 + chunk)
        fl = fl_all[sl]
        us = []
        for f in (fa, fb):
            m = f[0:19, sl].astype(np.float64) + f[19:38, sl]
            rho = np.where(fl, m.sum(0), 1.0)
            us.append(np.einsum("ia,i...->a...", _C19, m) / rho)
        dmax = max(dmax, float(np.abs(us[0] - us[1])[:, fl].max()))
        umax = max(umax, float(np.abs(us[1])[:, fl].max()))
    return dmax, umax


def measure_precision(lbm, torch, stream, world, nsteps):
    """256^3 periodic workload: FP32 and FP16 population storage from the same start,
    MLUPS of each and the FP16 - FP32 differences of conversion, gas saturation and u,
    next to the spread of two FP32 runs from starts 1e-6 apart and a second FP16 run
    from the perturbed start (a second draw of the FP16 rounding noise's effect)."""
    from paper_2608_15781_b300.configs import WORKLOADS

    wl = WORKLOADS["periodic256"]
    solid = wl.mask()
    out = {"workload": f"periodic256 (256^3, shell 12, porosity 0.5, seed 3), {nsteps} steps from rest"}
    # the last run: FP32 from a start perturbed by 1e-6 (the trajectories' own spread)
    rng = np.random.default_rng(0)
    perturbed = (1.0 + 1e-6 * rng.standard_normal(solid.shape)).astype(np.float32)
    ref = None
    n_bad = 0
    for name, storage, rho_r in (("fp32", 0, np.ones(solid.shape, np.float32)),
                                 ("fp16", 1, np.ones(solid.shape, np.float32)),
                                 ("fp32_spread_1e-6_start", 0, perturbed),
                                 ("fp16_1e-6_start", 1, perturbed)):
        L = lbm.Lattice(solid, dataclasses.replace(wl.params, storage=storage), bc_z=0, stream=stream.cuda_stream)
        L.step(3)
        L.init_fields(rho_r, np.zeros(solid.shape, np.float32), np.full(solid.shape, wl.params.c_init, np.float32))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        ob = L.observables()
        f = L.get_state()
        L.close()
        n_bad += int(ob["n_bad"])
        if ref is None:
            ref = (ob, f)
            out["fp32_mlups"] = round(whole_job_mlups(world, solid.size, nsteps, ms), 2)
            out["conversion_fp32"] = ob["conversion"]
            out["gas_saturation_fp32"] = ob["gas_saturation"]
            continue
        key = name if name.startswith("fp32") else f"{name}_vs_fp32"
        if name == "fp16":
            out[f"{name}_mlups"] = round(whole_job_mlups(world, solid.size, nsteps, ms), 2)
        d = {"abs_diff_conversion": abs(ob["conversion"] - ref[0]["conversion"]),
             "abs_diff_gas_saturation": abs(ob["gas_saturation"] - ref[0]["gas_saturation"])}
        d["max_abs_diff_u"], umax = velocity_difference(f, ref[1], solid)
        out.setdefault("max_abs_u_fp32", umax)
        out[key] = d
        del f
    out["n_bad"] = n_bad
    return out


PRECISION_CROP = os.path.join(ROOT, "tests", "golden", "precision_crop64_fp64.txt")


def read_precision_crop(path=PRECISION_CROP):
    """The FP64 oracle reference of the precision workload's 64^3 crop (written by
    tests/golden/make_precision_crop.py): observables per step and the velocity at sampled nodes."""
    obs, vel, part = [], [], None
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            if line.startswith("[observables]"):
                part = "obs"
                continue
            if line.startswith("[velocity]"):
                part = "vel"
                continue
            v = line.split()
            if part == "obs" and v:
                obs.append([int(v[0])] + [float(x) for x in v[1:]])
            elif part == "vel" and v:
                vel.append([int(v[0]), int(v[1]), int(v[2])] + [float(x) for x in v[3:]])
    return obs, vel


def measure_precision_crop(lbm, torch, stream, draws=3):
    """FP32 and FP16 population storage against the FP64 oracle on the 64^3 crop of the
    precision workload (same start, same steps): conversion, gas saturation and the
    velocity at the reference's sampled fluid nodes.  Next to them, the conversion error of
    runs whose start differs from the reference's by a relative 1e-6 (every f^r_i times
    1 + 1e-6 N(0, 1), `draws` seeds): the trajectory's own sensitivity, which sets the
    scale that any inexact run is judged on."""
    if not os.path.exists(PRECISION_CROP):
        return {"unavailable": "reference file tests/golden/precision_crop64_fp64.txt not present"}
    from paper_2608_15781_b300.configs import WORKLOADS

    obs, vel = read_precision_crop()
    wl = WORKLOADS["periodic256"]
    solid = wl.mask()[:64, :64, :64].copy()
    steps = [r[0] for r in obs]
    zyx = np.array([r[:3] for r in vel], dtype=np.int64)
    u_ref = np.array([r[3:] for r in vel])
    umax = float(np.abs(u_ref).max())
    out = {"workload": f"x, y, z < 64 crop of periodic256 run periodic, {steps[-1]} steps from rest; "
                       f"FP64 oracle reference at {len(vel)} sampled fluid nodes",
           "max_abs_u_fp64_sample": umax}

    def run(storage, draw=None):
        L = lbm.Lattice(solid, dataclasses.replace(wl.params, storage=storage), bc_z=0, stream=stream.cuda_stream)
        if draw is not None:
            f0 = L.get_state().astype(np.float64)
            f0[0:19] *= 1.0 + 1e-6 * np.random.default_rng(100 + draw).standard_normal(f0[0:19].shape)
            L.set_state(f0.astype(np.float32))
        dc, ds, done = [], [], 0
        for row in obs:
            L.step(row[0] - done)
            done = row[0]
            ob = L.observables()
            dc.append(abs(ob["conversion"] - row[1]))
            ds.append(abs(ob["gas_saturation"] - row[2]))
        f = L.get_state().astype(np.float64)
        L.close()
        return dc, ds, f

    for name, storage in (("fp32", 0), ("fp16", 1)):
        dc, ds, f = run(storage)
        fm = f[0:19] + f[19:38]
        rho = fm.sum(axis=0)
        u = np.stack([np.tensordot(_C19[:, a], fm, axes=(0, 0)) for a in range(3)]) / np.where(solid, 1.0, rho)
        du = np.abs(u[:, zyx[:, 0], zyx[:, 1], zyx[:, 2]].T - u_ref)
        out[name] = {"abs_err_conversion_final": dc[-1], "abs_err_conversion_max": max(dc),
                     "abs_err_gas_saturation_final": ds[-1], "abs_err_gas_saturation_max": max(ds),
                     "max_abs_err_u": float(du.max()), "max_abs_err_u_rel_to_max_u": float(du.max() / umax)}
    for name, storage in (("fp32_1e-6_starts", 0), ("fp16_1e-6_starts", 1)):
        errs = [max(run(storage, d)[0]) for d in range(draws)]
        out[name] = {"abs_err_conversion_max_per_draw": errs, "abs_err_conversion_max": max(errs)}
    return out


def superficial_velocity_x(f, solid, accel_x):
    """<u_x> = sum over fluid nodes of the physical velocity j_x / rho + a / 2, divided by all nodes
    (the volume average of Darcy's law; single phase, so the force shift is the body force alone)."""
    fm = f[0:19].astype(np.float64) + f[19:38]
    rho = np.where(solid, 1.0, fm.sum(axis=0))
    ux = np.tensordot(_C19[:, 0], fm, axes=(0, 0)) / rho + 0.5 * accel_x
    return float(ux[~solid].sum() / solid.size)


def measure_paper_mode(lbm, torch, stream, nsteps=50000, every=500, Da=1.0):
    """The paper's reactive-flow analysis (Sec. 4.2 and 5.1) on GPU runs through the C ABI.

    1. Permeability kappa = nu <u> / a of the structure from a single-phase run under
       the body force (tau = 1, steady Darcy flow).
    2. Nucleation sites (one site with one solid nearest neighbour per 64^3 block),
       A_r, and the viscosity that gives the Damkohler number Da (the paper varies
       Da through nu).
    3. The paper-mode reactive run (rho^r -> rho^p at the sites, xi = 1, sigma = 0.3,
       reactant-only start): m^r(t), m^p(t) and the reacted amount per step, turned
       into the effectiveness factor alpha(t), its running mean and the fit of
       m^r(t) = m^m exp(-xi A_r alpha t / (phi V))."""
    from paper_2608_15781_b300 import analysis as AN
    from paper_2608_15781_b300.configs import WORKLOADS

    wl = WORKLOADS["paper128"]
    solid = wl.mask()
    p0 = wl.params
    a = p0.accel[0]
    mor = AN.morphology(solid)
    V, phi = mor["volume"], mor["porosity"]
    nu1 = AN.kinematic_viscosity(1.0)
    L = lbm.Lattice(solid, dataclasses.replace(p0, tau=1.0, xi=0.0), stream=stream.cuda_stream)
    u_mean = []
    for _ in range(2):
        L.step(3000)
        u_mean.append(superficial_velocity_x(L.get_state(), solid, a))
    L.close()
    kappa = AN.permeability(nu1, u_mean[-1], a)
    sites = AN.nucleation_sites(solid, block=64, seed=0)
    A_r = AN.reactive_surface_area(sites, solid)
    length = solid.shape[2]                       # along the body force (x)
    nu = AN.viscosity_for_damkohler(Da, p0.xi, A_r, length, kappa, V, a)
    tau = AN.tau_for_viscosity(nu)
    L = lbm.Lattice(solid, dataclasses.replace(p0, tau=tau), reactive=sites, stream=stream.cuda_stream)
    ob = L.observables()
    m_m = ob["mass_r"] + ob["mass_p"]
    t, m_r, m_p, rate = [], [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for k in range(nsteps // every):
        e0.record(stream)
        L.step(every)
        e1.record(stream)
        ob = L.observables()
        ms += e0.elapsed_time(e1)
        t.append((k + 1) * every)
        m_r.append(ob["mass_r"])
        m_p.append(ob["mass_p"])
        rate.append(ob["rate"])
    n_bad = int(ob["n_bad"])
    L.close()
    t = np.array(t, dtype=np.float64)
    m_r = np.array(m_r)
    alpha = AN.effectiveness_factor(rate, m_r, p0.xi, A_r, phi, V)
    alpha_bar = AN.running_average(alpha)
    alpha_fit = AN.fit_effectiveness(t, m_r, m_m, p0.xi, A_r, phi, V)
    pick = [i for i in range(len(t)) if (i + 1) % max(1, len(t) // 10) == 0]
    return {"workload": f"paper128 (128^3 periodic GRF, shell 6, porosity {phi:.3f}, seed 6), reactant-only start",
            "permeability": kappa, "mean_u_x_at_3000_6000_steps": u_mean, "nucleation_sites": int(sites.sum()),
            "A_r": A_r, "Da": Da, "nu": nu, "tau": tau, "sigma": p0.sigma, "xi": p0.xi, "accel_x": a,
            "steps": int(t[-1]), "MLUPS": round(V * t[-1] / (ms * 1e-3) / 1e6, 1),
            "alpha_fit": alpha_fit, "alpha_bar_final": float(alpha_bar[-1]),
            "series_step_mr_over_mm_alpha_alphabar": [[int(t[i]), float(m_r[i] / m_m), float(alpha[i]),
                                                       float(alpha_bar[i])] for i in pick],
            "mass_conservation_rel": float(abs(m_r[-1] + m_p[-1] - m_m) / m_m), "n_bad": n_bad}


def measure_series(lbm, torch, stream, wl, params, nsteps, every):
    """The headline column run for nsteps steps: conversion and gas saturation every `every` steps.

    The column starts at rest, so the outlet sees no net inflow until the pressure
    front from the inlet has crossed the porous column; meanwhile the gas generated
    near the open outlet, pressurised by surface tension, draws a little liquid in
    through it (outlet flux < 0, conversion 1 - Phi_out / Phi_in > 1).
    ``transient_steps`` is the first sample from which the conversion stays in [0, 1]."""
    solid = wl.mask()
    L = lbm.Lattice(solid, params, bc_z=wl.bc_z, stream=stream.cuda_stream)
    series = []
    for k in range(nsteps // every):
        L.step(every)
        ob = L.observables()
        series.append([(k + 1) * every, round(ob["conversion"], 6), round(ob["gas_saturation"], 6)])
    L.close()
    transient = None
    for i in range(len(series)):
        if all(0.0 <= r[1] <= 1.0 for r in series[i:]):
            transient = series[i][0]
            break
    shown = [r for r in series if r[0] % (nsteps // 10) == 0 or r[0] <= 1000 and r[0] % 200 == 0]
    return {"workload": wl.name, "steps": every * len(series), "sample_every": every,
            "series_step_conversion_saturation": shown, "transient_steps": transient,
            "n_bad": int(ob["n_bad"])}


def measure_adjoint(lbm, torch, stream, world, nsteps):
    """Gradient of the outlet conversion of the 96^3 column after nsteps steps with respect to
    the per-solid-node contact angle and the inlet velocity: checkpointed forward
    (ceil(sqrt(nsteps)) spacing) plus the reverse sweep, timed with CUDA events."""
    from paper_2608_15781_b300.configs import WORKLOADS

    wl = WORKLOADS["column96"]
    solid = wl.mask()
    N = int(solid.size)
    L = lbm.Lattice(solid, wl.params, bc_z=wl.bc_z, stream=stream.cuda_stream)
    L.step(200)                       # a developed inflow with gas at the reactive walls
    f0 = L.get_state()
    nf = L.info()["n_fluid"]
    L.set_state(f0)                   # warm-up of both phases (allocates the checkpoints)
    L.adjoint_forward(min(nsteps, 100))
    L.adjoint_backward()
    L.set_state(f0)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    J = L.adjoint_forward(nsteps)
    e1.record(stream)
    dth, du, _ = L.adjoint_backward()
    e2.record(stream)
    torch.cuda.synchronize()
    t_f = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    t_b = max_over_ranks(e1.elapsed_time(e2), world, "cuda")
    # the gradient's reproducibility: the same run from starts moved by 1e-6 (relative, random),
    # i.e. how much of it is fixed by the objective rather than by rounding-level detail
    rng = np.random.default_rng(1)
    draws = []
    for _ in range(2):
        L.set_state((f0 * (1.0 + 1e-6 * rng.standard_normal(f0.shape))).astype(np.float32))
        Jk = L.adjoint_forward(nsteps)
        dthk, duk, _ = L.adjoint_backward()
        draws.append({"objective": Jk, "dJ_du_in": duk,
                      "dJ_dtheta_rel_change": float(np.linalg.norm(dthk - dth) / np.linalg.norm(dth))})
    K = int(np.ceil(np.sqrt(nsteps)))
    nstate = (nsteps + K - 1) // K + K + 3
    # reverse sweep per step and fluid node: recompute step (361 B) + adjoint step
    # (read f_t and lambda_{t+1}, write lambda_t: 3 x 180 B)
    rev_bytes = nf * (361 + 540) * nsteps
    peak, _ = measured_peaks()
    L.close()
    return {"value": round(whole_job_mlups(world, N, nsteps, t_f + t_b), 2), "unit": "MLUPS (forward+backward)",
            "workload": f"column96 (96^3, shell 6, porosity 0.5, u_in 0.004, k 2e-3), {nf} fluid, after 200 steps",
            "steps": nsteps, "checkpoint_every": K, "checkpoint_states": nstate,
            "ms_forward": round(t_f, 2), "ms_backward": round(t_b, 2), "objective": J,
            "dJ_du_in": du, "max_abs_dJ_dtheta_deg": float(np.abs(dth).max()),
            "starts_moved_by_1e-6": draws,
            "reverse_effective_gbs": round(rev_bytes / (t_b * 1e-3) / 1e9, 1),
            "reverse_frac_of_peak": round(rev_bytes / (t_b * 1e-3) / 1e9 / peak, 4)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
