#!/usr/bin/env python3
"""Throughput of the sparse-block-grid reaction-diffusion step on one B300.

Default workload (`--workload reactive512`): the two-species reactive run
on a 512^3 Boolean packing of polydisperse spheres (pore fraction 0.40):
species A diffuses (D = 1) and reacts to B at the pore surface (Sec. 3.5's
surface sink, k = 0.05 times the smoothed delta weight of phi), B diffuses
(D = 0.5) and decays (0.001); FP32 state, FP64 checks.  One bench step is
one whole run: 2000 forward-Euler steps from the initial field with an FP64
mass/flux/min/max check of both species every 100 steps.

Metric: species-voxel updates per second (GVox/s) = 2 * n_active * 2000 *
runs / time.  `value` is measured with CUDA events on the stream the library
uses, inputs resident in HBM; each check is enqueued behind its steps
(sbg_reduce_async) and read on the host while the next steps run.  `e2e`
repeats the runs through the C ABI's host-pointer path (the initial fields
uploaded by sbg_state_set from page-locked host memory, the final fields read
back by sbg_state_get).  `roofline` reports the step kernel's algorithmic
bytes (16 B per active voxel, plus 4 B per slot of the blocks that hold
surface-band voxels) per launch over its average launch time, against the
measured HBM copy bandwidth.

`--workload grf256`: the 256^3 tortuosity solve (thresholded Gaussian random
field, porosity 0.35, c = 1 / c = 0 held on the x faces, SBG_F32R state); one
bench step = one check interval of 256 steps plus the residual and flux
check.  With `--converge` it runs the whole solve to R < 1e-8 and reports the
wall time, D_eff, tau and psi.

Other workloads print one JSON line each:
  --workload inhom512      inhomogeneous diffusion (Eq. 6 factor) from one face, 2000 steps (512^3)
  --workload frap256       simulated FRAP (bleached cube, pore and bulk recovery, D_eff fit) (256^3)
  --workload mms           the unit-disk manufactured solution of Sec. 3.1, 32^2..1024^2, errors and orders
  --workload redist512     Sussman redistancing of a 512^3 indicator on the device (200 iterations)
  --workload gradient256   checkpointed adjoint of 1000 steps (256^3): adjoint / forward time,
                           memory, FP64 central-difference checks (--fd)
  --workload batch64       64 uneven geometries: one batched launch per step vs per-geometry
                           launches (fixed steps; --converge: steady solves to 1e-6)

`--impl reference` times the FP64 dense CPU oracle on the host cores on the
same workload (a bounded number of steps per bench step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CHECK_EVERY = 256  # RD steps per check, the SBG_F32R refresh interval
REACT_CHECK_EVERY = 100  # RD steps between the FP64 mass/flux checks of a reactive run
# per active voxel and step: read and write the state; f32r reads the correction d and the source r
# and writes d
BYTES_PER_VOXEL = {"f32": 8, "f32x2": 16, "f64": 16, "f32r": 12}
METRIC = "active-voxel updates/s per RD step (grf256 tortuosity solve)"
KERNEL_SOURCES = ["paper_2304_11165_b300/csrc/sbg_step_pipe.cu", "paper_2304_11165_b300/csrc/sbg_step.cuh",
                  "paper_2304_11165_b300/csrc/sbg_ptx.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="bench steps (default: 5 whole runs for reactive512, 200 check intervals for grf256)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sbg", choices=["sbg", "reference"])
    ap.add_argument("--workload", default="reactive512",
                    choices=["grf256", "reactive512", "inhom512", "frap256", "mms", "redist512", "gradient256",
                             "batch64"])
    ap.add_argument("--n", type=int, default=None, help="box side (default: the workload's)")
    ap.add_argument("--block", type=int, default=4)
    ap.add_argument("--parallel", default="replicas", choices=["replicas", "slab"],
                    help="reactive512 with --gpus N > 1: N independent replicas (weak scaling) or one box cut "
                         "into N x-slabs with a ghost-plane exchange after every step (strong scaling)")
    ap.add_argument("--rd-steps", type=int, default=None,
                    help="reactive512: RD steps per run (default: the workload's 2000; smaller for profiling)")
    ap.add_argument("--dtype", default="f32r", choices=["f32", "f32x2", "f32r"])
    ap.add_argument("--variant", default=None,
                    choices=["auto", "plain", "pipelined", "prefetch", "async", "stream", "wave", "wave4"],
                    help="step kernel (default: stream for reactive512, grf256, inhom512 and frap256, async for the others)")
    ap.add_argument("--order", default=None, choices=["tiled", "planes"],
                    help="block order of the grid (default: planes for reactive512, tiled for the others)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--fd", action="store_true", help="gradient256: FP64 central differences")
    ap.add_argument("--converge", action="store_true",
                    help="grf256: the steady solve to 1e-8 (and 1e-10); batch64: steady solves to 1e-6")
    ap.add_argument("--sides", default="64,96,128,192,256", help="batch64: box sides")
    ap.add_argument("--count", type=int, default=64, help="batch64: number of geometries")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_sha(sources=None):
    h = hashlib.sha256()
    for p in sources or KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(name, sources=None):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    summary is missing or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    tb = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not sha or not tb or sha.group(1) != kernel_sha(sources):
        return None
    return int(tb.group(1))


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def _timed_steps(P, u, seconds):
    """(steps, seconds) of a bounded oracle run: one step to size it, then as
    many as fit in `seconds` (at least one)."""
    t0 = time.perf_counter()
    u = P.run(u, 1)
    one = time.perf_counter() - t0
    nsteps = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    P.run(u, nsteps)
    return nsteps, time.perf_counter() - t0


def _single_thread(P, u, seconds, nsteps=None):
    """The same oracle on one OpenMP thread (the process's OpenMP runtime is
    set to one thread for the run and restored after), or None when the
    runtime cannot be reached; `nsteps` fixes the number of steps instead of
    sizing the run to `seconds`."""
    import ctypes
    import oracle
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None
    n0 = oracle.num_threads()
    gomp.omp_set_num_threads(1)
    try:
        if oracle.num_threads() != 1:
            return None
        if nsteps:
            t0 = time.perf_counter()
            P.run(u, nsteps)
            return nsteps, time.perf_counter() - t0
        return _timed_steps(P, u, seconds)
    finally:
        gomp.omp_set_num_threads(n0)


def cpu_baseline(phi, u0, phys, n_active, seconds, single_thread_steps=None):
    """The FP64 dense oracle as it stands, on the host cores, on a bounded
    number of steps of the same workload; beside it the same oracle on one
    thread for a few seconds (or for exactly `single_thread_steps` steps)."""
    import oracle
    P = oracle.Problem(phi, phys)
    u = P.shape_state(u0)
    cores = oracle.num_threads()
    nsteps, dt = _timed_steps(P, u, seconds)
    updates = int(phys.nspecies) * n_active
    one = _single_thread(P, u, min(3.0, seconds / 4), single_thread_steps)
    return {"value": updates * nsteps / dt / 1e9, "unit": "GVox/s", "cores": cores,
            "kind": "oracle",
            "sample": "%d FP64 dense steps of the full %s box (all %d voxels visited per step)"
                      % (nsteps, "x".join(str(d) for d in phys.dims), int(np.prod(phys.dims))),
            "host_cpu_count": os.cpu_count(), "omp_num_threads_env": os.environ.get("OMP_NUM_THREADS"),
            "single_thread": None if one is None else
            {"value": updates * one[0] / one[1] / 1e9, "unit": "GVox/s", "steps": one[0]}}


NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e, NVIDIA's nominal figure (context beside the measured copy peak)


def roofline_extras(r):
    """Adds to an HBM roofline object the fraction of the nominal HBM
    bandwidth and, where an ncu traffic figure exists, the DRAM throughput it
    implies over the same event-timed launch."""
    if not r or r.get("bound") != "hbm" or r.get("achieved") is None:
        return r
    r["peak_nominal"] = NOMINAL_HBM_GBS
    r["frac_nominal"] = r["achieved"] / NOMINAL_HBM_GBS
    us = r.get("avg_launch_us")
    if r.get("traffic") and us:
        r["dram_gbs_from_traffic"] = r["traffic"] / (us * 1e-6) / 1e9
        r["dram_frac_from_traffic"] = r["dram_gbs_from_traffic"] / r["peak"]
    return r


def interval_stats(ms, steps_per_interval):
    """Mean and standard error of the per-interval stepping times (each
    interval: `steps_per_interval` RD steps, CUDA events on the stream), per
    RD step, as the paper reports its timings."""
    if not ms:
        return None
    per = [m / steps_per_interval for m in ms]
    mean = statistics.mean(per)
    se = statistics.stdev(per) / len(per) ** 0.5 if len(per) > 1 else None
    return {"n_intervals": len(per), "rd_steps_per_interval": steps_per_interval,
            "mean_us_per_rd_step": mean * 1e3, "stderr_us": None if se is None else se * 1e3}


def emit(line):
    if isinstance(line.get("roofline"), dict):
        roofline_extras(line["roofline"])
    print(json.dumps(line), flush=True)


def max_over_ranks(x, device=None):
    """The largest x over all ranks (a timed region's duration), or x itself
    without a process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, max_ms):
    """Whole-job throughput of `world` independent replicas: the units all
    ranks processed over the slowest rank's time, per second."""
    return units_per_rank * world / (max_ms / 1e3)


# ---------------------------------------------------------------------------
REACT_METRIC = "species-voxel updates/s (two-species reactive run, reactive512)"


def reactive_workload_name(n, phys, nsteps, per):
    return ("reactive512: %d^3 Boolean sphere packing (lognormal radii, median 12, sigma 0.3), "
            "pore fraction %.3f; A: D=1, surface reaction A->B k=0.05 in 0<phi<1; B: D=0.5, "
            "decay 0.001; A=1 for x<32; closed box; dt=%.6f (0.9 x limit); one bench step = "
            "one run of %d steps with an FP64 mass/flux/min/max check (no residual) every %d"
            % (n, phys.extra["pore_fraction"], phys.dt, nsteps, per))


def run_reference(args):
    """The reference arm: the FP64 dense oracle as it stands, on the host
    cores, on the same workload, metric and unit as the library's line; each
    bench step is a bounded sample (two dense steps of the whole box for
    reactive512, two for grf256)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload not in ("grf256", "reactive512"):
        emit({"impl": "reference", "unavailable": "the reference arm times the reactive512 and grf256 workloads"})
        return 0
    import oracle
    per_step = 2
    if args.workload == "reactive512":
        from workloads import reactive512
        n = args.n or 512
        phi, u0, phys = reactive512(n=n)
        metric, counted = REACT_METRIC, 2
        workload = reactive_workload_name(n, phys, phys.steps, REACT_CHECK_EVERY)
    else:
        from workloads import grf256
        phi, u0, phys = grf256(n=args.n or 256)
        metric, counted = METRIC, 1
        workload = "grf256 tortuosity solve (%d^3 GRF, porosity 0.35)" % phys.dims[0]
    P = oracle.Problem(phi, phys)
    n_active = int(P.active.sum())
    u = P.shape_state(u0)
    for _ in range(args.warmup):
        u = P.run(u, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = P.run(u, per_step)
    dt = time.perf_counter() - t0
    value = counted * n_active * per_step * args.steps / dt / 1e9
    sample = "%d FP64 dense steps of the full %s box per bench step" % (
        per_step, "x".join(str(d) for d in phys.dims))
    emit({"impl": "reference", "metric": metric, "value": value, "unit": "GVox/s",
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": workload, "box": list(phys.dims), "steps_per_bench_step": per_step},
          "cpu_baseline": {"value": value, "unit": "GVox/s", "cores": oracle.num_threads(), "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": "GVox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return 0


# ---------------------------------------------------------------------------
def run_grf256(args):
    if args.converge:
        return run_grf256_converge(args)
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    import paper_2304_11165_b300._abi as abi
    from workloads import grf256

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    n = args.n or 256
    phi, u0, phys = grf256(n=n)
    stream = torch.cuda.current_stream(dev)
    g = Grid(phi, block=args.block, stream=stream)
    n_active = g.n_active
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(phi, u0, phys, n_active, args.cpu_seconds)

    st = State(g, 1, args.dtype).set_kernel(args.variant)
    p = make_params(phys)
    st.set(torch.from_numpy(u0.astype(np.float32)).to(dev), stream=stream)
    for _ in range(args.warmup):
        st.step(p, CHECK_EVERY, stream=stream)
        st.effective_D(p, stream=stream)
    torch.cuda.synchronize(dev)

    # device-resident timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    # each interval's check (residual, fluxes, mass; for SBG_F32R also the refresh of r) is
    # enqueued behind its steps and read back while the next interval runs (the convergence
    # decision lags one interval, as a pipelined solver's does)
    red_buf = [torch.zeros(abi.NRED, dtype=torch.float64).pin_memory() for _ in range(2)]
    red_done = [torch.cuda.Event() for _ in range(2)]
    residuals = []
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        st.step(p, CHECK_EVERY, stream=stream)
        ev[i][1].record(stream)
        st.reduce_async(p, red_buf[i % 2], stream=stream)
        red_done[i % 2].record(stream)
        if i > 0:
            red_done[(i - 1) % 2].synchronize()
            residuals.append(st.parse_reduction(red_buf[(i - 1) % 2])[0]["residual"])
    end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = start.elapsed_time(end)
    interval_ms = [a.elapsed_time(b) for a, b in ev]  # the stepping of each bench step
    step_kernel_ms = sum(interval_ms) / (args.steps * CHECK_EVERY)
    total_ms = max_over_ranks(total_ms, dev)
    value = replica_throughput(n_active * CHECK_EVERY * args.steps, world, total_ms) / 1e9

    # end to end through the C ABI's host-pointer path: every bench step sets its dense input field
    # from page-locked host memory (sbg_state_set with on_device = 0: the library copies it to the
    # device and scatters it), steps, and reads its check into host memory
    u0_host = torch.from_numpy(u0.astype(np.float32)).pin_memory()
    st2 = State(g, 1, args.dtype).set_kernel(args.variant)
    e_buf = [torch.zeros(abi.NRED, dtype=torch.float64).pin_memory() for _ in range(2)]
    e_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_steps(n):
        for i in range(n):
            st2.set(u0_host, stream=stream)
            st2.step(p, CHECK_EVERY, stream=stream)
            st2.reduce_async(p, e_buf[i % 2], stream=stream)  # device -> host copy of the step's result
            e_done[i % 2].record(stream)
            if i > 0:
                e_done[(i - 1) % 2].synchronize()  # the previous step's result, read on the host
                st2.parse_reduction(e_buf[(i - 1) % 2])
        e_done[(n - 1) % 2].synchronize()

    e2e_steps(2)
    torch.cuda.synchronize(dev)
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    e2e_steps(args.steps)
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max_over_ranks(e_start.elapsed_time(e_end), dev)
    e2e_value = replica_throughput(n_active * CHECK_EVERY * args.steps, world, e2e_ms) / 1e9

    peak, peak_kind = load_peaks()
    algo_bytes = n_active * BYTES_PER_VOXEL[args.dtype]
    achieved = algo_bytes / (step_kernel_ms / 1e3) / 1e9
    d_eff, tau, psi = st.effective_D(p, stream=stream)
    if args.variant == "plain":
        kernel_name = "k_step_x2" if args.dtype == "f32x2" else "k_step"
    elif args.variant == "stream" and args.block == 4:
        kernel_name = "k_step_stream_x2" if args.dtype == "f32x2" else "k_step_stream"
    else:  # the two-rows-per-thread kernel: single-array modes, and SBG_F32X2 with cp.async halos
        rows2 = (args.dtype in ("f32", "f32r") and args.variant != "prefetch") or args.variant == "async"
        kernel_name = "k_step_rows2" if rows2 else "k_step_pipe"
    traffic = None
    if (n, args.block) == (256, 4):
        traffic = profile_traffic("%s_%s_%s_grf256.md" % (kernel_name, args.variant, args.dtype),
                                  step_kernel_sources(kernel_name))
    line = {
        "metric": METRIC, "value": value, "unit": "GVox/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": "grf256 tortuosity solve: %d^3 GRF (correlation length 8, porosity 0.35), "
                               "c=1/c=0 on the x faces, D=1, dt=0.15" % n,
                   "block": args.block, "kernel": args.variant, "rd_steps_per_bench_step": CHECK_EVERY,
                   "n_active": n_active, "n_blocks": g.n_blocks, "porosity": psi,
                   "step_working_set_bytes": g.n_blocks * args.block ** 3 * BYTES_PER_VOXEL[args.dtype],
                   "l2": ("one step reads and writes %.0f MB of %d-slot arrays: about the size of the 126 MB "
                          "L2, so part of the step is served from L2 (the roofline case is reactive512)"
                          % (g.n_blocks * args.block ** 3 * BYTES_PER_VOXEL[args.dtype] / 1e6,
                             g.n_blocks * args.block ** 3)),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_us": step_kernel_ms * 1e3},
        "e2e": {"value": e2e_value, "unit": "GVox/s", "h2d_bytes_per_step": int(u0.size * 4),
                "d2h_bytes_per_step": abi.NRED * 8},
        # per bench step: CHECK_EVERY step kernels (replayed 64-step graphs) and the check:
        # reduction, its final pass and (SBG_F32R) the fold of the correction
        "gpu_launches": (CHECK_EVERY + (3 if args.dtype == "f32r" else 2)) * args.steps,
        "clocks": clocks,
        "interval_stats": interval_stats(interval_ms, CHECK_EVERY),
        "result": {"note": "the state after warm-up and timed intervals is not converged; --converge runs "
                           "the solve to R < 1e-8",
                   "residual_first_last_timed_check": [residuals[0], residuals[-1]] if residuals else None},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        emit(line)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_grf256_converge(args):
    """The tortuosity workflow of Eq. 2 / Sec. 3.3 on grf256: the steady-state
    solve from the initial field to a relative residual below 1e-8 (the
    config's criterion), timed on the host clock around sbg_run_to_steady,
    then continued to 1e-10; D_eff, tau and psi at both points against the
    FP64 oracle's conjugate-gradient steady state stored in
    tests/golden/grf256_steady.json."""
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    from workloads import grf256
    torch.cuda.set_device(0)
    n = args.n or 256
    phi, u0, phys = grf256(n=n)
    stream = torch.cuda.current_stream()
    g = Grid(phi, block=args.block, stream=stream)
    p = make_params(phys)
    st = State(g, 1, args.dtype).set_kernel(args.variant)
    check = 2048
    cap = 4_000_000  # steps per phase (the solve to 1e-8 takes a few hundred thousand)
    st.set(u0.astype(np.float32), stream=stream)  # warm-up: graphs, clocks; then restart
    st.run_to_steady(p, 1e-3, check_every=check, max_steps=cap, stream=stream, raise_on_max=False)
    st.set(u0.astype(np.float32), stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    steps1, rel1 = st.run_to_steady(p, 1e-8, check_every=check, max_steps=cap, stream=stream, raise_on_max=False)
    torch.cuda.synchronize()
    wall1 = time.perf_counter() - t0
    d1, tau1, psi1 = st.effective_D(p, stream=stream)
    # the relative residual of a call is measured against the residual at its start: 1e-10 of
    # the initial residual is 1e-10 / rel1 of the residual where the first phase stopped
    t0 = time.perf_counter()
    steps2, rel2 = st.run_to_steady(p, 1e-10 / max(rel1, 1e-300), check_every=check, max_steps=cap,
                                    stream=stream, raise_on_max=False)
    rel2 *= rel1
    torch.cuda.synchronize()
    wall2 = time.perf_counter() - t0
    clocks = sampler.stop()
    d2, tau2, psi2 = st.effective_D(p, stream=stream)
    gold = None
    gpath = os.path.join(ROOT, "tests", "golden", "grf256_steady.json")
    if n == 256 and os.path.exists(gpath):
        gold = json.load(open(gpath))
    line = {"metric": "wall time of the tortuosity solve to R < 1e-8 (grf256)", "value": wall1, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "grf256 tortuosity solve: %d^3 GRF (correlation length 8, porosity 0.35), "
                                   "c=1/c=0 on the x faces, D=1, dt=0.15, check every %d steps" % (n, check),
                       "block": args.block, "kernel": args.variant, "n_active": g.n_active},
            "result": {"to_1e-8": {"steps": steps1, "rel_residual": rel1, "wall_s": wall1, "D_eff": d1,
                                   "tau": tau1, "psi": psi1,
                                   "gvox_s": g.n_active * steps1 / wall1 / 1e9},
                       "to_1e-10": {"extra_steps": steps2, "rel_residual": rel2, "extra_wall_s": wall2,
                                    "D_eff": d2, "tau": tau2, "psi": psi2}},
            "clocks": clocks}
    if gold is not None:
        line["result"]["oracle_cg"] = {"D_eff": gold["D_eff"], "tau": gold["tau"], "psi": gold["psi"],
                                       "cg_relres": gold["cg_relres"]}
        line["result"]["to_1e-8"]["D_eff_rel_err"] = abs(d1 - gold["D_eff"]) / gold["D_eff"]
        line["result"]["to_1e-10"]["D_eff_rel_err"] = abs(d2 - gold["D_eff"]) / gold["D_eff"]
    emit(line)
    return 0


def step_kernel_name(ns, variant):
    """The step kernel a state of `ns` FP32 species runs for a kernel variant."""
    if variant == "stream":
        return "k_step_stream"
    if variant in ("wave", "wave4"):
        return "k_step_wave"
    return two_array_kernel(variant) if ns == 2 else ("k_step" if variant == "plain" else "k_step_rows2")


STREAM_SOURCES = ["paper_2304_11165_b300/csrc/sbg_step_stream.cu", "paper_2304_11165_b300/csrc/sbg_row.cuh",
                  "paper_2304_11165_b300/csrc/sbg_step.cuh"]
WAVE_SOURCES = ["paper_2304_11165_b300/csrc/sbg_step_wave.cu", "paper_2304_11165_b300/csrc/sbg_row.cuh",
                "paper_2304_11165_b300/csrc/sbg_step.cuh", "paper_2304_11165_b300/csrc/sbg_ptx.cuh"]


def step_kernel_sources(kernel_name):
    """Source files whose hash keys a committed ncu summary of that kernel."""
    return {"k_step_stream": STREAM_SOURCES, "k_step_stream_inh": STREAM_SOURCES, "k_step_stream_x2": STREAM_SOURCES,
            "k_step_wave": WAVE_SOURCES}.get(kernel_name, KERNEL_SOURCES)


def steps_per_launch(variant):
    """RD steps one launch of the step kernel advances (the wavefront kernel runs
    2 or 4 steps per launch)."""
    return {"wave": 2, "wave4": 4}.get(variant, 1)


def two_array_kernel(variant):
    """Step kernel of the FP32 modes with two haloed arrays (two species; u and
    the diffusivity factor) for a kernel variant."""
    return {"plain": "k_step", "pipelined": "k_step_pipe", "prefetch": "k_step_pipe",
            "stream": "k_step_stream_inh"}.get(variant, "k_step_rows2")


# ---------------------------------------------------------------------------


def reactive_algo_bytes(n_active, n_band_blocks, block):
    """Algorithmic bytes of one two-species step: both species read and
    written (16 B per active voxel) plus the surface weight read in every
    slot of the blocks that hold surface-band voxels (4 B per slot)."""
    return 16 * n_active + 4 * n_band_blocks * block ** 3


def reactive_state_bytes(n_blocks, block):
    """Bytes one step kernel touches in HBM besides the weights: two species
    read from one buffer and written to the other, every slot of every block."""
    return 2 * 2 * 4 * n_blocks * block ** 3


def run_reactive512(args):
    """The default bench line: the two-species reactive run of Sec. 3.5's
    surface-sink model on the 512^3 Boolean sphere packing.  One bench step
    is one whole run: the state reset to the initial field, 2000 FTCS steps
    of A and B with the surface transfer and B's decay, and an FP64
    mass/flux/min/max check of both species every 100 steps (sbg_check_async:
    the reduction without the residual, which a transient run does not use;
    enqueued behind its steps and read on the host while the next 100 run).
    `value` counts species-voxel updates (two per active voxel and step) over
    the device time of K runs with every input resident in HBM; `e2e` repeats
    the runs through the C ABI's host-pointer path: the initial fields copied
    from page-locked host memory by sbg_state_set (on_device = 0), the checks
    read into host memory, and the final fields of both species copied back
    by sbg_state_get (on_device = 0)."""
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    import paper_2304_11165_b300._abi as abi
    from workloads import reactive512

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n or 512
    phi, u0, phys = reactive512(n=n)
    nsteps = args.rd_steps or phys.steps
    per = min(REACT_CHECK_EVERY, nsteps)
    nsteps -= nsteps % per
    stream = torch.cuda.current_stream(dev)
    t_build = time.perf_counter()
    g = Grid(phi, block=args.block, stream=stream, order=args.order)
    torch.cuda.synchronize(dev)
    build_ms = (time.perf_counter() - t_build) * 1e3
    p = make_params(phys)
    u0_f32 = np.ascontiguousarray(u0.astype(np.float32))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(phi, u0, phys, g.n_active, args.cpu_seconds, single_thread_steps=1)
    st0 = State(g, 2, "f32").set_all(torch.from_numpy(u0_f32).to(dev), stream=stream)
    st = State(g, 2, "f32").set_kernel(args.variant)
    red_buf = [torch.zeros(2 * abi.NRED, dtype=torch.float64).pin_memory() for _ in range(2)]
    red_done = [torch.cuda.Event() for _ in range(2)]

    def one_run(state, ev=None, set_from_host=None, get_to_host=None):
        """One whole reactive run; returns the masses read at its checks."""
        if set_from_host is None:
            state.copy_from(st0, stream=stream)
        else:
            for s in range(2):
                state.set(set_from_host[s], species=s, stream=stream)
        masses = []
        for i in range(nsteps // per):
            if ev is not None:
                ev[i][0].record(stream)
            state.step(p, per, stream=stream)
            if ev is not None:
                ev[i][1].record(stream)
            state.check_async(p, red_buf[i % 2], stream=stream)
            red_done[i % 2].record(stream)
            if i > 0:
                red_done[(i - 1) % 2].synchronize()
                r = state.parse_reduction(red_buf[(i - 1) % 2])
                masses.append((r[0]["mass"], r[1]["mass"]))
        last = nsteps // per - 1
        red_done[last % 2].synchronize()
        r = state.parse_reduction(red_buf[last % 2])
        masses.append((r[0]["mass"], r[1]["mass"]))
        if get_to_host is not None:
            for s in range(2):
                state.get(s, out=get_to_host[s], stream=stream)
        return masses

    for _ in range(args.warmup):
        one_run(st)
    torch.cuda.synchronize(dev)

    nint = nsteps // per
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nint)]
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    masses = None
    for k in range(args.steps):
        masses = one_run(st, ev[k])
    end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(start.elapsed_time(end), dev)
    interval_ms = [a.elapsed_time(b) for evk in ev for a, b in evk]
    per_launch_ms = sum(interval_ms) / (args.steps * nsteps)
    updates_per_run = 2 * g.n_active * nsteps
    value = replica_throughput(updates_per_run * args.steps, world, total_ms) / 1e9

    # end to end through the C ABI's host-pointer path
    host_in = [torch.from_numpy(u0_f32[s]).pin_memory() for s in range(2)]
    host_out = [torch.empty(u0_f32.shape[1:], dtype=torch.float32).pin_memory() for _ in range(2)]
    st_e = State(g, 2, "f32").set_kernel(args.variant)
    one_run(st_e, set_from_host=host_in, get_to_host=host_out)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for _ in range(args.steps):
        one_run(st_e, set_from_host=host_in, get_to_host=host_out)
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    e_wall_ms = (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(max(e_start.elapsed_time(e_end), e_wall_ms), dev)
    e2e_value = replica_throughput(updates_per_run * args.steps, world, e2e_ms) / 1e9
    # the e2e run's final fields against the device-resident run's (same kernels, same inputs)
    same_as_device_run = bool(np.array_equal(host_out[0].numpy(), st.get(0).astype(np.float32)) and
                              np.array_equal(host_out[1].numpy(), st.get(1).astype(np.float32)))

    peak, peak_kind = load_peaks()
    algo_bytes = reactive_algo_bytes(g.n_active, g.info["n_band_blocks"], args.block)
    spl = steps_per_launch(args.variant)
    # per_launch_ms is the mean time of one RD step; a launch of the wavefront kernel runs spl of them
    achieved = algo_bytes / (per_launch_ms / 1e3) / 1e9
    kernel_name = step_kernel_name(2, args.variant)
    launches_per_interval = per // spl + per % spl
    red0 = st0.reduce(p)
    line = {
        "metric": REACT_METRIC,
        "value": value, "unit": "GVox/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": reactive_workload_name(n, phys, nsteps, per),
                   "block": args.block, "kernel": args.variant, "order": args.order, "n_active": g.n_active,
                   "n_blocks": g.n_blocks, "n_band_blocks": g.info["n_band_blocks"], "build_ms": build_ms,
                   "step_working_set_bytes": reactive_state_bytes(g.n_blocks, args.block)
                   + 4 * g.info["n_band_blocks"] * args.block ** 3,
                   "l2": "each step reads %.0f MB and writes %.0f MB of state (plus the weights), far beyond the "
                         "126 MB L2; no flush needed" % (reactive_state_bytes(g.n_blocks, args.block) / 2e6,
                                                        reactive_state_bytes(g.n_blocks, args.block) / 2e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profile_traffic("%s_%s_f32_reactive512.md" % (kernel_name, args.variant),
                                                step_kernel_sources(kernel_name)) if n == 512 else None,
                     "algorithmic_bytes_per_launch": algo_bytes * spl, "avg_launch_us": per_launch_ms * 1e3 * spl,
                     "steps_per_launch": spl,
                     "algorithmic_bytes_rule": "per RD step: 16 B per active voxel (A and B read and written) + 4 B "
                                               "per slot of the blocks holding surface-band voxels (w read); a "
                                               "launch of the wavefront kernel runs steps_per_launch steps and "
                                               "moves the state through HBM once"},
        "e2e": {"value": e2e_value, "unit": "GVox/s", "h2d_bytes_per_step": int(u0_f32.nbytes),
                "d2h_bytes_per_step": int(u0_f32.nbytes) + nint * 2 * abi.NRED * 8,
                "path": "sbg_state_set / sbg_state_get with host pointers (page-locked), sbg_check_async "
                        "into page-locked host memory", "final_fields_equal_device_run": same_as_device_run},
        # per run: the state copy (memcpy, not a kernel), per check interval `per` step kernels and the
        # check (per species: reduction and final pass)
        "gpu_launches": args.steps * nint * (launches_per_interval + 2 * 2),
        "clocks": clocks,
        "interval_stats": interval_stats(interval_ms, per),
        "result": {"mass_A_B_initial": [red0[0]["mass"], red0[1]["mass"]], "mass_A_B_end": list(masses[-1]),
                   "A_plus_B_end_over_initial": (masses[-1][0] + masses[-1][1]) / (red0[0]["mass"] + red0[1]["mass"])},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        emit(line)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
def run_reactive512_slab(args):
    """The reactive run with the box cut into WORLD_SIZE x-slabs (one per rank
    and GPU), balanced by active blocks; after every step each rank sends its
    boundary planes to its neighbours over NCCL and writes theirs into its
    ghost planes; the FP64 checks every 100 steps are combined over the ranks.
    One bench step is one whole 2000-step run.  `value` counts the species-
    voxel updates of the whole box over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    from paper_2304_11165_b300 import slab as sl
    from workloads import reactive512
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    n = args.n or 512
    phi, u0, phys = reactive512(n=n)
    nsteps = args.rd_steps or phys.steps
    per = min(REACT_CHECK_EVERY, nsteps)
    nsteps -= nsteps % per
    bounds = sl.partition(phi, world, block=args.block)
    slab = sl.Slab.of(bounds, rank)
    comm = sl.TorchComm(device=dev)
    n_active = int((phi > np.float32(np.finfo(np.float32).eps)).sum())

    def one_run():
        eng = sl.LibraryEngine(slab, phi, phys, u0.astype(np.float32), dtype="f32", block=args.block,
                               order=args.order, variant=args.variant)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(nsteps // per):
            if world > 1:
                sl.run(slab, eng, comm, 2, per)
            else:
                eng.step(per)
            checks = sl.global_checks(slab, eng, comm, 2) if world > 1 else \
                [eng.checks(0), eng.checks(1)]
        t1.record()
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1), checks

    for _ in range(args.warmup):
        one_run()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ms = 0.0
    checks = None
    for _ in range(args.steps):
        m, checks = one_run()
        ms += m
    clocks = sampler.stop()
    ms = max_over_ranks(ms, dev if world > 1 else None)
    value = 2 * n_active * nsteps * args.steps / (ms / 1e3) / 1e9
    if rank == 0:
        emit({"metric": REACT_METRIC, "value": value, "unit": "GVox/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": reactive_workload_name(n, phys, nsteps, per), "block": args.block,
                         "kernel": args.variant, "order": args.order, "parallelism": "x-slabs",
                         "x_bounds": bounds.tolist(),
                         "exchange": "after every step: the first and last owned x planes of both species to the "
                                     "neighbour slabs (NCCL send/recv), written into their ghost planes"},
              "result": {"mass_A_B_end": [checks[0][_abi_red_mass()], checks[1][_abi_red_mass()]]},
              "clocks": clocks})
    if world > 1:
        dist.destroy_process_group()
    return 0


def _abi_red_mass():
    import paper_2304_11165_b300._abi as abi
    return abi.RED_MASS


# ---------------------------------------------------------------------------
def run_inhom512(args):
    """Inhomogeneous diffusion (Eq. 6 factor, face-mean fluxes) of a solute
    entering from the x = 0 face of the 512^3 packed bed: one FP32 species,
    2000 steps.  Algorithmic bytes: u read and written and the factor read,
    12 B per active voxel."""
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    from workloads import inhom512
    torch.cuda.set_device(0)
    n = args.n or 512
    phi, u0, phys, (d_min, d_max, g1, g2) = inhom512(n=n)
    stream = torch.cuda.current_stream()
    g = Grid(phi, block=args.block, stream=stream)
    g.set_diffusivity_sigmoid(phi, d_min, d_max, g1, g2, stream=stream)
    st = State(g, 1, "f32").set_kernel(args.variant).set(u0, stream=stream)
    p = make_params(phys)
    red0 = st.reduce(p)
    per = 100
    st.step(p, 3 * per, stream=stream)  # warm-up, then restart from the initial state
    st.set(u0, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ms = 0.0
    masses = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(phys.steps // per):
        a.record(stream)
        st.step(p, per, stream=stream)
        b.record(stream)
        red = st.reduce(p)  # synchronises
        kernel_ms += a.elapsed_time(b)
        masses.append(red[0]["mass"])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    updates = g.n_active * phys.steps
    peak, peak_kind = load_peaks()
    algo_bytes = g.n_active * 12
    per_launch_ms = kernel_ms / phys.steps
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        eps = oracle.eps_sigmoid(phi, d_min, d_max, g1, g2)
        P = oracle.Problem(phi, phys, eps=eps)
        u = P.shape_state(u0)
        t0 = time.perf_counter()
        u = P.run(u, 1)
        one = time.perf_counter() - t0
        nsteps = max(1, int(args.cpu_seconds / max(one, 1e-6)))
        t0 = time.perf_counter()
        P.run(u, nsteps)
        dt = time.perf_counter() - t0
        cpu = {"value": g.n_active * nsteps / dt / 1e9, "unit": "GVox/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "%d FP64 dense steps of the full %d^3 box" % (nsteps, n)}
    emit({"metric": "active-voxel updates/s (inhomogeneous diffusion, Eq. 6 factor)",
          "value": updates / (total_ms / 1e3) / 1e9, "unit": "GVox/s", "n_gpus": 1, "steps": phys.steps,
          "ms_per_step": total_ms / phys.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
          "config": {"workload": "inhom512: %d^3 Boolean sphere packing, pore fraction %.3f, D = eps(phi) from "
                                 "Eq. 6 (D_min 0, D_max 1, gamma2 4, gamma1 %.3g), c = 1 held on x = 0, %d steps"
                                 % (n, phys.extra["pore_fraction"], g1, phys.steps),
                     "block": args.block, "kernel": args.variant, "n_active": g.n_active, "n_blocks": g.n_blocks},
          "roofline": {"bound": "hbm", "kernel": two_array_kernel(args.variant),
                       "achieved": algo_bytes / (per_launch_ms / 1e3) / 1e9,
                       "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                       "frac": algo_bytes / (per_launch_ms / 1e3) / 1e9 / peak,
                       "traffic": profile_traffic("%s_%s_inhom512.md" % (two_array_kernel(args.variant), args.variant),
                                                  step_kernel_sources(two_array_kernel(args.variant))),
                       "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_us": per_launch_ms * 1e3},
          "result": {"mass_start": red0[0]["mass"], "mass_end": masses[-1]},
          "clocks": clocks, "cpu_baseline": cpu})
    return 0


# ---------------------------------------------------------------------------
def run_frap256(args):
    """Simulated FRAP (Sec. 3.3) in the grf256 geometry: the recovery of a
    bleached centred cube of edge 64 in the closed pore space and in the bulk
    box, 16384 steps each with the box mass recorded on the device every 128
    steps, then the least-squares time-scale fit for D_eff and tau.  One
    bench line for the whole estimate; the step kernel's algorithmic bytes
    are 12 B per active voxel (SBG_F32R: d and r read, d written), and its
    average launch time is taken over both curves (the 258 box sums between
    the steps included)."""
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    from paper_2304_11165_b300.api import frap_effective_D
    from paper_2304_11165_b300.frap import recovery
    from workloads import frap256
    torch.cuda.set_device(0)
    n = args.n or 256
    phi, u0, phys, lo, hi = frap256(n=n)
    sps, ns = phys.extra["steps_per_sample"], phys.extra["samples"]
    stream = torch.cuda.current_stream()
    p = make_params(phys)
    grids = [Grid(phi, block=args.block, stream=stream),
             Grid(np.full(phi.shape, 1.0e3, np.float32), block=args.block, stream=stream)]
    states = [State(g, 1, args.dtype).set_kernel(args.variant) for g in grids]
    for st in states:  # warm-up (graph capture, clocks), then restart from the bleached state
        st.set(u0, stream=stream)
        st.step(p, 3 * sps, stream=stream)
        st.set(u0, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t0 = time.perf_counter()
    ev[0].record(stream)
    t, F = recovery(states[0], p, lo, hi, sps, ns, stream=stream)
    ev[1].record(stream)
    _, Fb = recovery(states[1], p, lo, hi, sps, ns, stream=stream)
    ev[2].record(stream)
    d_eff, tau_frap, s, rss = frap_effective_D(t, F, t, Fb, float(phys.D[0]), 1e-3, 1.0)
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
    steps = sps * ns
    n_act = [g.n_active for g in grids]
    updates = sum(n_act) * steps
    peak, peak_kind = load_peaks()
    bpv = BYTES_PER_VOXEL[args.dtype]
    algo_bytes = [na * bpv for na in n_act]
    achieved = sum(algo_bytes) * steps / (sum(ms) / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(phi, u0, phys, n_act[0], args.cpu_seconds)
    emit({"metric": "active-voxel updates/s (simulated FRAP: pore and bulk recovery runs and fit)",
          "value": updates / wall / 1e9, "unit": "GVox/s", "n_gpus": 1, "steps": 2 * steps,
          "ms_per_step": wall * 1e3 / (2 * steps), "higher_is_better": True, "dtype": args.dtype,
          "data": "synthetic",
          "config": {"workload": "frap256: %d^3 GRF (correlation length 8, porosity 0.35), closed box, D = 1, "
                                 "dt = 0.15, bleached centred cube of edge %d, %d steps per curve, box mass "
                                 "every %d steps; bulk reference of the same box"
                                 % (n, phys.extra["side"], steps, sps),
                     "block": args.block, "kernel": args.variant, "n_active": n_act,
                     "timing": "host clock around both curves and the fit (each curve synchronises once)"},
          "roofline": {"bound": "hbm", "kernel": {"stream": "k_step_stream", "prefetch": "k_step_pipe",
                                                  "pipelined": "k_step_pipe"}.get(args.variant, "k_step_rows2"),
                       "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                       "frac": achieved / peak, "traffic": None,
                       "algorithmic_bytes_per_launch": algo_bytes,
                       "avg_launch_us": [m * 1e3 / steps for m in ms]},
          "result": {"D_eff": d_eff, "tau_frap": tau_frap, "scale": s, "rss": rss,
                     "F_end": [float(F[-1]), float(Fb[-1])], "curve_ms": ms},
          "clocks": clocks, "cpu_baseline": cpu})
    return 0


# ---------------------------------------------------------------------------
def run_mms(args):
    """The verification case of Sec. 3.1 (unit disk, no flux on r = 1, the
    appendix's manufactured source S(r) exp(-B t), dt = h^2/8, t = 0.025) on
    grids of 32^2 to 1024^2 in FP32 and FP64 through the external-source
    step: L2 and Linf errors against the exact solution and the observed
    orders.  `value` is the least-squares FP32 L2 order over all grids (the
    paper reports about 1.5 for its FP32 runs)."""
    import math
    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    from workloads import mms_disk
    torch.cuda.set_device(0)
    sizes = [32, 64, 128, 256, 512, 1024]
    table = {}
    total_ms = 0.0
    total_updates = 0
    for dtype in ("f32", "f64"):
        rows = []
        for n in sizes:
            phi, u0, S, r, phys, nsteps = mms_disk(n)
            B, t_end = phys.extra["B"], phys.extra["t_final"]
            fac = np.array([math.exp(-B * k * phys.dt) for k in range(nsteps)])
            g = Grid(phi, block=args.block)
            st = State(g, 1, dtype).set(u0).set_source(S)
            p = make_params(phys)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st.step_source(p, fac)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            u = st.get()[0]
            exact = (r ** 3 / 3 - r ** 4 / 4) * math.exp(-B * t_end)
            act = phi[0] > np.finfo(np.float32).eps
            e = u[act] - exact[act]
            rows.append({"n": n, "steps": nsteps, "l2": float(math.sqrt(np.mean(e ** 2))),
                         "linf": float(np.max(np.abs(e))), "ms": ms})
            total_ms += ms
            total_updates += int(act.sum()) * nsteps
            st.close()
            g.close()
        for i in range(1, len(rows)):
            rows[i]["order_l2"] = math.log(rows[i - 1]["l2"] / rows[i]["l2"], 2.0)
            rows[i]["order_linf"] = math.log(rows[i - 1]["linf"] / rows[i]["linf"], 2.0)
        table[dtype] = rows
    # least-squares slope of log2(L2 error) against log2(1/h) over all grids
    ln = np.log2(np.array(sizes, dtype=float))
    le = np.log2(np.array([r["l2"] for r in table["f32"]]))
    order = float(-np.polyfit(ln, le, 1)[0])
    emit({"metric": "L2 error order, unit-disk manufactured solution (Sec. 3.1)",
          "value": order, "unit": "order", "n_gpus": 1,
          "steps": sum(r["steps"] for r in table["f32"]), "higher_is_better": True, "dtype": "f32",
          "data": "synthetic",
          "config": {"workload": "mms_disk: unit disk in [-2, 2]^2, n^2 cell centres, n = 32..1024, D = 1, "
                                 "dt = h^2/8, t = 0.025, B = 20, exact SDF", "block": args.block,
                     "kernel": "plain (one launch per step: the source factor is a kernel argument)"},
          "result": table, "throughput_gvox_s": total_updates / (total_ms / 1e3) / 1e9})
    return 0


# ---------------------------------------------------------------------------
def run_redist512(args):
    """Sussman redistancing on the device of the binary indicator (+1 pore,
    -1 solid) of a 512^3 GRF pore space (correlation length 8, porosity
    0.35), FP32, 200 iterations at cfl 0.3 with the band test every 16.
    Metric: voxel updates per second.  Algorithmic bytes per iteration: the
    field read once and written once, 8 B per voxel (the neighbours come from
    L1/L2)."""
    import torch
    from paper_2304_11165_b300 import redistance
    from workloads import gaussian_random_field, threshold_to_porosity
    from workloads.configs import SEED_GRF256
    torch.cuda.set_device(0)
    n = args.n or 512
    iters = 200
    pore = threshold_to_porosity(gaussian_random_field((n, n, n), 8.0, SEED_GRF256), 0.35)
    ind_host = np.where(pore, 1.0, -1.0).astype(np.float32)
    ind = torch.from_numpy(ind_host).cuda()
    stream = torch.cuda.current_stream()
    redistance(ind, max_iter=3 * 16, stream=stream)  # warm-up
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    phi, it, res = redistance(ind, max_iter=iters, check_every=16, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = a.elapsed_time(b)
    nvox = n ** 3
    per_iter_ms = ms / it
    algo_bytes = 8 * nvox
    peak, peak_kind = load_peaks()
    achieved = algo_bytes / (per_iter_ms / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        oracle.sussman(ind_host, iters=1)
        dt = time.perf_counter() - t0
        cpu = {"value": nvox / dt / 1e9, "unit": "GVox/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one FP64 dense iteration of the full %d^3 field" % n}
    emit({"metric": "voxel updates/s (Sussman redistancing, FP32, dense on the device)",
          "value": nvox * it / (ms / 1e3) / 1e9, "unit": "GVox/s", "n_gpus": 1, "steps": it,
          "ms_per_step": per_iter_ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
          "config": {"workload": "redist512: indicator (+1 pore / -1 solid) of a %d^3 GRF (correlation length 8, "
                                 "porosity 0.35), cfl 0.3, %d iterations, band test every 16" % (n, iters),
                     "l2": "the 0.5 GB field pair exceeds the 126 MB L2"},
          "roofline": {"bound": "hbm", "kernel": "k_sussman", "achieved": achieved, "peak": peak,
                       "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                       "traffic": profile_traffic("k_sussman_redist512.md",
                                                  ["paper_2304_11165_b300/csrc/sbg_redistance.cu"]),
                       "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_us": per_iter_ms * 1e3},
          "result": {"iterations": it, "last_residual": res,
                     "phi_range": [float(phi.min().item()), float(phi.max().item())]},
          "clocks": clocks, "cpu_baseline": cpu})
    return 0


# ---------------------------------------------------------------------------
def run_gradient256(args):
    import dataclasses

    import torch
    from paper_2304_11165_b300 import Grid, State, make_params
    from paper_2304_11165_b300.autograd import adjoint, forward_record
    from workloads import gradient_setup
    torch.cuda.set_device(0)
    n = args.n or 256
    phi, u0, phys, x_cut = gradient_setup(n=n)
    nsteps, K = phys.steps, 64
    stream = torch.cuda.current_stream()
    torch.cuda.reset_peak_memory_stats()
    g = Grid(phi, block=args.block)
    p = make_params(phys)
    active = State(g, 1, "f32").set(np.ones(phi.shape, np.float32)).get() != 0
    slab = active.copy()
    slab[:, :, :x_cut + 1] = False
    lamN = np.where(slab, 1.0 / slab.sum(), 0.0)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    st = State(g, 1, "f32").set_kernel(args.variant).set(u0)
    st.step(p, 3 * 64)  # warm-up: module load, launch set-up, step-graph capture
    st.set(u0)
    _, fwd_ms = timed(lambda: st.step(p, nsteps))
    st.set(u0)
    tape, rec_ms = timed(lambda: forward_record(st, p, nsteps, K))
    loss = float((st.get() * lamN).sum())
    lam = State(g, 1, "f32").set(lamN)
    grad, adj_ms = timed(lambda: adjoint(tape, lam))
    lam0 = lam.get()
    lam.set(lamN)
    grad2, adj2_ms = timed(lambda: adjoint(tape, lam))  # second call: recompute buffer already allocated
    info = tape.info()
    mem = {"tape_bytes": info["device_bytes"], "grid_bytes": g.info["device_bytes"],
           "state_bytes": 3 * g.n_blocks * args.block ** 3 * 4 * 2,
           "torch_max_allocated": torch.cuda.max_memory_allocated()}
    mem["total_bytes"] = mem["tape_bytes"] + mem["grid_bytes"] + mem["state_bytes"] + mem["torch_max_allocated"]
    out = {"metric": "adjoint time / forward time (gradient of the outlet-slab mean, 1000 steps)",
           "value": adj2_ms / fwd_ms, "unit": "ratio", "higher_is_better": False, "n_gpus": 1,
           "dtype": "f32 state, f64 gradient sums", "data": "synthetic",
           "config": {"workload": "gradient256: %d^3 GRF geometry, A0=1, A=0 held on x=%d, surface sink k=0.05, "
                                  "%d steps, checkpoints every %d, loss = mean of A over pore voxels x > %d"
                                  % (n, n - 1, nsteps, K, x_cut),
                      "block": args.block, "n_active": g.n_active, "checkpoints": info["checkpoints"]},
           "times_ms": {"forward": fwd_ms, "forward_recording_checkpoints": rec_ms, "adjoint_first_call": adj_ms,
                        "adjoint": adj2_ms},
           "gvox_forward": g.n_active * nsteps / (fwd_ms / 1e3) / 1e9,
           "gvox_adjoint_incl_recompute": g.n_active * nsteps / (adj2_ms / 1e3) / 1e9,
           "memory": mem, "loss": loss,
           "gradient": {"dL_dD": grad[0], "dL_dk": grad[2], "repeat_equal": bool(np.array_equal(grad, grad2))}}
    if args.fd:
        def loss64(ph, u_init):
            s = State(g, 1, "f64").set(u_init)
            s.step(make_params(ph), nsteps)
            return float((s.get() * lamN).sum())
        fd = {}
        for name, base in (("D", phys.D[0]), ("k", phys.k_surf)):
            h = 1e-3 * base
            if name == "D":
                plus, minus = dataclasses.replace(phys, D=(base + h, 0.0)), dataclasses.replace(phys, D=(base - h, 0.0))
            else:
                plus, minus = dataclasses.replace(phys, k_surf=base + h), dataclasses.replace(phys, k_surf=base - h)
            val = (loss64(plus, u0) - loss64(minus, u0)) / (2 * h)
            gval = grad[0] if name == "D" else grad[2]
            fd[name] = {"fd_fp64": val, "adjoint_fp32": gval, "rel_diff": abs(gval - val) / abs(val)}
        rng = np.random.default_rng(5)
        v = rng.standard_normal(phi.shape) * (lam0 != 0)
        h = 1e-3
        dirv = (loss64(phys, u0 + h * v) - loss64(phys, u0 - h * v)) / (2 * h)
        ad = float((lam0 * v).sum())
        fd["c0_direction"] = {"fd_fp64": dirv, "adjoint_fp32": ad, "rel_diff": abs(ad - dirv) / abs(dirv)}
        out["finite_differences"] = fd
    emit(out)
    return 0


# ---------------------------------------------------------------------------
def run_batch64(args):
    import torch
    from paper_2304_11165_b300 import Grid, State, autotune, make_params
    from workloads import batch_geometries
    from workloads.configs import initial_with_faces
    torch.cuda.set_device(0)
    sides = tuple(int(s) for s in args.sides.split(","))
    t0 = time.time()
    geos = list(batch_geometries(count=args.count, sides=sides))
    gen_s = time.time() - t0
    phis = [phi for _, phi, _ in geos]
    phys0 = geos[0][2]
    p = make_params(phys0)
    best, table = autotune.tune(phis, phys0, args.dtype)
    B, variant, ctas = best["block"], best["variant"], best["ctas_per_sm"]
    stream = torch.cuda.current_stream()

    def init(state, gi, phys):
        state.set(initial_with_faces(phys.dims, 0.0, phys), geom=gi, stream=stream)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    nsteps = 1024
    gb = Grid.batch(phis, block=B)
    na, _, _ = gb.geometry_info()
    sb = State(gb, 1, args.dtype).set_kernel(variant, ctas)
    for gi, (_, _, ph) in enumerate(geos):
        init(sb, gi, ph)
    sb.step(p, 64)
    _, batch_ms = timed(lambda: sb.step(p, nsteps))
    seq = {}
    for kv in ("plain", variant):
        total = 0.0
        for gi, (_, phi, ph) in enumerate(geos):
            g1 = Grid(phi, block=B)
            s1 = State(g1, 1, args.dtype).set_kernel(kv, ctas if kv == variant else 0)
            init(s1, 0, ph)
            s1.step(p, 64)
            _, ms = timed(lambda: s1.step(p, nsteps))
            total += ms
            s1.close()
            g1.close()
        seq[kv] = total
    upd = float(na.sum()) * nsteps
    out = {"metric": "aggregate active-voxel updates/s, 64 uneven geometries (batched vs per-geometry launches)",
           "value": upd / (batch_ms / 1e3) / 1e9, "unit": "GVox/s", "higher_is_better": True, "n_gpus": 1,
           "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": "batch64: %d geometries, sides %s, spheres/GRF alternating, porosity U(0.2,0.6), "
                                  "tortuosity physics" % (len(geos), list(sides)),
                      "autotuned": best, "autotune_table": table, "n_active_total": int(na.sum()),
                      "box_voxels_total": int(sum(phi.size for phi in phis)), "generation_s": gen_s},
           "fixed_steps": {"steps": nsteps, "batched_ms": batch_ms,
                           "sequential_plain_ms": seq["plain"], "sequential_same_kernel_ms": seq[variant],
                           "gvox_batched": upd / (batch_ms / 1e3) / 1e9,
                           "gvox_sequential_plain": upd / (seq["plain"] / 1e3) / 1e9,
                           "gvox_sequential_same_kernel": upd / (seq[variant] / 1e3) / 1e9}}
    if args.converge:
        for gi, (_, _, ph) in enumerate(geos):
            init(sb, gi, ph)
        t = time.perf_counter()
        steps_b, rel_b = sb.batch_run_to_steady(p, 1e-6, check_every=512, max_steps=3_000_000, raise_on_max=False)
        torch.cuda.synchronize()
        wall_b = time.perf_counter() - t
        deff_b = [sb.effective_D(p, geom=gi)[0] for gi in range(len(geos))]
        t = time.perf_counter()
        steps_s, deff_s = [], []
        for gi, (_, phi, ph) in enumerate(geos):
            g1 = Grid(phi, block=B)
            s1 = State(g1, 1, args.dtype).set_kernel("plain")
            init(s1, 0, ph)
            st_, _ = s1.run_to_steady(p, 1e-6, check_every=512, max_steps=3_000_000, raise_on_max=False)
            steps_s.append(st_)
            deff_s.append(s1.effective_D(p)[0])
            s1.close()
            g1.close()
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t
        work_b = float(sum(int(na[i]) * int(steps_b[i]) for i in range(len(geos))))
        work_s = float(sum(int(na[i]) * int(steps_s[i]) for i in range(len(geos))))
        dd = [abs(a - b) / max(abs(b), 1e-30) for a, b in zip(deff_b, deff_s) if abs(b) > 1e-12]
        out["converge"] = {"tol": 1e-6, "batched_wall_s": wall_b, "sequential_plain_wall_s": wall_s,
                           "gvox_batched": work_b / wall_b / 1e9, "gvox_sequential_plain": work_s / wall_s / 1e9,
                           "max_rel_residual_batched": float(np.max(rel_b)),
                           "steps_min_max": [int(np.min(steps_b)), int(np.max(steps_b))],
                           "max_rel_diff_deff_batched_vs_sequential": max(dd) if dd else 0.0}
    emit(out)
    return 0


def main():
    args = parse()
    if args.variant is None:
        args.variant = "stream" if args.workload in ("reactive512", "grf256", "inhom512", "frap256") else "async"
    if args.order is None:
        args.order = "planes" if args.workload == "reactive512" else "tiled"
    if args.steps is None:
        args.steps = 200 if args.workload == "grf256" else 5
    if args.impl == "reference":
        return run_reference(args)
    if args.workload not in ("grf256", "reactive512") and int(os.environ.get("RANK", "0")) != 0:
        return 0
    if args.workload == "reactive512" and args.parallel == "slab":
        return run_reactive512_slab(args)
    return {"grf256": run_grf256, "reactive512": run_reactive512, "inhom512": run_inhom512,
            "frap256": run_frap256, "mms": run_mms, "redist512": run_redist512,
            "gradient256": run_gradient256, "batch64": run_batch64}[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
