#!/usr/bin/env python3
"""Throughput of the sparse-block-grid reaction-diffusion step on one B300.

Workload (default): the 256^3 tortuosity solve - a thresholded Gaussian
random field (correlation length 8, porosity 0.35), c = 1 / c = 0 held on the
x faces, D = 1, dt = 0.15, compensated-FP32 state (FP32 arithmetic, value =
hi + lo) with FP64 reductions.  One bench step = one check interval of the
steady-state solve: 128 forward-Euler steps plus the FP64 residual and flux
reduction that decides convergence.

Metric: active-voxel updates per second (GVox/s) = n_active * 128 * steps /
time.  `value` is measured with CUDA events on the stream the library uses,
inputs resident in HBM; `e2e` repeats the measurement through the public API
with the dense initial field uploaded from pinned host memory every step and
D_eff read back.  `roofline` reports the step kernel's algorithmic bytes
(16 B per active voxel: hi and lo read and written) per launch over its
average launch time, against the measured HBM copy bandwidth.

`--impl reference` times the FP64 dense CPU oracle on the host cores on the
same workload (a bounded number of steps per bench step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CHECK_EVERY = 128
BYTES_PER_VOXEL = {"f32": 8, "f32x2": 16, "f64": 16}
METRIC = "active-voxel updates/s per RD step (grf256 tortuosity solve)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sbg", choices=["sbg", "reference"])
    ap.add_argument("--n", type=int, default=256, help="box side")
    ap.add_argument("--block", type=int, default=4)
    ap.add_argument("--dtype", default="f32x2", choices=["f32", "f32x2", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def workload(n):
    from workloads import grf256
    phi, u0, phys = grf256(n=n)
    return phi, u0, phys


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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def cpu_baseline(phi, u0, phys, n_active, seconds, nsteps_hint=None):
    """The FP64 dense oracle as it stands, on the host cores, on a bounded
    number of steps of the same workload."""
    import oracle
    P = oracle.Problem(phi, phys)
    u = P.shape_state(u0)
    t0 = time.perf_counter()
    u = P.run(u, 1)
    one = time.perf_counter() - t0
    nsteps = nsteps_hint or max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    P.run(u, nsteps)
    dt = time.perf_counter() - t0
    return {"value": n_active * nsteps / dt / 1e9, "unit": "GVox/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d FP64 dense steps of the full %s box (all %d voxels visited per step)"
                      % (nsteps, "x".join(str(d) for d in phys.dims), int(np.prod(phys.dims)))}, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    phi, u0, phys = workload(args.n)
    import oracle
    P = oracle.Problem(phi, phys)
    n_active = int(P.active.sum())
    u = P.shape_state(u0)
    per_step = 2
    for _ in range(args.warmup):
        u = P.run(u, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = P.run(u, per_step)
    dt = time.perf_counter() - t0
    value = n_active * per_step * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GVox/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grf256 tortuosity solve (256^3 GRF, porosity 0.35)",
                       "box": list(phys.dims), "steps_per_bench_step": per_step},
            "cpu_baseline": {"value": value, "unit": "GVox/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "%d FP64 dense steps of the full box per bench step" % per_step},
            "e2e": {"value": value, "unit": "GVox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # CPU baseline first (before heavy GPU use; the oracle runs in this process's threads)
    phi, u0, phys = workload(args.n)
    from paper_2304_11165_b300 import Grid, State, make_params
    import paper_2304_11165_b300._abi as abi

    stream = torch.cuda.current_stream(dev)
    g = Grid(phi, block=args.block, stream=stream)
    n_active = g.n_active
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline(phi, u0, phys, n_active, args.cpu_seconds)

    st = State(g, 1, args.dtype)
    p = make_params(phys)
    u0_dev = torch.from_numpy(u0.astype(np.float32)).to(dev)
    st.set(u0_dev, stream=stream)

    def bench_step():
        st.step(p, CHECK_EVERY, stream=stream)
        return st.effective_D(p, stream=stream)

    for _ in range(args.warmup):
        bench_step()
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
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        st.step(p, CHECK_EVERY, stream=stream)
        ev[i][1].record(stream)
        st.effective_D(p, stream=stream)
    end.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    total_ms = start.elapsed_time(end)
    step_kernel_ms = sum(a.elapsed_time(b) for a, b in ev) / (args.steps * CHECK_EVERY)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    updates = n_active * CHECK_EVERY * args.steps * world
    value = updates / (total_ms / 1e3) / 1e9

    # end-to-end through the public API: dense field from pinned host memory every step
    u0_host = torch.from_numpy(u0.astype(np.float32)).pin_memory()
    st2 = State(g, 1, args.dtype)
    for _ in range(2):
        st2.set(u0_host, stream=stream)
        st2.step(p, CHECK_EVERY, stream=stream)
        st2.effective_D(p, stream=stream)
    torch.cuda.synchronize(dev)
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for _ in range(args.steps):
        st2.set(u0_host, stream=stream)
        st2.step(p, CHECK_EVERY, stream=stream)
        st2.effective_D(p, stream=stream)
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e_start.elapsed_time(e_end)
    e2e_value = n_active * CHECK_EVERY * args.steps * world / (e2e_ms / 1e3) / 1e9

    peak, peak_kind = load_peaks()
    algo_bytes = n_active * BYTES_PER_VOXEL[args.dtype]
    achieved = algo_bytes / (step_kernel_ms / 1e3) / 1e9
    d_eff, tau, psi = st.effective_D(p, stream=stream)
    kernel_name = "k_step_x2" if args.dtype == "f32x2" else "k_step"
    launches_per_step = CHECK_EVERY + 2
    line = {
        "metric": METRIC, "value": value, "unit": "GVox/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": "grf256 tortuosity solve: %d^3 GRF (correlation length 8, porosity 0.35), "
                               "c=1/c=0 on the x faces, D=1, dt=0.15" % args.n,
                   "block": args.block, "rd_steps_per_bench_step": CHECK_EVERY,
                   "n_active": n_active, "n_blocks": g.n_blocks, "porosity": psi,
                   "state_bytes": st.grid.info["n_blocks"] * args.block ** 3 * BYTES_PER_VOXEL[args.dtype] * 2,
                   "l2": "working set (two state buffers) larger than the 126 MB L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_us": step_kernel_ms * 1e3},
        "e2e": {"value": e2e_value, "unit": "GVox/s", "h2d_bytes_per_step": int(u0.size * 4),
                "d2h_bytes_per_step": abi.NRED * 8},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "result": {"D_eff_after_warmup_and_timed_steps": d_eff, "tau": tau},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
