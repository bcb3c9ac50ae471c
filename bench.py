"""Throughput of the moment-encoded LBM step on GB300 (one JSON line).

Workload (the metric's configuration): decaying turbulence on a 256^3 periodic
grid, tau = 0.52, seeded random-phase divergence-free field with k^-5/3 shell
energy for 1 <= |k| <= 16 scaled to max|u| = 0.08, rho = 1, S = u u.  A step is
one melbm_step(1): the fluid kernel over all cells (this workload has no
boundary list and no outflow plane).  The headline value is the 16-bit storage
form; the FP32-storage form is timed on the same GPU in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

For N > 1 the script runs under torchrun, one rank per GPU; every rank advances
its own 256^3 replica (the update has no data-path exchange here), timing is the
max over ranks and the value is the whole-job cell updates per second (weak
scaling).  --impl reference times the FP64 CPU oracle on a bounded slab of the
same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM peak, 16-bit vs FP32 moment storage on 1 GB300 at stated error"
BYTES_PER_CELL = {"q16": 40, "f32": 80, "q16_d3q19": 40}  # state read once + written once
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json: torch copy, read+write bytes)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (earlier GB300 copy measurement)"


def source_hash():
    h = hashlib.sha256()
    for f in ("fluid.cu", "fluid_kernel.cuh", "melbm_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2602_05295_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_record(storage):
    """The fluid kernel's committed ncu figures for this storage (DRAM bytes and
    warp instructions per 256^3 launch), or {} when the kernel source changed
    since the capture."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "fluid_traffic.json")))
        rec = t.get(storage)
        if rec and rec.get("source_hash") == source_hash():
            return rec
    except Exception:
        pass
    return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank].strip() if vis else str(local_rank)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        busy = sorted(sm)[len(sm) // 4:] or sm  # drop the idle tail before the region
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def turbulence_inputs():
    from paper_2602_05295_gb300 import workloads as W
    wl = W.TURB256
    u = W.random_phase_field(wl.shape, 0.08)
    return wl, W.flat(u).astype(np.float32)


def time_storage(torch, melbm, wl, u_np, storage, steps, warmup, clocks=None, lattice=27):
    N = wl.cells
    sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602, lattice=lattice)
    u = torch.from_numpy(u_np).cuda()
    rho = torch.ones(N, dtype=torch.float32, device="cuda")
    sim.set_state(rho, u)
    for _ in range(warmup):
        sim.step(1)
    st = sim.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(torch)
    torch.cuda.synchronize()
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        t0.record(st)
        for k in range(steps):
            ev[k][0].record(st)
            sim.step(1)
            ev[k][1].record(st)
        t1.record(st)
        torch.cuda.synchronize()
    barrier(torch)
    total_ms = t0.elapsed_time(t1)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    mem = sim.memory_bytes()
    sim.close()
    return total_ms, kern_ms, mem


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def barrier(torch):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(torch, v):
    """The maximum of v over the ranks (the slowest replica sets the job time)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return v


def job_mlups(cells_per_rank, steps, world, job_ms):
    """Whole-job throughput of weak-scaled replicas: the cell updates of all ranks
    over the job time (the maximum over ranks)."""
    return cells_per_rank * steps * world / (job_ms / 1e3) / 1e6


def e2e_raw_run(torch, melbm, wl, u_np, steps, warmup, pipelined=True):
    """End to end through the public API with host buffers, in the library's own
    state format: every step uploads the 16-bit stored state (20 B/cell) from
    pinned host memory, takes one step and reads the new stored state back into
    pinned host memory.  Pipelined: melbm_upload_raw_state_async /
    melbm_step / melbm_download_raw_state_async, so that a step's download runs
    beside the next step's upload (one sync at the end of the timed region);
    otherwise the blocking melbm_set_raw_state / melbm_get_raw_state."""
    N = wl.cells
    sim = melbm.Simulator(wl.shape, wl.tau, "q16", seed=2602)
    rho = torch.ones(N, dtype=torch.float32, device="cuda")
    sim.set_state(rho, torch.from_numpy(u_np).cuda())
    nb = sim.state_bytes()
    h_in = sim.get_raw_state(torch.empty(nb, dtype=torch.uint8).pin_memory())
    h_out = torch.empty(nb, dtype=torch.uint8).pin_memory()

    def one():
        if pipelined:
            sim.upload_raw_state_async(h_in, 0)
            sim.step(1)
            sim.download_raw_state_async(h_out)
        else:
            sim.set_raw_state(h_in, 0)
            sim.step(1)
            sim.get_raw_state(h_out)

    for _ in range(warmup):
        one()
    sim.sync_transfers()
    barrier(torch)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        one()
    sim.sync_transfers()
    torch.cuda.synchronize()
    el = max_over_ranks(torch, time.perf_counter() - t)
    sim.close()
    return el, nb, nb


def e2e_run(torch, melbm, wl, u_np, steps, warmup):
    """End to end through the public API with host buffers: every step uploads
    the full FP32 moment state from pinned host memory (melbm_set_state), takes
    one step and reads the moments back into pinned host memory."""
    N = wl.cells
    sim = melbm.Simulator(wl.shape, wl.tau, "q16", seed=2602)
    rho = torch.ones(N, dtype=torch.float32).pin_memory()
    u = torch.from_numpy(u_np).pin_memory()
    S = torch.empty(6, N, dtype=torch.float32)
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        S[k] = u[a] * u[b]
    S = S.pin_memory()
    orho = torch.empty(N, dtype=torch.float32).pin_memory()
    ou = torch.empty(3, N, dtype=torch.float32).pin_memory()
    oS = torch.empty(6, N, dtype=torch.float32).pin_memory()

    def one():
        sim.set_state(rho, u, S)
        sim.step(1)
        sim.get_moments(orho, ou, oS)

    for _ in range(warmup):
        one()
    barrier(torch)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    el = max_over_ranks(torch, time.perf_counter() - t)
    sim.close()
    return el, 40 * N, 40 * N


def channel_run(torch, melbm, steps, warmup):
    """The 512x256x256 sphere channel (300 spheres, walls, inflow u = (0.05, 0, 0),
    outflow; 16-bit storage): device time of `steps` steps (bounce kernel, fluid
    kernel with the boundary tables, inflow and outflow passes) after `warmup`."""
    from paper_2602_05295_gb300 import workloads as W
    wl = W.CHANNEL512
    N = wl.cells
    mask, _ = W.sphere_pack(wl.shape)
    sim = melbm.Simulator(wl.shape, wl.tau, "q16", seed=2602)
    u = torch.zeros(3, N, dtype=torch.float32, device="cuda")
    u[0] = 0.05
    sim.set_state(torch.ones(N, dtype=torch.float32, device="cuda"), u)
    sim.set_solid(torch.from_numpy(mask.ravel()).cuda())
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    cells, _ = sim.boundary_list()
    for _ in range(warmup):
        sim.step(1)
    st = sim.stream
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(torch)
    torch.cuda.synchronize()
    t0.record(st)
    for _ in range(steps):
        sim.step(1)
    t1.record(st)
    torch.cuda.synchronize()
    barrier(torch)
    total = t0.elapsed_time(t1)
    listed = int(cells.numel())
    mem = sim.memory_bytes()
    sim.close()
    return total, listed, mem


def cpu_oracle_run(steps=12, warmup=1, planes=128):
    """FP64 oracle on a 256 x 256 x `planes` periodic slab of the workload's field
    (about ten seconds on 16 cores)."""
    import oracle
    from paper_2602_05295_gb300 import workloads as W
    oracle.build()
    wl = W.TURB256
    nx, ny, _ = wl.shape
    u = W.random_phase_field(wl.shape, 0.08)[:, :planes]
    shape = (nx, ny, planes)
    uf = W.flat(u)
    m = oracle.initial_state_from_velocity(uf)
    cur = m
    for _ in range(warmup):
        cur = oracle.step(cur, shape, wl.tau)
    t = time.perf_counter()
    for _ in range(steps):
        cur = oracle.step(cur, shape, wl.tau)
    el = time.perf_counter() - t
    cells = nx * ny * planes
    out = {"value": cells * steps / el / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": f"{steps} FP64 oracle steps (after {warmup} warm-up) of a periodic "
                     f"{nx}x{ny}x{planes} slab of the 256^3 turbulence field ({cells} cells)"}
    # the same oracle on one thread, on a thinner slab
    threads = oracle.num_threads()
    p1, s1 = 8, 2
    m1 = oracle.initial_state_from_velocity(W.flat(u[:, :p1]))
    oracle.set_threads(1)
    try:
        m1 = oracle.step(m1, (nx, ny, p1), wl.tau)
        t1 = time.perf_counter()
        oracle.step(m1, (nx, ny, p1), wl.tau, n=s1)
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(threads)
    out["single_thread"] = {"value": nx * ny * p1 * s1 / el1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": f"{s1} FP64 oracle steps (after 1 warm-up) of a periodic "
                                      f"{nx}x{ny}x{p1} slab ({nx * ny * p1} cells)"}
    out["boundary_workloads"] = cpu_oracle_boundary_samples()
    return out, el


def cpu_oracle_boundary_samples():
    """The FP64 oracle on z-slabs of the two obstacle workloads (sphere channel,
    large procedural scene): its step with the cell types of the slab (solid,
    fluid-boundary, inflow, outflow) from the uniform inflow state."""
    import oracle
    from paper_2602_05295_gb300 import workloads as W
    res = []
    for wl, make, u_in, planes, steps in ((W.CHANNEL512, W.sphere_pack, 0.05, 16, 6),
                                          (W.LARGE1000, W.procedural_obstacle, 0.06, 8, 3)):
        nx, ny, nz = wl.shape
        mask, _ = make(wl.shape)
        z0 = nz // 2 - planes // 2
        slab = np.ascontiguousarray(mask[z0:z0 + planes])
        typ = oracle.classify(slab, True, True)[0]
        shape = (nx, ny, planes)
        u = np.zeros((3, nx * ny * planes))
        u[0] = u_in
        m = oracle.initial_state_from_velocity(u)
        inflow = [1.0, u_in, 0.0, 0.0]
        m = oracle.step(m, shape, wl.tau, typ=typ, inflow=inflow)
        t = time.perf_counter()
        oracle.step(m, shape, wl.tau, typ=typ, inflow=inflow, n=steps)
        el = time.perf_counter() - t
        cells = nx * ny * planes
        res.append({"workload": wl.name, "value": cells * steps / el / 1e6, "unit": "MLUPS",
                    "cores": oracle.num_threads(), "kind": "oracle",
                    "sample": f"{steps} FP64 oracle steps (after 1 warm-up) of planes "
                              f"{z0}..{z0 + planes - 1} of the {nx}x{ny}x{nz} grid "
                              f"({cells} cells, the slab periodic in z, inflow/outflow/solid "
                              f"types of the slab)"})
    return res


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    from paper_2602_05295_gb300 import workloads as W
    wl = W.TURB256
    planes = 16
    nx, ny, _ = wl.shape
    shape = (nx, ny, planes)
    u = W.flat(W.random_phase_field(wl.shape, 0.08)[:, :planes])
    cur = oracle.initial_state_from_velocity(u)
    for _ in range(args.warmup):
        cur = oracle.step(cur, shape, wl.tau)
    t = time.perf_counter()
    for _ in range(args.steps):
        cur = oracle.step(cur, shape, wl.tau)
    el = time.perf_counter() - t
    cells = nx * ny * planes
    v = cells * args.steps / el / 1e6
    sample = (f"each step: one FP64 oracle step of a periodic {nx}x{ny}x{planes} slab "
              f"({cells} cells) of the 256^3 turbulence field")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "turbulence256 slab (CPU oracle)", "tau": wl.tau},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2602_05295_gb300 import build, melbm
    build.build()
    melbm.lib()
    wl, u_np = turbulence_inputs()
    N = wl.cells
    peak, peak_src = hbm_peak()

    clocks = Clocks(local)
    q_total, q_kern, q_mem = time_storage(torch, melbm, wl, u_np, "q16", args.steps, args.warmup,
                                          clocks)
    q_total = max_over_ranks(torch, q_total)
    f_total, f_kern, f_mem = time_storage(torch, melbm, wl, u_np, "f32", args.steps, args.warmup)
    f_total = max_over_ranks(torch, f_total)
    # the same workload on the D3Q19 lattice (16-bit), a shorter run
    d_steps = max(3, min(args.steps, 200))
    d_total, d_kern, _ = time_storage(torch, melbm, wl, u_np, "q16", d_steps, args.warmup,
                                      lattice=19)
    d_total = max_over_ranks(torch, d_total)
    c_steps = max(3, min(args.steps, 200))
    c_total, c_listed, c_mem = channel_run(torch, melbm, c_steps, args.warmup)
    c_total = max_over_ranks(torch, c_total)

    clk = clocks.summary()
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    def roof(storage, kern_ms):
        avg_s = statistics.mean(kern_ms) / 1e3
        achieved = BYTES_PER_CELL[storage] * N / avg_s / 1e9
        rec = ncu_record(storage)
        out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": achieved / peak, "frac_of_nominal_8000": achieved / 8000.0,
               "traffic": rec.get("bytes_per_launch_256cube"), "peak_source": peak_src,
               "kernel": "fluid_kernel<q16, D3Q19>" if storage == "q16_d3q19"
               else f"fluid_kernel<{storage}>", "kernel_ms": avg_s * 1e3,
               "algorithmic_bytes_per_launch": BYTES_PER_CELL[storage] * N}
        inst, mhz = rec.get("warp_inst_per_launch_256cube"), clk.get("sm_mhz")
        if inst and mhz:
            # instruction-issue ceiling: one warp instruction per scheduler per cycle
            ipeak = sms * 4 * mhz * 1e6
            out["issue"] = {"achieved": inst / avg_s, "peak": ipeak, "unit": "warp inst/s",
                            "frac": inst / avg_s / ipeak, "warp_inst_per_launch": inst,
                            "peak_from": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (median sampled)"}
        return out

    value = job_mlups(N, args.steps, world, q_total)
    f_value = job_mlups(N, args.steps, world, f_total)
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": q_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "turbulence256: 256^3 periodic, tau=0.52, k^-5/3 random-phase "
                               "field max|u|=0.08, rho=1", "storage": "q16",
                   "l2": "inputs larger than L2 (state 335 MB q16 / 671 MB f32 > 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof("q16", q_kern),
        "fp32_storage": {"value": f_value, "unit": "MLUPS", "ms_per_step": f_total / args.steps,
                         "roofline": roof("f32", f_kern)},
        "d3q19_q16": {"value": job_mlups(N, d_steps, world, d_total), "unit": "MLUPS",
                      "steps": d_steps, "ms_per_step": d_total / d_steps,
                      "roofline": roof("q16_d3q19", d_kern)},
        "channel512_q16": {
            "value": job_mlups(512 * 256 * 256, c_steps, world, c_total), "unit": "MLUPS",
            "steps": c_steps, "ms_per_step": c_total / c_steps, "listed_cells": c_listed,
            "memory_bytes": c_mem,
            "workload": "512x256x256 channel, 300 seeded spheres (13.5% solid) and walls, "
                        "inflow u=(0.05,0,0), outflow, tau=0.55, 16-bit storage: bounce kernel, "
                        "fluid kernel with boundary tables, inflow and outflow passes per step"},
        "memory_bytes": {"q16": q_mem, "f32": f_mem},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if not args.no_e2e:
        ks = max(3, min(args.steps, 10))
        el, bi, bo = e2e_raw_run(torch, melbm, wl, u_np, ks, 3)
        out["e2e"] = {"value": N * ks * world / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi,
                      "d2h_bytes_per_step": bo,
                      "what": "per step: melbm_upload_raw_state_async from pinned host (the 16-bit "
                              "stored state), melbm_step(1), melbm_download_raw_state_async into "
                              "pinned host; one melbm_sync_transfers at the end"}
        el, bi, bo = e2e_raw_run(torch, melbm, wl, u_np, ks, 3, pipelined=False)
        out["e2e_serial"] = {
            "value": N * ks * world / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo,
            "what": "per step: melbm_set_raw_state, melbm_step(1), melbm_get_raw_state "
                    "(blocking), pinned host"}
        el, bi, bo = e2e_run(torch, melbm, wl, u_np, ks, 3)
        out["e2e_fp32_moments"] = {
            "value": N * ks * world / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo,
            "what": "per step: melbm_set_state from pinned host (FP32 rho,u,S), "
                    "melbm_step(1), melbm_get_moments into pinned host"}
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, _ = cpu_oracle_run()
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
