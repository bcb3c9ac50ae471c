"""Run the five synthetic workloads on the GPU and print one JSON line each.

    python -m paper_2602_05295_gb300.configs [--only NAME] [--steps K]

For every workload: throughput (MLUPS over all cells, and over fluid cells where
solids exist), device memory of the 16-bit and FP32 forms, and a check that needs
no reference solution: the Taylor-Green decay rate (tgv32), total-mass drift
(FP64 reductions), boundary-list size and solid fraction (channel512, large1000),
gradient norms and timing of the checkpointed adjoint (adjoint128), and the
error-vs-bits sweep of the adaptive bit allocation on the turbulence field
(bits_sweep).
Timing uses CUDA events on the simulator's stream after warm-up steps.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time

import numpy as np
import torch

from . import melbm
from . import workloads as W


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed_steps(sim, steps, warmup=3):
    sim.step(warmup)
    a, b = _events()
    a.record(sim.stream)
    sim.step(steps)
    b.record(sim.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _state_from_velocity(u):
    return (torch.ones(u.shape[-1], dtype=torch.float32, device="cuda"),
            torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda())


def run_tgv32(steps):
    wl = W.TGV32
    u, k = W.taylor_green(wl.shape, 0.05)
    rho, ut = _state_from_velocity(W.flat(u))
    sim = melbm.Simulator(wl.shape, wl.tau, "f32")
    sim.set_state(rho, ut)
    nx, ny, nz = wl.shape
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    mode = (np.sin(k * x) * np.cos(k * y) * np.ones((nz, 1, 1))).ravel()
    amps, ts = [], []
    for t in range(0, wl.steps + 1, 10):
        if t:
            sim.step(10)
        if t >= 20:
            _, uu, _ = sim.get_moments()
            ux = uu[0].cpu().numpy().astype(np.float64)
            amps.append((ux * mode).sum() / (mode * mode).sum())
            ts.append(t)
    nu_fit = -np.polyfit(ts, np.log(amps), 1)[0] / (2 * k * k)
    nu = (wl.tau - 0.5) / 3.0
    ms = _timed_steps(sim, steps)
    return {"workload": wl.name, "storage": "f32", "cells": wl.cells, "ms_per_step": ms,
            "MLUPS": wl.cells / ms / 1e3, "nu_fit_over_nu": nu_fit / nu}


def run_turbulence256(steps):
    wl = W.TURB256
    rho, u = _state_from_velocity(W.flat(W.random_phase_field(wl.shape, 0.08)))
    out = []
    for storage in ("q16", "f32"):
        sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602)
        sim.set_state(rho, u)
        M0, E0 = sim.reduce()
        ms = _timed_steps(sim, steps)
        M1, E1 = sim.reduce()
        out.append({"workload": wl.name, "storage": storage, "cells": wl.cells, "ms_per_step": ms,
                    "MLUPS": wl.cells / ms / 1e3, "memory_bytes": sim.memory_bytes(),
                    "steps_run": steps + 3, "mass_drift": (M1 - M0) / M0, "ke_ratio": E1 / E0})
        sim.close()
    return out


def run_turbulence256_d3q19(steps):
    """The 256^3 turbulence workload on the D3Q19 lattice (same stored moments and
    storage forms; the 19-velocity reconstruction), beside the D3Q27 figures of
    run_turbulence256."""
    wl = W.TURB256
    rho, u = _state_from_velocity(W.flat(W.random_phase_field(wl.shape, 0.08)))
    out = []
    for storage in ("q16", "f32"):
        sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602, lattice=19)
        sim.set_state(rho, u)
        M0, E0 = sim.reduce()
        ms = _timed_steps(sim, steps)
        M1, E1 = sim.reduce()
        out.append({"workload": wl.name + "_d3q19", "storage": storage, "cells": wl.cells,
                    "ms_per_step": ms, "MLUPS": wl.cells / ms / 1e3,
                    "memory_bytes": sim.memory_bytes(), "steps_run": steps + 3,
                    "mass_drift": (M1 - M0) / M0, "ke_ratio": E1 / E0})
        sim.close()
    return out


def _channel(wl, mask, inflow_u, steps, storage="q16", lattice=27):
    sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602, lattice=lattice)
    N = wl.cells
    u = np.zeros((3, N), np.float32)
    u[0] = inflow_u
    rho, ut = _state_from_velocity(u)
    sim.set_state(rho, ut)
    mt = torch.from_numpy(mask.ravel()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_solid(mt)
    sim.set_inflow(1.0, (inflow_u, 0.0, 0.0))
    sim.set_outflow()
    cells, _ = sim.boundary_list()  # the first call that needs the list classifies
    torch.cuda.synchronize()
    classify_ms = 1e3 * (time.perf_counter() - t0)
    # the same classification again (its arrays are reused): the kernels and the
    # one host synchronisation that reads the list length
    sim.set_solid(mt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    count = ctypes.c_int64()
    rc = melbm.lib().melbm_get_boundary_list(sim._h, None, None, 0, ctypes.byref(count))
    reclassify_ms = 1e3 * (time.perf_counter() - t0)
    assert rc == melbm.OK and count.value == cells.numel()
    types = sim.types()
    fluid = int((types != melbm.SOLID).sum().item())
    M0, _ = sim.reduce()
    ms = _timed_steps(sim, steps)
    M1, E1 = sim.reduce()
    rec = {"workload": wl.name + ("_d3q19" if lattice == 19 else ""), "storage": storage,
           "cells": N, "fluid_cells": fluid,
           "solid_fraction": 1.0 - fluid / N, "boundary_list": int(cells.numel()),
           "classify_ms": classify_ms, "reclassify_ms": reclassify_ms, "ms_per_step": ms,
           "MLUPS": N / ms / 1e3,
           "fluid_MLUPS": fluid / ms / 1e3, "memory_bytes": sim.memory_bytes(),
           "mass_change_open_boundaries": (M1 - M0) / M0}
    sim.close()
    return rec


def run_channel512(steps):
    wl = W.CHANNEL512
    mask, spheres = W.sphere_pack(wl.shape)
    rec = _channel(wl, mask, 0.05, steps)
    rec["spheres"] = int(len(spheres))
    return rec


def run_channel512_d3q19(steps):
    """The sphere channel on the D3Q19 lattice (the paper runs one scene with solids
    on D3Q19): halfway bounce-back over its 19 directions."""
    wl = W.CHANNEL512
    mask, spheres = W.sphere_pack(wl.shape)
    rec = _channel(wl, mask, 0.05, steps, lattice=19)
    rec["spheres"] = int(len(spheres))
    return rec


def run_scene720_d3q19(steps):
    """A scene the size of the paper's D3Q19 scene (720 x 360 x 360, 93 M cells) with
    a procedural obstacle, on D3Q19 with 16-bit storage: the recompute design and
    the paper's mixed scheme, per-step time and memory."""
    wl = W.SCENE720
    mask, _ = W.scene720_obstacle(wl.shape)
    out = []
    for storage in ("q16", "mixed"):
        rec = _channel(wl, mask, 0.05, steps, storage=storage, lattice=19)
        rec["workload"] = wl.name
        out.append(rec)
    return out


def run_channel512_moving(steps):
    """The sphere channel with the moment-based wall model: every sphere (the first
    254) is a body spinning about its own centre (surface speed 0.01, axis z), the
    walls at rest; throughput and the time of one force-and-torque evaluation."""
    wl = W.CHANNEL512
    _, spheres = W.sphere_pack(wl.shape)
    body = W.sphere_bodies(wl.shape, spheres)
    N = wl.cells
    sim = melbm.Simulator(wl.shape, wl.tau, "q16", seed=2602)
    u = np.zeros((3, N), np.float32)
    u[0] = 0.05
    rho, ut = _state_from_velocity(u)
    sim.set_state(rho, ut)
    sim.set_solid(torch.from_numpy(body.ravel()).cuda())
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    sim.set_wall_model(1)
    for k, (cx, cy, cz, r) in enumerate(spheres[:254]):
        sim.set_body_motion(k + 1, (0, 0, 0), (0, 0, 0.01 / r), (cx, cy, cz))
    ms = _timed_steps(sim, steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ft = sim.solid_force(1)
    force_ms = 1e3 * (time.perf_counter() - t0)
    cells, _ = sim.boundary_list()
    rec = {"workload": "channel512_moving", "storage": "q16", "wall_model": "moment-based, 254 spinning spheres",
           "cells": N, "boundary_list": int(cells.numel()), "ms_per_step": ms, "MLUPS": N / ms / 1e3,
           "solid_force_ms": force_ms, "sphere1_force_torque": [float(v) for v in ft]}
    sim.close()
    return rec


def run_large1000(steps):
    """The 160 M-cell obstacle scene in both storage forms: throughput and the
    device memory each handle holds (melbm_memory_bytes)."""
    wl = W.LARGE1000
    mask, _ = W.procedural_obstacle(wl.shape)
    out = []
    for storage in ("q16", "f32"):
        out.append(_channel(wl, mask, 0.06, steps, storage=storage))
        torch.cuda.empty_cache()
    return out


def _flux_profile(sim, fluid, shape):
    """Q(x) = sum over the fluid cells of plane x of rho u_x (FP64), shape (nx,)."""
    nx, ny, nz = shape
    rho, u, _ = sim.get_moments()
    q = (rho.double() * u[0].double()) * fluid
    out = q.reshape(nz, ny, nx).sum((0, 1)).cpu().numpy()
    del rho, u
    return out


def _full_run(wl, mask, inflow_u, every=100):
    """The workload run to its full length in 16-bit and in FP32 storage from the
    same start (uniform inflow velocity, rho = 1): the FP64 mass and kinetic-energy
    histories every `every` steps, the mass-flux profile Q(x) at the end, the
    device memory of each handle and the MLUPS of the whole run (CUDA events around
    the steps only)."""
    N = wl.cells
    u = np.zeros((3, N), np.float32)
    u[0] = inflow_u
    rho, ut = _state_from_velocity(u)
    mt = torch.from_numpy(mask.ravel()).cuda()
    runs = {}
    for storage in ("q16", "f32"):
        sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602)
        sim.set_state(rho, ut)
        sim.set_solid(mt)
        sim.set_inflow(1.0, (inflow_u, 0.0, 0.0))
        sim.set_outflow()
        fluid = (sim.types() != melbm.SOLID).double()
        inlet_cells = int((sim.types().reshape(wl.shape[2], wl.shape[1], wl.shape[0])[:, :, 0]
                           == melbm.INFLOW).sum().item())
        M, E = [], []
        m0, e0 = sim.reduce()
        M.append(m0)
        E.append(e0)
        ms_total = 0.0
        for t in range(every, wl.steps + 1, every):
            a, b = _events()
            a.record(sim.stream)
            sim.step(every)
            b.record(sim.stream)
            torch.cuda.synchronize()
            ms_total += a.elapsed_time(b)
            m, e = sim.reduce()
            M.append(m)
            E.append(e)
        Q = _flux_profile(sim, fluid, wl.shape)
        runs[storage] = {"mass": np.array(M), "ke": np.array(E), "Q": Q,
                         "memory_bytes": sim.memory_bytes(), "ms_per_step": ms_total / wl.steps,
                         "inlet_cells": inlet_cells}
        sim.close()
        del fluid
        torch.cuda.empty_cache()
    q, f = runs["q16"], runs["f32"]
    nx = wl.shape[0]
    Q_in = 1.0 * inflow_u * f["inlet_cells"]
    inner = slice(1, nx - 1)
    rec = {"workload": wl.name + "_full", "steps": wl.steps, "cells": N,
           "record_every": every,
           "ke_rel_diff_max": float(np.abs(q["ke"] / f["ke"] - 1).max()),
           "ke_end_over_start": {s: float(r["ke"][-1] / r["ke"][0]) for s, r in runs.items()},
           "mass_change": {s: float((r["mass"][-1] - r["mass"][0]) / r["mass"][0])
                           for s, r in runs.items()},
           "mass_rel_diff_max": float(np.abs(q["mass"] / f["mass"] - 1).max()),
           "flux_inflow_prescribed": Q_in,
           "flux_mean_over_x": {s: float(r["Q"][inner].mean()) for s, r in runs.items()},
           "flux_spread_over_x": {s: float((r["Q"][inner].max() - r["Q"][inner].min())
                                           / r["Q"][inner].mean()) for s, r in runs.items()},
           "flux_profile_rel_diff_max": float(np.abs(q["Q"][inner] / f["Q"][inner] - 1).max()),
           "memory_bytes": {s: r["memory_bytes"] for s, r in runs.items()},
           "MLUPS": {s: N / r["ms_per_step"] / 1e3 for s, r in runs.items()},
           "ke_history": {s: [float(v) for v in r["ke"]] for s, r in runs.items()},
           "mass_history": {s: [float(v) for v in r["mass"]] for s, r in runs.items()}}
    return rec


def run_channel512_full(steps):
    """The sphere channel for its full 2000 steps, 16-bit against FP32 storage."""
    wl = W.CHANNEL512
    mask, _ = W.sphere_pack(wl.shape)
    return _full_run(wl, mask, 0.05)


def run_large1000_full(steps):
    """The 160 M-cell obstacle scene for its full 1000 steps, 16-bit against FP32
    storage, with the measured device memory of both handles."""
    wl = W.LARGE1000
    mask, _ = W.procedural_obstacle(wl.shape)
    return _full_run(wl, mask, 0.06)


def run_adjoint128(steps, K=20):
    from .autograd import MELBMFunction, kinetic_energy_in_region
    wl = W.ADJOINT128
    N = wl.cells
    u0 = torch.from_numpy(W.flat(W.random_phase_field(wl.shape, 0.05)).astype(np.float32)).cuda()
    F = torch.from_numpy(W.flat(W.force_field(wl.shape, 1e-5)).astype(np.float32)).cuda()
    z, y, x = np.mgrid[0:128, 0:128, 0:128]
    region = torch.from_numpy(((x >= 48) & (x < 80) & (y >= 48) & (y < 80) & (z >= 48)
                               & (z < 80)).ravel()).cuda()
    sim = melbm.Simulator(wl.shape, wl.tau, "f32")
    u0.requires_grad_(True)
    F.requires_grad_(True)
    times = []
    for _ in range(2):  # the first call also allocates the checkpoints and segment states
        u0.grad = F.grad = None
        a, b, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), \
            torch.cuda.Event(enable_timing=True)
        a.record()
        m = MELBMFunction.apply(u0, F, sim, wl.steps, K)
        L = kinetic_energy_in_region(m, region)
        b.record()
        L.backward()
        c.record()
        torch.cuda.synchronize()
        times.append((a.elapsed_time(b), b.elapsed_time(c)))
    storage = (f"f32 + 16-bit checkpoints (K={K})" if K < wl.steps
               else "f32, every state kept (no recompute)")
    return {"workload": wl.name + ("" if K < wl.steps else "_keep_all"), "storage": storage,
            "cells": N,
            "steps": wl.steps, "loss": float(L.item()), "forward_ms": times[1][0],
            "backward_ms": times[1][1], "first_call_forward_ms": times[0][0],
            "first_call_backward_ms": times[0][1], "grad_u0_norm": float(u0.grad.norm().item()),
            "grad_F_norm": float(F.grad.norm().item()), "memory_bytes": sim.memory_bytes()}


def run_adjoint128_keep_all(steps):
    """The same gradient with K = 200: one segment, every FP32 state kept on the
    device (200 x 84 MB), so the backward pass runs no recompute."""
    return run_adjoint128(steps, K=W.ADJOINT128.steps)


def run_mixed_vs_recompute(steps):
    """The paper's mixed-precision scheme (16-bit post-collision + FP32
    post-streaming, atomic solid correction, re-quantisation pass) against this
    library's recompute design (16-bit post-streaming ping-pong, boundary list
    recomputed from the input) on the periodic 256^3 turbulence and on the
    512x256x256 sphere channel (D3Q27 and D3Q19): throughput and device memory."""
    out = []
    wl = W.TURB256
    rho, u = _state_from_velocity(W.flat(W.random_phase_field(wl.shape, 0.08)))
    for storage in ("q16", "mixed"):
        sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602)
        sim.set_state(rho, u)
        ms = _timed_steps(sim, steps)
        out.append({"workload": "mixed_vs_recompute", "case": wl.name, "storage": storage,
                    "ms_per_step": ms, "MLUPS": wl.cells / ms / 1e3, "memory_bytes": sim.memory_bytes()})
        sim.close()
    wl = W.CHANNEL512
    mask, _ = W.sphere_pack(wl.shape)
    for lattice in (27, 19):
        for storage in ("q16", "mixed"):
            rec = _channel(wl, mask, 0.05, steps, storage=storage, lattice=lattice)
            out.append({"workload": "mixed_vs_recompute", "case": rec["workload"],
                        "storage": storage, "ms_per_step": rec["ms_per_step"],
                        "MLUPS": rec["MLUPS"], "memory_bytes": rec["memory_bytes"]})
    return out


def run_bits_sweep(steps):
    """Adaptive bit allocation b_rho_u / b_S (Sec. 6.2.2) on the 256^3 turbulence
    field: velocity error against the FP32-storage run after 100 steps (relative
    l2 and max over the field), mass drift, throughput, and the packed-equivalent
    bits per cell 4 b_rho_u + 6 b_S (the codes are kept in 16-bit halves)."""
    wl = W.TURB256
    rho, u = _state_from_velocity(W.flat(W.random_phase_field(wl.shape, 0.08)))
    T = 100

    def run(storage, bits=None):
        sim = melbm.Simulator(wl.shape, wl.tau, storage, seed=2602)
        if bits:
            sim.set_bits(*bits)
        sim.set_state(rho, u)
        M0, _ = sim.reduce()
        sim.step(T)
        M1, _ = sim.reduce()
        _, uu, _ = sim.get_moments()
        ms = _timed_steps(sim, steps)
        sim.close()
        return uu.double(), (M1 - M0) / M0, ms

    uref, _, ms_f = run("f32")
    out = [{"workload": "bits_sweep", "config": "fp32", "bits_per_cell": 320, "MLUPS": wl.cells / ms_f / 1e3}]
    nref = torch.linalg.vector_norm(uref).item()
    for bits in ((16, 16), (16, 15), (15, 14), (14, 13), (13, 12), (12, 11)):
        uq, drift, ms = run("q16", bits)
        d = uq - uref
        out.append({"workload": "bits_sweep", "config": f"{bits[0]}/{bits[1]}",
                    "bits_per_cell": 4 * bits[0] + 6 * bits[1], "steps": T,
                    "u_rel_l2_vs_fp32": torch.linalg.vector_norm(d).item() / nref,
                    "u_max_vs_fp32": d.abs().max().item() / uref.abs().max().item(),
                    "mass_drift": drift, "MLUPS": wl.cells / ms / 1e3})
    return out


RUNNERS = {"tgv32": run_tgv32, "turbulence256": run_turbulence256,
           "turbulence256_d3q19": run_turbulence256_d3q19, "channel512": run_channel512,
           "channel512_d3q19": run_channel512_d3q19, "scene720_d3q19": run_scene720_d3q19,
           "channel512_moving": run_channel512_moving, "large1000": run_large1000, "adjoint128": run_adjoint128,
           "adjoint128_keep_all": run_adjoint128_keep_all, "bits_sweep": run_bits_sweep,
           "mixed_vs_recompute": run_mixed_vs_recompute, "channel512_full": run_channel512_full,
           "large1000_full": run_large1000_full}
# run only when asked for by name (--only): each takes minutes
ON_REQUEST = {"channel512_full", "large1000_full"}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--only", default=None)
    p.add_argument("--steps", type=int, default=100)
    args = p.parse_args()
    melbm.lib()
    for name, fn in RUNNERS.items():
        if (args.only and name != args.only) or (not args.only and name in ON_REQUEST):
            continue
        recs = fn(args.steps)
        for r in (recs if isinstance(recs, list) else [recs]):
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
