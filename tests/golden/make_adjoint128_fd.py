"""Write tests/golden/adjoint128_fd.json: FP64 central differences of the oracle
for the adjoint workload at its full size.

Workload: 128^3 periodic grid, tau = 0.55, 200 steps, initial state
(rho = 1, u0, S = u0 u0) with u0 the seeded random-phase field (max |u| = 0.05)
and the seeded body force F (max |F| = 1e-5); loss L = sum over [48, 80)^3 of
rho |u|^2 / 2 of the final state.  For each of 16 seeded directions
v = (vu, vF) (standard normal, scaled by max|u0| and max|F|, drawn in order from
numpy's default_rng(38)) the derivative dL/dv is the central difference
(L(theta + eps v) - L(theta - eps v)) / (2 eps), eps = 1e-4, each L one FP64
oracle forward run.

Only the oracle and the seeded input generators are called; nothing of the CUDA
path.  Usage: ``python tests/golden/make_adjoint128_fd.py [--threads T]``.  The
file is rewritten after every direction, and directions already present are
kept, so an interrupted run resumes.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_05295_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "adjoint128_fd.json")
DIRECTION_SEED = 38
NDIR = 16
EPS = 1e-4
LO, HI = 48, 80


def problem():
    """(shape, tau, nsteps, u0, F, region, loss) of the adjoint workload."""
    wl = W.ADJOINT128
    shape, tau, nsteps = wl.shape, wl.tau, wl.steps
    u0 = W.flat(W.random_phase_field(shape, 0.05))
    F = W.flat(W.force_field(shape, 1e-5))
    nx, ny, nz = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    region = ((x >= LO) & (x < HI) & (y >= LO) & (y < HI) & (z >= LO) & (z < HI)).ravel()

    def loss(m):
        return 0.5 * (m[0] * (m[1:4] ** 2).sum(0))[region].sum()

    return shape, tau, nsteps, u0, F, region, loss


def directions(u0, F, n=NDIR):
    """The n seeded directions (vu, vF), in order."""
    rng = np.random.default_rng(DIRECTION_SEED)
    su, sF = np.abs(u0).max(), np.abs(F).max()
    for _ in range(n):
        vu = rng.standard_normal(u0.shape) * su
        vF = rng.standard_normal(F.shape) * sF
        yield vu, vF


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    if args.threads:
        oracle.set_threads(args.threads)
    shape, tau, nsteps, u0, F, region, loss = problem()
    rec = {}
    if os.path.exists(OUT):
        rec = json.load(open(OUT))
    rec.update({
        "about": "FP64 central differences of the oracle for the 128^3 adjoint workload; "
                 "written by tests/golden/make_adjoint128_fd.py (oracle only)",
        "shape": list(shape), "tau": tau, "nsteps": nsteps, "region": [LO, HI],
        "u0": "random_phase_field(shape, 0.05)", "F": "force_field(shape, 1e-5)",
        "direction_seed": DIRECTION_SEED, "eps": EPS,
    })
    rec.setdefault("fd", [None] * NDIR)
    rec.setdefault("loss_plus", [None] * NDIR)
    rec.setdefault("loss_minus", [None] * NDIR)
    for k, (vu, vF) in enumerate(directions(u0, F)):
        if rec["fd"][k] is not None:
            continue
        t0 = time.time()
        lp, _ = oracle.forward_loss(u0 + EPS * vu, F + EPS * vF, shape, tau, nsteps, loss)
        lm, _ = oracle.forward_loss(u0 - EPS * vu, F - EPS * vF, shape, tau, nsteps, loss)
        rec["fd"][k] = (lp - lm) / (2 * EPS)
        rec["loss_plus"][k], rec["loss_minus"][k] = lp, lm
        with open(OUT + ".tmp", "w") as f:
            json.dump(rec, f, indent=1)
        os.replace(OUT + ".tmp", OUT)
        print(f"direction {k}: fd = {rec['fd'][k]:.12e} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
