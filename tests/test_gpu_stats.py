"""Statistics of the full-length runs: the 256^3 decaying turbulence (1000 steps,
tau = 0.52), the 512x256x256 sphere channel (2000 steps) and the 1000x400x400
obstacle scene (1000 steps).

The flow is chaotic: the 16-bit and FP32 runs start from the same state but
their rounding differs, so pointwise agreement only holds early (the parity
tests check FP32 against the FP64 oracle pointwise at t <= 100).  Over the full
run the 16-bit form is compared with the FP32 form through what the
quantisation must not change: the kinetic-energy history (FP64 reductions,
within 1%), the shell-averaged energy spectrum E(k) for 1 <= k <= 16 (within 5%
per shell) and the total mass (drift within 1e-6).
"""
import numpy as np
import pytest
import torch

from paper_2602_05295_gb300 import melbm as M
from paper_2602_05295_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def shell_spectrum(u, shape, kmax=16):
    """E(k) = sum over |k| in [k - 1/2, k + 1/2) of |u_hat|^2 / 2 (per cell)."""
    nx, ny, nz = shape
    uu = u.reshape(3, nz, ny, nx).to(torch.float64)
    uh = torch.fft.fftn(uu, dim=(1, 2, 3)) / (nx * ny * nz)
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(0)
    kz = torch.fft.fftfreq(nz, d=1.0 / nz, device=u.device, dtype=torch.float64)
    ky = torch.fft.fftfreq(ny, d=1.0 / ny, device=u.device, dtype=torch.float64)
    kx = torch.fft.fftfreq(nx, d=1.0 / nx, device=u.device, dtype=torch.float64)
    kk = torch.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    shell = torch.round(kk).to(torch.int64).flatten()
    spec = torch.bincount(shell, weights=e.flatten(), minlength=kmax + 1)
    return spec[:kmax + 1].cpu().numpy()


def test_turbulence256_statistics_16bit_vs_fp32():
    wl = W.TURB256
    u0 = torch.from_numpy(W.flat(W.random_phase_field(wl.shape, 0.08)).astype(np.float32)).cuda()
    rho0 = torch.ones(wl.cells, device="cuda")
    ke, drift, spec = {}, {}, {}
    for storage in ("f32", "q16"):
        sim = M.Simulator(wl.shape, wl.tau, storage, seed=2602)
        sim.set_state(rho0, u0)
        m0, e0 = sim.reduce()
        curve = [e0]
        for _ in range(10):
            sim.step(100)
            m, e = sim.reduce()
            curve.append(e)
        ke[storage] = np.array(curve)
        drift[storage] = (m - m0) / m0
        _, u, _ = sim.get_moments()
        spec[storage] = shell_spectrum(u, wl.shape)
        sim.close()
    # the run decays: the comparison is not between two constant curves
    assert ke["f32"][-1] < 0.9 * ke["f32"][0]
    rel_ke = np.abs(ke["q16"] / ke["f32"] - 1.0)
    assert rel_ke.max() <= 0.01, rel_ke
    assert abs(drift["q16"]) <= 1e-6, drift
    k = np.arange(1, 17)
    rel_spec = np.abs(spec["q16"][k] / spec["f32"][k] - 1.0)
    assert rel_spec.max() <= 0.05, rel_spec


@pytest.mark.parametrize("name", ["channel512", "large1000"])
def test_full_length_channel_runs_16bit_vs_fp32(name):
    """The two channel workloads run to their full length (2000 / 1000 steps) in
    16-bit and in FP32 storage from the same start.  The wake behind the obstacles
    is unsteady, so the forms are compared through what the quantisation must not
    change: the kinetic-energy history (FP64 reductions every 100 steps, within
    1%), the total-mass history -- set by what the inflow brings in and the
    outflow lets out -- (within 1e-5 relative; the open boundaries respond to the
    rounding, so this is looser than the 1e-6 drift bound of a closed box), and the
    mass-flux profile Q(x) = sum over each plane of rho u_x at the end (within
    1e-3).  The 16-bit handle also holds at most 60% of the FP32 one's memory."""
    from paper_2602_05295_gb300 import configs as C
    rec = C.run_channel512_full(0) if name == "channel512" else C.run_large1000_full(0)
    ke = rec["ke_history"]["f32"]
    assert max(ke) > 1.02 * min(ke)  # the energy history is not flat
    assert rec["ke_rel_diff_max"] <= 0.01, rec["ke_rel_diff_max"]
    assert rec["mass_rel_diff_max"] <= 1e-5, rec["mass_rel_diff_max"]
    assert rec["flux_profile_rel_diff_max"] <= 1e-3, rec["flux_profile_rel_diff_max"]
    assert rec["memory_bytes"]["q16"] <= 0.6 * rec["memory_bytes"]["f32"], rec["memory_bytes"]
