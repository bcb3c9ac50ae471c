"""The hand-written adjoint (melbm_forward_checkpointed / melbm_backward) against
the oracle's FP64 discrete adjoint and FP64 central finite differences."""
import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05295_gb300 import melbm
    melbm.lib()
    return melbm


def cuda(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def gpu_grad(M, shape, tau, u0, F, g, nsteps, K, mask=None, inflow=None, outflow=False,
             lattice=27):
    sim = M.Simulator(shape, tau, "f32", lattice=lattice)
    if mask is not None:
        sim.set_solid(cuda(mask.ravel(), torch.uint8))
    if inflow is not None:
        sim.set_inflow(inflow[0], inflow[1:])
    if outflow:
        sim.set_outflow()
    if F is not None:
        sim.set_force(cuda(F))
    sim.forward_checkpointed(cuda(u0), nsteps, K)
    gu, gF = sim.backward(cuda(g), dL_dF=torch.empty(3, sim.N, device="cuda"))
    torch.cuda.synchronize()
    return gu.cpu().numpy().astype(np.float64), gF.cpu().numpy().astype(np.float64)


def rel(a, b, keep=None):
    if keep is not None:
        a, b = a[:, keep], b[:, keep]
    return np.abs(a - b).max() / np.abs(b).max()


def test_adjoint_matches_oracle_periodic_with_force(M, orc):
    shape = (20, 18, 14)
    N = int(np.prod(shape))
    rng = np.random.default_rng(30)
    u0 = W.flat(W.random_phase_field(shape, 0.05, kmax=4, seed=31))
    F = W.flat(W.force_field(shape, 1e-4, seed=32))
    g = rng.standard_normal((10, N))
    gu, gF = gpu_grad(M, shape, 0.55, u0, F, g, 6, 6)
    ou, oF = orc.adjoint(u0, F, shape, 0.55, 6, lambda m: g, K=6)
    assert rel(gu, ou) < 1e-4, rel(gu, ou)
    assert rel(gF, oF) < 1e-4, rel(gF, oF)


@pytest.mark.parametrize("shape", [(37, 29, 9), (4, 3, 5), (64, 15, 33)])
def test_adjoint_matches_oracle_periodic_without_force(M, orc, shape):
    """No body force (the force-free kernel); ragged tiles, grids smaller than one
    tile in every direction, several z-chunks."""
    N = int(np.prod(shape))
    rng = np.random.default_rng(40)
    u0 = 0.05 * rng.standard_normal((3, N))
    g = rng.standard_normal((10, N))
    gu, _ = gpu_grad(M, shape, 0.58, u0, None, g, 4, 4)
    ou, _ = orc.adjoint(u0, np.zeros((3, N)), shape, 0.58, 4, lambda m: g, K=4)
    assert rel(gu, ou) < 1e-4, rel(gu, ou)


def test_adjoint_matches_oracle_with_bounce_back_inflow_outflow(M, orc):
    shape = (24, 14, 12)
    N = int(np.prod(shape))
    mask = W.channel_walls(shape)
    mask[4:8, 5:9, 10:13] = 1
    typ, _, _, _ = orc.classify(mask, True, True)
    rng = np.random.default_rng(33)
    u0 = 0.02 * rng.standard_normal((3, N))
    u0[0] += 0.04
    F = W.flat(W.force_field(shape, 1e-4, seed=34))
    g = rng.standard_normal((10, N))
    inflow = [1.0, 0.04, 0.0, 0.0]
    gu, gF = gpu_grad(M, shape, 0.6, u0, F, g, 5, 5, mask=mask, inflow=inflow, outflow=True)
    ou, oF = orc.adjoint(u0, F, shape, 0.6, 5, lambda m: g, K=5, typ=typ, inflow=inflow)
    keep = typ != orc.SOLID
    assert rel(gu, ou, keep) < 1e-4, rel(gu, ou, keep)
    assert rel(gF, oF, keep) < 1e-4, rel(gF, oF, keep)


def test_checkpointed_adjoint_against_fp64_central_differences(M, orc):
    """Config adjoint128 scaled down (32^3, 40 steps, checkpoints every 10 stored
    16-bit): directional derivatives of the kinetic energy in a 8^3 subregion along
    16 seeded directions in (u0, F) match FP64 central differences of the oracle."""
    shape = (32, 32, 32)
    N = 32 ** 3
    tau, nsteps, K = 0.55, 40, 10
    u0 = W.flat(W.random_phase_field(shape, 0.05, kmax=8, seed=35))
    F = W.flat(W.force_field(shape, 1e-5, seed=36))
    z, y, x = np.mgrid[0:32, 0:32, 0:32]
    region = ((x >= 12) & (x < 20) & (y >= 12) & (y < 20) & (z >= 12) & (z < 20)).ravel()

    def loss(m):
        return 0.5 * (m[0] * (m[1:4] ** 2).sum(0))[region].sum()

    from paper_2602_05295_gb300.autograd import MELBMFunction, kinetic_energy_in_region
    sim = M.Simulator(shape, tau, "f32")
    u0_t = cuda(u0).requires_grad_(True)
    F_t = cuda(F).requires_grad_(True)
    m_T = MELBMFunction.apply(u0_t, F_t, sim, nsteps, K)
    L = kinetic_energy_in_region(m_T, cuda(region, torch.bool))
    L.backward()
    gu = u0_t.grad.cpu().numpy().astype(np.float64)
    gF = F_t.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(37)
    scale_u, scale_F = np.abs(u0).max(), np.abs(F).max()
    fds, ads = [], []
    for _ in range(16):
        vu = rng.standard_normal(u0.shape) * scale_u
        vF = rng.standard_normal(F.shape) * scale_F
        eps = 1e-4
        lp, _ = orc.forward_loss(u0 + eps * vu, F + eps * vF, shape, tau, nsteps, loss)
        lm, _ = orc.forward_loss(u0 - eps * vu, F - eps * vF, shape, tau, nsteps, loss)
        fds.append((lp - lm) / (2 * eps))
        ads.append((gu * vu).sum() + (gF * vF).sum())
    fds, ads = np.array(fds), np.array(ads)
    # A random direction can give a derivative far below the others, where a
    # per-direction relative error only measures that smallness; the errors are
    # taken against the set's scale: relative l2 over the 16 derivatives, and each
    # error against the largest derivative.
    assert np.linalg.norm(ads - fds) / np.linalg.norm(fds) < 1e-4
    assert np.abs(ads - fds).max() / np.abs(fds).max() < 1e-4


def test_adjoint128_full_size_directional_derivatives(M, orc):
    """Workload adjoint128 at full size: 128^3, tau = 0.55, 200 steps, 16-bit
    checkpoints every 20 steps, loss = kinetic energy in [48, 80)^3.  Two seeded
    directions in (u0, F) against FP64 central differences of the oracle (each
    oracle forward is 4e8 cell updates, so the 16-direction check runs at 32^3)."""
    from paper_2602_05295_gb300.autograd import MELBMFunction, kinetic_energy_in_region
    wl = W.ADJOINT128
    shape, tau, nsteps = wl.shape, wl.tau, wl.steps
    u0 = W.flat(W.random_phase_field(shape, 0.05))
    F = W.flat(W.force_field(shape, 1e-5))
    z, y, x = np.mgrid[0:128, 0:128, 0:128]
    region = ((x >= 48) & (x < 80) & (y >= 48) & (y < 80) & (z >= 48) & (z < 80)).ravel()

    def loss(m):
        return 0.5 * (m[0] * (m[1:4] ** 2).sum(0))[region].sum()

    sim = M.Simulator(shape, tau, "f32")
    u0_t = cuda(u0).requires_grad_(True)
    F_t = cuda(F).requires_grad_(True)
    L = kinetic_energy_in_region(MELBMFunction.apply(u0_t, F_t, sim, nsteps, 20),
                                 cuda(region, torch.bool))
    L.backward()
    gu = u0_t.grad.cpu().numpy().astype(np.float64)
    gF = F_t.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(38)
    fds, ads = [], []
    for _ in range(2):
        vu = rng.standard_normal(u0.shape) * np.abs(u0).max()
        vF = rng.standard_normal(F.shape) * np.abs(F).max()
        eps = 1e-4
        lp, _ = orc.forward_loss(u0 + eps * vu, F + eps * vF, shape, tau, nsteps, loss)
        lm, _ = orc.forward_loss(u0 - eps * vu, F - eps * vF, shape, tau, nsteps, loss)
        fds.append((lp - lm) / (2 * eps))
        ads.append((gu * vu).sum() + (gF * vF).sum())
    fds, ads = np.array(fds), np.array(ads)
    assert np.abs(ads - fds).max() / np.abs(fds).max() < 1e-4, (ads, fds)


@pytest.mark.parametrize("case", ["periodic", "channel"])
def test_d3q19_adjoint_against_fp64_central_differences(M, orc, case):
    """The adjoint on the D3Q19 lattice (its closure of the tensor moments
    transposed, bounce-back over its 19 directions): directional derivatives of a
    linear functional of the final state along 12 seeded directions in (u0, F)
    match FP64 central differences of the D3Q19 oracle."""
    shape = (22, 18, 14)
    N = int(np.prod(shape))
    tau, nsteps = 0.58, 6
    rng = np.random.default_rng(50)
    u0 = W.flat(W.random_phase_field(shape, 0.05, kmax=4, seed=51))
    F = W.flat(W.force_field(shape, 1e-4, seed=52))
    mask = typ = inflow = None
    if case == "channel":
        mask = W.channel_walls(shape)
        mask[5:8, 6:10, 9:12] = 1
        typ, _, _, _ = orc.classify(mask, True, True)
        inflow = [1.0, 0.03, 0.0, 0.0]
        F[:, typ == orc.SOLID] = 0
        keep = typ != orc.SOLID
    else:
        keep = np.ones(N, bool)
    g = rng.standard_normal((10, N)) * keep

    def loss(m):
        return (g * m).sum()

    gu, gF = gpu_grad(M, shape, tau, u0, F, g, nsteps, nsteps, mask=mask, inflow=inflow,
                      outflow=case == "channel", lattice=19)
    fds, ads = [], []
    for _ in range(12):
        vu = rng.standard_normal(u0.shape) * np.abs(u0).max() * keep
        vF = rng.standard_normal(F.shape) * np.abs(F).max() * keep
        eps = 1e-4
        lp, _ = orc.forward_loss(u0 + eps * vu, F + eps * vF, shape, tau, nsteps, loss, typ=typ,
                                 inflow=inflow, lattice=19)
        lm, _ = orc.forward_loss(u0 - eps * vu, F - eps * vF, shape, tau, nsteps, loss, typ=typ,
                                 inflow=inflow, lattice=19)
        fds.append((lp - lm) / (2 * eps))
        ads.append((gu * vu).sum() + (gF * vF).sum())
    fds, ads = np.array(fds), np.array(ads)
    assert np.linalg.norm(ads - fds) / np.linalg.norm(fds) < 1e-4, (ads, fds)
    assert np.abs(ads - fds).max() / np.abs(fds).max() < 1e-4
    # the D3Q27 adjoint of the same problem differs: the lattice matters
    gu27, _ = gpu_grad(M, shape, tau, u0, F, g, nsteps, nsteps, mask=mask, inflow=inflow,
                       outflow=case == "channel")
    assert np.abs(gu27 - gu).max() > 1e-3 * np.abs(gu).max()
