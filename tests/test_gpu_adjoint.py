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


def test_pipelined_recompute_with_boundaries_matches_oracle(M, orc):
    """Several checkpoint segments (8 steps, K = 3: three segments, so both segment
    buffers are used and each earlier segment is recomputed on the second stream
    beside the adjoint of the later one) in a walled channel with an obstacle,
    inflow, outflow and a body force: the gradients match the oracle's FP64 adjoint
    (whose checkpoints are exact; the 16-bit ones move the recomputed states by half
    a code step), and a second backward call on the same forward pass gives the
    same bits."""
    shape = (24, 14, 12)
    N = int(np.prod(shape))
    mask = W.channel_walls(shape)
    mask[4:8, 5:9, 10:13] = 1
    typ, _, _, _ = orc.classify(mask, True, True)
    rng = np.random.default_rng(43)
    u0 = 0.02 * rng.standard_normal((3, N))
    u0[0] += 0.04
    F = W.flat(W.force_field(shape, 1e-4, seed=44))
    g = rng.standard_normal((10, N))
    inflow = [1.0, 0.04, 0.0, 0.0]
    sim = M.Simulator(shape, 0.6, "f32")
    sim.set_solid(cuda(mask.ravel(), torch.uint8))
    sim.set_inflow(inflow[0], inflow[1:])
    sim.set_outflow()
    sim.set_force(cuda(F))
    sim.forward_checkpointed(cuda(u0), 8, 3)
    runs = []
    for _ in range(2):
        gu, gF = sim.backward(cuda(g), dL_dF=torch.empty(3, N, device="cuda"))
        torch.cuda.synchronize()
        runs.append((gu.cpu().numpy().astype(np.float64), gF.cpu().numpy().astype(np.float64)))
    sim.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    gu, gF = runs[0]
    ou, oF = orc.adjoint(u0, F, shape, 0.6, 8, lambda m: g, K=3, typ=typ, inflow=inflow)
    keep = typ != orc.SOLID
    assert rel(gu, ou, keep) < 1e-4, rel(gu, ou, keep)
    assert rel(gF, oF, keep) < 1e-4, rel(gF, oF, keep)


def test_checkpointed_adjoint_against_fp64_central_differences(M, orc):
    """Config adjoint128 scaled down (32^3, 40 steps): directional derivatives of
    the kinetic energy in a 8^3 subregion along 16 seeded directions in (u0, F)
    against FP64 central differences of the oracle, per direction.  With every
    FP32 state kept (K = 40, no recompute) each direction is within 1e-4 of its
    own derivative.  With 16-bit checkpoints every 10 steps the recomputed
    segments start from rounded states, which moves the linearisation point by up
    to half a code step; that shifts every directional derivative by up to ~1e-5
    of the largest one, so a direction whose derivative is far below the others
    meets 1e-4 of its own value plus that floor: |ad - fd| <= 1e-4 |fd| +
    1e-5 max|fd| (the stated bound of the checkpointed adjoint)."""
    shape = (32, 32, 32)
    tau, nsteps = 0.55, 40
    u0 = W.flat(W.random_phase_field(shape, 0.05, kmax=8, seed=35))
    F = W.flat(W.force_field(shape, 1e-5, seed=36))
    z, y, x = np.mgrid[0:32, 0:32, 0:32]
    region = ((x >= 12) & (x < 20) & (y >= 12) & (y < 20) & (z >= 12) & (z < 20)).ravel()

    def loss(m):
        return 0.5 * (m[0] * (m[1:4] ** 2).sum(0))[region].sum()

    from paper_2602_05295_gb300.autograd import MELBMFunction, kinetic_energy_in_region

    def grads(K):
        sim = M.Simulator(shape, tau, "f32")
        u0_t = cuda(u0).requires_grad_(True)
        F_t = cuda(F).requires_grad_(True)
        m_T = MELBMFunction.apply(u0_t, F_t, sim, nsteps, K)
        kinetic_energy_in_region(m_T, cuda(region, torch.bool)).backward()
        return u0_t.grad.cpu().numpy().astype(np.float64), F_t.grad.cpu().numpy().astype(np.float64)

    gu, gF = grads(10)
    gu_all, gF_all = grads(nsteps)
    rng = np.random.default_rng(37)
    scale_u, scale_F = np.abs(u0).max(), np.abs(F).max()
    fds, ads, ads_all = [], [], []
    for _ in range(16):
        vu = rng.standard_normal(u0.shape) * scale_u
        vF = rng.standard_normal(F.shape) * scale_F
        eps = 1e-4
        lp, _ = orc.forward_loss(u0 + eps * vu, F + eps * vF, shape, tau, nsteps, loss)
        lm, _ = orc.forward_loss(u0 - eps * vu, F - eps * vF, shape, tau, nsteps, loss)
        fds.append((lp - lm) / (2 * eps))
        ads.append((gu * vu).sum() + (gF * vF).sum())
        ads_all.append((gu_all * vu).sum() + (gF_all * vF).sum())
    fds, ads, ads_all = np.array(fds), np.array(ads), np.array(ads_all)
    rel_all = np.abs(ads_all - fds) / np.abs(fds)
    assert rel_all.max() < 1e-4, rel_all
    bound = 1e-4 * np.abs(fds) + 1e-5 * np.abs(fds).max()
    assert np.all(np.abs(ads - fds) <= bound), (np.abs(ads - fds) / np.abs(fds), fds)


def test_adjoint128_full_size_directional_derivatives(M):
    """Workload adjoint128 at its stated size: 128^3, tau = 0.55, 200 steps, 16-bit
    checkpoints every 20 steps, loss = kinetic energy in [48, 80)^3.  The gradient
    in (u0, F) along each of the 16 seeded directions matches the FP64 central
    difference of the oracle (tests/golden/adjoint128_fd.json, written by
    tests/golden/make_adjoint128_fd.py from the oracle alone) within 1e-4 of that
    direction's own derivative."""
    import json
    import os
    from paper_2602_05295_gb300.autograd import MELBMFunction, kinetic_energy_in_region
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "adjoint128_fd.json")))
    assert None not in gold["fd"], "the golden file is incomplete"
    wl = W.ADJOINT128
    shape, tau, nsteps = wl.shape, wl.tau, wl.steps
    assert list(shape) == gold["shape"] and tau == gold["tau"] and nsteps == gold["nsteps"]
    u0 = W.flat(W.random_phase_field(shape, 0.05))
    F = W.flat(W.force_field(shape, 1e-5))
    lo, hi = gold["region"]
    z, y, x = np.mgrid[0:128, 0:128, 0:128]
    region = ((x >= lo) & (x < hi) & (y >= lo) & (y < hi) & (z >= lo) & (z < hi)).ravel()
    sim = M.Simulator(shape, tau, "f32")
    u0_t = cuda(u0).requires_grad_(True)
    F_t = cuda(F).requires_grad_(True)
    L = kinetic_energy_in_region(MELBMFunction.apply(u0_t, F_t, sim, nsteps, 20),
                                 cuda(region, torch.bool))
    L.backward()
    gu = u0_t.grad.cpu().numpy().astype(np.float64)
    gF = F_t.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(gold["direction_seed"])
    su, sF = np.abs(u0).max(), np.abs(F).max()
    ads = []
    for _ in range(len(gold["fd"])):
        vu = rng.standard_normal(u0.shape) * su
        vF = rng.standard_normal(F.shape) * sF
        ads.append((gu * vu).sum() + (gF * vF).sum())
    ads, fds = np.array(ads), np.array(gold["fd"])
    rel = np.abs(ads - fds) / np.abs(fds)
    assert rel.max() < 1e-4, (rel, ads, fds)


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
