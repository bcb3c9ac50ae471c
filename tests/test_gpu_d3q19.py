"""The D3Q19 lattice on the GPU (Table 1's D3Q19 scene): the fluid kernel with the
19-velocity reconstruction (third-order terms projected on what the lattice
carries) and the boundary update over its 19 directions, against the FP64 D3Q19
oracle.

Tolerances as in the D3Q27 parity tests: FP32 storage <= 1e-5 (field-normalised)
after several steps; 16-bit storage <= 2e-3 of max|u| after 100 steps with the
total mass drift <= 1e-6; one 16-bit step code for code up to FP32-vs-FP64
rounding at a code boundary.
"""
import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05295_gb300 import melbm
    melbm.lib()
    return melbm


def to_gpu(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def eq_state(rho, u):
    m = np.zeros((10, u.shape[1]))
    m[0] = rho
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b]
    return m


def make(M, shape, tau, storage, m, seed=0):
    sim = M.Simulator(shape, tau, storage, seed=seed, lattice=19)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    return sim


def read(sim):
    rho, u, S = sim.get_moments()
    return np.concatenate([rho.cpu().numpy()[None], u.cpu().numpy(), S.cpu().numpy()]).astype(np.float64)


def errors(g, r):
    e_rho = np.abs(g[0] - r[0]).max()
    e_u = np.abs(g[1:4] - r[1:4]).max() / max(np.abs(r[1:4]).max(), 1e-30)
    e_s = np.abs(g[4:] - r[4:]).max() / max(np.abs(r[4:]).max(), 1e-30)
    return e_rho, e_u, e_s


@pytest.mark.parametrize("shape", [(37, 23, 19), (61, 15, 40), (64, 30, 12), (4, 4, 4), (1, 1, 1),
                                   (2, 3, 1), (65, 2, 3)])
def test_d3q19_random_state_fp32_matches_oracle(M, orc, shape):
    rng = np.random.default_rng(41)
    N = int(np.prod(shape))
    m = eq_state(1.0 + 0.01 * rng.standard_normal(N), 0.05 * rng.standard_normal((3, N)))
    m[4:] += 0.002 * rng.standard_normal((6, N))
    sim = make(M, shape, 0.57, "f32", m)
    sim.step(5)
    e = errors(read(sim), orc.step19(m, shape, 0.57, n=5))
    assert max(e) < 1e-5, e


def test_d3q19_differs_from_d3q27(M, orc):
    """The two lattices give different updates of the same state (the kernel did
    not fall back to the 27-velocity path): their difference is far above the
    FP32 tolerance, and the GPU follows the D3Q19 one."""
    shape = (32, 20, 12)
    rng = np.random.default_rng(42)
    N = int(np.prod(shape))
    m = eq_state(1.0 + 0.01 * rng.standard_normal(N), 0.08 * rng.standard_normal((3, N)))
    m[4:] += 0.01 * rng.standard_normal((6, N))
    sim = make(M, shape, 0.6, "f32", m)
    sim.step(1)
    g = read(sim)
    r19 = orc.step19(m, shape, 0.6)
    r27 = orc.step(m, shape, 0.6)
    assert errors(r27, r19)[2] > 100 * 1e-5
    assert max(errors(g, r19)) < 1e-5


def test_d3q19_force_fp32_matches_oracle(M, orc):
    shape = (40, 17, 12)
    u = W.random_phase_field(shape, 0.05, kmax=4, seed=3)
    m = eq_state(1.0, W.flat(u))
    F = W.flat(W.force_field(shape, 1e-4, seed=4))
    sim = make(M, shape, 0.55, "f32", m)
    sim.set_force(to_gpu(F))
    sim.step(20)
    e = errors(read(sim), orc.step19(m, shape, 0.55, F=F, n=20))
    assert max(e) < 1e-5, e


def test_d3q19_taylor_green_fp32_100_steps(M, orc):
    wl = W.TGV32
    u, _ = W.taylor_green(wl.shape, 0.05)
    m = eq_state(1.0, W.flat(u))
    sim = make(M, wl.shape, wl.tau, "f32", m)
    sim.step(wl.steps)
    e = errors(read(sim), orc.step19(m, wl.shape, wl.tau, n=wl.steps))
    assert max(e) < 1e-5, e


@pytest.mark.parametrize("bits", [(16, 16), (13, 12)])
def test_d3q19_q16_tracks_fp64_and_conserves_mass(M, orc, bits):
    shape = (64, 48, 40)
    u = W.random_phase_field(shape, 0.08, kmax=8, seed=6)
    m = eq_state(1.0, W.flat(u))
    sim = M.Simulator(shape, 0.52, "q16", seed=11, lattice=19)
    sim.set_bits(*bits)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    g0 = read(sim)
    M0, _ = sim.reduce()
    sim.step(100)
    g = read(sim)
    ref = orc.step19(g0, shape, 0.52, n=100)
    scale = 2.0 ** (16 - bits[0])
    e = errors(g, ref)
    assert e[1] < 2e-3 * scale, (bits, e)
    M1, _ = sim.reduce()
    assert abs(M1 - M0) / M0 < 1e-6 * scale


def test_d3q19_q16_one_step_codes_match_emulation(M, orc):
    shape = (45, 20, 18)
    u = W.random_phase_field(shape, 0.08, kmax=6, seed=7)
    m = eq_state(1.0, W.flat(u))
    sim = make(M, shape, 0.52, "q16", m, seed=5)
    codes0 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    sim.step(1)
    codes1 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    ref = orc.q16_step(codes0.astype(np.uint16), shape, 0.52, 1, 5, lattice=19).astype(np.int64)
    d = np.abs(codes1 - ref)
    assert d.max() <= 1
    assert (d > 0).mean() < 0.02


@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_d3q19_turbulence256_sampled_one_step(M, orc, storage):
    """At 256^3 (the launch configuration of the D3Q19 measurement), one GPU step
    agrees with the oracle's update of sampled cells from the GPU's own input."""
    wl = W.TURB256
    u = W.random_phase_field(wl.shape, 0.08)
    m = eq_state(1.0, W.flat(u)).astype(np.float32)
    sim = make(M, wl.shape, wl.tau, storage, m, seed=3)
    sim.step(3)
    g_in = read(sim)
    sim.step(1)
    g_out = read(sim)
    rng = np.random.default_rng(45)
    cells = np.concatenate([rng.integers(0, wl.cells, 4000), np.arange(0, 256),
                            np.arange(wl.cells - 300, wl.cells)])
    ref = orc.step19_cells(g_in, wl.shape, wl.tau, cells)
    got = g_out[:, cells]
    du = np.abs(got[1:4] - ref[1:4]).max()
    drho = np.abs(got[0] - ref[0]).max()
    if storage == "f32":
        assert du < 5e-7 and drho < 5e-7, (du, drho)
    else:
        assert du <= 0.8 / 65535 * 1.01 and drho <= 0.7 / 65535 * 1.01, (du, drho)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("q16", 2e-3)])
def test_d3q19_channel_with_obstacles_matches_oracle(M, orc, storage, tol):
    """Walls in y and z, two obstacles, inflow at x = 0 and outflow at x = nx-1, on
    the 19-velocity lattice: halfway bounce-back over its 19 directions."""
    shape = (48, 26, 22)
    nx, ny, nz = shape
    mask = W.channel_walls(shape)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    mask[(x - 18) ** 2 + (y - 12) ** 2 + (z - 10) ** 2 <= 25] = 1
    mask[(abs(x - 30) <= 2) & (abs(y - 15) <= 3) & (abs(z - 12) <= 2)] = 1
    typ, _, _, _ = orc.classify(mask, True, True)
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0] = 0.05
    m = eq_state(np.ones(N), u)
    F = W.flat(W.force_field(shape, 1e-5, seed=9))
    F[:, typ == orc.SOLID] = 0
    sim = make(M, shape, 0.55, storage, m, seed=9)
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    sim.set_force(to_gpu(F))
    assert np.array_equal(sim.types().cpu().numpy(), typ)
    g0 = read(sim)
    sim.step(100)
    g = read(sim)
    ref = orc.step19(g0, shape, 0.55, F=F, typ=typ, inflow=[1.0, 0.05, 0.0, 0.0], n=100)
    keep = typ != orc.SOLID
    e_u = np.abs(g[1:4][:, keep] - ref[1:4][:, keep]).max() / np.abs(ref[1:4][:, keep]).max()
    e_rho = np.abs(g[0][keep] - ref[0][keep]).max()
    assert e_u < tol and e_rho < tol, (e_u, e_rho)
    # the obstacles matter: the periodic D3Q19 update of the same state differs
    per = orc.step19(g0, shape, 0.55, F=F, n=100)
    assert np.abs(per[1:4][:, keep] - ref[1:4][:, keep]).max() > 0.2 * np.abs(ref[1:4][:, keep]).max()


def test_d3q19_q16_channel_one_step_codes_match_emulation(M, orc):
    shape = (40, 20, 18)
    nx, ny, nz = shape
    mask = W.channel_walls(shape)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    mask[(x - 15) ** 2 + (y - 10) ** 2 + (z - 9) ** 2 <= 16] = 1
    typ, _, _, _ = orc.classify(mask, True, True)
    u = W.random_phase_field(shape, 0.05, kmax=4, seed=12)
    m = eq_state(1.0, W.flat(u))
    sim = make(M, shape, 0.6, "q16", m, seed=4)
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.04, 0.0, 0.0))
    sim.set_outflow()
    codes0 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    sim.step(1)
    codes1 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    ref = orc.q16_step(codes0.astype(np.uint16), shape, 0.6, 1, 4, typ=typ,
                       inflow=[1.0, 0.04, 0.0, 0.0], lattice=19).astype(np.int64)
    keep = typ != orc.SOLID
    d = np.abs(codes1[:, keep] - ref[:, keep])
    assert d.max() <= 1
    assert (d > 0).mean() < 0.02


def test_d3q19_channel512_sampled_one_step(M, orc):
    """The full-size sphere channel on D3Q19 (16-bit): one GPU step against the
    oracle's D3Q19 update of sampled listed, inflow, outflow and fluid cells."""
    wl = W.CHANNEL512
    mask, _ = W.sphere_pack(wl.shape)
    N = wl.cells
    rng = np.random.default_rng(28)
    u = np.zeros((3, N), np.float32)
    u[0] = 0.05
    u += (0.01 * rng.standard_normal((3, N))).astype(np.float32)
    sim = M.Simulator(wl.shape, wl.tau, "q16", seed=8, lattice=19)
    sim.set_state(to_gpu(np.ones(N, np.float32)), to_gpu(u))
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    typ = sim.types().cpu().numpy()
    listed, _ = sim.boundary_list()
    listed = listed.cpu().numpy().astype(np.int64)
    sim.step(2)
    g_in = read(sim)
    sim.step(1)
    g_out = read(sim)
    cells = np.unique(np.concatenate([
        rng.choice(listed, 3000, replace=False), rng.integers(0, N, 2000),
        np.nonzero(typ == orc.INFLOW)[0][:300], np.nonzero(typ == orc.OUTFLOW)[0][:300]]))
    cells = cells[typ[cells] != orc.SOLID]
    ref = orc.step19_cells(g_in, wl.shape, wl.tau, cells, typ=typ, inflow=[1.0, 0.05, 0.0, 0.0])
    got = g_out[:, cells]
    du = np.abs(got[1:4] - ref[1:4]).max()
    drho = np.abs(got[0] - ref[0]).max()
    assert du <= 0.8 / 65535 * 1.01 and drho <= 0.7 / 65535 * 1.01, (du, drho)


def test_d3q19_refusals_and_recovery(M):
    shape = (16, 8, 8)
    N = 16 * 8 * 8
    with pytest.raises(M.MelbmError):
        M.Simulator(shape, 0.6, "f32", lattice=15)
    sim = M.Simulator(shape, 0.6, "f32", lattice=19)
    sim.set_wall_model(1)
    with pytest.raises(M.MelbmError):  # the adjoint covers halfway bounce-back only
        sim.forward_checkpointed(torch.zeros(3, N, device="cuda"), 4, 2)
    sim.set_wall_model(0)
    sim.set_solid(torch.zeros(N, dtype=torch.uint8, device="cuda"))
    sim.step(2)
    assert sim.time_index == 2
