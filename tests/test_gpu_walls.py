"""Solid coupling on the GPU (Sec. 3.2): the moment-based reconstruction at moving
walls and the momentum-exchange force and torque, against the FP64 oracle, on the
D3Q27 and the D3Q19 lattice.

Geometry: channel walls in y and z (body 2, at rest) and a box obstacle (body 1)
that translates and rotates (its geometry stays; only the wall velocity u^p at
each link's halfway point follows the rigid motion).
"""
import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
MOTION = {1: ([0.02, -0.01, 0.005], [0.0, 0.0, 0.002], [20.0, 10.0, 8.0]),
          2: ([0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])}


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05295_gb300 import melbm
    melbm.lib()
    return melbm


def to_gpu(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def geometry(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    body = np.zeros((nz, ny, nx), np.uint8)
    body[(y == 0) | (y == ny - 1) | (z == 0) | (z == nz - 1)] = 2
    body[(abs(x - 20) <= 3) & (abs(y - 10) <= 2) & (abs(z - 8) <= 3)] = 1
    return body.ravel()


def state(shape, seed=4):
    u = W.flat(W.random_phase_field(shape, 0.04, kmax=4, seed=seed))
    m = np.zeros((10, u.shape[1]))
    m[0] = 1.0
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b]
    return m


def make(M, shape, tau, storage, m, body, model=1, lattice=27):
    sim = M.Simulator(shape, tau, storage, seed=3, lattice=lattice)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    sim.set_solid(to_gpu(body, torch.uint8))
    sim.set_wall_model(model)
    for b, (V, Om, r0) in MOTION.items():
        sim.set_body_motion(b, V, Om, r0)
    return sim


def read(sim):
    rho, u, S = sim.get_moments()
    return np.concatenate([rho.cpu().numpy()[None], u.cpu().numpy(), S.cpu().numpy()]).astype(np.float64)


def ostep(orc, lattice):
    return orc.step19 if lattice == 19 else orc.step


@pytest.mark.parametrize("lattice", [27, 19])
@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("q16", 2e-3)])
def test_moving_walls_track_the_oracle(M, orc, storage, tol, lattice):
    shape = (40, 20, 16)
    body = geometry(shape)
    m = state(shape)
    sim = make(M, shape, 0.6, storage, m, body, lattice=lattice)
    g0 = read(sim)
    typ = sim.types().cpu().numpy()
    fluid = typ != orc.SOLID
    step = ostep(orc, lattice)
    ref = step(g0, shape, 0.6, typ=typ, wall=orc.Wall(1, body, MOTION), n=100)
    sim.step(100)
    g = read(sim)
    e_rho = np.abs(g[0] - ref[0])[fluid].max()
    e_u = np.abs(g[1:4] - ref[1:4])[:, fluid].max() / np.abs(ref[1:4])[:, fluid].max()
    assert e_u < tol and e_rho < tol, (e_rho, e_u)
    # the obstacle drags the fluid: the walls moved it away from the rest state
    bb = step(g0, shape, 0.6, typ=typ, wall=orc.Wall(0, body), n=100)
    assert np.abs(bb[1:4] - ref[1:4])[:, fluid].max() > 10 * tol


@pytest.mark.parametrize("lattice", [27, 19])
@pytest.mark.parametrize("model", [0, 1])
def test_solid_force_and_torque_match_the_oracle(M, orc, model, lattice):
    shape = (40, 20, 16)
    body = geometry(shape)
    m = state(shape, seed=5)
    F = 1e-5 * np.random.default_rng(6).standard_normal((3, m.shape[1]))
    sim = make(M, shape, 0.6, "f32", m, body, model, lattice=lattice)
    sim.set_force(to_gpu(F))
    sim.step(10)
    g = read(sim)
    typ = sim.types().cpu().numpy()
    wall = orc.Wall(model, body, MOTION)
    # each of the ~3e4 link terms (~0.1) carries the FP32 rounding of the
    # populations (~3e-7 relative); their random sum stays below ~1e-5 absolute
    # (x up to ~20 cells of lever arm for the torque)
    for b in (0, 1, 2):
        got = sim.solid_force(b)
        ref = orc.solid_force(g, shape, 0.6, typ, wall, F=F, body_id=b, lattice=lattice)
        assert np.abs(got[:3] - ref[:3]).max() < 1e-5 * np.abs(ref[:3]).max() + 5e-5, (model, b, got, ref)
        assert np.abs(got[3:] - ref[3:]).max() < 1e-5 * np.abs(ref[3:]).max() + 1e-3, (model, b, got, ref)


@pytest.mark.parametrize("lattice", [27, 19])
def test_momentum_exchange_identity_on_the_gpu(M, orc, lattice):
    """P(t+1) - P(t) = sum F - F_solid, with the FP32 state's rounding as the only error."""
    shape = (40, 20, 16)
    body = geometry(shape)
    m = state(shape, seed=7)
    F = 1e-5 * np.random.default_rng(8).standard_normal((3, m.shape[1]))
    sim = make(M, shape, 0.6, "f32", m, body, lattice=lattice)
    sim.set_force(to_gpu(F))
    typ = sim.types().cpu().numpy()
    fluid = typ != orc.SOLID
    g0 = read(sim)
    Fs = sim.solid_force(0)
    sim.step(1)
    g1 = read(sim)
    dP = (g1[0] * g1[1:4])[:, fluid].sum(1) - (g0[0] * g0[1:4])[:, fluid].sum(1)
    expect = F.astype(np.float32).astype(np.float64)[:, fluid].sum(1) - Fs[:3]
    assert np.abs(dP - expect).max() < 1e-3 * np.abs(Fs[:3]).max(), (dP, expect)


@pytest.mark.parametrize("lattice", [27, 19])
def test_comoving_walls_keep_uniform_flow(M, lattice):
    shape = (40, 20, 16)
    body = geometry(shape)
    N = body.size
    U = np.array([0.03, -0.01, 0.02])
    m = np.zeros((10, N))
    m[0] = 1.0
    m[1:4] = U[:, None]
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = U[a] * U[b]
    sim = M.Simulator(shape, 0.6, "f32", lattice=lattice)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    sim.set_solid(to_gpu(body, torch.uint8))
    sim.set_wall_model(1)
    sim.set_body_motion(1, U)
    sim.set_body_motion(2, U)
    sim.step(20)
    g = read(sim)
    fluid = sim.types().cpu().numpy() != 4
    assert np.abs(g[1:4][:, fluid] - U[:, None]).max() < 1e-6


def test_adjoint_refuses_the_moving_wall_model(M):
    sim = M.Simulator((8, 8, 8), 0.6, "f32")
    sim.set_wall_model(1)
    with pytest.raises(M.MelbmError):
        sim.forward_checkpointed(torch.zeros(3, 512, device="cuda"), 4, 2)
    with pytest.raises(M.MelbmError):
        sim.set_wall_model(2)
    with pytest.raises(M.MelbmError):
        sim.set_body_motion(0, (0, 0, 0))
