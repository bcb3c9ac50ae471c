"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Metrics (field-normalised, per group): density error is absolute (rho ~ 1);
velocity error is max_x |u_gpu - u_ref| / max_x |u_ref| over all three
components; stress error likewise over the six S components.  Solid cells are
excluded (their content is unspecified).  Tolerances: FP32 storage <= 1e-5
after 100 steps; 16-bit storage <= 2e-3 on velocity against FP64 with total
mass drift <= 1e-6; classification bit-exact; codec bit-exact.
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


def eq_state(rho, u):
    N = u.shape[1]
    m = np.zeros((10, N))
    m[0] = rho
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b]
    return m


def to_gpu(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def make_sim(M, shape, tau, storage, m, seed=0):
    sim = M.Simulator(shape, tau, storage, seed=seed)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    return sim


def read(sim):
    rho, u, S = sim.get_moments()
    torch.cuda.synchronize()
    return np.concatenate([rho.cpu().numpy()[None], u.cpu().numpy(), S.cpu().numpy()]).astype(np.float64)


def errors(g, r, keep=None):
    if keep is not None:
        g, r = g[:, keep], r[:, keep]
    e_rho = np.abs(g[0] - r[0]).max()
    e_u = np.abs(g[1:4] - r[1:4]).max() / max(np.abs(r[1:4]).max(), 1e-30)
    e_s = np.abs(g[4:] - r[4:]).max() / max(np.abs(r[4:]).max(), 1e-30)
    return e_rho, e_u, e_s


# ------------------------------------------------------------------ codec
def test_codec_bit_exact_against_oracle(M, orc):
    rng = np.random.default_rng(20)
    shape = (37, 11, 5)
    N = 37 * 11 * 5
    lo, hi = orc.ranges()
    v = (lo[:, None] - 0.05 * (hi - lo)[:, None]
         + 1.1 * (hi - lo)[:, None] * rng.uniform(size=(10, N))).astype(np.float32)
    v[:, 0] = np.nan
    v[:, 1] = lo
    v[:, 2] = hi
    v[:, 3] = -0.0
    v_orc = v.copy()
    v_orc[0] = v[0] - np.float32(1.0)  # the codec's density variable, exact in FP32
    for det in (True, False):
        for t, seed in ((0, 0), (17, 2602), (2 ** 31 + 5, 0xDEADBEEF)):
            words = M.q16_encode(to_gpu(v), shape, t, seed, deterministic=det)
            codes = M.words_to_codes(words).cpu().numpy()
            ref = orc.encode(v_orc, shape, t, seed, deterministic=det)
            assert np.array_equal(codes, ref.astype(np.int64)), (det, t, seed)
    dec = M.q16_decode(words).cpu().numpy().astype(np.float64)
    ref_dec = orc.decode(ref)
    assert np.abs(dec - ref_dec).max() <= 2e-7  # FP32 decode of rho = 1 + (rho - 1)


# ------------------------------------------------------------------ periodic fluid
def test_taylor_green_fp32_100_steps(M, orc):
    wl = W.TGV32
    u, k = W.taylor_green(wl.shape, 0.05)
    m = eq_state(1.0, W.flat(u))
    sim = make_sim(M, wl.shape, wl.tau, "f32", m)
    sim.step(wl.steps)
    g = read(sim)
    r = orc.step(m, wl.shape, wl.tau, n=wl.steps)
    e = errors(g, r)
    assert e[0] < 1e-5 and e[1] < 1e-5 and e[2] < 1e-5, e


@pytest.mark.parametrize("shape", [(37, 23, 19), (61, 15, 40), (30, 14, 33), (4, 4, 4), (1, 1, 1),
                                   (2, 3, 1), (65, 2, 3)])
def test_random_state_fp32_matches_oracle(M, orc, shape):
    rng = np.random.default_rng(21)
    N = int(np.prod(shape))
    m = eq_state(1.0 + 0.01 * rng.standard_normal(N), 0.05 * rng.standard_normal((3, N)))
    m[4:] += 0.002 * rng.standard_normal((6, N))
    sim = make_sim(M, shape, 0.57, "f32", m)
    sim.step(5)
    g = read(sim)
    r = orc.step(m, shape, 0.57, n=5)
    e = errors(g, r)
    assert max(e) < 1e-5, e


def test_force_fp32_matches_oracle(M, orc):
    shape = (40, 17, 12)
    N = int(np.prod(shape))
    rng = np.random.default_rng(22)
    u = W.random_phase_field(shape, 0.05, kmax=4, seed=3)
    m = eq_state(1.0, W.flat(u))
    F = W.flat(W.force_field(shape, 1e-4, seed=4))
    sim = make_sim(M, shape, 0.55, "f32", m)
    sim.set_force(to_gpu(F))
    sim.step(20)
    g = read(sim)
    r = orc.step(m, shape, 0.55, F=F, n=20)
    e = errors(g, r)
    assert max(e) < 1e-5, e


def test_q16_tracks_fp64_and_conserves_mass(M, orc):
    shape = (64, 48, 40)
    u = W.random_phase_field(shape, 0.08, kmax=8, seed=6)
    m = eq_state(1.0, W.flat(u))
    sim = make_sim(M, shape, 0.52, "q16", m, seed=11)
    g0 = read(sim)
    M0, _ = sim.reduce()
    ref = g0.copy()
    sim.step(100)
    g = read(sim)
    ref = orc.step(ref, shape, 0.52, n=100)
    e = errors(g, ref)
    assert e[1] < 2e-3, e
    M1, _ = sim.reduce()
    assert abs(M1 - M0) / M0 < 1e-6


def test_q16_one_step_codes_match_emulation(M, orc):
    """From identical codes, one GPU step and one oracle 16-bit step (same dither
    counter) agree code for code except where FP32 and FP64 round a value to
    opposite sides of a code boundary (|difference| <= 1)."""
    shape = (45, 20, 18)
    u = W.random_phase_field(shape, 0.08, kmax=6, seed=7)
    m = eq_state(1.0, W.flat(u))
    sim = make_sim(M, shape, 0.52, "q16", m, seed=5)
    raw0 = sim.get_raw_state().view(torch.int32).reshape(5, -1)
    codes0 = M.words_to_codes(raw0).cpu().numpy().astype(np.uint16)
    sim.step(1)
    codes1 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    ref = orc.q16_step(codes0, shape, 0.52, 1, 5).astype(np.int64)
    d = np.abs(codes1 - ref)
    assert d.max() <= 1
    assert (d > 0).mean() < 0.02


# ------------------------------------------------------------------ classification
@pytest.mark.parametrize("shape,dens,inflow,outflow", [
    ((33, 17, 9), 0.15, True, True), ((64, 8, 8), 0.02, False, True), ((5, 4, 3), 0.4, True, False),
    ((130, 31, 7), 0.3, False, False)])
def test_classification_bit_exact(M, orc, shape, dens, inflow, outflow):
    mask = W.random_mask(shape, dens, seed=sum(shape))
    sim = M.Simulator(shape, 0.6, "q16")
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    if inflow:
        sim.set_inflow(1.0, (0.05, 0, 0))
    if outflow:
        sim.set_outflow()
    cells, words = sim.boundary_list()
    types = sim.types().cpu().numpy()
    t, l, c, w = orc.classify(mask, inflow, outflow)
    assert np.array_equal(types, t)
    assert np.array_equal(cells.cpu().numpy().astype(np.uint32), c)
    assert np.array_equal(words.cpu().numpy().astype(np.uint32), w)


def test_classification_of_config_channel512_bit_exact(M, orc):
    mask, _ = W.sphere_pack(W.CHANNEL512.shape)
    sim = M.Simulator(W.CHANNEL512.shape, 0.55, "q16")
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.05, 0, 0))
    sim.set_outflow()
    cells, words = sim.boundary_list()
    t, l, c, w = orc.classify(mask, True, True)
    assert np.array_equal(cells.cpu().numpy().astype(np.uint32), c)
    assert np.array_equal(words.cpu().numpy().astype(np.uint32), w)
    assert np.array_equal(sim.types().cpu().numpy(), t)


@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_channel512_sampled_one_step(M, orc, storage):
    """At the full 512 x 256 x 256 sphere-channel size (the configuration the
    channel workload times), one GPU step agrees with the oracle's update of
    sampled cells -- listed boundary cells, inflow and outflow cells and plain
    fluid cells -- computed from the GPU's own input state."""
    wl = W.CHANNEL512
    mask, _ = W.sphere_pack(wl.shape)
    N = wl.cells
    rng = np.random.default_rng(27)
    u = np.zeros((3, N), np.float32)
    u[0] = 0.05
    u += (0.01 * rng.standard_normal((3, N))).astype(np.float32)
    sim = M.Simulator(wl.shape, wl.tau, storage, seed=8)
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
    nx = wl.shape[0]
    cells = np.unique(np.concatenate([
        rng.choice(listed, 3000, replace=False), rng.integers(0, N, 2000),
        np.nonzero(typ == orc.INFLOW)[0][:300], np.nonzero(typ == orc.OUTFLOW)[0][:300]]))
    cells = cells[typ[cells] != orc.SOLID]
    ref = orc.step_cells(g_in, wl.shape, wl.tau, cells, typ=typ, inflow=[1.0, 0.05, 0.0, 0.0])
    got = g_out[:, cells]
    du = np.abs(got[1:4] - ref[1:4]).max()
    drho = np.abs(got[0] - ref[0]).max()
    if storage == "f32":
        assert du < 5e-7 and drho < 5e-7, (du, drho)
    else:
        assert du <= 0.8 / 65535 * 1.01 and drho <= 0.7 / 65535 * 1.01, (du, drho)
    assert np.all(cells % nx < nx)


def test_large1000_sampled_one_step(M, orc):
    """The largest workload, 1000 x 400 x 400 (160 M cells, 16-bit, tau = 0.505)
    with its procedural obstacle, inflow and outflow: one GPU step against the
    oracle's update of sampled listed, inflow, outflow and fluid cells."""
    wl = W.LARGE1000
    mask, _ = W.procedural_obstacle(wl.shape)
    N = wl.cells
    rng = np.random.default_rng(29)
    sim = M.Simulator(wl.shape, wl.tau, "q16", seed=8)
    u = torch.zeros(3, N, device="cuda")
    u[0] = 0.06
    u += 0.01 * torch.randn(3, N, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    sim.set_state(torch.ones(N, device="cuda"), u)
    del u
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.06, 0.0, 0.0))
    sim.set_outflow()
    typ = sim.types().cpu().numpy()
    listed, _ = sim.boundary_list()
    listed = listed.cpu().numpy().astype(np.int64)
    sim.step(2)
    g_in = read(sim)
    sim.step(1)
    cells = np.unique(np.concatenate([
        rng.choice(listed, 3000, replace=False), rng.integers(0, N, 2000),
        np.nonzero(typ == orc.INFLOW)[0][:300], np.nonzero(typ == orc.OUTFLOW)[0][:300]]))
    cells = cells[typ[cells] != orc.SOLID]
    ref = orc.step_cells(g_in, wl.shape, wl.tau, cells, typ=typ, inflow=[1.0, 0.06, 0.0, 0.0])
    del g_in
    rho, uu, _ = sim.get_moments()
    idx = torch.from_numpy(cells).cuda()
    got_rho = rho[idx].double().cpu().numpy()
    got_u = uu[:, idx].double().cpu().numpy()
    du = np.abs(got_u - ref[1:4]).max()
    drho = np.abs(got_rho - ref[0]).max()
    assert du <= 0.8 / 65535 * 1.01 and drho <= 0.7 / 65535 * 1.01, (du, drho)


# ------------------------------------------------------------------ boundaries
def _channel_case(shape=(48, 26, 22)):
    nx, ny, nz = shape
    mask = W.channel_walls(shape)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    mask[(x - 18) ** 2 + (y - 12) ** 2 + (z - 10) ** 2 <= 25] = 1
    mask[(x - 30) ** 2 + (y - 15) ** 2 + (z - 12) ** 2 <= 9] = 1
    mask[5:8, 4:9, 36:40] = 1
    return mask


@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_channel_with_obstacles_matches_oracle(M, orc, storage):
    shape = (48, 26, 22)
    mask = _channel_case(shape)
    typ, _, _, _ = orc.classify(mask, True, True)
    N = int(np.prod(shape))
    m = eq_state(np.ones(N), np.zeros((3, N)))
    m[1] = 0.05
    m[4] = 0.05 ** 2
    inflow = [1.0, 0.05, 0.0, 0.0]
    sim = make_sim(M, shape, 0.55, storage, m, seed=9)
    sim.set_solid(to_gpu(mask.ravel(), torch.uint8))
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    g0 = read(sim)
    nsteps = 100
    sim.step(nsteps)
    g = read(sim)
    ref = orc.step(g0 if storage == "q16" else m, shape, 0.55, typ=typ, inflow=inflow, n=nsteps)
    keep = typ != orc.SOLID
    e = errors(g, ref, keep)
    if storage == "f32":
        assert max(e) < 1e-5, e
    else:
        assert e[1] < 2e-3, e


@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_open_channel_without_solids_matches_oracle(M, orc, storage):
    """Inflow and outflow without a solid mask: no boundary tables, the plain fluid
    kernel, then the inflow face reset and the outflow copy (periodic in y and z)."""
    shape = (30, 12, 10)
    N = int(np.prod(shape))
    typ = orc.classify(np.zeros(shape[::-1], np.uint8), True, True)[0]
    rng = np.random.default_rng(31)
    u = 0.01 * rng.standard_normal((3, N))
    u[0] += 0.04
    m = eq_state(1 + 0.005 * rng.standard_normal(N), u)
    inflow = [1.0, 0.05, 0.0, 0.0]
    sim = make_sim(M, shape, 0.6, storage, m, seed=5)
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    g0 = read(sim)
    sim.step(50)
    g = read(sim)
    ref = orc.step(g0 if storage == "q16" else m, shape, 0.6, typ=typ, inflow=inflow, n=50)
    e = errors(g, ref, np.ones(N, bool))
    if storage == "f32":
        assert max(e) < 1e-5, e
    else:
        assert e[1] < 2e-3, e


def test_fluid_kernel_matches_per_cell_boundary_kernel(M):
    """The fluid kernel with boundary tables that mark nothing (an all-fluid
    solid mask) and an inflow face that lists the x = 0 plane gives, off that
    face, the plain kernel's result: zero-bit tables, an empty bounce pass and the
    staged-record path change no cell."""
    shape = (20, 18, 16)
    N = int(np.prod(shape))
    rng = np.random.default_rng(23)
    m = eq_state(1 + 0.01 * rng.standard_normal(N), 0.05 * rng.standard_normal((3, N)))
    a = make_sim(M, shape, 0.6, "f32", m)
    b = make_sim(M, shape, 0.6, "f32", m)
    mask = np.zeros(shape[::-1], np.uint8)
    b.set_solid(to_gpu(mask.ravel(), torch.uint8))
    b.set_inflow(1.0, (0.0, 0.0, 0.0))  # lists the x = 0 plane only
    a.step(1)
    b.step(1)
    ga, gb = read(a), read(b)
    keep = np.ones(N, bool)
    keep[::shape[0]] = False  # x = 0 plane reset by inflow in b
    e = errors(ga, gb, keep)
    assert max(e) < 2e-6, e


# ------------------------------------------------------------------ reductions, state I/O
def test_reduce_matches_oracle_and_host_io(M, orc):
    shape = (33, 21, 17)
    N = int(np.prod(shape))
    rng = np.random.default_rng(24)
    m = eq_state(1 + 0.01 * rng.standard_normal(N), 0.05 * rng.standard_normal((3, N)))
    for storage in ("f32", "q16"):
        sim = make_sim(M, shape, 0.6, storage, m)
        sim.step(3)
        g = read(sim)
        Mg, Eg = sim.reduce()
        Mo, Eo = orc.reduce(g)
        # the GPU sums rho - 1 as stored; g holds rho rounded to FP32
        tol = 1e-9
        assert abs(Mg - Mo) / Mo < tol and abs(Eg - Eo) / Eo < 1e-6, (Mg, Mo, Eg, Eo)
        # host-pointer path gives the same values as the device path
        rho = torch.empty(N, dtype=torch.float32).pin_memory()
        u = torch.empty(3, N, dtype=torch.float32).pin_memory()
        S = torch.empty(6, N, dtype=torch.float32).pin_memory()
        sim.get_moments(rho, u, S)
        h = np.concatenate([rho.numpy()[None], u.numpy(), S.numpy()])
        assert np.array_equal(h, g.astype(np.float32))
        sim2 = M.Simulator(shape, 0.6, storage)
        sim2.set_state(rho, u, S)
        raw = sim.get_raw_state()
        sim3 = M.Simulator(shape, 0.6, storage)
        sim3.set_raw_state(raw, sim.time_index)
        sim.step(2)
        sim3.step(2)
        assert torch.equal(sim.get_raw_state(), sim3.get_raw_state())


def test_error_paths(M):
    sim = M.Simulator((8, 8, 8), 0.6, "f32")
    with pytest.raises(M.MelbmError):  # only face 0 takes an inflow
        M._check(M.lib().melbm_set_inflow(sim._h, 1, 1.0, 0.0, 0.0, 0.0), sim._h)
    with pytest.raises(M.MelbmError):
        sim.step(-1)
    with pytest.raises(ValueError):
        sim.set_solid(torch.zeros(7, dtype=torch.uint8, device="cuda"))
    with pytest.raises(M.MelbmError):
        M.Simulator((8, 8, 8), 0.4, "f32")
    sim.step(0)
    assert sim.time_index == 0


# ------------------------------------------------------------------ full-size sampled parity
@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_turbulence256_sampled_one_step(M, orc, storage):
    """At the full 256^3 size and in the launch configuration the benchmark uses,
    one GPU step agrees with the oracle's update of sampled cells computed from
    the GPU's own input state."""
    wl = W.TURB256
    u = W.random_phase_field(wl.shape, 0.08)
    m = eq_state(1.0, W.flat(u)).astype(np.float32)
    sim = make_sim(M, wl.shape, wl.tau, storage, m, seed=3)
    sim.step(3)
    g_in = read(sim)
    sim.step(1)
    g_out = read(sim)
    rng = np.random.default_rng(25)
    cells = np.concatenate([rng.integers(0, wl.cells, 4000), np.arange(0, 256),
                            np.arange(wl.cells - 300, wl.cells)])
    ref = orc.step_cells(g_in, wl.shape, wl.tau, cells)
    got = g_out[:, cells]
    du = np.abs(got[1:4] - ref[1:4]).max()
    drho = np.abs(got[0] - ref[0]).max()
    if storage == "f32":
        assert du < 5e-7 and drho < 5e-7, (du, drho)
    else:
        step_u = 0.8 / 65535
        assert du <= step_u * 1.01 and drho <= 0.7 / 65535 * 1.01


def test_q16_mass_drift_over_1000_steps(M):
    """Dithered 16-bit storage keeps total mass within 1e-6 over the 1000 steps of
    the turbulence workload (at 96^3 with the same tau and velocity scale)."""
    shape = (96, 96, 96)
    u = W.random_phase_field(shape, 0.08, seed=8)
    m = eq_state(1.0, W.flat(u))
    sim = make_sim(M, shape, 0.52, "q16", m, seed=17)
    M0, E0 = sim.reduce()
    sim.step(1000)
    M1, E1 = sim.reduce()
    assert abs(M1 - M0) / M0 < 1e-6, (M0, M1)
    assert 0 < E1 < E0


_ALLOC_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import torch
from paper_2602_05295_gb300 import melbm as M
sim = M.Simulator((16, 8, 8), 0.6, "q16")       # its allocations come first
try:
    sim.set_force(torch.zeros(3, 1024, device="cuda"))
    print("no failure")
except M.MelbmError as e:
    print("failed", e.code)
sim.step(3)                                        # the handle still works
rho, _, _ = sim.get_moments()
print("steps", sim.time_index, float(rho.mean()))
"""


def test_injected_allocation_failure_leaves_the_handle_usable(M):
    """MELBM_FAIL_ALLOC_AFTER=4 lets melbm_create take its four allocations and
    fails the next (the force field): MELBM_ENOMEM, and the simulation keeps
    running without the force."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MELBM_FAIL_ALLOC_AFTER="4")
    r = subprocess.run([sys.executable, "-c", _ALLOC_SCRIPT.format(root=root)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    assert lines[0] == "failed 2", r.stdout
    assert lines[1].startswith("steps 3") and abs(float(lines[1].split()[2]) - 1.0) < 1e-6


def test_literal_xyz_ablation_build_matches_the_oracle_switch(M, orc, tmp_path):
    """Reading C1 as a build switch: a library built with MELBM_HERMITE_XYZ_LITERAL
    (the printed 1/(2 c_s^6) on the xyz term) follows the oracle's literal_xyz
    step, and differs from the default reading by far more than FP32 rounding."""
    import ctypes
    from paper_2602_05295_gb300 import build as B
    path = B.build(extra_flags=["-DMELBM_HERMITE_XYZ_LITERAL"], lib_path=str(tmp_path / "lib.so"))
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.melbm_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_float, ctypes.c_int, ctypes.POINTER(P)]
    L.melbm_set_state.argtypes = [P, P, P, P]
    L.melbm_step.argtypes = [P, ctypes.c_int]
    L.melbm_get_moments.argtypes = [P, P, P, P]
    L.melbm_destroy.argtypes = [P]
    shape = (37, 23, 19)
    N = int(np.prod(shape))
    rng = np.random.default_rng(61)
    m = eq_state(1.0 + 0.01 * rng.standard_normal(N), 0.08 * rng.standard_normal((3, N)))
    m[4:] += 0.01 * rng.standard_normal((6, N))
    h = P()
    assert L.melbm_create(*shape, 27, ctypes.c_float(0.57), 0, ctypes.byref(h)) == 0
    d = [to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:])]
    assert L.melbm_set_state(h, *(P(t.data_ptr()) for t in d)) == 0
    assert L.melbm_step(h, 5) == 0
    out = [torch.empty(k, N, device="cuda") for k in (1, 3, 6)]
    assert L.melbm_get_moments(h, *(P(t.data_ptr()) for t in out)) == 0
    torch.cuda.synchronize()
    L.melbm_destroy(h)
    g = np.concatenate([t.cpu().numpy() for t in out]).astype(np.float64)
    lit = orc.step(m, shape, 0.57, n=5, literal_xyz=True)
    std = orc.step(m, shape, 0.57, n=5)
    assert max(errors(g, lit)) < 1e-5, errors(g, lit)
    assert max(errors(std, lit)) > 100 * 1e-5


_BOUNDARY_FAIL_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_2602_05295_gb300 import melbm as M, workloads as W
shape = (24, 16, 12)
sim = M.Simulator(shape, 0.6, "q16")
mask = torch.from_numpy(W.channel_walls(shape).ravel()).cuda()
try:
    sim.set_solid(mask)
    print("no failure")
except M.MelbmError as e:
    print("set_solid", e.code)
for call in (lambda: sim.step(1), lambda: sim.solid_force(0)):
    try:
        call()
        print("ran")
    except M.MelbmError as e:
        print("refused", e.code)
print("time", sim.time_index)
"""


@pytest.mark.parametrize("after", [7, 12, 13, 14])
def test_failed_boundary_setup_leaves_no_partial_lists(M, after):
    """melbm_set_solid only records the mask (and copies it, the handle's fifth
    allocation after its four state and reduction buffers); the classification
    runs at the first call that needs it.  A device allocation failing there
    (MELBM_FAIL_ALLOC_AFTER; the classification allocates the type array, the
    solid-bit and boundary-bit tables, three scratch arrays, the two list arrays,
    the list-index table and the side table, so 7, 12, 13 and 14 fail the
    boundary bits, the second list array, the list-index table and the side
    table) is that call's MELBM_ENOMEM, and the handle then refuses to step or to
    sum solid forces (MELBM_ESTATE) instead of running with partial tables."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MELBM_FAIL_ALLOC_AFTER=str(after))
    r = subprocess.run([sys.executable, "-c", _BOUNDARY_FAIL_SCRIPT.format(root=root)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    assert lines == ["no failure", "refused 2", "refused 4", "time 0"], r.stdout
