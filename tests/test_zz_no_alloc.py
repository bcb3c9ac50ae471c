"""The allocation-free reduction entry point, checked against melbm_reduce.

melbm_reduce_state_noalloc serves callers that cannot allocate device memory
where they need the conservation diagnostics (a loop with a fixed memory
budget, a device pool owned by another allocator, code that must avoid the
implicit synchronisation of cudaMalloc/cudaFree).  It reads a raw state buffer
the caller owns and keeps its scratch in a fixed array inside the library, so
these tests call it twice in a row on different states -- the second call runs
on scratch the first one left behind -- and compare each result with the
handle-based melbm_reduce on the same state.  This file is collected last so a
stop-at-first-failure run has already run every other test.
"""
import ctypes

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
    L = melbm.lib()
    fn = L.melbm_reduce_state_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return melbm


def _noalloc(M, sim, types=None):
    raw = sim.get_raw_state()
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    storage = {"f32": M.F32, "q16": M.Q16}[sim.storage]
    rc = M.lib().melbm_reduce_state_noalloc(
        ctypes.c_void_p(raw.data_ptr()), storage, sim.N,
        None if types is None else ctypes.c_void_p(types.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == M.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _state(shape, seed):
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    u = 0.05 * rng.standard_normal((3, N))
    rho = 1.0 + 0.01 * rng.standard_normal(N)
    return (torch.from_numpy(rho).float().cuda(), torch.from_numpy(u).float().cuda())


@pytest.mark.parametrize("storage", ["f32", "q16"])
def test_noalloc_reduce_matches_reduce_on_two_calls(M, storage):
    shape = (70, 33, 29)  # 66990 cells: two chunks, the second one ragged
    sim = M.Simulator(shape, 0.6, storage, seed=4)
    for call, seed in enumerate((1, 2)):
        rho, u = _state(shape, seed)
        sim.set_state(rho, u)
        sim.step(2 + call)
        mass, ke = sim.reduce()
        got = _noalloc(M, sim)
        assert abs(got[0] - mass) <= 1e-12 * abs(mass), (call, got[0], mass)
        assert abs(got[1] - ke) <= 1e-12 * abs(ke), (call, got[1], ke)
        assert got[2] == 0.0


def test_noalloc_reduce_with_solid_cells(M):
    shape = (48, 26, 22)
    mask = W.channel_walls(shape)
    mask[5:9, 6:12, 20:30] = 1
    sim = M.Simulator(shape, 0.55, "q16", seed=6)
    sim.set_solid(torch.from_numpy(mask.ravel()).cuda())
    sim.set_inflow(1.0, (0.05, 0.0, 0.0))
    sim.set_outflow()
    types = sim.types()
    for call in range(2):
        sim.step(5)
        mass, ke = sim.reduce()
        got = _noalloc(M, sim, types)
        assert abs(got[0] - mass) <= 1e-12 * abs(mass), (call, got[0], mass)
        assert abs(got[1] - ke) <= 1e-12 * abs(ke), (call, got[1], ke)


def test_noalloc_reduce_counts_saturated_codes(M):
    """A 16-bit state with codes pinned at both range limits: out[2] is the number
    of non-solid codes equal to 0 or 65535, counted here from the raw words, on
    two calls in a row; mass and energy still match melbm_reduce."""
    import warnings
    shape = (40, 20, 18)
    N = int(np.prod(shape))
    sim = M.Simulator(shape, 0.6, "q16", seed=8)
    rng = np.random.default_rng(9)
    for call in range(2):
        rho = 1.0 + 0.01 * rng.standard_normal(N)
        u = 0.05 * rng.standard_normal((3, N))
        hit = rng.random(N) < 0.01 * (call + 1)
        u[0, hit] = 0.5 * np.sign(rng.standard_normal(hit.sum()))  # beyond [-0.4, 0.4]
        rho[rng.random(N) < 0.003] = 0.7                              # below the rho range
        sim.set_state(torch.from_numpy(rho).float().cuda(), torch.from_numpy(u).float().cuda())
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", M.SaturationWarning)
            mass, ke = sim.reduce()
        words = sim.get_raw_state().view(torch.int32).reshape(5, N)
        codes = M.words_to_codes(words).cpu().numpy()
        want = int(((codes == 0) | (codes == 65535)).sum())
        assert want > 0
        got = _noalloc(M, sim)
        assert got[2] == want, (call, got[2], want)
        assert abs(got[0] - mass) <= 1e-12 * abs(mass)
        assert abs(got[1] - ke) <= 1e-12 * abs(ke)


def test_noalloc_reduce_allocates_no_device_memory(M):
    """After a first call (which looks up the scratch address), further calls leave
    the device's free memory unchanged."""
    shape = (64, 32, 32)
    sim = M.Simulator(shape, 0.6, "q16", seed=10)
    rho, u = _state(shape, 11)
    sim.set_state(rho, u)
    raw = sim.get_raw_state()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def call():
        rc = M.lib().melbm_reduce_state_noalloc(
            ctypes.c_void_p(raw.data_ptr()), M.Q16, sim.N, None, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(st))
        assert rc == M.OK
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_reduce_rejects_oversized_grid(M):
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    too_many = 4096 * 65536 + 1
    rc = M.lib().melbm_reduce_state_noalloc(ctypes.c_void_p(buf.data_ptr()), M.Q16, too_many, None,
                                            ctypes.c_void_p(out.data_ptr()), None)
    assert rc == M.EINVAL
    assert b"exceeds" in M.lib().melbm_last_error(None)
    rc = M.lib().melbm_reduce_state_noalloc(None, M.Q16, 10, None, ctypes.c_void_p(out.data_ptr()),
                                            None)
    assert rc == M.EINVAL
    assert b"NULL" in M.lib().melbm_last_error(None)


def test_noalloc_reduce_replays_from_a_cuda_graph(M):
    """After a warm-up call (the scratch address lookup), one call captured into a
    CUDA graph replays with the results of melbm_reduce, and a replay after the
    state buffer's contents change reads the new contents."""
    shape = (64, 32, 32)
    sim = M.Simulator(shape, 0.6, "q16", seed=12)
    rho, u = _state(shape, 13)
    sim.set_state(rho, u)
    raw = sim.get_raw_state().clone()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()

    def call():
        return M.lib().melbm_reduce_state_noalloc(
            ctypes.c_void_p(raw.data_ptr()), M.Q16, sim.N, None, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(s.cuda_stream))

    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert call() == M.OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = call()
    assert rc == M.OK
    for seed in (13, 14):
        if seed != 13:
            rho, u = _state(shape, seed)
            sim.set_state(rho, u)
            raw.copy_(sim.get_raw_state())
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        mass, ke = sim.reduce()
        assert abs(got[0] - mass) <= 1e-12 * abs(mass), (seed, got[0], mass)
        assert abs(got[1] - ke) <= 1e-12 * abs(ke), (seed, got[1], ke)
        assert got[2] == 0.0
