"""Asynchronous raw-state transfers (melbm_upload_raw_state_async,
melbm_download_raw_state_async, melbm_sync_transfers) against the blocking
set_raw_state / step / get_raw_state sequence: the states must be byte-identical
whatever the transfers overlap with, on periodic grids and on a channel with
obstacles, inflow and outflow, in both storages."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPE = (64, 40, 36)


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05295_gb300 import melbm
    melbm.lib()
    return melbm


def make(M, storage, channel, lattice=27):
    nx, ny, nz = SHAPE
    N = nx * ny * nz
    sim = M.Simulator(SHAPE, 0.55, storage, seed=5, lattice=lattice)
    g = np.random.default_rng(3)
    u = (0.03 * g.standard_normal((3, N))).astype(np.float32)
    sim.set_state(torch.ones(N, device="cuda"), torch.from_numpy(u).cuda())
    if channel:
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        mask = np.zeros((nz, ny, nx), np.uint8)
        mask[:, 0, :] = mask[:, ny - 1, :] = 1
        mask[(x - 24) ** 2 + (y - 20) ** 2 + (z - 18) ** 2 <= 36] = 1
        sim.set_solid(torch.from_numpy(mask.ravel()).cuda())
        sim.set_inflow(1.0, (0.05, 0.0, 0.0))
        sim.set_outflow()
    return sim


def pinned(nb):
    return torch.zeros(nb, dtype=torch.uint8).pin_memory()


def inputs(sim, k):
    """k distinct packed states in pinned host memory with their time indices."""
    out = []
    for i in range(k):
        sim.step(3)
        h = pinned(sim.state_bytes())
        sim.get_raw_state(h)
        out.append((h, sim.time_index))
    return out


@pytest.mark.parametrize("storage,channel,lattice", [
    ("q16", False, 27), ("f32", False, 27), ("q16", True, 27), ("f32", True, 27),
    ("q16", True, 19)])
def test_upload_step_download_pipeline_matches_blocking(M, storage, channel, lattice):
    sim = make(M, storage, channel, lattice)
    ins = inputs(sim, 4)
    nb = sim.state_bytes()
    ref = []
    for h, t in ins:
        sim.set_raw_state(h, t)
        sim.step(1)
        ref.append(sim.get_raw_state(pinned(nb)))
    outs = [pinned(nb) for _ in ins]
    for (h, t), o in zip(ins, outs):
        sim.upload_raw_state_async(h, t)
        sim.step(1)
        sim.download_raw_state_async(o)
    sim.sync_transfers()
    for i, (r, o) in enumerate(zip(ref, outs)):
        assert torch.equal(r, o), f"state {i} differs"
    assert sim.time_index == ins[-1][1] + 1
    # the handle's blocking calls see the last stepped state
    assert torch.equal(sim.get_raw_state(pinned(nb)), ref[-1])
    sim.close()


def test_downloads_overlapping_steps_and_blocking_calls(M):
    """Downloads issued between steps (one and several at a time) return the state
    they were issued on; an upload followed at once by a download returns the
    upload; blocking calls after pending transfers see the right state."""
    sim = make(M, "q16", True)
    (h0, t0), = inputs(sim, 1)
    nb = sim.state_bytes()
    # blocking reference: s0, s1 = one step, s3 = two more, and the reductions
    sim.set_raw_state(h0, t0)
    s0 = sim.get_raw_state(pinned(nb))
    sim.step(1)
    s1 = sim.get_raw_state(pinned(nb))
    sim.step(2)
    s3 = sim.get_raw_state(pinned(nb))
    m3, e3 = sim.reduce()
    rho3, u3, _ = sim.get_moments()
    # asynchronous
    d_up, d0, d1, d3 = (pinned(nb) for _ in range(4))
    sim.upload_raw_state_async(h0, t0)
    sim.download_raw_state_async(d_up)
    sim.download_raw_state_async(d0)
    sim.step(1)
    sim.download_raw_state_async(d1)
    sim.step(2)  # overwrites both buffers: waits for every download
    sim.download_raw_state_async(d3)
    m, e = sim.reduce()  # joins the transfers
    rho, u, _ = sim.get_moments()
    sim.sync_transfers()
    assert torch.equal(d_up, h0) and torch.equal(d0, s0)
    assert torch.equal(d1, s1) and torch.equal(d3, s3)
    assert (m, e) == (m3, e3)
    assert torch.equal(rho, rho3) and torch.equal(u, u3)
    sim.close()


def test_upload_then_blocking_reads_and_refusals(M):
    sim = make(M, "f32", False)
    (h0, t0), (h1, t1) = inputs(sim, 2)
    nb = sim.state_bytes()
    sim.set_raw_state(h1, t1)
    ref = sim.get_moments()
    sim.set_raw_state(h0, t0)
    sim.upload_raw_state_async(h1, t1)
    got = sim.get_moments()  # waits for the upload
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    assert sim.time_index == t1
    with pytest.raises(M.MelbmError):  # wrong size
        M._check(M.lib().melbm_upload_raw_state_async(
            sim._h, ctypes.c_void_p(h0.data_ptr()), nb - 4, 0), sim._h)
    with pytest.raises(M.MelbmError):
        sim.upload_raw_state_async(h0, -1)
    sim.sync_transfers()
    sim.close()
    mixed = M.Simulator((32, 16, 16), 0.6, "mixed")
    buf = pinned(32 * 16 * 16 * 20)
    with pytest.raises(M.MelbmError):
        M._check(M.lib().melbm_download_raw_state_async(
            mixed._h, ctypes.c_void_p(buf.data_ptr()), buf.numel()), mixed._h)
    mixed.sync_transfers()  # no transfers were issued: a no-op
    mixed.close()


@pytest.mark.parametrize("seed", [7, 11])
def test_random_interleavings_match_blocking(M, seed):
    """A seeded random sequence of uploads (including back to back), steps of one
    and two, downloads and reductions gives the same states and sums through the
    asynchronous calls as through the blocking ones."""
    import random
    sim = make(M, "q16", True)
    ins = inputs(sim, 3)
    nb = sim.state_bytes()
    rng = random.Random(seed)
    ops = [rng.choice(["up", "up", "step1", "step1", "step2", "down", "down", "reduce"])
           for _ in range(40)]

    def run(asynchronous):
        sim.set_raw_state(*ins[0])
        outs, k = [], 0
        for op in ops:
            if op == "up":
                h, t = ins[k % len(ins)]
                k += 1
                if asynchronous:
                    sim.upload_raw_state_async(h, t)
                else:
                    sim.set_raw_state(h, t)
            elif op == "step1":
                sim.step(1)
            elif op == "step2":
                sim.step(2)
            elif op == "down":
                o = pinned(nb)
                if asynchronous:
                    sim.download_raw_state_async(o)
                else:
                    sim.get_raw_state(o)
                outs.append(o)
            else:
                outs.append(sim.reduce())
        o = pinned(nb)
        if asynchronous:
            sim.download_raw_state_async(o)
        else:
            sim.get_raw_state(o)
        outs.append(o)
        sim.sync_transfers()
        return outs, sim.time_index

    ref, t_ref = run(False)
    got, t_got = run(True)
    assert t_ref == t_got and len(ref) == len(got)
    for i, (r, g) in enumerate(zip(ref, got)):
        if isinstance(r, tuple):
            assert r == g, (i, r, g)
        else:
            assert torch.equal(r, g), f"output {i} differs"
    sim.close()


def test_spare_buffer_is_accounted_and_freed(M):
    sim = make(M, "f32", False)
    before = sim.memory_bytes()
    (h0, t0), = inputs(sim, 1)
    sim.upload_raw_state_async(h0, t0)
    sim.sync_transfers()
    assert sim.memory_bytes() == before + sim.state_bytes()
    sim.close()


def test_set_stream_orders_pending_work(M):
    """Work enqueued on the previous stream is ordered before work on the new one:
    a read issued right after switching streams sees every pending step."""
    shape = (128, 128, 128)
    N = 128 ** 3
    g = np.random.default_rng(5)
    u = torch.from_numpy((0.03 * g.standard_normal((3, N))).astype(np.float32)).cuda()
    rho = torch.ones(N, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    ref_sim = M.Simulator(shape, 0.55, "q16", seed=2, stream=s1)
    ref_sim.set_state(rho, u)
    torch.cuda.synchronize()
    ref_sim.step(60)
    ref = ref_sim.get_raw_state(pinned(ref_sim.state_bytes()))
    ref_sim.close()
    sim = M.Simulator(shape, 0.55, "q16", seed=2, stream=s1)
    sim.set_state(rho, u)
    torch.cuda.synchronize()
    sim.step(60)  # still running on s1 when the stream changes
    M._check(M.lib().melbm_set_stream(sim._h, ctypes.c_void_p(s2.cuda_stream)), sim._h)
    got = sim.get_raw_state(pinned(sim.state_bytes()))
    assert torch.equal(ref, got)
    sim.close()
