"""Per-row barriers of the 16-bit fluid kernel.

The 16-bit kernel without boundary tables synchronises its rows through per-row
mbarriers instead of one block-wide barrier per plane pair: a row waits for its
two neighbour rows (the y exchange) and for warp 0 (the x-halo buffer), and warp
0 for the whole block.  Two checks:

* bit-exactness at full size: the same state stepped by that kernel and by the
  kernel with boundary tables (an all-zero solid mask: no solid cell and no
  record, the same arithmetic, one block-wide barrier per plane pair) must give
  the same stored words after every block has crossed its barriers many times;
* the bounded waits: MELBM_TEST_STALL_BARRIER=1 at melbm_create initialises warp
  0's barriers for twice the arrivals they receive, so the waits on them run out
  (no GPU fault, no hang).  The kernel then sets the handle's fault word, the next
  melbm_reduce / melbm_step report it, the handle refuses to step until a new
  state is set, and the GPU context stays usable for other handles.
"""
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
    return melbm


def _turbulence(shape, umax, seed):
    u = W.random_phase_field(shape, umax, seed=seed)
    N = int(np.prod(shape))
    return torch.ones(N, device="cuda"), torch.from_numpy(W.flat(u).astype(np.float32)).cuda()


@pytest.mark.parametrize("lattice", [27, 19])
def test_row_barriers_match_block_barrier_at_full_size(M, lattice):
    shape = (256, 256, 256)
    rho, u = _turbulence(shape, 0.08, 2602)
    out = []
    for tables in (False, True):
        sim = M.Simulator(shape, 0.52, "q16", lattice=lattice, seed=2602)
        if tables:  # all-fluid mask: the tables' kernel, block-wide barriers
            sim.set_solid(torch.zeros(sim.N, dtype=torch.uint8, device="cuda"))
        sim.set_state(rho, u)
        sim.step(40)
        out.append(sim.get_raw_state())
        sim.close()
    assert torch.equal(out[0], out[1])


def test_row_barriers_on_small_and_ragged_grids(M):
    """Grids whose blocks hold few plane pairs, ragged x and y tiles and tiny nz,
    against the tables' kernel as above."""
    for shape in ((33, 15, 9), (70, 29, 40), (32, 14, 64), (5, 3, 3)):
        rho = (1.0 + 0.01 * torch.randn(int(np.prod(shape)), generator=torch.Generator().manual_seed(1))).cuda()
        u = (0.03 * torch.randn(3 * int(np.prod(shape)), generator=torch.Generator().manual_seed(2))).cuda()
        out = []
        for tables in (False, True):
            sim = M.Simulator(shape, 0.6, "q16", seed=5)
            if tables:
                sim.set_solid(torch.zeros(sim.N, dtype=torch.uint8, device="cuda"))
            sim.set_state(rho, u)
            sim.step(12)
            out.append(sim.get_raw_state())
            sim.close()
        assert torch.equal(out[0], out[1]), shape


def test_barrier_wait_that_runs_out_is_reported(M, monkeypatch):
    shape = (32, 14, 64)
    N = int(np.prod(shape))
    rho = torch.ones(N, device="cuda")
    u = torch.zeros(3 * N, device="cuda")
    monkeypatch.setenv("MELBM_TEST_STALL_BARRIER", "1")
    stalled = M.Simulator(shape, 0.6, "q16", seed=3)
    monkeypatch.delenv("MELBM_TEST_STALL_BARRIER")
    stalled.set_state(rho, u)
    stalled.step(1)  # the launch itself succeeds; its waits run out on the GPU
    with pytest.raises(M.MelbmError) as e:
        stalled.reduce()
    assert e.value.code == M.ECUDA and "barrier wait" in str(e.value)
    with pytest.raises(M.MelbmError) as e:  # the state is undefined until a new one
        stalled.step(1)
    assert e.value.code == M.ESTATE
    # the context stays usable: a handle without the stall steps normally
    ok = M.Simulator(shape, 0.6, "q16", seed=3)
    ok.set_state(rho, u)
    ok.step(3)
    mass, _ = ok.reduce()
    assert abs(mass - N) < 1e-3
    # a new state clears the refusal; the stalled handle's next step reports again
    stalled.set_state(rho, u)
    stalled.step(1)
    with pytest.raises(M.MelbmError) as e:
        stalled.reduce()
    assert e.value.code == M.ECUDA
    stalled.close()
    ok.close()
