"""Adaptive bit allocation on the GPU (Sec. 6.2.2: rho and u on b_rho_u bits, rho
S^neq on b_S bits, each on the Sec. 5.4 grid with 2^b - 1 steps).

* the codec is bit-exact against the oracle for every configuration;
* one step from identical codes matches the oracle's quantised step code for
  code up to FP32-vs-FP64 rounding at a code boundary;
* 100 steps track the FP64 oracle within a bound that scales with the grid step
  of the configuration, and dithering keeps the mass drift at the noise level;
* melbm_set_bits re-encodes the state, and reduce flags codes on 0 or 2^b - 1.
"""
import warnings

import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONFIGS = [(16, 15), (15, 14), (14, 13), (13, 12), (12, 11)]
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05295_gb300 import melbm
    melbm.lib()
    return melbm


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def eq_state(rho, u):
    m = np.zeros((10, u.shape[1]))
    m[0] = rho
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b]
    return m


def read(sim):
    rho, u, S = sim.get_moments()
    return np.concatenate([rho.cpu().numpy()[None], u.cpu().numpy(), S.cpu().numpy()]).astype(np.float64)


@pytest.mark.parametrize("bits", CONFIGS)
def test_codec_bits_bit_exact_against_oracle(M, orc, bits):
    rng = np.random.default_rng(21)
    shape = (37, 11, 5)
    N = 37 * 11 * 5
    lo, hi = orc.ranges()
    v = (lo[:, None] - 0.05 * (hi - lo)[:, None]
         + 1.1 * (hi - lo)[:, None] * rng.uniform(size=(10, N))).astype(np.float32)
    v[:, 0] = np.nan
    v[:, 1] = lo
    v[:, 2] = hi
    v_orc = v.copy()
    v_orc[0] = v[0] - np.float32(1.0)
    for det in (True, False):
        for t, seed in ((0, 0), (17, 2602)):
            words = M.codec_encode(to_gpu(v), shape, t, seed, bits, deterministic=det)
            codes = M.words_to_codes(words).cpu().numpy()
            ref = orc.encode(v_orc, shape, t, seed, deterministic=det, bits=bits)
            assert np.array_equal(codes, ref.astype(np.int64)), (bits, det, t)
    Q = np.array([2 ** bits[0] - 1] * 4 + [2 ** bits[1] - 1] * 6)
    assert np.array_equal(codes[:, 2], Q)  # the range maxima map to 2^b - 1
    dec = M.codec_decode(words, bits).cpu().numpy().astype(np.float64)
    assert np.abs(dec - orc.decode(ref, bits)).max() <= 2e-7


@pytest.mark.parametrize("bits", [(16, 15), (12, 11)])
def test_bits_one_step_codes_match_emulation(M, orc, bits):
    shape = (45, 20, 18)
    u = W.random_phase_field(shape, 0.08, kmax=6, seed=7)
    m = eq_state(1.0, W.flat(u))
    sim = M.Simulator(shape, 0.52, "q16", seed=5)
    sim.set_bits(*bits)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    codes0 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    sim.step(1)
    codes1 = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    ref = orc.q16_step(codes0.astype(np.uint16), shape, 0.52, 1, 5, bits=bits).astype(np.int64)
    d = np.abs(codes1 - ref)
    assert d.max() <= 1
    assert (d > 0).mean() < 0.02


@pytest.mark.parametrize("bits", [(16, 16)] + CONFIGS)
def test_bits_track_fp64_and_conserve_mass(M, orc, bits):
    """The quantisation noise per step is one grid step at most (dithered), so the
    velocity error after 100 steps scales with the step of b_rho_u (the 16/16
    bound of the parity tests, 2e-3 of max|u|, times 2^(16 - b_rho_u)), and the
    relative mass drift with the step of rho (1e-6 at 16 bits)."""
    shape = (64, 48, 40)
    u = W.random_phase_field(shape, 0.08, kmax=8, seed=6)
    m = eq_state(1.0, W.flat(u))
    sim = M.Simulator(shape, 0.52, "q16", seed=11)
    sim.set_bits(*bits)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    g0 = read(sim)
    M0, _ = sim.reduce()
    sim.step(100)
    g = read(sim)
    ref = orc.step(g0, shape, 0.52, n=100)
    scale = 2.0 ** (16 - bits[0])
    e_u = np.abs(g[1:4] - ref[1:4]).max() / np.abs(ref[1:4]).max()
    assert e_u < 2e-3 * scale, (bits, e_u)
    M1, _ = sim.reduce()
    assert abs(M1 - M0) / M0 < 1e-6 * scale, (bits, M0, M1)


def test_set_bits_reencodes_the_state_and_reduce_flags_the_range_ends(M):
    shape = (32, 16, 8)
    N = 32 * 16 * 8
    u = W.random_phase_field(shape, 0.05, kmax=4, seed=3)
    m = eq_state(1.0, W.flat(u))
    sim = M.Simulator(shape, 0.6, "q16", seed=1)
    sim.set_state(to_gpu(m[0]), to_gpu(m[1:4]), to_gpu(m[4:10]))
    a = read(sim)
    sim.set_bits(12, 11)
    b = read(sim)
    step_u = 0.8 / (2 ** 12 - 1)
    assert np.abs(b[1:4] - a[1:4]).max() <= step_u * 1.01
    with pytest.raises(Exception):
        sim.set_bits(7, 11)
    with pytest.raises(Exception):
        M.Simulator(shape, 0.6, "f32").set_bits(16, 15)
    # a velocity beyond the range saturates at 2^12 - 1, which reduce reports
    uu = np.zeros((3, N))
    uu[0, 0] = 0.5
    sim.set_state(to_gpu(np.ones(N)), to_gpu(uu))
    codes = M.words_to_codes(sim.get_raw_state().view(torch.int32).reshape(5, -1)).cpu().numpy()
    assert codes[1, 0] == 2 ** 12 - 1
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        sim.reduce()
    assert any(issubclass(x.category, M.SaturationWarning) for x in w)
