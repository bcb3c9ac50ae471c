"""FP64 CPU oracle of the moment-encoded LBM update -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA path
(``paper_2602_05295_gb300``) and never imports it.

The arithmetic lives in ``melbm_oracle.cpp`` (plain C++ in FP64, one routine per
equation of arXiv 2602.05295); this module builds it with g++, loads it with
ctypes and adds the numpy glue that the paper states as plain formulas:

* stored variables of the 16-bit form (Sec. 5.4, range reduction):
  ``(rho, u, rho S^neq)`` with ``rho S^neq_ab = rho (S_ab - u_a u_b)``;
* the 16-bit emulation step: decode (FP64 dequantisation), one FP64 step,
  re-encode in FP32 with the dither of the same counter as the kernels use;
* complex-step linearisation of the step map (amplification matrix G(k),
  Sec. 5.2 brute-force form) and the multi-step discrete adjoint with
  recomputation from FP64 checkpoints.

Public state layout: component-major ``(10, N)`` float64 arrays with components
``(rho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz)`` and ``n = x + nx (y + ny z)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "melbm_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

FLUID, FLUID_BOUNDARY, INFLOW, OUTFLOW, SOLID = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP, -O2, no machine-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I, I64, D, U32 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
            L.orc_num_threads.restype = I
            L.orc_set_threads.argtypes = [I]
            L.orc_lattice.argtypes = [P, P]
            L.orc_collide.argtypes = [I64, P, P, D, P]
            L.orc_reconstruct.argtypes = [I64, P, I, P]
            L.orc_moments.argtypes = [I64, P, P, P]
            L.orc_classify.argtypes = [I, I, I, P, I, I, P, P, P, P]
            L.orc_classify.restype = I64
            for name in ("orc_step_f64", "orc_step_c128"):
                getattr(L, name).argtypes = [I, I, I, D, P, P, P, P, I, P]
            L.orc_step_cells_f64.argtypes = [I, I, I, D, P, P, P, P, P, I64, P]
            L.orc_step_planted_f64.argtypes = [I, I, I, D, P, P, P, P, I, P]
            L.orc_step_vjp_f64.argtypes = [I, I, I, D, P, P, P, P, P, P]
            L.orc_reduce.argtypes = [I64, P, P, P, P]
            L.orc_dither.argtypes = [U32, U32, U32, U32, U32, P]
            L.orc_encode.argtypes = [I, I, I, P, U32, U32, I, P]
            L.orc_decode.argtypes = [I64, P, P]
            L.orc_encode_bits.argtypes = [I, I, I, P, U32, U32, I, I, I, P]
            L.orc_step_wall_f64.argtypes = [I, I, I, D, P, P, P, P, I, P, P, P]
            L.orc_step19_f64.argtypes = [I, I, I, D, P, P, P, P, P]
            L.orc_step19_cells_f64.argtypes = [I, I, I, D, P, P, P, P, P, I64, P]
            L.orc_step19_wall_f64.argtypes = [I, I, I, D, P, P, P, P, I, P, P, P]
            L.orc_solid_force19_f64.argtypes = [I, I, I, D, P, P, P, I, P, P, I, P]
            L.orc_reconstruct19.argtypes = [P, P, P, P]
            L.orc_solid_force_f64.argtypes = [I, I, I, D, P, P, P, I, P, P, I, P]
            L.orc_decode_bits.argtypes = [I64, P, I, I, P]
            L.orc_codec_constants_bits.argtypes = [I, I, I, P]
            L.orc_mean_code_over_dither_bits.argtypes = [ctypes.c_float, I, I, I]
            L.orc_mean_code_over_dither_bits.restype = D
            L.orc_code_coordinate_bits.argtypes = [ctypes.c_float, I, I, I]
            L.orc_code_coordinate_bits.restype = D
            L.orc_ranges.argtypes = [P, P]
            L.orc_codec_constants.argtypes = [I, P]
            L.orc_mean_code_over_dither.argtypes = [ctypes.c_float, I]
            L.orc_mean_code_over_dither.restype = D
            L.orc_code_coordinate.argtypes = [ctypes.c_float, I]
            L.orc_code_coordinate.restype = D
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- lattice / cell
def lattice():
    c = np.zeros((27, 3), np.int32)
    w = np.zeros(27)
    lib().orc_lattice(_p(c), _p(w))
    return c, w


def collide(m, F=None, tau=0.6):
    """App. A collision of cells given as rows of 10 moments."""
    m = np.atleast_2d(_f64(m))
    out = np.empty_like(m)
    Fa = None if F is None else np.atleast_2d(_f64(F))
    lib().orc_collide(m.shape[0], _p(m), _p(Fa), float(tau), _p(out))
    return out


def reconstruct(m, literal_xyz=False):
    """Eq. three_order_f: the 27 populations of cells given as rows of 10 moments."""
    m = np.atleast_2d(_f64(m))
    f = np.empty((m.shape[0], 27))
    lib().orc_reconstruct(m.shape[0], _p(m), int(literal_xyz), _p(f))
    return f


def moments(f, F=None):
    """Eq. rho_u_stress of cells given as rows of 27 populations."""
    f = np.atleast_2d(_f64(f))
    out = np.empty((f.shape[0], 10))
    Fa = None if F is None else np.atleast_2d(_f64(F))
    lib().orc_moments(f.shape[0], _p(f), _p(Fa), _p(out))
    return out


# ---------------------------------------------------------------- classification
def classify(mask, inflow=False, outflow=False):
    """Cell types, 27-bit solid-link masks and the ascending boundary list.

    ``mask`` is a (nz, ny, nx) uint8 array (nonzero = solid)."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = mask.shape
    N = mask.size
    typ = np.empty(N, np.uint8)
    link = np.empty(N, np.uint32)
    cells = np.empty(N, np.uint32)
    words = np.empty(N, np.uint32)
    L = lib().orc_classify(nx, ny, nz, _p(mask), int(inflow), int(outflow), _p(typ), _p(link),
                           _p(cells), _p(words))
    return typ, link, cells[:L].copy(), words[:L].copy()


# ---------------------------------------------------------------- steps
def _inflow_arr(inflow):
    if inflow is None:
        return None
    return np.asarray(inflow, np.float64).reshape(4)


class Wall:
    """Solid walls (Sec. 3.2): model 0 = halfway bounce-back, 1 = moment-based
    reconstruction with rigid body motion; ``body`` = uint8 body id per cell (the
    solid mask values, None: every solid is body 1); ``motion`` = {id: (V, Om, r0)}."""

    def __init__(self, model=1, body=None, motion=None):
        self.model = int(model)
        self.body = None if body is None else np.ascontiguousarray(body, np.uint8)
        self.table = np.zeros((256, 9))
        for b, (V, Om, r0) in (motion or {}).items():
            self.table[b] = np.concatenate([V, Om, r0])


def step(m, shape, tau, F=None, typ=None, inflow=None, n=1, literal_xyz=False, wall=None):
    """n FP64 steps of the public state ``m`` (10, N) on the grid ``shape`` = (nx, ny, nz)."""
    nx, ny, nz = shape
    cur = _f64(m).copy()
    out = np.empty_like(cur)
    Fa = _f64(F)
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    ia = _inflow_arr(inflow)
    for _ in range(n):
        if wall is None:
            lib().orc_step_f64(nx, ny, nz, float(tau), _p(cur), _p(Fa), _p(ta), _p(ia),
                               int(literal_xyz), _p(out))
        else:
            lib().orc_step_wall_f64(nx, ny, nz, float(tau), _p(cur), _p(Fa), _p(ta), _p(ia),
                                    wall.model, _p(wall.body), _p(wall.table), _p(out))
        cur, out = out, cur
    return cur


PLANT_OUT_FROM_OLD, PLANT_OUT_FROM_SELF, PLANT_IN_S_ZERO = 1, 2, 3


def step_planted(m, shape, tau, planted, F=None, typ=None, inflow=None):
    """One D3Q27 step with a deliberately wrong special-cell rule (``PLANT_*``),
    for the tests that show their pins reject it."""
    nx, ny, nz = shape
    cur = _f64(m)
    out = np.empty_like(cur)
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    lib().orc_step_planted_f64(nx, ny, nz, float(tau), _p(cur), _p(_f64(F)), _p(ta),
                               _p(_inflow_arr(inflow)), int(planted), _p(out))
    return out


def step19(m, shape, tau, F=None, n=1, typ=None, inflow=None, wall=None):
    """n FP64 D3Q19 steps of the public state ``m`` (10, N); ``typ``/``inflow``/
    ``wall`` as for ``step`` (None: periodic)."""
    nx, ny, nz = shape
    cur = _f64(m).copy()
    out = np.empty_like(cur)
    Fa = _f64(F)
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    ia = None if inflow is None else np.ascontiguousarray(inflow, np.float64)
    for _ in range(n):
        if wall is None:
            lib().orc_step19_f64(nx, ny, nz, float(tau), _p(cur), _p(Fa), _p(ta), _p(ia), _p(out))
        else:
            lib().orc_step19_wall_f64(nx, ny, nz, float(tau), _p(cur), _p(Fa), _p(ta), _p(ia),
                                      wall.model, _p(wall.body), _p(wall.table), _p(out))
        cur, out = out, cur
    return cur


def step19_cells(m, shape, tau, cells, F=None, typ=None, inflow=None):
    """The D3Q19 update of the listed cells: (10, len(cells))."""
    nx, ny, nz = shape
    ma = _f64(m)
    ca = np.ascontiguousarray(cells, np.int64)
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    ia = None if inflow is None else np.ascontiguousarray(inflow, np.float64)
    out = np.empty((len(ca), 10))
    lib().orc_step19_cells_f64(nx, ny, nz, float(tau), _p(ma), _p(_f64(F)), _p(ta), _p(ia), _p(ca),
                               len(ca), _p(out))
    return out.T.copy()


def reconstruct19(m10):
    """(f[19], c[19, 3], w[19]) of the D3Q19 reconstruction of one moment set."""
    f = np.empty(19)
    c = np.empty((19, 3), np.int32)
    w = np.empty(19)
    lib().orc_reconstruct19(_p(np.ascontiguousarray(m10, np.float64)), _p(f), _p(c), _p(w))
    return f, c, w


def solid_force(m, shape, tau, typ, wall, F=None, body_id=0, lattice=27):
    """(Fx, Fy, Fz, Tx, Ty, Tz) the next step transfers to body ``body_id`` (0: all
    solids) by momentum exchange; torque about the body's r0."""
    nx, ny, nz = shape
    out = np.zeros(6)
    fn = lib().orc_solid_force19_f64 if lattice == 19 else lib().orc_solid_force_f64
    fn(nx, ny, nz, float(tau), _p(_f64(m)), _p(_f64(F)), _p(np.ascontiguousarray(typ, np.uint8)),
       wall.model, _p(wall.body), _p(wall.table), int(body_id), _p(out))
    return out


def step_complex(m, shape, tau, F=None, typ=None, inflow=None, literal_xyz=False):
    """One step on complex128 inputs (complex-step derivatives)."""
    nx, ny, nz = shape
    mc = np.ascontiguousarray(m, np.complex128)
    out = np.empty_like(mc)
    Fc = None if F is None else np.ascontiguousarray(F, np.complex128)
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    lib().orc_step_c128(nx, ny, nz, float(tau), _p(mc), _p(Fc), _p(ta), _p(_inflow_arr(inflow)),
                        int(literal_xyz), _p(out))
    return out


def step_cells(m, shape, tau, cells, F=None, typ=None, inflow=None):
    """The new state at selected cells only: returns (10, len(cells))."""
    nx, ny, nz = shape
    ma = _f64(m)
    cells = np.ascontiguousarray(cells, np.int64)
    out = np.empty((cells.size, 10))
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    lib().orc_step_cells_f64(nx, ny, nz, float(tau), _p(ma), _p(_f64(F)), _p(ta),
                             _p(_inflow_arr(inflow)), _p(cells), cells.size, _p(out))
    return out.T.copy()


def step_vjp(m, shape, tau, lam_out, F=None, typ=None):
    """Discrete adjoint of one step: returns (dL/dm, dL/dF)."""
    nx, ny, nz = shape
    ma = _f64(m)
    lo = _f64(lam_out)
    li = np.empty_like(ma)
    gF = np.zeros((3, ma.shape[1]))
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    lib().orc_step_vjp_f64(nx, ny, nz, float(tau), _p(ma), _p(_f64(F)), _p(ta), _p(lo), _p(li),
                           _p(gF))
    return li, gF


def reduce(m, typ=None):
    """FP64 total mass and kinetic energy over non-solid cells."""
    ma = _f64(m)
    M = ctypes.c_double()
    E = ctypes.c_double()
    ta = None if typ is None else np.ascontiguousarray(typ, np.uint8)
    lib().orc_reduce(ma.shape[1], _p(ma), _p(ta), ctypes.byref(M), ctypes.byref(E))
    return M.value, E.value


# ---------------------------------------------------------------- 16-bit form
def ranges():
    lo = np.empty(10)
    hi = np.empty(10)
    lib().orc_ranges(_p(lo), _p(hi))
    return lo, hi


def dither(x, y, z, t, seed):
    d = np.empty(10, np.float32)
    lib().orc_dither(x, y, z, t, seed, _p(d))
    return d


# Bit widths (b_rho_u, b_S) of the adaptive allocation (Sec. 6.2.2); (16, 16) is
# the uniform 16-bit codec.
BITS16 = (16, 16)


def codec_constants(k, bits=BITS16):
    """(qc, step, c, K, b) of component k's grid (FP32 values)."""
    out = np.empty(5)
    lib().orc_codec_constants_bits(int(k), int(bits[0]), int(bits[1]), _p(out))
    return out


def mean_code_over_dither(value32, k, bits=BITS16):
    """Expected code of an FP32 codec input over all dither values of component k."""
    return lib().orc_mean_code_over_dither_bits(float(value32), int(k), int(bits[0]), int(bits[1]))


def code_coordinate(value32, k, bits=BITS16):
    """Exact position of an FP32 codec input on the code axis (FP64)."""
    return lib().orc_code_coordinate_bits(float(value32), int(k), int(bits[0]), int(bits[1]))


def public_to_stored(m):
    """(rho, u, S) -> (rho, u, rho S^neq) with rho S^neq = rho (S - u u) (Sec. 5.4)."""
    m = _f64(m)
    rho, u = m[0], m[1:4]
    S = m[4:10]
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    out = np.empty_like(m)
    out[0] = rho
    out[1:4] = u
    for k, (a, b) in enumerate(pairs):
        out[4 + k] = rho * (S[k] - u[a] * u[b])
    return out


def stored_for_codec(s):
    """FP64 stored variables -> the FP32 codec input (component 0 = rho - 1,
    formed in FP64 before the cast)."""
    v = np.array(s, dtype=np.float64, copy=True)
    v[0] = v[0] - 1.0
    return v.astype(np.float32)


def stored_to_public(s):
    s = _f64(s)
    rho, u = s[0], s[1:4]
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    out = np.empty_like(s)
    out[0] = rho
    out[1:4] = u
    for k, (a, b) in enumerate(pairs):
        out[4 + k] = s[4 + k] / rho + u[a] * u[b]
    return out


def encode(stored32, shape, t, seed, deterministic=False, bits=BITS16):
    """FP32 stored variables (10, N), component 0 = rho - 1, -> codes (10, N) of
    b_rho_u / b_S bits (uint16)."""
    nx, ny, nz = shape
    v = np.ascontiguousarray(stored32, np.float32)
    q = np.empty(v.shape, np.uint16)
    lib().orc_encode_bits(nx, ny, nz, _p(v), int(t) & 0xFFFFFFFF, int(seed) & 0xFFFFFFFF,
                          int(deterministic), int(bits[0]), int(bits[1]), _p(q))
    return q


def decode(q, bits=BITS16):
    q = np.ascontiguousarray(q, np.uint16)
    v = np.empty(q.shape, np.float64)
    lib().orc_decode_bits(q.shape[1], _p(q), int(bits[0]), int(bits[1]), _p(v))
    return v


def q16_step(codes, shape, tau, t_out, seed, F=None, typ=None, inflow=None, bits=BITS16, lattice=27):
    """One step of the quantised form: decode, FP64 step, FP32 re-encode with the
    dither of time index ``t_out``.  Solid cells keep their codes; outflow cells
    take the codes of (nx-2, y, z).  ``lattice=19``: the periodic D3Q19 step."""
    pub = stored_to_public(decode(codes, bits))
    if lattice == 19:
        new = step19(pub, shape, tau, F=F, typ=typ, inflow=inflow)
    else:
        new = step(pub, shape, tau, F=F, typ=typ, inflow=inflow)
    q = encode(stored_for_codec(public_to_stored(new)), shape, t_out, seed, bits=bits)
    if typ is not None:
        solid = typ == SOLID
        q[:, solid] = codes[:, solid]
        out_cells = np.nonzero(typ == OUTFLOW)[0]
        q[:, out_cells] = q[:, out_cells - 1]
    return q


# ---------------------------------------------------------------- linearisation
def amplification_matrix(rho0, U, tau, kvecs, h=1e-30):
    """Brute-force moment-space amplification matrices G(k) of one step,
    linearised by complex step about the uniform state (rho0, U, U U) on a
    periodic 4^3 grid: G(k) = sum_d J(d) exp(-i k.d) with J(d) the response at
    offset d to a unit perturbation at the origin.  Returns (len(k), 10, 10)."""
    n = 4
    N = n ** 3
    shape = (n, n, n)
    base = np.zeros((10, N))
    base[0] = rho0
    U = np.asarray(U, float)
    base[1:4] = U[:, None]
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        base[4 + k] = U[a] * U[b]
    J = np.zeros((N, 10, 10))  # J[cell, out, in]
    for j in range(10):
        mc = base.astype(np.complex128)
        mc[j, 0] += 1j * h
        out = step_complex(mc, shape, tau)
        J[:, :, j] = (out.imag / h).T
    # offsets of each cell, wrapped into {-1, 0, 1, 2}
    idx = np.arange(N)
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    off = np.stack([np.where(v > n // 2, v - n, v) for v in (x, y, z)], axis=1).astype(float)
    kv = np.atleast_2d(np.asarray(kvecs, float))
    phase = np.exp(-1j * kv @ off.T)  # (K, N)
    return np.einsum("kn,nij->kij", phase, J)


# ---------------------------------------------------------------- adjoint
def forward_loss(u0, F, shape, tau, nsteps, loss_fn, typ=None, inflow=None, lattice=27):
    """Initial state (1, u0, u0 u0) -> n FP64 steps -> loss_fn(final state)."""
    m = initial_state_from_velocity(u0)
    stepper = step19 if lattice == 19 else step
    m = stepper(m, shape, tau, F=F, typ=typ, inflow=inflow, n=nsteps)
    return loss_fn(m), m


def initial_state_from_velocity(u0):
    u0 = _f64(u0)
    N = u0.shape[1]
    m = np.empty((10, N))
    m[0] = 1.0
    m[1:4] = u0
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        m[4 + k] = u0[a] * u0[b]
    return m


def initial_state_vjp(u0, lam0):
    """dL/du0 from dL/dm0 through m0 = (1, u0, u0 u0)."""
    u0 = _f64(u0)
    g = lam0[1:4].copy()
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for k, (a, b) in enumerate(pairs):
        g[a] += lam0[4 + k] * u0[b]
        g[b] += lam0[4 + k] * u0[a]
    return g


def adjoint(u0, F, shape, tau, nsteps, dloss_dm, K=10, typ=None, inflow=None):
    """Gradient of loss(m_T) w.r.t. (u0, F) by the discrete adjoint of the FP64
    step, recomputing each K-step segment from an FP64 checkpoint."""
    m = initial_state_from_velocity(u0)
    ckpt = {}
    for t in range(nsteps):
        if t % K == 0:
            ckpt[t] = m.copy()
        m = step(m, shape, tau, F=F, typ=typ, inflow=inflow)
    lam = _f64(dloss_dm(m)).copy()
    gF = np.zeros((3, m.shape[1]))
    seg_starts = sorted(ckpt)
    for s in reversed(seg_starts):
        e = min(s + K, nsteps)
        states = [ckpt[s]]
        for _ in range(s, e - 1):
            states.append(step(states[-1], shape, tau, F=F, typ=typ, inflow=inflow))
        for t in reversed(range(s, e)):
            lam, g = step_vjp(states[t - s], shape, tau, lam, F=F, typ=typ)
            gF += g
    return initial_state_vjp(u0, lam), gF
