"""Thin ctypes binding of ``include/melbm.h`` (argument marshalling only).

Every step of the update runs in the CUDA kernels of ``libmelbm.so``; this module
only converts torch tensors to pointers, checks shapes and turns status codes
into exceptions.  There is no CPU fallback: if the library is missing or the
device is not a CUDA GPU, the calls raise.

Field tensors are float32, contiguous, with ``N = nx * ny * nz`` cells in the
order ``n = x + nx (y + ny z)``: ``rho`` has N elements, ``u`` 3N
(``(3, N)`` or ``(3, nz, ny, nx)``), ``S`` 6N ordered (xx, yy, zz, xy, xz, yz).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ESTATE, WSATURATED = 0, 1, 2, 3, 4, 5
F32, Q16, MIXED = 0, 1, 2
FLUID, FLUID_BOUNDARY, INFLOW, OUTFLOW, SOLID = 0, 1, 2, 3, 4
_STORAGE = {"f32": F32, "q16": Q16, "mixed": MIXED}

_lib = None


class MelbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"melbm error {code}: {msg}")
        self.code = code


class SaturationWarning(UserWarning):
    pass


def lib():
    """Load libmelbm.so (build it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        _build.build()
    L = ctypes.CDLL(path)
    P, I, I64, U32, F, D = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                            ctypes.c_float, ctypes.c_double)
    sig = {
        "melbm_create": [I, I, I, I, F, I, ctypes.POINTER(P)],
        "melbm_destroy": [P],
        "melbm_set_stream": [P, P],
        "melbm_set_seed": [P, U32],
        "melbm_set_state": [P, P, P, P],
        "melbm_get_moments": [P, P, P, P],
        "melbm_set_solid": [P, P],
        "melbm_set_inflow": [P, I, F, F, F, F],
        "melbm_set_outflow": [P, I],
        "melbm_get_boundary_list": [P, P, P, I64, ctypes.POINTER(I64)],
        "melbm_get_types": [P, P],
        "melbm_set_force": [P, P],
        "melbm_step": [P, I],
        "melbm_reduce": [P, ctypes.POINTER(D), ctypes.POINTER(D)],
        "melbm_time_index": [P, ctypes.POINTER(I64)],
        "melbm_memory_bytes": [P, ctypes.POINTER(I64)],
        "melbm_state_bytes": [P, ctypes.POINTER(I64)],
        "melbm_get_raw_state": [P, P, I64],
        "melbm_set_raw_state": [P, P, I64, I64],
        "melbm_upload_raw_state_async": [P, P, I64, I64],
        "melbm_download_raw_state_async": [P, P, I64],
        "melbm_sync_transfers": [P],
        "melbm_forward_checkpointed": [P, P, I, I],
        "melbm_backward": [P, P, P, P],
        "melbm_q16_encode": [P, I, I, I, U32, U32, I, P, P],
        "melbm_q16_decode": [P, I64, P, P],
        "melbm_set_bits": [P, I, I],
        "melbm_set_wall_model": [P, I],
        "melbm_set_body_motion": [P, I, P, P, P],
        "melbm_solid_force": [P, I, P],
        "melbm_codec_encode": [P, I, I, I, U32, U32, I, I, I, P, P],
        "melbm_codec_decode": [P, I64, I, I, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = I
    L.melbm_last_error.argtypes = [P]
    L.melbm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points the loaded library exports (checked by tests)."""
    L = lib()
    names = []
    for line in open(os.path.join(os.path.dirname(_build.HERE), "include", "melbm.h")):
        line = line.strip()
        if line.startswith("MELBM_API"):
            names.append(line.split("(")[0].split()[-1].lstrip("*"))
    return [n for n in names if hasattr(L, n)]


def _check(code, handle=None):
    if code == OK:
        return code
    msg = lib().melbm_last_error(handle).decode(errors="replace")
    if code == WSATURATED:
        import warnings
        warnings.warn(msg, SaturationWarning)
        return code
    raise MelbmError(code, msg)


def _ptr(t, numel=None, dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Simulator:
    """One moment-encoded LBM simulation on the current CUDA device.

    ``storage`` is ``"f32"``, ``"q16"`` (the paper's 16-bit form) or ``"mixed"``
    (the paper's mixed-precision scheme with solids, kept for comparison).
    ``lattice`` is 27 (D3Q27) or 19 (D3Q19: the same storage forms, boundaries,
    walls and adjoint over the 19 velocities).  Work is enqueued on ``stream``
    (default: torch's current stream at construction)."""

    def __init__(self, shape, tau, storage="q16", stream=None, seed=0, lattice=27):
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.tau = float(tau)
        self.storage = storage
        self.lattice = int(lattice)
        h = ctypes.c_void_p()
        _check(lib().melbm_create(nx, ny, nz, self.lattice, ctypes.c_float(tau), _STORAGE[storage],
                                  ctypes.byref(h)))
        self._h = h
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().melbm_set_stream(h, _stream_ptr(self.stream)), h)
        _check(lib().melbm_set_seed(h, ctypes.c_uint32(seed & 0xFFFFFFFF)), h)

    # -------------------------------------------------------------- life cycle
    def close(self):
        if getattr(self, "_h", None):
            lib().melbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- state
    def set_state(self, rho, u, S=None):
        N = self.N
        _check(lib().melbm_set_state(self._h, _ptr(rho, N, name="rho"), _ptr(u, 3 * N, name="u"),
                                     _ptr(S, 6 * N, name="S")), self._h)

    def get_moments(self, rho=None, u=None, S=None, device=None):
        """Returns (rho[N], u[3, N], S[6, N]) as float32 tensors (allocated on
        ``device`` -- default the current CUDA device -- unless given)."""
        N = self.N
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        rho = torch.empty(N, dtype=torch.float32, device=dev) if rho is None else rho
        u = torch.empty(3, N, dtype=torch.float32, device=dev) if u is None else u
        S = torch.empty(6, N, dtype=torch.float32, device=dev) if S is None else S
        _check(lib().melbm_get_moments(self._h, _ptr(rho, N), _ptr(u, 3 * N), _ptr(S, 6 * N)),
               self._h)
        return rho, u, S

    def state_bytes(self):
        b = ctypes.c_int64()
        _check(lib().melbm_state_bytes(self._h, ctypes.byref(b)), self._h)
        return b.value

    def get_raw_state(self, dst=None):
        nb = self.state_bytes()
        if dst is None:
            dst = torch.empty(nb, dtype=torch.uint8, device="cuda")
        _check(lib().melbm_get_raw_state(self._h, _ptr(dst, nb, torch.uint8), nb), self._h)
        return dst

    def set_raw_state(self, src, time_index):
        nb = self.state_bytes()
        _check(lib().melbm_set_raw_state(self._h, _ptr(src, nb, torch.uint8), nb, int(time_index)),
               self._h)

    def upload_raw_state_async(self, src, time_index):
        """Make the packed state in ``src`` (pinned host uint8 for overlap) the
        current state, without blocking; ``src`` must stay unchanged until
        :meth:`sync_transfers`."""
        nb = self.state_bytes()
        _check(lib().melbm_upload_raw_state_async(self._h, _ptr(src, nb, torch.uint8), nb,
                                                  int(time_index)), self._h)

    def download_raw_state_async(self, dst):
        """Copy the current packed state into ``dst`` without blocking; ``dst`` is
        valid after :meth:`sync_transfers`."""
        nb = self.state_bytes()
        _check(lib().melbm_download_raw_state_async(self._h, _ptr(dst, nb, torch.uint8), nb),
               self._h)
        return dst

    def sync_transfers(self):
        _check(lib().melbm_sync_transfers(self._h), self._h)

    # -------------------------------------------------------------- boundaries
    def set_solid(self, mask):
        _check(lib().melbm_set_solid(self._h, _ptr(mask, self.N, torch.uint8, "mask")), self._h)

    def set_inflow(self, rho, u):
        ux, uy, uz = (float(v) for v in u)
        _check(lib().melbm_set_inflow(self._h, 0, rho, ux, uy, uz), self._h)

    def set_outflow(self):
        _check(lib().melbm_set_outflow(self._h, 1), self._h)

    def set_force(self, F):
        _check(lib().melbm_set_force(self._h, _ptr(F, 3 * self.N, name="F")), self._h)

    def set_wall_model(self, model):
        """0: halfway bounce-back; 1: moment-based reconstruction at moving walls."""
        _check(lib().melbm_set_wall_model(self._h, int(model)), self._h)

    def set_body_motion(self, body, V=(0, 0, 0), Omega=(0, 0, 0), r0=(0, 0, 0)):
        """Rigid motion of body ``body`` (the solid mask value, 1..255)."""
        arr = [(ctypes.c_float * 3)(*map(float, v)) for v in (V, Omega, r0)]
        _check(lib().melbm_set_body_motion(self._h, int(body), *[ctypes.cast(a, ctypes.c_void_p) for a in arr]),
               self._h)

    def solid_force(self, body=0):
        """(Fx, Fy, Fz, Tx, Ty, Tz) the next step transfers to body ``body`` (0: all)."""
        out = (ctypes.c_double * 6)()
        _check(lib().melbm_solid_force(self._h, int(body), ctypes.cast(out, ctypes.c_void_p)), self._h)
        return np.array(list(out))

    def set_bits(self, bits_rho_u, bits_S):
        """Bit widths b_rho_u / b_S of the quantised form (8..16 each); re-encodes
        the current state."""
        _check(lib().melbm_set_bits(self._h, int(bits_rho_u), int(bits_S)), self._h)

    def boundary_list(self):
        cnt = ctypes.c_int64()
        _check(lib().melbm_get_boundary_list(self._h, None, None, 0, ctypes.byref(cnt)), self._h)
        L = cnt.value
        cells = torch.empty(max(L, 1), dtype=torch.int32, device="cuda")
        words = torch.empty(max(L, 1), dtype=torch.int32, device="cuda")
        _check(lib().melbm_get_boundary_list(self._h, ctypes.c_void_p(cells.data_ptr()),
                                             ctypes.c_void_p(words.data_ptr()), L,
                                             ctypes.byref(cnt)), self._h)
        return cells[:L], words[:L]

    def types(self):
        t = torch.empty(self.N, dtype=torch.uint8, device="cuda")
        _check(lib().melbm_get_types(self._h, ctypes.c_void_p(t.data_ptr())), self._h)
        return t

    # -------------------------------------------------------------- stepping
    def step(self, n=1):
        _check(lib().melbm_step(self._h, int(n)), self._h)

    def reduce(self):
        M, E = ctypes.c_double(), ctypes.c_double()
        _check(lib().melbm_reduce(self._h, ctypes.byref(M), ctypes.byref(E)), self._h)
        return M.value, E.value

    @property
    def time_index(self):
        t = ctypes.c_int64()
        _check(lib().melbm_time_index(self._h, ctypes.byref(t)), self._h)
        return t.value

    def memory_bytes(self):
        b = ctypes.c_int64()
        _check(lib().melbm_memory_bytes(self._h, ctypes.byref(b)), self._h)
        return b.value

    # -------------------------------------------------------------- adjoint
    def forward_checkpointed(self, u0, nsteps, K):
        _check(lib().melbm_forward_checkpointed(self._h, _ptr(u0, 3 * self.N, name="u0"),
                                                int(nsteps), int(K)), self._h)

    def backward(self, dL_dm, dL_du0=None, dL_dF=None):
        N = self.N
        dL_du0 = torch.empty(3, N, dtype=torch.float32, device="cuda") if dL_du0 is None else dL_du0
        _check(lib().melbm_backward(self._h, _ptr(dL_dm, 10 * N, name="dL_dm"), _ptr(dL_du0, 3 * N),
                                    _ptr(dL_dF, 3 * N)), self._h)
        return dL_du0, dL_dF


# ------------------------------------------------------------------ codec
def q16_encode(stored, shape, t, seed, deterministic=False, stream=None):
    """FP32 stored variables (10, N) -> int32 words (5, N) holding two 16-bit codes."""
    nx, ny, nz = shape
    N = nx * ny * nz
    words = torch.empty(5, N, dtype=torch.int32, device=stored.device)
    _check(lib().melbm_q16_encode(_ptr(stored, 10 * N), nx, ny, nz, ctypes.c_uint32(t & 0xFFFFFFFF),
                                  ctypes.c_uint32(seed & 0xFFFFFFFF), int(deterministic),
                                  ctypes.c_void_p(words.data_ptr()), _stream_ptr(stream)))
    return words


def q16_decode(words, stream=None):
    N = words.shape[-1]
    out = torch.empty(10, N, dtype=torch.float32, device=words.device)
    _check(lib().melbm_q16_decode(_ptr(words, 5 * N, torch.int32), N, ctypes.c_void_p(out.data_ptr()),
                                  _stream_ptr(stream)))
    return out


def codec_encode(stored, shape, t, seed, bits, deterministic=False, stream=None):
    """FP32 stored variables (10, N) -> int32 words (5, N) of b_rho_u / b_S-bit codes."""
    nx, ny, nz = shape
    N = nx * ny * nz
    words = torch.empty(5, N, dtype=torch.int32, device=stored.device)
    _check(lib().melbm_codec_encode(_ptr(stored, 10 * N), nx, ny, nz,
                                    ctypes.c_uint32(t & 0xFFFFFFFF),
                                    ctypes.c_uint32(seed & 0xFFFFFFFF), int(deterministic),
                                    int(bits[0]), int(bits[1]),
                                    ctypes.c_void_p(words.data_ptr()), _stream_ptr(stream)))
    return words


def codec_decode(words, bits, stream=None):
    N = words.shape[-1]
    out = torch.empty(10, N, dtype=torch.float32, device=words.device)
    _check(lib().melbm_codec_decode(_ptr(words, 5 * N, torch.int32), N, int(bits[0]), int(bits[1]),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def words_to_codes(words):
    """(5, N) int32 words -> (10, N) int64 codes (low half = even component)."""
    w = words.to(torch.int64) & 0xFFFFFFFF
    lo = w & 0xFFFF
    hi = (w >> 16) & 0xFFFF
    return torch.stack([lo, hi], 1).reshape(10, -1)
