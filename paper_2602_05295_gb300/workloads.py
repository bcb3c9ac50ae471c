"""Seeded synthetic inputs for the five benchmark workloads.

This module holds input generators only -- velocity fields, force fields and
solid masks -- and none of the lattice Boltzmann arithmetic, so that the CUDA
path and the FP64 oracle can be fed identical inputs.  Every generator is a
pure function of its arguments and a numpy ``default_rng`` seed.

Array conventions: velocity and force fields are float arrays of shape
``(3, nz, ny, nx)``; masks are ``uint8`` arrays of shape ``(nz, ny, nx)`` with
1 = solid; the linear cell index is ``n = x + nx (y + ny z)``.

The paper's own scenes rely on triangle meshes (motorcycle, car, skeleton,
delta wing, porous solids) that are not available; the sphere packing and the
procedural box/ellipsoid obstacle stand in for them at the paper's grid sizes
(512x256x256 and 1000x400x400).
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED = 2602


# ----------------------------------------------------------------- configurations
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    shape: tuple  # (nx, ny, nz)
    tau: float
    steps: int
    storage: str  # "f32", "q16" or "both"
    description: str

    @property
    def cells(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


TGV32 = Workload("tgv32", (32, 32, 32), 0.6, 100, "f32",
                 "Taylor-Green vortex, 32^3 periodic, u0=0.05, k=2pi/32, rho=1")
TURB256 = Workload("turbulence256", (256, 256, 256), 0.52, 1000, "both",
                   "decaying turbulence, 256^3 periodic, k^-5/3 random-phase field, max|u|=0.08")
CHANNEL512 = Workload("channel512", (512, 256, 256), 0.55, 2000, "q16",
                      "channel past 300 random spheres, inflow u=(0.05,0,0), walls in y and z")
LARGE1000 = Workload("large1000", (1000, 400, 400), 0.505, 1000, "q16",
                     "1000x400x400 flow past 40 random boxes/ellipsoids, inflow u=(0.06,0,0)")
ADJOINT128 = Workload("adjoint128", (128, 128, 128), 0.55, 200, "f32",
                      "adjoint, 128^3 periodic, random-phase u0 (max 0.05), trainable force")

# the grid size of the paper's one D3Q19 scene (Table 1), with a procedural obstacle
# standing in for its mesh
SCENE720 = Workload("scene720_d3q19", (720, 360, 360), 0.55, 1000, "q16",
                    "D3Q19, 720x360x360 flow past 30 random boxes/ellipsoids, inflow u=(0.05,0,0)")

ALL = (TGV32, TURB256, CHANNEL512, LARGE1000, ADJOINT128)


def scene720_obstacle(shape=SCENE720.shape):
    """The obstacle of the 720 x 360 x 360 scene: 30 boxes/ellipsoids, half-extents
    in [8, 45], centres in x [100, 430), y [80, 280), z [80, 280), plus walls."""
    return procedural_obstacle(shape, count=30, hmin=8.0, hmax=45.0, seed=SEED + 9,
                               region=((100, 430), (80, 280), (80, 280)))


# ----------------------------------------------------------------- velocity fields
def taylor_green(shape, u0=0.05, wavelength=None):
    """u = u0 (sin kx cos ky, -cos kx sin ky, 0), z-invariant, k = 2 pi / wavelength."""
    nx, ny, nz = shape
    lam = nx if wavelength is None else wavelength
    k = 2.0 * np.pi / lam
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y)
    return u, k


def random_phase_field(shape, umax, kmin=1, kmax=16, slope=-5.0 / 3.0, seed=SEED):
    """Divergence-free random-phase field with shell energy ~ k^slope for kmin<=|k|<=kmax.

    Each Fourier amplitude is a complex Gaussian with a uniform random phase,
    projected perpendicular to k; |u_hat|^2 ~ k^(slope-2) so that the shell
    energy E(k) ~ 4 pi k^2 |u_hat|^2 ~ k^slope.  The real part of the inverse
    FFT is taken (Hermitian symmetrisation), then the field is scaled so that
    max |u| = umax."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    band = (kk >= kmin) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[band] = kk[band] ** ((slope - 2.0) / 2.0)
    uh = np.empty((3,) + kk.shape, np.complex128)
    for a in range(3):
        g = rng.standard_normal(kk.shape)
        ph = rng.uniform(0.0, 2.0 * np.pi, kk.shape)
        uh[a] = g * np.exp(1j * ph) * amp
    # project perpendicular to k
    kvec = [np.broadcast_to(kx, kk.shape), np.broadcast_to(ky, kk.shape),
            np.broadcast_to(kz, kk.shape)]
    safe = np.where(k2 > 0, k2, 1.0)
    dot = (kvec[0] * uh[0] + kvec[1] * uh[1] + kvec[2] * uh[2]) / safe
    for a in range(3):
        uh[a] -= kvec[a] * dot
    u = np.empty((3, nz, ny, nx))
    for a in range(3):
        u[a] = np.fft.ifftn(uh[a]).real
    mag = np.sqrt((u * u).sum(0)).max()
    return u * (umax / mag)


def force_field(shape, fmax=1e-5, seed=SEED + 5):
    """Seeded normal force field scaled to max |F_a| = fmax."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((3, nz, ny, nx))
    return F * (fmax / np.abs(F).max())


# ----------------------------------------------------------------- solid masks
def channel_walls(shape):
    """One-cell solid layers at y in {0, ny-1} and z in {0, nz-1}."""
    nx, ny, nz = shape
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, 0, :] = 1
    m[:, ny - 1, :] = 1
    m[0, :, :] = 1
    m[nz - 1, :, :] = 1
    return m


def sphere_pack(shape, count=300, rmin=4.0, rmax=20.0, seed=SEED + 3, max_tries=200000):
    """Non-overlapping spheres by rejection sampling; r^3 uniform in [rmin^3, rmax^3].

    Centres are uniform in [r+8, nx-r-8] x [r+2, ny-r-2] x [r+2, nz-r-2].
    Returns (mask, spheres) with spheres an (count, 4) array of (cx, cy, cz, r)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    spheres = []
    tries = 0
    while len(spheres) < count and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin ** 3, rmax ** 3) ** (1.0 / 3.0)
        c = np.array([rng.uniform(r + 8, nx - r - 8), rng.uniform(r + 2, ny - r - 2),
                      rng.uniform(r + 2, nz - r - 2)])
        ok = True
        for s in spheres:
            if np.sum((c - s[:3]) ** 2) < (r + s[3]) ** 2:
                ok = False
                break
        if ok:
            spheres.append(np.array([c[0], c[1], c[2], r]))
    spheres = np.array(spheres)
    m = channel_walls(shape)
    for cx, cy, cz, r in spheres:
        x0, x1 = int(np.floor(cx - r)), int(np.ceil(cx + r)) + 1
        y0, y1 = int(np.floor(cy - r)), int(np.ceil(cy + r)) + 1
        z0, z1 = int(np.floor(cz - r)), int(np.ceil(cz + r)) + 1
        x0, y0, z0 = max(x0, 0), max(y0, 0), max(z0, 0)
        x1, y1, z1 = min(x1, nx), min(y1, ny), min(z1, nz)
        xs = np.arange(x0, x1)[None, None, :]
        ys = np.arange(y0, y1)[None, :, None]
        zs = np.arange(z0, z1)[:, None, None]
        inside = (xs - cx) ** 2 + (ys - cy) ** 2 + (zs - cz) ** 2 <= r * r
        m[z0:z1, y0:y1, x0:x1] |= inside.astype(np.uint8)
    return m, spheres


def sphere_bodies(shape, spheres, max_bodies=254):
    """Body ids for a sphere pack (the solid mask values): sphere k < max_bodies is
    body k + 1, the channel walls and any further spheres are body 255."""
    nx, ny, nz = shape
    m = channel_walls(shape) * np.uint8(255)
    for k, (cx, cy, cz, r) in enumerate(spheres):
        x0, x1 = max(int(np.floor(cx - r)), 0), min(int(np.ceil(cx + r)) + 1, nx)
        y0, y1 = max(int(np.floor(cy - r)), 0), min(int(np.ceil(cy + r)) + 1, ny)
        z0, z1 = max(int(np.floor(cz - r)), 0), min(int(np.ceil(cz + r)) + 1, nz)
        xs = np.arange(x0, x1)[None, None, :]
        ys = np.arange(y0, y1)[None, :, None]
        zs = np.arange(z0, z1)[:, None, None]
        inside = (xs - cx) ** 2 + (ys - cy) ** 2 + (zs - cz) ** 2 <= r * r
        sub = m[z0:z1, y0:y1, x0:x1]
        sub[inside] = np.uint8(k + 1 if k < max_bodies else 255)
    return m


def procedural_obstacle(shape, count=40, hmin=10.0, hmax=60.0, seed=SEED + 4,
                        region=((100, 600), (100, 300), (75, 325))):
    """Union of seeded boxes and ellipsoids (probability 1/2 each) with half-extents
    uniform in [hmin, hmax], centres uniform in `region`, clipped to `region`."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    m = channel_walls(shape)
    (rx0, rx1), (ry0, ry1), (rz0, rz1) = region
    shapes = []
    for _ in range(count):
        kind = "box" if rng.uniform() < 0.5 else "ellipsoid"
        h = rng.uniform(hmin, hmax, 3)
        c = np.array([rng.uniform(rx0, rx1), rng.uniform(ry0, ry1), rng.uniform(rz0, rz1)])
        shapes.append((kind, c, h))
        x0, x1 = max(int(np.floor(c[0] - h[0])), rx0), min(int(np.ceil(c[0] + h[0])) + 1, rx1)
        y0, y1 = max(int(np.floor(c[1] - h[1])), ry0), min(int(np.ceil(c[1] + h[1])) + 1, ry1)
        z0, z1 = max(int(np.floor(c[2] - h[2])), rz0), min(int(np.ceil(c[2] + h[2])) + 1, rz1)
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        xs = np.arange(x0, x1)[None, None, :]
        ys = np.arange(y0, y1)[None, :, None]
        zs = np.arange(z0, z1)[:, None, None]
        if kind == "box":
            inside = ((np.abs(xs - c[0]) <= h[0]) & (np.abs(ys - c[1]) <= h[1])
                      & (np.abs(zs - c[2]) <= h[2]))
        else:
            inside = (((xs - c[0]) / h[0]) ** 2 + ((ys - c[1]) / h[1]) ** 2
                      + ((zs - c[2]) / h[2]) ** 2) <= 1.0
        m[z0:z1, y0:y1, x0:x1] |= inside.astype(np.uint8)
    return m, shapes


def random_mask(shape, density=0.2, seed=SEED + 7):
    """Uniform random solid mask (classification tests)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=(nz, ny, nx)) < density).astype(np.uint8)


def flat(field):
    """(c, nz, ny, nx) -> (c, N) with n = x + nx (y + ny z)."""
    field = np.asarray(field)
    return field.reshape(field.shape[0], -1)
