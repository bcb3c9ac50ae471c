"""The identity behind the boundary update (host logic on the FP64 oracle, no GPU).

With solids, the fluid kernel lets every solid cell enter the stream at rest
(post-collision populations f+_i = w_i, i.e. zero moments about the rest state)
and keeps the raw post-streaming sums (sum f, sum c f, sum (c c - I/3) f) of each
FLUID_BOUNDARY cell; the boundary kernel then adds, for every solid link i of
the cell, what halfway bounce-back returns there instead, f+_opp(i)(x) - w_i, from
the cell's own post-collision state (split design of Sec. 4.2).  This test
restates that decomposition with the oracle's primitives -- a periodic step of a
state whose solid cells are at rest, and the collision (App. A) and
reconstruction (Eq. three_order_f, or the D3Q19 projection) of each boundary cell
-- and checks that it gives the raw sums of the oracle's full step with
bounce-back, on random masks with inflow and outflow, for both lattices and on
grids small enough for the periodic wrap to alias neighbours.  A planted slip
(returning f+_i(x) instead of f+_opp(i)(x)) must fail."""
import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
C = np.array([((i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1) for i in range(27)])


def raw_sums(m, F):
    """(rho, rho u - F/2, rho S) of public moments m (10, N): the sums
    sum f, sum c f and sum (c c - I/3) f of Eq. rho_u_stress."""
    r = np.empty_like(m)
    r[0] = m[0]
    r[1:4] = m[0] * m[1:4] - 0.5 * F
    r[4:] = m[0] * m[4:]
    return r


def random_state(N, rng):
    m = np.zeros((10, N))
    m[0] = 1.0 + 0.01 * rng.standard_normal(N)
    m[1:4] = 0.05 * rng.standard_normal((3, N))
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = m[1 + a] * m[1 + b] + 0.002 * rng.standard_normal(N)
    return m


def populations(orc, m_cell, F_cell, tau, q19):
    """Post-collision populations f+ of one cell, indexed by the 27 directions
    (zero for the corners on D3Q19)."""
    mc = orc.collide(m_cell[None], F_cell[None], tau)[0]
    if not q19:
        return orc.reconstruct(mc[None])[0]
    f19, c19, _ = orc.reconstruct19(mc)
    f = np.zeros(27)
    for fi, c in zip(f19, c19):
        f[(c[0] + 1) + 3 * (c[1] + 1) + 9 * (c[2] + 1)] = fi
    return f


def decomposed(orc, shape, m, F, tau, typ, inflow, q19, bounce=lambda i: 26 - i):
    """The raw sums of every FLUID_BOUNDARY cell by the split: periodic step with
    the solids at rest, plus the bounced populations of the cell's solid links."""
    nx, ny, nz = shape
    N = nx * ny * nz
    solid = typ == orc.SOLID
    m_rest = m.copy()
    m_rest[:, solid] = 0.0
    m_rest[0, solid] = 1.0
    F_rest = F.copy()
    F_rest[:, solid] = 0.0
    step = orc.step19 if q19 else orc.step
    fluid = raw_sums(step(m_rest, shape, tau, F=F_rest), F_rest)
    _, w = orc.lattice()
    if q19:
        w = np.zeros(27)
        n2 = (C * C).sum(1)
        w[n2 == 0], w[n2 == 1], w[n2 == 2] = 1 / 3, 1 / 18, 1 / 36
    fb = np.nonzero(typ == orc.FLUID_BOUNDARY)[0]
    out = {}
    for n in fb.tolist():
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        f = populations(orc, m[:, n], F[:, n], tau, q19)
        r = fluid[:, n].copy()
        for i in range(27):
            if q19 and (C[i] ** 2).sum() > 2:
                continue
            s = ((x - C[i][0]) % nx) + nx * (((y - C[i][1]) % ny) + ny * ((z - C[i][2]) % nz))
            if not solid[s]:
                continue
            g = f[bounce(i)] - w[i]  # what bounce-back returns, minus the rest population pulled
            c = C[i]
            r[0] += g
            r[1:4] += c * g
            r[4:] += np.array([c[a] * c[b] - (a == b) / 3.0 for a, b in PAIRS]) * g
        out[n] = r
    return out


@pytest.mark.parametrize("shape", [(9, 7, 6), (6, 5, 4), (5, 3, 3)])
@pytest.mark.parametrize("q19", [False, True])
def test_split_boundary_update_equals_the_full_step(orc, shape, q19):
    rng = np.random.default_rng(sum(shape) + 11 * q19)
    nx, ny, nz = shape
    N = nx * ny * nz
    tau = 0.6
    for dens, (inflow_on, outflow_on) in ((0.15, (True, True)), (0.3, (False, False))):
        mask = (rng.random((nz, ny, nx)) < dens).astype(np.uint8)
        typ, _, _, _ = orc.classify(mask, inflow_on, outflow_on)
        m = random_state(N, rng)
        F = 1e-4 * rng.standard_normal((3, N))
        inflow = [1.0, 0.03, 0.0, 0.01] if inflow_on else None
        step = orc.step19 if q19 else orc.step
        truth = raw_sums(step(m, shape, tau, F=F, typ=typ, inflow=inflow), F)
        got = decomposed(orc, shape, m, F, tau, typ, inflow, q19)
        assert got, "no FLUID_BOUNDARY cell"
        for n, r in got.items():
            assert np.abs(r - truth[:, n]).max() < 1e-14, (n, r, truth[:, n])


def test_a_planted_bounce_mistake_is_caught(orc):
    """Returning f+_i(x) instead of f+_opp(i)(x) on the solid links breaks the identity."""
    shape = (7, 5, 4)
    rng = np.random.default_rng(5)
    N = 7 * 5 * 4
    mask = W.channel_walls(shape)
    typ, _, _, _ = orc.classify(mask)
    m = random_state(N, rng)
    F = np.zeros((3, N))
    truth = raw_sums(orc.step(m, shape, 0.6, F=F, typ=typ), F)
    got = decomposed(orc, shape, m, F, 0.6, typ, None, False, bounce=lambda i: i)
    err = max(np.abs(r - truth[:, n]).max() for n, r in got.items())
    assert err > 1e-4, err
