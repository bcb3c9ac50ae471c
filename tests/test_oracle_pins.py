"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_constants.json), closed forms (Hermite moment
identities, Taylor-Green decay, Poiseuille profile, hydrodynamic modes),
invariants (conservation, fixed points, lattice symmetries) and brute force
(classification, complex-step derivatives).  A plausible slip anywhere in the
oracle -- a dropped term, a wrong sign or index, a transposed operand -- fails
at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2602_05295_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
CS2 = 1.0 / 3.0


def sget(S, a, b):
    return S[PAIRS.index(tuple(sorted((a, b))))]


def random_cells(n, rng, du=0.1, ds=0.01, drho=0.05):
    m = np.zeros((n, 10))
    m[:, 0] = 1.0 + drho * rng.standard_normal(n)
    m[:, 1:4] = du * rng.standard_normal((n, 3))
    for k, (a, b) in enumerate(PAIRS):
        m[:, 4 + k] = m[:, 1 + a] * m[:, 1 + b] + ds * rng.standard_normal(n)
    return m


def random_state(shape, rng, du=0.05, ds=0.002, drho=0.01):
    N = int(np.prod(shape))
    return random_cells(N, rng, du, ds, drho).T.copy()


def eq_state(rho, u):
    """(rho, u, S = u u) for u of shape (3, N)."""
    N = u.shape[1]
    m = np.zeros((10, N))
    m[0] = rho
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b]
    return m


# ------------------------------------------------------------------ lattice
def test_lattice_weights_marginalise_to_paper_d2q9(orc):
    """App. D prints the D2Q9 weights; the D3Q27 weights summed over c_z give them."""
    c, w = orc.lattice()
    g = GOLD["d2q9"]
    for cx, cy, num, den in zip(g["cx"], g["cy"], g["w_num"], g["w_den"]):
        sel = (c[:, 0] == cx) & (c[:, 1] == cy)
        assert abs(w[sel].sum() - num / den) < 1e-15
    assert abs(w.sum() - 1.0) < 1e-15
    # isotropy up to 4th order with c_s^2 = 1/3 (paper value)
    cs2 = g["cs2_num"] / g["cs2_den"]
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((w * c[:, a] * c[:, b]).sum() - cs2 * (a == b)) < 1e-15
    assert abs((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum() - cs2 ** 2) < 1e-15
    assert abs((w * c[:, 0] ** 4).sum() - 3 * cs2 ** 2) < 1e-15
    # opposite direction is 26 - i
    assert np.all(c[::-1] == -c)


# ------------------------------------------------------------------ P1 moment identities
def test_reconstruction_moments_identity(orc):
    """m(h(rho,u,S)) = (rho, u, S): the Hermite reconstruction reproduces the
    moments it is built from (Eq. three_order_f with Eq. rho_u_stress)."""
    rng = np.random.default_rng(1)
    m = random_cells(64, rng)
    f = orc.reconstruct(m)
    back = orc.moments(f)
    assert np.abs(back - m).max() < 1e-14


def test_reconstruction_third_moments(orc):
    """The third Hermite moments of h equal rho T_abg for all seven triples
    (reading: the xyz triple carries 1/c_s^6); with the printed factor the xyz
    moment comes out halved, which is why that reading is taken."""
    rng = np.random.default_rng(2)
    m = random_cells(32, rng)
    c, _ = orc.lattice()
    for literal in (False, True):
        f = orc.reconstruct(m, literal_xyz=literal)
        for (a, b, g) in [(0, 0, 1), (0, 1, 1), (0, 0, 2), (0, 2, 2), (1, 2, 2), (1, 1, 2), (0, 1, 2)]:
            H3 = (c[:, a] * c[:, b] * c[:, g]
                  - CS2 * (c[:, a] * (b == g) + c[:, b] * (a == g) + c[:, g] * (a == b)))
            got = (f * H3).sum(1)
            S = m[:, 4:].T
            u = m[:, 1:4].T
            T = (sget(S, a, b) * u[g] + sget(S, a, g) * u[b] + sget(S, b, g) * u[a]
                 - 2 * u[a] * u[b] * u[g])
            want = m[:, 0] * T
            err = np.abs(got - want).max()
            if (a, b, g) == (0, 1, 2) and literal:
                assert np.abs(got - 0.5 * want).max() < 1e-15
            else:
                assert err < 1e-15, ((a, b, g), literal, err)


def test_reconstruction_equals_full_tensor_hermite(orc):
    """Textbook form: f = w rho [1 + c.u/cs2 + H2:S/(2 cs2^2) + H3:T/(6 cs2^3)] with
    the sums over all 9 / 27 index tuples (Shan-Yuan-Chen truncation)."""
    rng = np.random.default_rng(3)
    m = random_cells(16, rng)
    c, w = orc.lattice()
    f = orc.reconstruct(m)
    for n in range(m.shape[0]):
        rho, u, S = m[n, 0], m[n, 1:4], m[n, 4:]
        Sm = np.array([[sget(S, a, b) for b in range(3)] for a in range(3)])
        T = np.einsum("ab,g->abg", Sm, u) + np.einsum("ag,b->abg", Sm, u) + \
            np.einsum("bg,a->abg", Sm, u) - 2 * np.einsum("a,b,g->abg", u, u, u)
        for i in range(27):
            ci = c[i].astype(float)
            H2 = np.outer(ci, ci) - CS2 * np.eye(3)
            H3 = (np.einsum("a,b,g->abg", ci, ci, ci)
                  - CS2 * (np.einsum("a,bg->abg", ci, np.eye(3)) + np.einsum("b,ag->abg", ci, np.eye(3))
                           + np.einsum("g,ab->abg", ci, np.eye(3))))
            want = w[i] * rho * (1 + ci @ u / CS2 + (H2 * Sm).sum() / (2 * CS2 ** 2)
                                 + (H3 * T).sum() / (6 * CS2 ** 3))
            assert abs(f[n, i] - want) < 1e-15


# ------------------------------------------------------------------ collision
def test_collision_conserves_and_relaxes(orc):
    """App. A without force: rho and u unchanged, trace of S set to |u|^2, the
    deviatoric non-equilibrium part multiplied by (1 - 1/tau); with force the
    velocity gains F/(2 rho) (App. A, printed factor 1/2)."""
    rng = np.random.default_rng(4)
    m = random_cells(50, rng)
    for tau in (0.51, 0.6, 1.0, 1.7):
        o = orc.collide(m, tau=tau)
        assert np.abs(o[:, :4] - m[:, :4]).max() < 1e-15
        u = m[:, 1:4]
        uu = np.stack([u[:, a] * u[:, b] for a, b in PAIRS], 1)
        neq_in = m[:, 4:] - uu
        neq_out = o[:, 4:] - uu
        tr_in = neq_in[:, :3].sum(1)
        dev_in = neq_in.copy()
        dev_in[:, :3] -= tr_in[:, None] / 3
        assert np.abs(neq_out[:, :3].sum(1)).max() < 1e-15
        assert np.abs(neq_out - (1 - 1 / tau) * dev_in).max() < 1e-15
    F = 1e-3 * rng.standard_normal((50, 3))
    o = orc.collide(m, F, tau=0.6)
    k = GOLD["collision"]["velocity_force_factor_num"] / GOLD["collision"]["velocity_force_factor_den"]
    assert np.abs(o[:, 1:4] - (m[:, 1:4] + k * F / m[:, :1])).max() < 1e-15


# ------------------------------------------------------------------ P2/P3 invariants
def test_conservation_periodic(orc):
    rng = np.random.default_rng(5)
    shape = (6, 5, 4)
    m = random_state(shape, rng)
    M0 = m[0].sum()
    P0 = (m[0] * m[1:4]).sum(1)
    out = orc.step(m, shape, 0.55, n=20)
    assert abs(out[0].sum() - M0) / M0 < 1e-13
    assert np.abs((out[0] * out[1:4]).sum(1) - P0).max() < 1e-13 * M0


def test_momentum_gain_equals_force(orc):
    """With a body force, total momentum rho u grows by sum F per step (App. A with
    Eq. rho_u_stress: F/2 in the recovery plus F/(2 rho) in the collision)."""
    rng = np.random.default_rng(6)
    shape = (5, 4, 6)
    N = 120
    m = random_state(shape, rng)
    F = 1e-4 * rng.standard_normal((3, N))
    P0 = (m[0] * m[1:4]).sum(1)
    n = 7
    out = orc.step(m, shape, 0.6, F=F, n=n)
    P1 = (out[0] * out[1:4]).sum(1)
    assert np.abs(P1 - P0 - n * F.sum(1)).max() < 1e-13
    assert abs(out[0].sum() - m[0].sum()) < 1e-12


def test_uniform_flow_is_fixed_point(orc):
    shape = (4, 4, 4)
    U = np.array([0.1, -0.05, 0.07])
    m = eq_state(1.02, np.repeat(U[:, None], 64, 1))
    out = orc.step(m, shape, 0.52, n=3)
    assert np.abs(out - m).max() < 2e-15


def test_closed_box_bounce_back_conserves_mass(orc):
    shape = (7, 6, 5)
    rng = np.random.default_rng(7)
    mask = W.channel_walls(shape)
    mask[:, :, 0] = 1
    mask[:, :, -1] = 1
    mask[2, 2, 3] = 1  # an interior obstacle
    typ, _, _, _ = orc.classify(mask)
    m = random_state(shape, rng)
    fl = typ != orc.SOLID
    M0 = m[0][fl].sum()
    out = orc.step(m, shape, 0.6, typ=typ, n=15)
    assert abs(out[0][fl].sum() - M0) / M0 < 1e-13
    assert np.array_equal(out[:, ~fl], m[:, ~fl])


# ------------------------------------------------------------------ symmetries
def _perm_state(m, n):
    """Cyclic axis relabelling x->y, y->z, z->x of a cubic n^3 state."""
    g = m.reshape(10, n, n, n)
    g = np.transpose(g, (0, 2, 3, 1))  # new[z', y', x'] = old[...]
    out = np.empty_like(g)
    out[0] = g[0]
    # u'[sigma(a)] = u[a], sigma = (1, 2, 0)
    out[1 + 1], out[1 + 2], out[1 + 0] = g[1], g[2], g[3]
    S = {p: g[4 + k] for k, p in enumerate(PAIRS)}
    sig = (1, 2, 0)
    for (a, b), val in S.items():
        pa, pb = sig[a], sig[b]
        out[4 + PAIRS.index(tuple(sorted((pa, pb))))] = val
    return out.reshape(10, -1)


def _mirror_x(m, n):
    g = m.reshape(10, n, n, n)
    g = np.roll(g[..., ::-1], 1, axis=-1).copy()
    for comp in (1, 4 + PAIRS.index((0, 1)), 4 + PAIRS.index((0, 2))):
        g[comp] = -g[comp]
    return g.reshape(10, -1)


def test_step_commutes_with_axis_permutation_and_mirror(orc):
    n = 5
    rng = np.random.default_rng(8)
    m = random_state((n, n, n), rng, du=0.08, ds=0.01)
    F = 1e-3 * rng.standard_normal((3, n ** 3))
    Fp = _perm_state(np.concatenate([np.zeros((1, n ** 3)), F, np.zeros((6, n ** 3))]), n)[1:4]
    a = orc.step(_perm_state(m, n), (n, n, n), 0.57, F=Fp)
    b = _perm_state(orc.step(m, (n, n, n), 0.57, F=F), n)
    assert np.abs(a - b).max() < 1e-15
    Fm = _mirror_x(np.concatenate([np.zeros((1, n ** 3)), F, np.zeros((6, n ** 3))]), n)[1:4]
    a = orc.step(_mirror_x(m, n), (n, n, n), 0.57, F=Fm)
    b = _mirror_x(orc.step(m, (n, n, n), 0.57, F=F), n)
    assert np.abs(a - b).max() < 1e-15


# ------------------------------------------------------------------ P4 Taylor-Green
def test_taylor_green_decay_rate(orc):
    """Config tgv32: amplitude ~ exp(-2 nu k^2 t), nu = c_s^2 (tau - 1/2)."""
    wl = W.TGV32
    u, k = W.taylor_green(wl.shape, 0.05)
    m = eq_state(1.0, W.flat(u))
    nx, ny, nz = wl.shape
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    mode = (np.sin(k * x) * np.cos(k * y) * np.ones((nz, 1, 1))).ravel()
    amps, ts = [], []
    cur = m
    for t in range(0, 101, 10):
        if t:
            cur = orc.step(cur, wl.shape, wl.tau, n=10)
        if t >= 20:
            amps.append((cur[1] * mode).sum() / (mode * mode).sum())
            ts.append(t)
    slope = np.polyfit(ts, np.log(amps), 1)[0]
    nu_fit = -slope / (2 * k * k)
    nu = CS2 * (wl.tau - 0.5)
    assert abs(nu_fit / nu - 1) < 0.01, nu_fit / nu


# ------------------------------------------------------------------ P5 Poiseuille
def test_poiseuille_profile_with_bounce_back(orc):
    """Body-force channel between solid layers y = 0 and y = ny-1: halfway
    bounce-back puts the walls at y = 0.5 and ny - 1.5."""
    ny = 34
    shape = (1, ny, 1)
    mask = np.zeros((1, ny, 1), np.uint8)
    mask[0, 0, 0] = mask[0, ny - 1, 0] = 1
    typ, _, _, _ = orc.classify(mask)
    tau = 0.8
    nu = CS2 * (tau - 0.5)
    H = ny - 2.0
    umax = 0.01
    Fx = 8 * nu * umax / H ** 2
    F = np.zeros((3, ny))
    F[0] = Fx
    F[:, typ == orc.SOLID] = 0
    m = eq_state(1.0, np.zeros((3, ny)))
    m = orc.step(m, shape, tau, F=F, typ=typ, n=12000)
    y = np.arange(ny)
    want = Fx / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    fl = typ != orc.SOLID
    err = np.sqrt(((m[1][fl] - want[fl]) ** 2).sum() / (want[fl] ** 2).sum())
    assert err < 0.02, err
    assert np.abs(m[2:4][:, fl]).max() < 1e-12


# ------------------------------------------------------------------ special cells (configs 3-4)
def _special_cell_violations(orc, m, out, typ, inflow, nx):
    """The special-cell rules of the channel configurations (reading C9 of the
    inflow / outflow / wall set-up): INFLOW cells hold exactly the inflow
    equilibrium (rho_in, u_in, u_in u_in); OUTFLOW cells (x = nx-1) hold the NEW
    state of (nx-2, y, z); SOLID cells keep their old value.  Returns the names
    of the rules the pair (m -> out) breaks."""
    bad = []
    rho_in, u_in = inflow[0], np.asarray(inflow[1:4], np.float64)
    want_in = np.concatenate([[rho_in], u_in, [u_in[a] * u_in[b] for a, b in PAIRS]])
    i_in = np.nonzero(typ == orc.INFLOW)[0]
    if not (len(i_in) and np.array_equal(out[:, i_in], np.repeat(want_in[:, None], len(i_in), 1))):
        bad.append("inflow")
    i_out = np.nonzero(typ == orc.OUTFLOW)[0]
    if not (len(i_out) and np.all(i_out % nx == nx - 1)
            and np.array_equal(out[:, i_out], out[:, i_out - 1])):
        bad.append("outflow")
    sol = typ == orc.SOLID
    if not np.array_equal(out[:, sol], m[:, sol]):
        bad.append("solid")
    return bad


def _special_cell_case(orc):
    shape = (9, 6, 5)
    rng = np.random.default_rng(27)
    mask = W.channel_walls(shape)
    mask[2, 3, 6] = 1  # an obstacle next to the plane x = nx-2
    typ, _, _, _ = orc.classify(mask, True, True)
    m = random_state(shape, rng)
    F = 1e-4 * rng.standard_normal((3, m.shape[1]))
    return shape, typ, m, F, [1.01, 0.03, -0.01, 0.02]


def test_inflow_outflow_solid_cells(orc):
    """One D3Q27 step of a walled channel with inflow, outflow and an obstacle:
    every special cell follows its rule, and the plane x = nx-2 does change in the
    step (so copying its pre-step state would be seen)."""
    shape, typ, m, F, inflow = _special_cell_case(orc)
    out = orc.step(m, shape, 0.6, F=F, typ=typ, inflow=inflow)
    assert _special_cell_violations(orc, m, out, typ, inflow, shape[0]) == []
    i_out = np.nonzero(typ == orc.OUTFLOW)[0]
    assert np.abs(out[:, i_out - 1] - m[:, i_out - 1]).min(axis=0).max() > 0
    assert np.abs(out[:, i_out - 1] - m[:, i_out - 1]).max() > 1e-4
    # the x = nx-2 plane is an ordinary update: the sampled-cell step (which has
    # no outflow pass) gives the same values there
    got = orc.step_cells(m, shape, 0.6, i_out - 1, F=F, typ=typ, inflow=inflow)
    assert np.abs(got - out[:, i_out - 1]).max() < 1e-15


@pytest.mark.parametrize("planted,rule", [(1, "outflow"), (2, "outflow"), (3, "inflow")])
def test_planted_special_cell_mistakes_are_caught(orc, planted, rule):
    """Plausible slips in the special-cell rules -- the outflow copying the
    pre-step state of x = nx-2 (1) or no copy, i.e. x = nx-1 itself (2), the
    inflow resetting S to 0 (3) -- each break the pin above."""
    shape, typ, m, F, inflow = _special_cell_case(orc)
    good = orc.step_planted(m, shape, 0.6, 0, F=F, typ=typ, inflow=inflow)
    assert np.array_equal(good, orc.step(m, shape, 0.6, F=F, typ=typ, inflow=inflow))
    bad = orc.step_planted(m, shape, 0.6, planted, F=F, typ=typ, inflow=inflow)
    assert _special_cell_violations(orc, m, bad, typ, inflow, shape[0]) == [rule]


# ------------------------------------------------------------------ P6 linear modes
def test_linear_modes_k0_and_hydrodynamic_limits(orc):
    tau = 0.6
    nu = CS2 * (tau - 0.5)
    G0 = orc.amplification_matrix(1.0, [0, 0, 0], tau, [[0, 0, 0]])[0]
    ev = np.sort(np.linalg.eigvals(G0).real)
    want = np.sort([1] * 4 + [1 - 1 / tau] * 5 + [0])
    assert np.abs(ev - want).max() < 1e-12
    kap = 2 * np.pi / 64
    for U in (0.0, 0.1):
        G = orc.amplification_matrix(1.0, [U, 0, 0], tau, [[kap, 0, 0]])[0]
        lam = np.linalg.eigvals(G)
        hyd = lam[np.argsort(-np.abs(lam))[:4]]
        omega = 1j * np.log(hyd)  # lambda = exp(-i omega)
        shear = omega[np.abs(omega.real - kap * U) < 0.3 * kap * np.sqrt(CS2)]
        assert len(shear) == 2
        # Eq. shear_mode: omega = k U cos(phi) - i k^2 nu
        assert np.abs(shear.real - kap * U).max() < 1e-3 * kap
        assert np.abs(-shear.imag / kap ** 2 / nu - 1).max() < 0.01
        ac = omega[np.abs(omega.real - kap * U) > 0.3 * kap * np.sqrt(CS2)]
        assert len(ac) == 2
        # Eq. acoustic_modes: omega = k (U cos(phi) +- c_s) - i k^2 ((D-1)/D nu + mu_v/2)
        speeds = np.sort(ac.real / kap - U)
        assert np.abs(speeds - np.array([-1, 1]) * np.sqrt(CS2)).max() < 2e-3
        # bulk viscosity of a trace relaxed at rate 1: mu_v = (2/3) c_s^2 (1/1 - 1/2) = 1/9.
        # Checked at rest only: with mean flow the third-order closure carries the
        # known O(U^2) Galilean defect of the acoustic damping (about 4% at U = 0.1).
        gam = -ac.imag / kap ** 2
        if U == 0.0:
            assert np.abs(gam / ((2 / 3) * nu + (1 / 9) / 2) - 1).max() < 5e-4
        else:
            assert np.abs(gam / ((2 / 3) * nu + (1 / 9) / 2) - 1).max() < 0.06


def test_linear_stability_within_paper_velocity_bound(orc):
    """max |lambda(k)| <= 1 over a k-grid for tau near 1/2 and |u| up to 0.3
    (the paper bounds velocities to [-0.4, 0.4] from its stability analysis)."""
    ks = np.linspace(-np.pi, np.pi, 9)
    kgrid = np.array(list(itertools.product(ks, ks, ks[4:])))
    for tau in (0.505, 0.52, 0.6):
        for U in ([0, 0, 0], [0.1, 0, 0], [0.3, 0, 0], [0.15, 0.15, 0.15]):
            G = orc.amplification_matrix(1.0, U, tau, kgrid)
            rad = np.abs(np.linalg.eigvals(G)).max()
            assert rad <= 1 + 1e-12, (tau, U, rad)


def test_linear_stability_at_the_papers_viscosities_and_diagonal_velocities(orc):
    """The von Neumann check of Sec. 5.3 (numerical spectral analysis) at its
    viscosities nu = 1e-3 and 1e-4 and its diagonal background flows u = (a, a):
    max |lambda(k)| <= 1 over k = (kx, ky, 0) in [0, pi]^2 for a = 0, 0.1, 0.2."""
    ks = np.linspace(0, np.pi, 13)
    kgrid = np.array([[a, b, 0.0] for a in ks for b in ks])
    for nu in (1e-3, 1e-4):
        tau = 0.5 + nu / CS2
        for a in (0.0, 0.1, 0.2):
            G = orc.amplification_matrix(1.0, [a, a, 0.0], tau, kgrid)
            rad = np.abs(np.linalg.eigvals(G)).max()
            assert rad <= 1 + 1e-12, (nu, a, rad)


# ------------------------------------------------------------------ P7 adjoint
def _bc_case(orc, rng):
    shape = (7, 5, 4)
    mask = np.zeros((4, 5, 7), np.uint8)
    mask[1, 2, 3] = 1
    mask[2, 1:3, 4] = 1
    mask[:, 0, :] = 1
    typ, _, _, _ = orc.classify(mask, inflow=True, outflow=True)
    m = random_state(shape, rng, du=0.05, ds=0.003)
    F = 1e-3 * rng.standard_normal((3, 140))
    return shape, typ, m, F


def test_adjoint_dot_product_against_complex_step(orc):
    rng = np.random.default_rng(9)
    shape, typ, m, F = _bc_case(orc, rng)
    inflow = [1.01, 0.04, 0.0, 0.0]
    tau = 0.58
    v = rng.standard_normal(m.shape)
    vF = rng.standard_normal(F.shape)
    w = rng.standard_normal(m.shape)
    h = 1e-30
    jv = orc.step_complex(m + 1j * h * v, shape, tau, F=F + 1j * h * vF, typ=typ, inflow=inflow).imag / h
    lam, gF = orc.step_vjp(m, shape, tau, w, F=F, typ=typ)
    lhs = (jv * w).sum()
    rhs = (v * lam).sum() + (vF * gF).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_multistep_adjoint_against_central_differences(orc):
    rng = np.random.default_rng(10)
    shape = (6, 5, 4)
    N = 120
    u0 = 0.04 * rng.standard_normal((3, N))
    F = 1e-4 * rng.standard_normal((3, N))
    tau, nsteps = 0.55, 6
    region = np.zeros(N, bool)
    region[::3] = True

    def loss(mm):
        return 0.5 * (mm[0] * (mm[1:4] ** 2).sum(0))[region].sum()

    def dloss(mm):
        g = np.zeros_like(mm)
        g[0][region] = 0.5 * (mm[1:4] ** 2).sum(0)[region]
        g[1:4][:, region] = (mm[0] * mm[1:4])[:, region]
        return g

    gu, gF = orc.adjoint(u0, F, shape, tau, nsteps, dloss, K=4)
    for trial in range(3):
        vu = rng.standard_normal(u0.shape)
        vF = rng.standard_normal(F.shape)
        eps_u, eps_F = 1e-5, 1e-7
        lp, _ = orc.forward_loss(u0 + eps_u * vu, F + eps_F * vF, shape, tau, nsteps, loss)
        lm, _ = orc.forward_loss(u0 - eps_u * vu, F - eps_F * vF, shape, tau, nsteps, loss)
        # directional derivative along (eps_u vu, eps_F vF), scaled by 1/eps_u
        fd = (lp - lm) / 2
        ad = eps_u * (gu * vu).sum() + eps_F * (gF * vF).sum()
        assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


# ------------------------------------------------------------------ moving solid walls
def _two_body_mask(shape, rng, dens=0.12):
    """Random solid cells split into bodies 1 and 2 (the mask value is the body id)."""
    nx, ny, nz = shape
    body = (rng.uniform(size=nx * ny * nz) < dens).astype(np.uint8)
    body[body > 0] = 1 + (rng.uniform(size=int(body.sum())) < 0.5)
    return body


def test_wall_momentum_exchange_balances_the_step(orc):
    """Sec. 3.2: the force on the solid is the momentum its links exchange with the
    fluid, sum -c_i (f_in + f_out).  For every state the step then changes the total
    fluid momentum by the body force minus that force, exactly:
    P(t+1) - P(t) = sum F - F_solid (both wall models, moving bodies, any state)."""
    rng = np.random.default_rng(31)
    shape = (9, 8, 7)
    N = 9 * 8 * 7
    body = _two_body_mask(shape, rng)
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    fluid = typ != orc.SOLID
    u = 0.05 * rng.standard_normal((3, N))
    m = np.zeros((10, N))
    m[0] = 1 + 0.01 * rng.standard_normal(N)
    m[1:4] = u
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        m[4 + k] = u[a] * u[b] + 0.003 * rng.standard_normal(N)
    F = 1e-4 * rng.standard_normal((3, N))
    motion = {1: ([0.02, -0.01, 0.0], [0.0, 0.0, 0.003], [4.0, 3.5, 3.0]),
              2: ([-0.01, 0.0, 0.015], [0.002, -0.001, 0.0], [1.0, 2.0, 5.0])}
    for model in (0, 1):
        wall = orc.Wall(model, body, motion)
        new = orc.step(m, shape, 0.6, F=F, typ=typ, wall=wall)
        P0 = (m[0] * m[1:4])[:, fluid].sum(1)
        P1 = (new[0] * new[1:4])[:, fluid].sum(1)
        Fs = orc.solid_force(m, shape, 0.6, typ, wall, F=F)
        assert np.abs(P1 - P0 - (F[:, fluid].sum(1) - Fs[:3])).max() < 1e-12, model
        F1 = orc.solid_force(m, shape, 0.6, typ, wall, F=F, body_id=1)
        F2 = orc.solid_force(m, shape, 0.6, typ, wall, F=F, body_id=2)
        assert np.allclose(F1[:3] + F2[:3], Fs[:3], rtol=0, atol=1e-13)
        # the same motion described about r0 + d (V + Om x d): the torque becomes
        # T(r0 + d) = T(r0) - d x F
        d = np.array([0.7, -1.3, 2.1])
        V1 = np.add(motion[1][0], np.cross(motion[1][1], d))
        m1 = {1: (V1, motion[1][1], list(np.add(motion[1][2], d))), 2: motion[2]}
        F1s = orc.solid_force(m, shape, 0.6, typ, orc.Wall(model, body, m1), F=F, body_id=1)
        assert np.allclose(F1s[3:], F1[3:] - np.cross(d, F1[:3]), rtol=0, atol=1e-12)


def test_moment_wall_moving_with_the_flow_keeps_uniform_flow(orc):
    """With the walls moving at the fluid's velocity U the reconstruction at p is
    the fluid's own equilibrium, so (rho, U, U U) stays a fixed point; halfway
    bounce-back (a wall at rest) does not keep it."""
    rng = np.random.default_rng(32)
    shape = (8, 7, 6)
    N = 8 * 7 * 6
    body = _two_body_mask(shape, rng)
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    fluid = typ != orc.SOLID
    U = np.array([0.04, -0.02, 0.03])
    m = np.zeros((10, N))
    m[0] = 1.0
    m[1:4] = U[:, None]
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        m[4 + k] = U[a] * U[b]
    moving = orc.Wall(1, body, {1: (U, [0, 0, 0], [0, 0, 0]), 2: (U, [0, 0, 0], [3, 3, 3])})
    new = orc.step(m, shape, 0.7, typ=typ, wall=moving)
    assert np.abs(new[:, fluid] - m[:, fluid]).max() < 1e-14
    bb = orc.step(m, shape, 0.7, typ=typ, wall=orc.Wall(0, body))
    assert np.abs(bb[1:4, fluid] - m[1:4, fluid]).max() > 1e-3


def test_moment_wall_couette_flow(orc):
    """Plane Couette flow between body 1 (y = 0, at rest) and body 2 (y = ny - 1,
    moving with U x): the steady profile is linear, and the force on each wall
    equals the viscous momentum flux rho nu du/dy times the wall area."""
    shape = (2, 14, 2)
    nx, ny, nz = shape
    N = nx * ny * nz
    y = (np.arange(N) // nx) % ny
    body = np.zeros(N, np.uint8)
    body[y == 0] = 1
    body[y == ny - 1] = 2
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    U, tau = 0.05, 0.8
    nu = (tau - 0.5) / 3
    wall = orc.Wall(1, body, {1: ([0, 0, 0], [0, 0, 0], [0, 0, 0]), 2: ([U, 0, 0], [0, 0, 0], [0, 0, 0])})
    m = np.zeros((10, N))
    m[0] = 1.0
    m = orc.step(m, shape, tau, typ=typ, wall=wall, n=6000)
    rows = np.arange(1, ny - 1)
    ux = np.array([m[1][y == r].mean() for r in rows])
    rho = np.array([m[0][y == r].mean() for r in rows])
    slope, icpt = np.polyfit(rows, ux, 1)
    assert np.abs(ux - (slope * rows + icpt)).max() < 1e-7 * U
    y0, y1 = -icpt / slope, (U - icpt) / slope  # where the profile meets the wall velocities
    assert abs(y0 - 0.5) < 1.0 and abs(y1 - (ny - 1.5)) < 1.0, (y0, y1)
    F2 = orc.solid_force(m, shape, tau, typ, wall, body_id=2)
    F1 = orc.solid_force(m, shape, tau, typ, wall, body_id=1)
    flux = rho.mean() * nu * slope * nx * nz
    assert abs(F2[0] + flux) < 1e-3 * flux and abs(F1[0] - flux) < 1e-3 * flux, (F1[0], F2[0], flux)


# ------------------------------------------------------------------ P8 codec
def test_codec_paper_formula_endpoints_and_round_trip(orc):
    """Sec. 5.4: ranges, b = 16 bits, dequantisation m_min + q (m_max - m_min)/(2^b - 1).
    The grid is anchored at the code nearest the centre of the values, which moves
    its end points by less than 2e-7 from the printed bounds."""
    q = GOLD["quantization"]
    lo, hi = orc.ranges()
    assert list(lo[:1]) == [q["rho_range"][0]] and list(hi[:1]) == [q["rho_range"][1]]
    assert np.all(lo[1:4] == q["u_range"][0]) and np.all(hi[1:4] == q["u_range"][1])
    assert np.all(lo[4:] == q["rhoS_neq_range"][0]) and np.all(hi[4:] == q["rhoS_neq_range"][1])
    raw = q["rhoS_raw_range"]
    assert (raw[1] - raw[0]) / (hi[4] - lo[4]) > q["resolution_gain_of_range_reduction_at_least"]
    levels = 2 ** q["bits"] - 1
    codes = np.arange(levels + 1, dtype=np.uint16)
    qq = np.tile(codes, (10, 1))
    dec = orc.decode(qq)
    assert np.abs(dec[:, 0] - lo).max() < 2e-7 and np.abs(dec[:, -1] - hi).max() < 2e-7
    step = (hi - lo) / levels
    assert np.abs(np.diff(dec, axis=1) - step[:, None]).max() < 1e-7 * step.max()
    # every code survives decode -> FP32 -> deterministic encode
    enc = orc.encode(orc.stored_for_codec(dec), (levels + 1, 1, 1), 0, 0, deterministic=True)
    assert np.array_equal(enc, qq)


def test_codec_error_bounds_and_saturation(orc):
    rng = np.random.default_rng(11)
    lo, hi = orc.ranges()
    N = 4096
    v = lo[:, None] + (hi - lo)[:, None] * rng.uniform(size=(10, N))
    v32 = orc.stored_for_codec(v)
    ref = v32.astype(np.float64)
    ref[0] += 1.0
    step = (hi - lo) / 65535
    det = orc.decode(orc.encode(v32, (16, 16, 16), 0, 0, deterministic=True))
    sto = orc.decode(orc.encode(v32, (16, 16, 16), 5, 99))
    # the decision is taken in FP32: w = m K + b carries half an ulp (<= 2^-9 code
    # for |w| < 2^16) plus the relative error of K times |w| (<= 2^-9 code)
    slack = 4e-3 * step[:, None]
    assert np.all(np.abs(det - ref) <= 0.5 * step[:, None] + slack)
    assert np.all(np.abs(sto - ref) < step[:, None] + slack)
    out = np.full((10, 3), 0, np.float32)
    out[:, 0] = (lo - 1.0) - np.array([1.0] + [0.0] * 9)
    out[:, 1] = (hi + 1.0) - np.array([1.0] + [0.0] * 9)
    out[:, 2] = np.nan
    q = orc.encode(out, (3, 1, 1), 0, 0)
    assert np.all(q[:, 0] == 0) and np.all(q[:, 1] == 65535) and np.all(q[:, 2] == 0)


def test_dither_is_uniform_and_rounding_unbiased(orc):
    """Dithering adds zero-mean uniform noise of one unit before rounding (Sec. 5.4),
    so the rounding is unbiased: the mean of decode(encode(m)) over cells is m."""
    ds = np.array([orc.dither(x, y, z, 7, 123) for x in range(8) for y in range(8) for z in range(8)])
    assert ds.min() > 0 and ds.max() < 1
    # the dither takes the midpoints (f + 1/2)/2^16 of equal cells of [0, 1)
    for k, bits in enumerate([16] * 10):
        f = ds[:, k] * 2 ** bits - 0.5
        assert np.array_equal(f, np.round(f)) and f.min() >= 0 and f.max() <= 2 ** bits - 1
    assert np.abs(ds.mean(0) - 0.5).max() < 0.05
    assert np.abs(ds.var(0) - 1 / 12).max() < 0.015
    lo, hi = orc.ranges()
    shape = (64, 64, 16)
    N = 64 * 64 * 16
    step = (hi - lo) / 65535
    for frac in (0.1, 0.37, 0.5, 0.83):
        val = lo + (1000 + frac) * step
        v = np.repeat(val[:, None], N, 1)
        dec = orc.decode(orc.encode(orc.stored_for_codec(v), shape, 3, 77))
        bias = (dec.mean(1) - val) / step
        sigma = 0.5 / np.sqrt(N)
        assert np.abs(bias).max() < 5 * sigma + 1e-3, bias


def test_dither_components_are_pairwise_independent(orc):
    """The ten dither values of a cell come from one 128-bit hash: eight 16-bit
    halves and two fields that are xors of halves of two other words.  Each is
    uniform, and no two components are dependent: over 32768 cells the 8 x 8 joint
    histogram of the top three bits of every pair of components is flat (chi-square
    with 63 degrees of freedom below 120; a component that repeated another's field,
    or the xor of its own word's halves with another, would give thousands)."""
    ds = np.array([orc.dither(x, y, z, 11, 5) for x in range(32) for y in range(32)
                   for z in range(32)])
    top = np.floor(ds * 8).astype(int)
    n = len(top)
    for i in range(10):
        for j in range(i + 1, 10):
            h = np.bincount(top[:, i] * 8 + top[:, j], minlength=64)
            chi2 = ((h - n / 64) ** 2 / (n / 64)).sum()
            assert chi2 < 120, (i, j, chi2)


def test_stochastic_rounding_is_unbiased_over_the_dither(orc):
    """Sec. 5.4: the dither is zero-mean uniform noise of one unit, so the expected
    code equals the value.  Enumerating every dither value: E[q] differs from the
    exact code coordinate by at most half a dither quantum (2^-17 code for the
    16-bit fields) plus the FP32 rounding of w, and by ~0 on average over values
    spread across code cells (a dither f/2^16 instead of (f + 1/2)/2^16 would
    under-round by 2^-17 code on average, a -8e-11 per-step drift of rho)."""
    rng = np.random.default_rng(14)
    devs = {0: [], 1: [], 4: []}
    for k, centre, spread in ((0, 0.0, 0.01), (1, 0.0, 0.05), (4, 0.0, 0.005)):
        for v in (centre + spread * rng.standard_normal(300)).astype(np.float32):
            w = orc.code_coordinate(v, k) - orc.codec_constants(k)[0]
            # half a dither quantum + the FP32 rounding of w (half an ulp, plus
            # the relative error of the FP32 constant K times |w|)
            bound = 2.0 ** -17 + float(np.spacing(np.float32(abs(w)))) / 2 + abs(w) * 2.0 ** -24
            dev = orc.mean_code_over_dither(v, k) - orc.code_coordinate(v, k)
            assert abs(dev) <= bound, (k, v, dev, bound)
            devs[k].append(dev)
    # On average the deviation is the tie effect only: when |w| < 2048 its FP32
    # value has >= 13 fractional bits, w + d can be an exact integer and the
    # exact floor keeps it (at most +6e-5 code on average).
    for k, d in devs.items():
        assert abs(np.mean(d)) < 6e-5, (k, np.mean(d))


# Adaptive bit allocation (Sec. 6.2.2): rho and u take b_rho_u bits, rho S^neq b_S
# bits, each on the grid of Sec. 5.4 with 2^b - 1 steps.
BIT_CONFIGS = [(16, 15), (15, 14), (14, 13), (13, 12), (12, 11)]


@pytest.mark.parametrize("bits", BIT_CONFIGS)
def test_codec_bits_grid_endpoints_and_round_trip(orc, bits):
    """Dequantisation m_min + q (m_max - m_min)/(2^b - 1) for q = 0 .. 2^b - 1 with b
    per group; every code survives decode -> FP32 -> deterministic encode, and the
    centre code is the one nearest the centre of the values."""
    lo, hi = orc.ranges()
    Q = np.array([2 ** bits[0] - 1] * 4 + [2 ** bits[1] - 1] * 6, np.int64)
    for k in (0, 1, 4):
        qc, step, c, K, b = orc.codec_constants(k, bits)
        centre = 1.0 if k == 0 else 0.0
        assert qc == np.floor((centre - lo[k]) * Q[k] / (hi[k] - lo[k]) + 0.5)
        assert abs(step - (hi[k] - lo[k]) / Q[k]) <= 1e-7 * step
    n = int(Q.max()) + 1
    codes = np.tile(np.arange(n, dtype=np.int64), (10, 1))
    codes = np.minimum(codes, Q[:, None]).astype(np.uint16)
    dec = orc.decode(codes, bits)
    assert np.abs(dec[:, 0] - lo).max() < 1e-6 and np.abs(dec[np.arange(10), Q] - hi).max() < 1e-6
    step = (hi - lo) / Q
    d = np.diff(dec, axis=1)
    for k in range(10):
        assert np.abs(d[k, :Q[k]] - step[k]).max() < 1e-6 * step[k]
    enc = orc.encode(orc.stored_for_codec(dec), (n, 1, 1), 0, 0, deterministic=True, bits=bits)
    assert np.array_equal(enc, codes)


@pytest.mark.parametrize("bits", BIT_CONFIGS)
def test_codec_bits_error_bounds_saturation_and_unbiased_rounding(orc, bits):
    rng = np.random.default_rng(12)
    lo, hi = orc.ranges()
    Q = np.array([2 ** bits[0] - 1] * 4 + [2 ** bits[1] - 1] * 6, np.float64)
    step = (hi - lo) / Q
    v = lo[:, None] + (hi - lo)[:, None] * rng.uniform(size=(10, 4096))
    v32 = orc.stored_for_codec(v)
    ref = v32.astype(np.float64)
    ref[0] += 1.0
    det = orc.decode(orc.encode(v32, (16, 16, 16), 0, 0, deterministic=True, bits=bits), bits)
    sto = orc.decode(orc.encode(v32, (16, 16, 16), 5, 99, bits=bits), bits)
    slack = 4e-3 * step[:, None]
    assert np.all(np.abs(det - ref) <= 0.5 * step[:, None] + slack)
    assert np.all(np.abs(sto - ref) < step[:, None] + slack)
    out = np.zeros((10, 3), np.float32)
    out[:, 0] = (lo - 1.0) - np.array([1.0] + [0.0] * 9)
    out[:, 1] = (hi + 1.0) - np.array([1.0] + [0.0] * 9)
    out[:, 2] = np.nan
    q = orc.encode(out, (3, 1, 1), 0, 0, bits=bits)
    assert np.all(q[:, 0] == 0) and np.all(q[:, 1] == Q) and np.all(q[:, 2] == 0)
    # expected code over every dither value = the exact code coordinate
    for k, spread in ((0, 0.01), (1, 0.05), (4, 0.005)):
        for val in (spread * rng.standard_normal(50)).astype(np.float32):
            w = orc.code_coordinate(val, k, bits) - orc.codec_constants(k, bits)[0]
            bound = 2.0 ** -17 + float(np.spacing(np.float32(abs(w)))) / 2 + abs(w) * 2.0 ** -24
            dev = orc.mean_code_over_dither(val, k, bits) - orc.code_coordinate(val, k, bits)
            assert abs(dev) <= bound, (bits, k, val, dev)


def test_codec_bits_16_16_is_the_uniform_codec(orc):
    rng = np.random.default_rng(13)
    lo, hi = orc.ranges()
    v32 = orc.stored_for_codec(lo[:, None] + (hi - lo)[:, None] * rng.uniform(size=(10, 512)))
    a = orc.encode(v32, (8, 8, 8), 3, 9)
    b = orc.encode(v32, (8, 8, 8), 3, 9, bits=(16, 16))
    assert np.array_equal(a, b)
    assert np.array_equal(orc.decode(a), orc.decode(a, (16, 16)))


def test_repeated_requantisation_conserves_mass_and_momentum(orc):
    """1000 decode/encode cycles of a field fluctuating about rho = 1, u = 0 (the
    round trip a stored state makes every step) leave the mean density and
    velocity unbiased to < 1e-9 per cycle.  Rounding to nearest after adding the
    dither, or FP32 constants applied to the full offset from m_min, give
    systematic drifts of 5e-9 to 1e-8 per cycle."""
    rng = np.random.default_rng(13)
    shape = (64, 64, 16)
    N = 65536
    m = np.zeros((10, N))
    m[0] = 1.0 + 0.01 * rng.standard_normal(N)
    m[1:4] = 0.03 * rng.standard_normal((3, N))
    m[4:] = 0.005 * rng.standard_normal((6, N))
    q = orc.encode(orc.stored_for_codec(m), shape, 0, 5)
    start = orc.decode(q)
    cur = start
    cycles = 1000
    for t in range(1, cycles + 1):
        q = orc.encode(orc.stored_for_codec(cur), shape, t, 5)
        cur = orc.decode(q)
    drift = (cur.mean(1) - start.mean(1)) / cycles
    assert abs(drift[0]) < 1e-9, drift[0]
    assert np.abs(drift[1:4]).max() < 1e-9, drift[1:4]


# ------------------------------------------------------------------ P9 classification
def _classify_bruteforce(mask, inflow, outflow):
    nz, ny, nx = mask.shape
    c = [(i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1) for i in range(27)]
    typ, link = [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                solid = bool(mask[z, y, x])
                bits = 0
                if not solid:
                    for i, (cx, cy, cz) in enumerate(c):
                        if mask[(z - cz) % nz, (y - cy) % ny, (x - cx) % nx]:
                            bits |= 1 << i
                if solid:
                    t = 4
                elif inflow and x == 0:
                    t = 2
                elif outflow and x == nx - 1 and nx >= 2 and not mask[z, y, x - 1]:
                    t = 3
                elif bits:
                    t = 1
                else:
                    t = 0
                typ.append(t)
                link.append(bits)
    cells = [n for n, t in enumerate(typ) if t in (1, 2)]
    words = [(typ[n] << 27) | link[n] for n in cells]
    return np.array(typ), np.array(link), np.array(cells), np.array(words)


@pytest.mark.parametrize("shape,dens,inflow,outflow", [
    ((5, 4, 3), 0.2, False, False), ((6, 5, 4), 0.3, True, True), ((7, 3, 5), 0.05, True, False),
    ((2, 2, 2), 0.5, False, True), ((1, 4, 4), 0.3, False, False)])
def test_classification_matches_brute_force(orc, shape, dens, inflow, outflow):
    mask = W.random_mask(shape, dens, seed=hash((shape, dens)) % 1000)
    t, l, c, w = orc.classify(mask, inflow, outflow)
    bt, bl, bc, bw = _classify_bruteforce(mask, inflow, outflow)
    assert np.array_equal(t, bt) and np.array_equal(l, bl)
    assert np.array_equal(c, bc) and np.array_equal(w, bw)


# ------------------------------------------------------------------ helpers pinned to the step
def test_step_cells_and_reduce_agree_with_full_step(orc):
    rng = np.random.default_rng(12)
    shape, typ, m, F = _bc_case(orc, rng)
    inflow = [1.0, 0.05, 0.0, 0.0]
    full = orc.step(m, shape, 0.6, F=F, typ=typ, inflow=inflow)
    cells = np.arange(140)
    part = orc.step_cells(m, shape, 0.6, cells, F=F, typ=typ, inflow=inflow)
    assert np.abs(part - full).max() < 1e-15
    M, E = orc.reduce(full, typ)
    fl = typ != orc.SOLID
    assert abs(M - full[0][fl].sum()) < 1e-12
    assert abs(E - (0.5 * full[0] * (full[1:4] ** 2).sum(0))[fl].sum()) < 1e-14


def test_q16_emulation_tracks_fp64(orc):
    """The 16-bit form stays within the stated bounds of FP64 over 10 steps:
    velocity within 2e-3 of max|u|, total mass within 1e-6 of the decoded initial
    mass.  The initial state is encoded with the dither of time index 0: rho = 1
    is not on the 16-bit grid of [0.8, 1.5], and deterministic rounding would
    shift every cell the same way (-3e-6)."""
    shape = (16, 16, 16)
    u = W.random_phase_field(shape, 0.05, kmax=4, seed=5)
    m = eq_state(1.0, W.flat(u))
    st = orc.public_to_stored(m)
    assert np.abs(orc.stored_to_public(st) - m).max() < 1e-16
    q = orc.encode(orc.stored_for_codec(st), shape, 0, 1)
    ref = orc.stored_to_public(orc.decode(q))
    M0 = ref[0].sum()
    for t in range(10):
        q = orc.q16_step(q, shape, 0.55, t + 1, 1)
        ref = orc.step(ref, shape, 0.55)
    pub = orc.stored_to_public(orc.decode(q))
    du = np.abs(pub[1:4] - ref[1:4]).max() / np.abs(ref[1:4]).max()
    assert du < 2e-3, du
    assert abs(pub[0].sum() - M0) / M0 < 1e-6


# ------------------------------------------------------------------ D3Q19
TRIPLES19 = [(0, 0, 1), (1, 2, 2), (0, 1, 1), (0, 2, 2), (0, 0, 2), (1, 1, 2)]


def _h3(c, a, b, g):
    c = c.astype(float)
    return (c[:, a] * c[:, b] * c[:, g]
            - CS2 * (c[:, a] * (b == g) + c[:, b] * (a == g) + c[:, g] * (a == b)))


def _T(m, a, b, g):
    S, u = m[4:], m[1:4]
    return (sget(S, a, b) * u[g] + sget(S, a, g) * u[b] + sget(S, b, g) * u[a]
            - 2 * u[a] * u[b] * u[g])


def test_d3q19_lattice_is_the_textbook_lattice(orc):
    """19 velocities |c|^2 <= 2, weights 1/3, 1/18, 1/36; summed over c_z they give
    App. D's D2Q9 weights; isotropic to 4th order with c_s^2 = 1/3."""
    _, c, w = orc.reconstruct19(np.array([1.0, 0, 0, 0, 0, 0, 0, 0, 0, 0]))
    n2 = (c ** 2).sum(1)
    assert len(c) == 19 and len({tuple(v) for v in c}) == 19 and n2.max() == 2
    assert np.all(w[n2 == 0] == 1 / 3) and np.all(w[n2 == 1] == 1 / 18) and np.all(w[n2 == 2] == 1 / 36)
    g = GOLD["d2q9"]
    for cx, cy, num, den in zip(g["cx"], g["cy"], g["w_num"], g["w_den"]):
        sel = (c[:, 0] == cx) & (c[:, 1] == cy)
        assert abs(w[sel].sum() - num / den) < 1e-15
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((w * c[:, a] * c[:, b]).sum() - CS2 * (a == b)) < 1e-15
    assert abs((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum() - CS2 ** 2) < 1e-15
    assert abs((w * c[:, 0] ** 4).sum() - 3 * CS2 ** 2) < 1e-15
    # the xyz Hermite polynomial vanishes on every D3Q19 velocity
    assert np.all(_h3(c, 0, 1, 2) == 0)


def test_d3q19_reconstruction_is_the_unique_moment_matching_polynomial(orc):
    """f / w lies in the span of {1, H1, H2, H3_aab for the six triples with a
    repeated index} and reproduces rho, rho u, rho S and rho T_aab: 16 linear
    conditions with a non-singular Gram matrix on the lattice, so f is fixed by
    them alone (independently of how the projection is written)."""
    rng = np.random.default_rng(31)
    _, c, w = orc.reconstruct19(np.zeros(10) + [1, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    cf = c.astype(float)
    basis = [np.ones(19)] + [cf[:, a] for a in range(3)]
    basis += [cf[:, a] * cf[:, b] - CS2 * (a == b) for a, b in PAIRS]
    basis += [_h3(c, *t) for t in TRIPLES19]
    B = np.array(basis).T  # (19, 16)
    G = B.T @ (w[:, None] * B)
    assert np.linalg.matrix_rank(G) == 16
    for m in random_cells(24, rng):
        f, _, _ = orc.reconstruct19(m)
        coef, *_ = np.linalg.lstsq(B, f / w, rcond=None)
        assert np.abs(B @ coef - f / w).max() < 1e-13
        rho = m[0]
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(cf.T @ f - rho * m[1:4]).max() < 1e-14
        for k, (a, b) in enumerate(PAIRS):
            assert abs(((cf[:, a] * cf[:, b] - CS2 * (a == b)) * f).sum() - rho * m[4 + k]) < 1e-14
        for t in TRIPLES19:
            assert abs((_h3(c, *t) * f).sum() - rho * _T(m, *t)) < 1e-14, t
        assert abs((_h3(c, 0, 1, 2) * f).sum()) < 1e-15


def test_d3q19_step_conserves_mass_and_gains_the_force(orc):
    rng = np.random.default_rng(32)
    shape = (6, 5, 4)
    m = random_state(shape, rng)
    F = 1e-4 * rng.standard_normal((3, 120))
    P0 = (m[0] * m[1:4]).sum(1)
    out = orc.step19(m, shape, 0.55, F=F, n=9)
    assert abs(out[0].sum() - m[0].sum()) / m[0].sum() < 1e-13
    assert np.abs((out[0] * out[1:4]).sum(1) - P0 - 9 * F.sum(1)).max() < 1e-13


def test_d3q19_uniform_flow_is_fixed_point_and_symmetries(orc):
    U = np.array([0.1, -0.05, 0.07])
    m = eq_state(1.02, np.repeat(U[:, None], 64, 1))
    assert np.abs(orc.step19(m, (4, 4, 4), 0.52, n=3) - m).max() < 2e-15
    n = 5
    rng = np.random.default_rng(33)
    m = random_state((n, n, n), rng, du=0.08, ds=0.01)
    F = 1e-3 * rng.standard_normal((3, n ** 3))
    pad = lambda v: np.concatenate([np.zeros((1, n ** 3)), v, np.zeros((6, n ** 3))])
    a = orc.step19(_perm_state(m, n), (n, n, n), 0.57, F=_perm_state(pad(F), n)[1:4])
    b = _perm_state(orc.step19(m, (n, n, n), 0.57, F=F), n)
    assert np.abs(a - b).max() < 1e-15
    a = orc.step19(_mirror_x(m, n), (n, n, n), 0.57, F=_mirror_x(pad(F), n)[1:4])
    b = _mirror_x(orc.step19(m, (n, n, n), 0.57, F=F), n)
    assert np.abs(a - b).max() < 1e-15


def test_d3q19_taylor_green_decay_rate(orc):
    """Same workload as the D3Q27 pin: the shear viscosity nu = c_s^2 (tau - 1/2)
    does not depend on the velocity set."""
    wl = W.TGV32
    u, k = W.taylor_green(wl.shape, 0.05)
    cur = eq_state(1.0, W.flat(u))
    nx, ny, nz = wl.shape
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    mode = (np.sin(k * x) * np.cos(k * y) * np.ones((nz, 1, 1))).ravel()
    amps, ts = [], []
    for t in range(0, 101, 10):
        if t:
            cur = orc.step19(cur, wl.shape, wl.tau, n=10)
        if t >= 20:
            amps.append((cur[1] * mode).sum() / (mode * mode).sum())
            ts.append(t)
    nu_fit = -np.polyfit(ts, np.log(amps), 1)[0] / (2 * k * k)
    assert abs(nu_fit / (CS2 * (wl.tau - 0.5)) - 1) < 0.01, nu_fit


def test_d3q19_sampled_cells_agree_with_full_step(orc):
    rng = np.random.default_rng(34)
    shape = (7, 5, 6)
    m = random_state(shape, rng)
    F = 1e-4 * rng.standard_normal((3, 210))
    full = orc.step19(m, shape, 0.6, F=F)
    cells = np.array([0, 1, 6, 7, 34, 35, 100, 209])
    assert np.abs(orc.step19_cells(m, shape, 0.6, cells, F=F) - full[:, cells]).max() < 1e-15


def test_d3q19_closed_box_bounce_back_conserves_mass(orc):
    shape = (7, 6, 5)
    rng = np.random.default_rng(35)
    mask = W.channel_walls(shape)
    mask[:, :, 0] = 1
    mask[:, :, -1] = 1
    mask[2, 2, 3] = 1
    typ, _, _, _ = orc.classify(mask)
    m = random_state(shape, rng)
    fl = typ != orc.SOLID
    M0 = m[0][fl].sum()
    out = orc.step19(m, shape, 0.6, typ=typ, n=15)
    assert abs(out[0][fl].sum() - M0) / M0 < 1e-13
    assert np.array_equal(out[:, ~fl], m[:, ~fl])


def test_d3q19_poiseuille_profile_with_bounce_back(orc):
    """The same body-force channel as the D3Q27 pin: halfway bounce-back on the
    19-velocity lattice puts the walls at y = 0.5 and ny - 1.5 as well."""
    ny = 34
    shape = (1, ny, 1)
    mask = np.zeros((1, ny, 1), np.uint8)
    mask[0, 0, 0] = mask[0, ny - 1, 0] = 1
    typ, _, _, _ = orc.classify(mask)
    tau = 0.8
    nu = CS2 * (tau - 0.5)
    umax = 0.01
    Fx = 8 * nu * umax / (ny - 2.0) ** 2
    F = np.zeros((3, ny))
    F[0] = Fx
    F[:, typ == orc.SOLID] = 0
    m = orc.step19(eq_state(1.0, np.zeros((3, ny))), shape, tau, F=F, typ=typ, n=12000)
    y = np.arange(ny)
    want = Fx / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    fl = typ != orc.SOLID
    err = np.sqrt(((m[1][fl] - want[fl]) ** 2).sum() / (want[fl] ** 2).sum())
    assert err < 0.02, err
    assert np.abs(m[2:4][:, fl]).max() < 1e-12


def test_d3q19_inflow_outflow_cells(orc):
    """Inflow cells take the inflow equilibrium, the outflow plane copies x = nx-2,
    solid cells keep their value."""
    shape = (9, 6, 5)
    rng = np.random.default_rng(36)
    mask = W.channel_walls(shape)
    typ, _, _, _ = orc.classify(mask, True, True)
    m = random_state(shape, rng)
    inflow = [1.01, 0.03, -0.01, 0.02]
    out = orc.step19(m, shape, 0.6, typ=typ, inflow=inflow)
    nx = shape[0]
    i_in = np.nonzero(typ == orc.INFLOW)[0]
    assert len(i_in) and np.allclose(out[0, i_in], 1.01) and np.allclose(out[1, i_in], 0.03)
    assert np.allclose(out[4, i_in], 0.03 ** 2) and np.allclose(out[7, i_in], 0.03 * -0.01)
    i_out = np.nonzero(typ == orc.OUTFLOW)[0]
    assert len(i_out) and np.all(i_out % nx == nx - 1)
    assert np.array_equal(out[:, i_out], out[:, i_out - 1])
    sol = typ == orc.SOLID
    assert np.array_equal(out[:, sol], m[:, sol])


def test_d3q19_sampled_cells_agree_with_full_step_with_boundaries(orc):
    shape = (9, 7, 6)
    rng = np.random.default_rng(37)
    mask = W.channel_walls(shape)
    mask[3, 3, 4] = 1
    typ, _, _, _ = orc.classify(mask, True, True)
    m = random_state(shape, rng)
    F = 1e-4 * rng.standard_normal((3, m.shape[1]))
    inflow = [1.0, 0.04, 0.0, 0.01]
    full = orc.step19(m, shape, 0.6, F=F, typ=typ, inflow=inflow)
    cells = np.arange(m.shape[1])
    got = orc.step19_cells(m, shape, 0.6, cells, F=F, typ=typ, inflow=inflow)
    assert np.abs(got - full).max() < 1e-15


def test_d3q19_wall_momentum_exchange_balances_the_step(orc):
    """The momentum-exchange identity on the 19-velocity lattice:
    P(t+1) - P(t) = sum F - F_solid for both wall models with moving bodies."""
    rng = np.random.default_rng(38)
    shape = (9, 8, 7)
    N = 9 * 8 * 7
    body = _two_body_mask(shape, rng)
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    fluid = typ != orc.SOLID
    u = 0.05 * rng.standard_normal((3, N))
    m = np.zeros((10, N))
    m[0] = 1 + 0.01 * rng.standard_normal(N)
    m[1:4] = u
    for k, (a, b) in enumerate(PAIRS):
        m[4 + k] = u[a] * u[b] + 0.003 * rng.standard_normal(N)
    F = 1e-4 * rng.standard_normal((3, N))
    motion = {1: ([0.02, -0.01, 0.0], [0.0, 0.0, 0.003], [4.0, 3.5, 3.0]),
              2: ([-0.01, 0.0, 0.015], [0.002, -0.001, 0.0], [1.0, 2.0, 5.0])}
    for model in (0, 1):
        wall = orc.Wall(model, body, motion)
        new = orc.step19(m, shape, 0.6, F=F, typ=typ, wall=wall)
        P0 = (m[0] * m[1:4])[:, fluid].sum(1)
        P1 = (new[0] * new[1:4])[:, fluid].sum(1)
        Fs = orc.solid_force(m, shape, 0.6, typ, wall, F=F, lattice=19)
        assert np.abs(P1 - P0 - (F[:, fluid].sum(1) - Fs[:3])).max() < 1e-12, model
        F1 = orc.solid_force(m, shape, 0.6, typ, wall, F=F, body_id=1, lattice=19)
        F2 = orc.solid_force(m, shape, 0.6, typ, wall, F=F, body_id=2, lattice=19)
        assert np.allclose(F1[:3] + F2[:3], Fs[:3], rtol=0, atol=1e-13)
        # the same motion described about r0 + d: T(r0 + d) = T(r0) - d x F
        d = np.array([0.7, -1.3, 2.1])
        V1 = np.add(motion[1][0], np.cross(motion[1][1], d))
        m1 = {1: (V1, motion[1][1], list(np.add(motion[1][2], d))), 2: motion[2]}
        F1s = orc.solid_force(m, shape, 0.6, typ, orc.Wall(model, body, m1), F=F, body_id=1,
                              lattice=19)
        assert np.allclose(F1s[3:], F1[3:] - np.cross(d, F1[:3]), rtol=0, atol=1e-12)
    # model 0 through the wall path equals the plain bounce-back step
    bb = orc.step19(m, shape, 0.6, F=F, typ=typ)
    assert np.abs(orc.step19(m, shape, 0.6, F=F, typ=typ, wall=orc.Wall(0, body)) - bb).max() == 0


def test_d3q19_moment_wall_moving_with_the_flow_keeps_uniform_flow(orc):
    rng = np.random.default_rng(39)
    shape = (8, 7, 6)
    N = 8 * 7 * 6
    body = _two_body_mask(shape, rng)
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    fluid = typ != orc.SOLID
    U = np.array([0.04, -0.02, 0.03])
    m = eq_state(1.0, np.repeat(U[:, None], N, 1))
    moving = orc.Wall(1, body, {1: (U, [0, 0, 0], [0, 0, 0]), 2: (U, [0, 0, 0], [3, 3, 3])})
    new = orc.step19(m, shape, 0.7, typ=typ, wall=moving)
    assert np.abs(new[:, fluid] - m[:, fluid]).max() < 1e-14
    bb = orc.step19(m, shape, 0.7, typ=typ, wall=orc.Wall(0, body))
    assert np.abs(bb[1:4, fluid] - m[1:4, fluid]).max() > 1e-3


def test_d3q19_sound_speed_and_acoustic_damping(orc):
    """A standing acoustic wave rho = 1 + eps cos(k x) on the 19-velocity lattice
    oscillates at c_s k with c_s^2 = 1/3 and decays at the rate of the D3Q27
    closure, Gamma = k^2 ((2/3) nu + mu_v / 2), mu_v = 1/9 (the trace of S is reset
    each step on both lattices)."""
    nx, tau, eps = 64, 0.6, 1e-5
    shape = (nx, 1, 1)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    m = eq_state(1.0 + eps * np.cos(k * x), np.zeros((3, nx)))
    amp = []
    cur = m
    T = 400
    for t in range(T + 1):
        amp.append(((cur[0] - 1.0) * np.cos(k * x)).sum() / (np.cos(k * x) ** 2).sum())
        cur = orc.step19(cur, shape, tau)
    a = np.array(amp) / eps
    # fit a damped cosine exp(-g t) cos(w t) through its zero crossings and peaks
    s = np.sign(a)
    zc = np.nonzero(s[1:] * s[:-1] < 0)[0]
    t0 = zc + a[zc] / (a[zc] - a[zc + 1])  # linear interpolation of each crossing
    w = np.pi / np.diff(t0).mean()
    cs_fit = w / k
    assert abs(cs_fit / np.sqrt(CS2) - 1) < 1e-3, cs_fit
    nu = CS2 * (tau - 0.5)
    gamma = k * k * (2.0 / 3.0 * nu + 1.0 / 18.0)
    env = np.abs(a[np.round(t0[:-1] + np.pi / w / 2).astype(int)])  # near the extrema
    tt = np.round(t0[:-1] + np.pi / w / 2)
    g_fit = -np.polyfit(tt, np.log(env), 1)[0]
    assert abs(g_fit / gamma - 1) < 1e-2, (g_fit, gamma)


@pytest.mark.parametrize("lattice", [27, 19])
def test_moving_wall_population_at_the_halfway_point(orc, lattice):
    """Sec. 3.2 for one isolated solid cell s of a rigid body in fluid at rest: each
    neighbour x = s + c has exactly one solid link, c, and after one step its
    moments are those of the rest populations with population c replaced by the
    reconstruction of (rho = 1, u^p, u^p u^p) at the halfway point p = s + c/2,
    u^p = V + Om x (p - r0) -- the wall point and velocity set independently of the
    step's own geometry."""
    n = 6
    shape = (n, n, n)
    N = n ** 3
    s = np.array([2, 2, 2])
    body = np.zeros(N, np.uint8)
    body[s[0] + n * (s[1] + n * s[2])] = 1
    V, Om, r0 = np.array([0.003, -0.002, 0.001]), np.array([0.01, -0.02, 0.03]), np.array([1.3, 2.7, 2.2])
    wall = orc.Wall(1, body, {1: (V, Om, r0)})
    typ = orc.classify((body > 0).reshape(shape[::-1]))[0]
    m = eq_state(1.0, np.zeros((3, N)))
    if lattice == 19:
        out = orc.step19(m, shape, 0.6, typ=typ, wall=wall)
        _, c, w = orc.reconstruct19(m[:, 0])
        def pop(i, mm):
            return orc.reconstruct19(mm)[0][i]
    else:
        out = orc.step(m, shape, 0.6, typ=typ, wall=wall)
        c, w = orc.lattice()
        def pop(i, mm):
            return orc.reconstruct(mm)[0, i]
    checked = 0
    for i, ci in enumerate(c):
        if not ci.any():
            continue
        x = s + ci
        nidx = x[0] + n * (x[1] + n * x[2])
        p = s + 0.5 * ci
        up = V + np.cross(Om, p - r0)
        mw = np.concatenate([[1.0], up, [up[a] * up[b] for a, b in PAIRS]])
        df = pop(i, mw) - w[i]  # the replaced population minus the rest one
        rho = 1.0 + df
        ci_f = ci.astype(float)
        want_u = ci_f * df / rho
        want_S = np.array([(ci_f[a] * ci_f[b] - CS2 * (a == b)) * df for a, b in PAIRS]) / rho
        assert abs(out[0, nidx] - rho) < 1e-15
        assert np.abs(out[1:4, nidx] - want_u).max() < 1e-15
        assert np.abs(out[4:, nidx] - want_S).max() < 1e-15
        checked += 1
    assert checked == len(c) - 1
