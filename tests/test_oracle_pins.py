"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
moment identity of the lattice, a conservation law, a closed-form solution,
a textbook count, or a value worked out by hand from the printed equations.
"""
import math
import os

import numpy as np
import pytest

from paper_2511_01629_gb300 import workloads as W

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(1234)


def _rand_u(D):
    u = np.zeros(3)
    u[:D] = RNG.uniform(-0.08, 0.08, D)
    return u


def _eye(D):
    e = np.zeros((3, 3))
    e[:D, :D] = np.eye(D)
    return e


# ---------------------------------------------------------------- lattice ---

@pytest.mark.parametrize("D", [2, 3])
def test_lattice_isotropy(oracle, D):
    """Sec. 2.2: weights sum to 1, zero first and third moments, second moment
    cs^2 I, fourth moment cs^4 (d_ij d_kl + d_ik d_jl + d_il d_jk)."""
    c, w, opp = oracle.lattice(D)
    c = c.astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    assert np.abs(np.einsum("q,qi,qj->ij", w, c, c) - CS2 * _eye(D)).max() < 1e-15
    assert np.abs(np.einsum("q,qi,qj,qk->ijk", w, c, c, c)).max() < 1e-15
    m4 = np.einsum("q,qi,qj,qk,ql->ijkl", w, c, c, c, c)
    e = _eye(D)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", e, e) + np.einsum("ik,jl->ijkl", e, e)
                      + np.einsum("il,jk->ijkl", e, e))
    assert np.abs(m4 - iso).max() < 1e-15
    assert np.all(c[opp] == -c)


def test_d2q9_numbering_matches_figure(oracle):
    """Fig. 1: c1..c4 = +x, +y, -x, -y; c5..c8 = (1,1), (-1,1), (-1,-1), (1,-1)."""
    c, w, _ = oracle.lattice(2)
    fig = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert [tuple(r[:2]) for r in c] == fig
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


# ------------------------------------------------------- per-node formulas ---

@pytest.mark.parametrize("D", [2, 3])
def test_feq_moments(oracle, D):
    """Eq. 12: sum feq = 0, sum feq c = u, sum feq c c = u u + p I."""
    c, _, _ = oracle.lattice(D)
    for _ in range(20):
        u, p = _rand_u(D), RNG.uniform(-0.05, 0.05)
        fe = oracle.feq(D, u, p)
        assert abs(fe.sum()) < 1e-16
        assert np.abs(fe @ c - u).max() < 1e-16
        Pi = np.einsum("q,qi,qj->ij", fe, c, c)
        assert np.abs(Pi - np.outer(u, u) - p * _eye(D)).max() < 1e-16


@pytest.mark.parametrize("D", [2, 3])
def test_macro_recovers_equilibrium(oracle, D):
    """Eq. 15 inverts Eq. 13: f = feq(u, p) returns (u, p); a force a shifts u
    by a/2 (Eq. 15a)."""
    for _ in range(20):
        u, p = _rand_u(D), RNG.uniform(-0.05, 0.05)
        fe = oracle.feq(D, u, p)
        u2, p2 = oracle.macro(D, fe)
        assert np.abs(u2 - u).max() < 1e-16 and abs(p2 - p) < 1e-16
        a = _rand_u(D) * 1e-2
        u3, _ = oracle.macro(D, fe, a)
        assert np.abs(u3 - (u + 0.5 * a)).max() < 1e-16


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.7])
def test_guo_force_moments(oracle, D, tau):
    """Eq. 14: sum F = 0, sum F c = (1 - 1/2tau) a, sum F c c = (1 - 1/2tau)(u a + a u)
    (lattice isotropy, Guo et al. 2002)."""
    c, _, _ = oracle.lattice(D)
    k = 1 - 1 / (2 * tau)
    for _ in range(10):
        u, a = _rand_u(D), _rand_u(D) * 1e-3
        F = oracle.force(D, tau, u, a)
        assert abs(F.sum()) < 1e-18
        assert np.abs(F @ c - k * a).max() < 1e-18
        m2 = np.einsum("q,qi,qj->ij", F, c, c)
        assert np.abs(m2 - k * (np.outer(u, a) + np.outer(a, u))).max() < 1e-18


@pytest.mark.parametrize("D", [2, 3])
def test_penalty_source_moments(oracle, D):
    """Eq. 17: S has zero mass and momentum and its second moment is E = alpha Pi_neq
    with Pi_neq = sum (f - feq) c c."""
    c, _, _ = oracle.lattice(D)
    Q = len(c)
    for _ in range(10):
        alpha = RNG.uniform(0.1, 1.5)
        f = RNG.uniform(-1e-3, 1e-3, Q)
        fe = oracle.feq(D, _rand_u(D), 1e-3)
        S = oracle.source(D, alpha, f, fe)
        E = alpha * np.einsum("q,qi,qj->ij", f - fe, c, c)
        tol = 1e-14 * np.abs(S).max()
        assert abs(S.sum()) < tol
        assert np.abs(S @ c).max() < tol
        assert np.abs(np.einsum("q,qi,qj->ij", S, c, c) - E).max() < tol


# ------------------------------------------------------------ indicators ---

def _golden_points():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "lattice_points.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_indicator_counts_circle(oracle):
    """Eq. 9 on the lattice: a disk of integer radius r centred on a node holds
    exactly the Gauss-circle number of nodes (OEIS A000328)."""
    for r, circle, _ in _golden_points():
        if r < 2:
            continue
        n = 2 * r + 9
        s = oracle.Sim(oracle.make_config(D=2, n=(n, n, 1), periodic=(1, 1, 1)))
        s.add_particles([[r + 3.0, r + 4.0]], [float(r)], [1.0])
        assert int((s.owner_map() == 0).sum()) == circle


def test_indicator_counts_sphere(oracle):
    """Eq. 9 in 3D: lattice points in a ball of integer radius (OEIS A000605)."""
    for r, _, sphere in _golden_points():
        if r < 2 or r > 7:
            continue
        n = 2 * r + 5
        s = oracle.Sim(oracle.make_config(D=3, n=(n, n, n), periodic=(1, 1, 1)))
        s.add_particles([[r + 2.0, r + 2.0, r + 2.0]], [float(r)], [1.0])
        assert int((s.owner_map() == 0).sum()) == sphere


def test_indicator_periodic_and_overlap(oracle):
    """Minimum image across a periodic face; overlapping particles give the node to
    the lowest index."""
    s = oracle.Sim(oracle.make_config(D=2, n=(20, 16, 1), periodic=(1, 0, 1)))
    s.add_particles([[0.2, 8.0], [3.0, 8.0]], [3.0, 3.0], [1.5, 1.5])
    own = s.owner_map()
    assert own[8, 19] == 0 and own[8, 18] == 0 and own[8, 17] == -1  # wraps in x
    assert own[8, 2] == 0 and own[8, 3] == 0  # (3,8): 2.8 from p0 -> p0 wins overlap
    assert own[8, 5] == 1 and own[8, 6] == 1 and own[8, 7] == -1
    s2 = oracle.Sim(oracle.make_config(D=2, n=(20, 16, 1), periodic=(1, 0, 1)))
    s2.add_particles([[3.0, 8.0], [0.2, 8.0]], [3.0, 3.0], [1.5, 1.5])
    assert s2.owner_map()[8, 2] == 0 and s2.owner_map()[8, 1] == 0


# ------------------------------------------------------------ projection ---

@pytest.mark.parametrize("D", [2, 3])
def test_rigid_projection_exact_on_rigid_field(oracle, D):
    """Eq. 22: for u = U + w x r on the solid nodes (noise elsewhere) and centres
    on symmetric lattice positions, the projection returns U and w exactly."""
    if D == 2:
        n, X, R = (40, 36, 1), [[10.0, 9.5], [27.5, 25.0]], [5.3, 6.1]
    else:
        n, X, R = (26, 24, 22), [[7.0, 7.5, 8.0], [18.5, 16.0, 13.5]], [4.2, 3.7]
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(0, 0, 0)))
    s.add_particles(X, R, [1.5, 2.0])
    own = s.owner_map()
    u = RNG.normal(size=own.shape + (D,)) * 1e-2
    Ut = [RNG.normal(size=3) * 1e-2 for _ in X]
    Wt = [RNG.normal(size=3) * 1e-3 for _ in X]
    if D == 2:
        for v in Ut:
            v[2] = 0
        for v in Wt:
            v[:2] = 0
    idx = np.argwhere(own >= 0)
    for ind in idx:
        p = own[tuple(ind)]
        xyz = ind[::-1].astype(float)  # (x, y[, z])
        r = np.zeros(3)
        r[:D] = xyz - np.asarray(X[p])
        u[tuple(ind)] = (Ut[p] + np.cross(Wt[p], r))[:D]
    U, Wv, cnt = s.rigid_projection(u)
    for p in range(len(X)):
        assert np.abs(U[p] - Ut[p]).max() < 1e-15
        assert np.abs(Wv[p] - Wt[p]).max() < 1e-15
        assert cnt[p] == int((own == p).sum())


# ------------------------------------------------------------ collisions ---

def test_collision_forces_by_hand(oracle):
    """Eqs. 19-21 evaluated by hand: C = (rho_s - rho_f)|g|.

    Pair: R = 5 and 5, delta = 1, eps_p = 2, d = 10.5, |g| = 2e-6.
      particle 0 (ratio 1.5): C = 1e-6, F = C/2 * (-10.5) * ((11 - 10.5)/1)^2 = -1.3125e-6
      particle 1 (ratio 2.0): C = 2e-6, F = +2.625e-6.
    Wall: R = 4 at y = 3.5 above the wall plane y = -1/2, eps_w = 1: image at -4.5,
      d' = 8 <= 2R + delta = 9, F_y = C * 8 * 1^2 = 8e-6 for C = 1e-6.
    """
    cfg = oracle.make_config(D=2, n=(100, 50, 1), periodic=(1, 1, 1), g_grav=(0, -2e-6),
                             delta=1.0, eps_p=2.0, eps_w=1.0)
    F = oracle.collision_forces(cfg, [[30.0, 20.0], [40.5, 20.0]], [5.0, 5.0], [1.5, 2.0])
    assert F[0] == pytest.approx([-1.3125e-6, 0, 0], abs=1e-20)
    assert F[1] == pytest.approx([2.625e-6, 0, 0], abs=1e-20)
    for d in (11.0, 11.5, 30.0):  # touching the range boundary or beyond: zero
        F = oracle.collision_forces(cfg, [[30.0, 20.0], [30.0 + d, 20.0]], [5.0, 5.0], [1.5, 2.0])
        assert np.all(F == 0)
    cfgw = oracle.make_config(D=2, n=(100, 50, 1), periodic=(1, 0, 1), g_grav=(0, -2e-6),
                              delta=1.0, eps_p=2.0, eps_w=1.0)
    F = oracle.collision_forces(cfgw, [[30.0, 3.5]], [4.0], [1.5])
    assert F[0] == pytest.approx([0, 8e-6, 0], abs=1e-20)
    F = oracle.collision_forces(cfgw, [[30.0, 45.5]], [4.0], [1.5])  # mirror at the top wall
    assert F[0] == pytest.approx([0, -8e-6, 0], abs=1e-20)
    F = oracle.collision_forces(cfgw, [[30.0, 4.0]], [4.0], [1.5])  # d' = 9: zero
    assert np.all(F == 0)
    cfg0 = oracle.make_config(D=2, n=(100, 50, 1), periodic=(1, 0, 1))  # no gravity: C = 0
    assert np.all(oracle.collision_forces(cfg0, [[30.0, 3.5]], [4.0], [1.5]) == 0)


def test_disk_column_workload_is_in_contact(oracle):
    """The contact workload of the GPU parity test engages Eq. 21 from the
    first step: every column disk feels a pair force (the bottom one is pushed
    down by its only neighbour, the top one up), and the disk beside the wall
    x = -1/2 is pushed in +x."""
    from paper_2511_01629_gb300 import workloads as W
    w = W.disk_column(seed=7)
    cfg = oracle.make_config(D=2, n=w.n, periodic=w.periodic, g_grav=w.g_grav, delta=w.delta,
                             eps_p=w.eps_p, eps_w=w.eps_w)
    F = oracle.collision_forces(cfg, w.pos, w.radius, w.ratio)
    col = len(w.radius) - 1
    assert np.all(np.abs(F[:col, 1]) > 0)
    assert F[0, 1] < 0 and F[col - 1, 1] > 0  # the ends are pushed outwards
    assert F[col, 0] > 0 and F[col, 1] == 0    # wall disk: +x only
    far = [[p[0], p[1] + 40.0 * k] for k, p in enumerate(w.pos[:2])]
    assert np.all(oracle.collision_forces(cfg, far, w.radius[:2], w.ratio[:2]) == 0)


# -------------------------------------------------------------- dynamics ---

def _uniform_state(oracle, D, n, U0):
    Q = 9 if D == 2 else 19
    fe = oracle.feq(D, U0, 0.0)
    N = int(np.prod(n))
    return np.repeat(fe[:, None], N, axis=1)


@pytest.mark.parametrize("D", [2, 3])
def test_neutral_particle_advects_with_uniform_flow(oracle, D):
    """A uniform flow feq(U0, 0) in a periodic box is a fixed point of Eq. 10 and a
    neutrally buoyant particle moving with it follows X0 + U0 t (Algorithm 1)."""
    if D == 2:
        n, U0, X0, R, v0 = (32, 24, 1), np.array([0.02, -0.013, 0]), [10.3, 12.7], 5.0, [0.05, 0.0]
    else:
        n, U0, X0, R, v0 = (16, 14, 12), np.array([0.02, -0.013, 0.01]), [6.3, 7.7, 5.2], 3.5, \
            [0.05, 0.0, 0.01]
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(1, 1, 1), tau=0.9))
    s.set_f(_uniform_state(oracle, D, n, U0))
    s.add_particles([X0], [R], [1.0], vel=[v0])
    s.step(1)  # Algorithm 1 averages U^0 = U0 with the initial velocity v0
    X1 = s.particles()["X"][0, :D]
    assert np.abs(X1 - (np.asarray(X0) + 0.5 * (U0[:D] + np.asarray(v0)))).max() < 1e-12
    steps = 40
    s.step(steps - 1)
    u, p, _ = s.fields()
    assert np.abs(u - U0[:D]).max() < 1e-14 and np.abs(p).max() < 1e-14
    part = s.particles()
    expect = (X1 + (steps - 1) * U0[:D]) % np.asarray(n[:D])
    assert np.abs(part["X"][0, :D] - expect).max() < 1e-11
    assert np.abs(part["U"][0, :D] - U0[:D]).max() < 1e-14
    assert np.abs(part["A"][0]).max() < 1e-11


@pytest.mark.parametrize("D", [2, 3])
def test_mass_invariant(oracle, D):
    """Streaming (periodic or bounce-back, moving walls included) conserves
    sum_x sum_a f, and collision multiplies it by (1 - 1/tau) since feq, F and S
    have zero sum (Eqs. 10, 12, 14, 17): the total follows (1-1/tau)^n."""
    tau = 0.8
    n = (18, 16, 1) if D == 2 else (10, 12, 9)
    wall = np.zeros((3, 2, 3))
    wall[1, 0, 0], wall[1, 1, 0] = -0.01, 0.02
    wk = W.random_small(7, D=D, n=n, periodic=(1, 0, 1), nparticles=2, rlo=2.5, rhi=3.5, tau=tau)
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(1, 0, 1), tau=tau, wall_u=wall,
                                      g_grav=wk.g_grav, g_drive=(1e-5, 0, 0)))
    Q = 9 if D == 2 else 19
    s.set_f(RNG.uniform(-1e-3, 1e-3, (Q,) + s.shape))
    s.add_particles(wk.pos, wk.radius, wk.ratio)
    tot = s.get_f().sum()
    for _ in range(6):
        s.step(1)
        new = s.get_f().sum()
        assert abs(new - (1 - 1 / tau) * tot) < 1e-16 * Q * s.N * 1e-3 * 10
        tot = new


@pytest.mark.parametrize("D", [2, 3])
def test_momentum_balance_periodic(oracle, D):
    """In a fully periodic box each step adds exactly sum_x a(x) to the total
    momentum of f* (Eq. 15a with the first moments of Eqs. 12, 14, 17): the
    drive on every node plus (1 - rho_f/rho_s) g + A_i on the solid nodes."""
    n = (20, 18, 1) if D == 2 else (12, 10, 11)
    wk = W.random_small(11, D=D, n=n, periodic=(1, 1, 1), nparticles=3, rlo=2.5, rhi=3.5)
    g = np.array([3e-5, -1e-4, 2e-5])[:D] if D == 3 else np.array([3e-5, -1e-4])
    drive = np.array([1e-5, 0, 0])
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(1, 1, 1), tau=0.9, g_grav=g,
                                      g_drive=drive[:D]))
    Q = 9 if D == 2 else 19
    c, _, _ = oracle.lattice(D)
    s.set_f(RNG.uniform(-1e-3, 1e-3, (Q,) + s.shape))
    s.add_particles(wk.pos, wk.radius, wk.ratio)
    g3 = np.zeros(3)
    g3[:D] = g
    for _ in range(5):
        mom0 = s.get_f().reshape(Q, -1).sum(axis=1) @ c
        A_in = s.particles()["A"]
        s.step(1)
        part = s.particles()
        expect = s.N * drive.copy()
        for p in range(s.np):
            expect += part["count"][p] * ((1 - 1 / wk.ratio[p]) * g3 + A_in[p])
        mom1 = s.get_f().reshape(Q, -1).sum(axis=1) @ c
        assert np.abs(mom1 - mom0 - expect).max() < 1e-15


def _poiseuille(oracle, D, tau, g, ny, steps):
    n = (2, ny, 1) if D == 2 else (2, ny, 2)
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(1, 0, 1), tau=tau, g_drive=(g, 0, 0)))
    s.step(steps)
    u, _, _ = s.fields()
    return u[..., 0].reshape(-1, ny, 2)[0, :, 0] if D == 3 else u[:, 0, 0]


@pytest.mark.parametrize("D", [2, 3])
def test_poiseuille_closed_form(oracle, D):
    """Steady channel flow under a body force between halfway bounce-back walls:
      * bulk second difference of u equals -g/nu, nu = cs^2 (tau - 1/2) (Eq. 16);
      * the profile is (g/2nu)(y+1/2)(H-1/2-y) plus the bounce-back slip
        (g/nu)(16L - 3)/24 with L = (tau - 1/2)^2, which vanishes at
        tau = 1/2 + sqrt(3)/4 (Ginzburg's closed form for halfway bounce-back).
    g is small so that the model's quadratic terms stay below round-off."""
    ny, g = 20, 1e-10
    y = np.arange(ny)
    for tau in (0.5 + math.sqrt(3) / 4, 0.8, 1.0):
        nu = CS2 * (tau - 0.5)
        ux = _poiseuille(oracle, D, tau, g, ny, 30000)
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.abs(d2 + g / nu).max() < 1e-9 * g / nu
        lam = (tau - 0.5) ** 2
        exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y) + g / nu * (16 * lam - 3) / 24
        assert np.abs(ux - exact).max() < 1e-10 * exact.max()


def test_poiseuille_startup_transient(oracle):
    """Start-up of the 100x200 channel (tau 0.8, g 1e-6) after 2000 steps against
    the Fourier-series solution of the diffusion problem with plates at
    y = -1/2 and H - 1/2; the lattice velocity at step n is the continuous one at
    t = n + 1/2 (Eq. 15a adds a/2 to the initial f = 0).  Agreement to O(dx^2)."""
    tau, g, H, steps = 0.8, 1e-6, 200, 2000
    nu = CS2 * (tau - 0.5)
    ux = _poiseuille(oracle, 2, tau, g, H, steps)
    eta = np.arange(H) + 0.5
    t = steps + 0.5
    series = np.zeros(H)
    for k in range(1, 400, 2):
        series += 4 * g * H ** 2 / (nu * math.pi ** 3 * k ** 3) * np.sin(k * math.pi * eta / H) \
            * math.exp(-nu * k * k * math.pi ** 2 * t / H ** 2)
    exact = g / (2 * nu) * eta * (H - eta) - series
    assert np.abs(ux - exact).max() < 1e-3 * exact.max()


def _couette(oracle, D, tau, u_lo, u_hi, H, steps, comp=0):
    """Steady flow between two walls moving along axis `comp` (x, or z in 3D)
    with velocities u_lo (plane y = -1/2) and u_hi (plane y = H - 1/2)."""
    wall = np.zeros((3, 2, 3))
    wall[1, 0, comp], wall[1, 1, comp] = u_lo, u_hi
    n = (2, H, 1) if D == 2 else (2, H, 2)
    s = oracle.Sim(oracle.make_config(D=D, n=n, periodic=(1, 0, 1), tau=tau, wall_u=wall))
    s.step(steps)
    u, _, _ = s.fields()
    return (u[:, 0, :] if D == 2 else u[0, :, 0, :])  # [y, D]


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("tau,steps", [(0.6, 30000), (0.8, 20000), (1.0, 20000), (1.7, 12000)])
@pytest.mark.parametrize("u_lo,u_hi", [(-5e-3, 5e-3), (0.0, 1e-2), (3e-3, -7e-3)])
def test_moving_wall_couette_closed_form(oracle, D, tau, steps, u_lo, u_hi):
    """Plane Couette flow under halfway bounce-back with the moving-wall term
    (reading of the wall treatment: planes at -1/2 and H - 1/2).  The steady
    profile is the straight line through the wall velocities at the planes,
      u_x(y) = u_lo + (u_hi - u_lo) (y + 1/2) / H,
    exact for the BGK lattice at any tau (the linear profile makes the
    second-order Chapman-Enskog terms vanish and halfway bounce-back of a linear
    field is exact), so it holds to round-off.  It fixes the wall term itself,
    not only a ratio: a wrong factor, sign or power of cs^2 in
    2 w_a (c_a . u_w) / cs^2 moves the line's ends."""
    H = 16
    u = _couette(oracle, D, tau, u_lo, u_hi, H, steps)
    y = np.arange(H)
    exact = u_lo + (u_hi - u_lo) * (y + 0.5) / H
    scale = max(abs(u_lo), abs(u_hi))
    assert np.abs(u[:, 0] - exact).max() < 1e-12 * scale
    assert np.abs(u[:, 1:]).max() < 1e-13 * scale  # no wall-normal or spanwise flow


def test_moving_wall_couette_spanwise_3d(oracle):
    """The same closed form with the walls moving along z in D3Q19 (the edge
    velocities with c_z != 0 carry the wall term)."""
    H = 16
    u = _couette(oracle, 3, 0.9, 2e-3, -6e-3, H, 20000, comp=2)
    exact = 2e-3 + (-6e-3 - 2e-3) * (np.arange(H) + 0.5) / H
    assert np.abs(u[:, 2] - exact).max() < 1e-12 * 6e-3
    assert np.abs(u[:, :2]).max() < 1e-13 * 6e-3


def _slab(oracle, tau, alpha, steps=30000, ny=60, y1=20, y2=40):
    wall = np.zeros((3, 2, 3))
    wall[1, 0, 0], wall[1, 1, 0] = -5e-6, 5e-6
    s = oracle.Sim(oracle.make_config(D=2, n=(2, ny, 1), periodic=(1, 0, 1), tau=tau, alpha=alpha,
                                      wall_u=wall))
    mask = np.zeros((ny, 2), np.int32)
    mask[y1:y2] = 1
    s.set_static_solid(mask)
    s.step(steps)
    u, _, _ = s.fields()
    gam = np.diff(u[:, 0, 0])
    return gam[3:y1 - 4].mean(), gam[y1 + 3:y2 - 4].mean(), gam


@pytest.mark.parametrize("tau,alpha", [(1.0, 0.5), (0.8, 0.5), (0.9, 0.9)])
def test_penalized_slab_effective_viscosity(oracle, tau, alpha):
    """Couette flow across a penalized layer (Eq. 17 on chi = 1): the stress is
    continuous, so the shear-rate ratio is nu / nu_eff.  The source keeps a
    fraction alpha*tau of the non-equilibrium second moment, i.e. relaxes it with
    tau_eff = tau / (1 - alpha tau), so nu_eff = cs^2 (tau_eff - 1/2).  (The
    printed nu/(1 - alpha tau) of Sec. 2.2 omits the -1/2 lattice term.)"""
    gf, gs, _ = _slab(oracle, tau, alpha)
    nu = CS2 * (tau - 0.5)
    nu_eff = CS2 * (tau / (1 - alpha * tau) - 0.5)
    assert gs / gf == pytest.approx(nu / nu_eff, rel=1e-10)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_penalized_slab_vanishing_strain_at_alpha_one_over_tau(oracle, tau):
    """With alpha = 1/tau (every run of Sec. 3) the strain rate inside the
    penalized layer vanishes: the layer moves rigidly."""
    gf, gs, gam = _slab(oracle, tau, 1.0 / tau)
    assert np.abs(gam[21:38]).max() < 1e-12 * abs(gf)


def test_algorithm1_trapezoid_and_collision_acceleration(oracle):
    """Algorithm 1 with a wall force F normal to the wall and motion otherwise only
    along the periodic axis: A^{n+1} = F/M for K = 1 (F(X*) = F(X^n) exactly) and
    F/(K M) for K sub-steps (the corrections add K terms (dt/K)^2 F / 2M; the
    sub-step displacement changes F by O(C), kept small by a weak gravity),
    with M = rho_s * (number of solid nodes).  The motion along x gets no
    collision acceleration."""
    for K in (1, 2, 3):
        cfg = oracle.make_config(D=2, n=(40, 30, 1), periodic=(1, 0, 1), tau=1.0,
                                 g_grav=(-1e-8, 0), delta=1.0, eps_w=1.0, K=K)
        s = oracle.Sim(cfg)
        ratio, R, y0 = 1.5, 4.0, 3.5
        s.add_particles([[20.0, y0]], [R], [ratio])
        Fw = oracle.collision_forces(cfg, [[20.0, y0]], [R], [ratio])[0]
        assert Fw[1] > 0
        s.step(1)
        part = s.particles()
        M = ratio * part["count"][0]
        assert part["A"][0, 1] == pytest.approx(Fw[1] / (K * M), rel=1e-12 if K == 1 else 1e-9)
        assert part["A"][0, 0] == 0.0  # no force along x: no correction, exactly


def test_orientation_trapezoid(oracle):
    """theta^{n+1} = theta^n + dt (w^n + w^{n-1}) / 2 (reading: the paper reports theta
    but gives no rule).  Fluid at rest and a centre on a node: the solid nodes all
    see the same acceleration, the symmetric node set has sum r = 0, so w^0 = 0
    and theta^1 is half the initial angular velocity."""
    s = oracle.Sim(oracle.make_config(D=2, n=(30, 30, 1), periodic=(1, 1, 1), g_grav=(0, -1e-4)))
    s.add_particles([[15.0, 15.0]], [5.0], [1.5], omega=[0.01])
    s.step(1)
    part = s.particles()
    assert abs(part["W"][0, 2]) < 1e-20
    assert part["theta"][0, 2] == pytest.approx(0.005, rel=1e-15)


def test_collision_acceleration_vanishes_without_forces(oracle):
    """Algorithm 1 with no collision force: X^{n+1} = X^n + Ubar, so A^{n+1} =
    (2/dt^2)(X^{n+1} - X^n - dt Ubar) is exactly zero, at any position.  (Its
    literal evaluation as a difference of positions of size ~10^3 would leave
    ulp(X) ~ 1e-13 of rounding noise instead; the oracle evaluates the bracket
    as the sum of the sub-step corrections it equals.)"""
    for K in (1, 3):
        s = oracle.Sim(oracle.make_config(D=2, n=(64, 1600, 1), periodic=(1, 0, 1), tau=1.0,
                                          g_grav=(0, -2e-6), K=K))
        s.add_particles([[31.3, 1280.123456789]], [12.0], [1.5], vel=[[1.234e-5, -3.21e-5]])
        for _ in range(5):
            s.step(1)
            assert np.all(s.particles()["A"] == 0.0)


def test_single_disk_is_insensitive_to_round_off(oracle):
    """Without collisions the settling-disk dynamics damp small perturbations:
    populations perturbed by 1e-12 (relative) stay within 1e-18 (absolute) of
    the unperturbed run over 300 steps.  A rounding-noise force of ulp(X) per
    step in A^{n+1} would instead decorrelate the two runs to ~1e-12 within
    ~150 steps."""
    w = W.single_disk(0, nx=100, ny=400, radius=8.0)
    cfg = oracle.make_config(D=2, n=w.n, periodic=w.periodic, tau=w.tau, alpha=w.alpha,
                             g_grav=w.g_grav)
    sims = []
    for eps in (0.0, 1e-12):
        sim = oracle.Sim(cfg, parallel=True)
        sim.add_particles(w.pos, w.radius, w.ratio)
        sim.step(1)
        if eps:
            f = sim.get_f()
            sim.set_f(f * (1 + eps * np.random.default_rng(0).standard_normal(f.shape)))
        sims.append(sim)
    for sim in sims:
        sim.step(299)
    d = np.abs(sims[1].fields()[0] - sims[0].fields()[0]).max()
    assert d < 1e-18, d
