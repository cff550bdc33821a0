"""The oracle on the paper's particle experiments (Secs. 3.1 and 3.4), pinned
by what the physics fixes rather than by the oracle itself:

  * plane Couette flow is unchanged by a half turn about the channel centre
    line, so a disk released at (x0, y0) and one released at
    (L - x0, H - 1 - y0) follow trajectories that are each other's half
    turn: X' = L - X, Y' = H - 1 - Y, U' = -U, omega' = omega;
  * a neutrally buoyant disk released off centre in Couette flow migrates
    towards the centre line and comes to rest there (Sec. 3.1) and, free of
    torque, turns at about
    half the shear rate, omega = -gamma / 2 (the rotation of a free circle in
    simple shear; the walls 1.5 D away slow it slightly);
  * two disks released one above the other draft, kiss and tumble
    (Sec. 3.4): the upper disk falls faster in the wake of the lower one,
    the two stay in contact range for a while, and then the upper one passes
    the lower one and they separate sideways;
  * an ellipse released at 45 degrees in a vertical channel (Sec. 3.3)
    turns broadside, swings off the centre line and back, and settles on it
    at Re ~ 11 (the paper reports 11 for this case).

The stored trajectories (tests/golden/make_oracle_references.py) are
recomputed here over their first rows, bit for bit.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2511_01629_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _config(w):
    return oracle.make_config(D=w.D, n=w.n, periodic=w.periodic, wall_u=w.wall_u, tau=w.tau,
                              alpha=w.alpha, g_grav=w.g_grav, g_drive=w.g_drive, delta=w.delta,
                              eps_p=w.eps_p, eps_w=w.eps_w, K=w.K)


def _couette_case():
    return W.couette_migration(H=40, diameter=10.0, length_d=20.0, U_w=1.0 / 12.0, steps=28000)


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name))


def _rows(w, every, upto):
    s = oracle.Sim(_config(w), parallel=True)
    s.add_particles(w.pos, w.radius, w.ratio)
    out = []
    for n in range(0, upto + 1, every):
        if n:
            s.step(every)
        p = s.particles()
        row = [n]
        for i in range(w.num_particles):
            row += [*p["X"][i, :2], *p["U"][i, :2], p["W"][i, 2], p["count"][i]]
        out.append(row)
    s.close()
    return np.array(out, dtype=np.float64)


def test_couette_reference_matches_the_oracle():
    ref = _load("couette_migration_h40.txt")
    got = _rows(_couette_case(), 200, 2000)
    assert np.array_equal(got, ref[: len(got)])


def test_dkt_reference_matches_the_oracle():
    ref = _load("dkt_l200.txt")
    got = _rows(W.dkt(), 100, 300)
    assert np.array_equal(got, ref[: len(got)])


def test_couette_disk_trajectory_is_symmetric_under_a_half_turn():
    """The walls move at -U_w/2 (bottom) and +U_w/2 (top): a half turn about
    the centre line maps the wall velocities, the lattice and the initial
    fluid at rest onto themselves, so it maps a disk's trajectory onto the
    trajectory of the turned disk.  A sign error in the moving-wall term of
    one face, or a wall plane off by a node, breaks it at once."""
    w = W.couette_migration(H=40, diameter=10.0, length_d=8.0, U_w=1.0 / 12.0, steps=600)
    L, H = w.n[0], w.n[1]
    x0, y0 = 17.25, 11.375
    runs = []
    for pos in ([x0, y0], [L - x0, H - 1 - y0]):
        s = oracle.Sim(_config(w))
        s.add_particles([pos], w.radius, w.ratio)
        s.step(w.steps)
        runs.append(s.particles())
        s.close()
    a, b = runs
    assert a["count"][0] == b["count"][0] > 0
    # the disk has moved and turned, and the two runs are each other's half turn
    assert abs(a["X"][0, 0] - x0) > 1.0 and abs(a["W"][0, 2]) > 1e-5
    dX = (L - a["X"][0, 0]) - b["X"][0, 0]
    dX -= L * np.round(dX / L)
    assert abs(dX) < 1e-9
    assert abs((H - 1 - a["X"][0, 1]) - b["X"][0, 1]) < 1e-9
    assert np.abs(a["U"][0, :2] + b["U"][0, :2]).max() < 1e-12
    assert abs(a["W"][0, 2] - b["W"][0, 2]) < 1e-12


def test_couette_disk_migrates_to_the_centre_line():
    """Stored run at the paper's particle and channel Reynolds numbers
    (gamma D^2 / nu = 1.25, U_w H / nu = 20) over the paper's shear time
    gamma t = 58: y/H rises in every window of gamma t = 5.8 from 0.25,
    passes 0.40 and stays below the centre line; omega / gamma averages
    -1/2 within 15 % once the shear profile has formed (gamma t > 29)."""
    r = _load("couette_migration_h40.txt")
    H, gamma = 40, 1.0 / 12.0 / 40
    yH = (r[:, 2] + 0.5) / H
    assert yH[0] == 0.25
    win = yH[::14]
    assert np.all(np.diff(win) > 0.005), win
    assert 0.40 < yH[-1] < 0.5
    assert np.all(yH < 0.5)
    late = r[:, 0] > 14000
    w_over_g = r[late, 5] / gamma
    assert -0.575 < w_over_g.mean() < -0.425, w_over_g.mean()
    # the node count stays that of a disk R = 5 (pi R^2 = 78.5)
    assert np.all(np.abs(r[1:, 6] - np.pi * 25) < 6)


def test_couette_disk_comes_to_rest_at_the_centre_line():
    """The same case run to gamma t = 417: the migration ends at the centre
    line (Sec. 3.1).  y/H rises in every window of gamma t ~ 21 until it is
    within 0.01 of 0.5, then stays on a plateau from gamma t ~ 170 on; the
    plateau lies less than one lattice unit below the centre line (the
    staircase of a D = 10 disk on the lattice shifts its equilibrium by a
    fraction of a node) and jitters by less than 0.1 node as the disk's node
    set changes with its x position.  The run is bit for bit the short stored
    run over their common rows."""
    r = _load("couette_migration_h40_long.txt")
    short = _load("couette_migration_h40.txt")
    common = short[np.isin(short[:, 0], r[:, 0])]
    assert len(common) == 15 and np.array_equal(common, r[: len(common)])
    H = 40
    yH = (r[:, 2] + 0.5) / H
    rising = yH[yH < 0.49]
    assert np.all(np.diff(rising[::5]) > 0), rising[::5]
    plateau = yH[r[:, 0] >= 80000]
    assert np.all(np.abs(plateau - 0.5) < 1.0 / H), plateau.min()
    assert np.all(plateau < 0.5)
    assert plateau.max() - plateau.min() < 0.1 / H
    # settled: the lateral velocity averages to zero on the plateau
    assert abs(r[r[:, 0] >= 80000, 4].mean()) < 2e-5


def test_dkt_reference_drafts_kisses_and_tumbles():
    """Stored DKT run (disk 0 starts above disk 1, both on the centre line):
    drafting — after the start the gap closes from 2 D to contact range while
    disk 0 falls faster; kissing — the centres stay within R_0 + R_1 + delta (the range of
    the collision force of Eq. 19) for at least 1,000 steps, over the first
    1,000 of them nearly in line (|x_0 - x_1| < R); tumbling — disk 0 then passes below disk 1 and the two
    separate sideways to more than 2 D apart, falling side by side."""
    d = _load("dkt_l200.txt")
    t = d[:, 0]
    X0, Y0, U0 = d[:, 1], d[:, 2], d[:, 4]
    X1, Y1, U1 = d[:, 7], d[:, 8], d[:, 10]
    R, delta = 10.0, 1.0
    dist = np.hypot(X0 - X1, Y0 - Y1)
    assert abs(dist[0] - 4 * R) < 1e-3  # 2 D apart (the 0.1 offset adds 1.25e-4)
    contact = dist <= 2 * R + delta
    first = int(np.argmax(contact))
    assert contact.any() and t[first] > 0
    # drafting: before contact the trailing disk is faster and the gap shrinks
    approach = (t > 500) & (t < t[first])
    assert np.all(U0[approach] < U1[approach])
    # (over the first few hundred steps, while both accelerate, the gap first opens by ~0.07)
    assert np.all(np.diff(dist[approach]) < 0)
    assert dist[: first + 1].max() < 4 * R + 0.1
    # kissing: a contiguous stretch in contact range, nearly in line
    last = first
    while last + 1 < len(d) and contact[last + 1]:
        last += 1
    assert t[last] - t[first] >= 1000, (t[first], t[last])
    inline = (t >= t[first]) & (t <= t[first] + 1000)
    assert np.all(np.abs(X0[inline] - X1[inline]) < R)
    assert np.all(Y0[inline] > Y1[inline])
    # tumbling: disk 0 ends up below disk 1, side by side and apart
    swap = int(np.argmax(Y0 < Y1))
    assert Y0[swap] < Y1[swap] and swap > last
    after = t > t[swap] + 1000
    assert np.all(np.abs(X0[after] - X1[after]) > 2 * (2 * R))
    assert np.all(Y0[after] < Y1[after])


def _ellipse_rows(upto):
    w = W.ellipse_settling()
    s = oracle.Sim(_config(w), parallel=True)
    s.add_ellipses(w.pos, w.radius, w.minor, w.theta, w.ratio)
    out = []
    for n in range(0, upto + 1, 100):
        if n:
            s.step(100)
        p = s.particles()
        out.append([n, *p["X"][0, :2], *p["U"][0, :2], p["W"][0, 2], p["theta"][0, 2], p["count"][0]])
    s.close()
    return np.array(out, dtype=np.float64)


def test_ellipse_reference_matches_the_oracle():
    ref = _load("ellipse_settling_l200.txt")
    got = _ellipse_rows(200)
    assert np.array_equal(got, ref[: len(got)])


def test_ellipse_reference_settles_broadside_on_the_centre_line():
    """Stored run of workloads.ellipse_settling (a = 25, b = 12.5, L = 8 a,
    ratio 1.1, 30,000 steps): the major axis starts at 45 degrees and ends
    horizontal (|sin theta| < 0.05 over the last 30 % of the run); the
    ellipse first drifts more than 10 lattice units off the centre line and
    comes back within 2; its settling velocity over the last 20 % gives
    Re = 2 a U / nu between 10 and 14 (nu = 1/6 at tau = 1)."""
    r = _load("ellipse_settling_l200.txt")
    t, x, uy, th = r[:, 0], r[:, 1], r[:, 4], r[:, 6]
    xc = 99.5
    assert abs(th[0] - math.pi / 4) < 1e-15
    late = t > 0.7 * t[-1]
    assert np.all(np.abs(np.sin(th[late])) < 0.05)
    assert np.abs(x - xc).max() > 10.0
    assert abs(x[-1] - xc) < 2.0
    tail = t > 0.8 * t[-1]
    Re = 2 * 25.0 * np.abs(uy[tail]).mean() * 6.0
    assert 10.0 < Re < 14.0, Re
    # the node count stays that of the ellipse (pi a b = 981.7)
    assert np.all(np.abs(r[1:, 7] - math.pi * 25 * 12.5) < 15)
