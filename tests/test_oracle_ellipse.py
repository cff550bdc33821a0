"""Pins of the oracle's ellipse particles (Sec. 3.3), each against something
other than the oracle's own formula:

  * the solid indicator against the focal definition of an ellipse (the
    nodes whose distances to the two foci sum to at most 2a), evaluated
    independently in numpy;
  * equal axes give the disk, a half turn gives the same solid and the same
    motion, and a quarter turn swaps the roles of the axes;
  * the node count against the area pi a b;
  * the collision forces: an ellipse aligned with a wall or with the line of
    centres acts like a disk of radius equal to its semi-axis along that
    line (the support distance), for both orientations;
  * Eq. 22 in 2D does not depend on the shape: a rigid rotation of the fluid
    inside any ellipse is recovered exactly as U = 0, omega = Omega.
"""
import math

import numpy as np
import pytest

import oracle


def _sim(n=(96, 80, 1), periodic=(0, 0, 1), tau=1.0, g=(0.0, -1e-5, 0.0), eps_w=1.0):
    return oracle.Sim(oracle.make_config(D=2, n=n, periodic=periodic, tau=tau, g_grav=g,
                                         eps_w=eps_w))


CASES = [
    # centre, a, b, theta
    ((40.3, 37.85), 20.0, 10.0, math.pi / 4),
    ((47.12, 41.07), 25.0, 12.5, 0.3),
    ((44.71, 38.33), 18.5, 4.25, -1.1),
    ((43.0, 40.0), 12.0, 11.0, 2.7),
    ((39.5, 42.25), 30.0, 7.5, math.pi / 2 + 0.05),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_ellipse_indicator_matches_the_focal_definition(case):
    (X, Y), a, b, th = CASES[case]
    s = _sim()
    s.add_ellipses([[X, Y]], [a], [b], [th], [1.1])
    own = s.owner_map()
    c = math.sqrt(a * a - b * b)
    F1 = (X + c * math.cos(th), Y + c * math.sin(th))
    F2 = (X - c * math.cos(th), Y - c * math.sin(th))
    j, i = np.mgrid[0:own.shape[0], 0:own.shape[1]].astype(np.float64)
    total = np.hypot(i - F1[0], j - F1[1]) + np.hypot(i - F2[0], j - F2[1])
    # no node is so close to the boundary that rounding could decide it
    assert np.abs(total - 2 * a).min() > 1e-9
    focal = total <= 2 * a
    assert focal.sum() > 0
    assert np.array_equal(own == 0, focal)


def test_ellipse_node_count_is_close_to_its_area():
    for (X, Y), a, b, th in CASES:
        s = _sim()
        s.add_ellipses([[X, Y]], [a], [b], [th], [1.1])
        cnt = int((s.owner_map() == 0).sum())
        area = math.pi * a * b
        # lattice-point count of a convex domain: error well below its perimeter
        perim = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))
        assert abs(cnt - area) < 0.25 * perim, (a, b, cnt, area)


def test_equal_axes_give_the_disk():
    """b = a is the disk (the disk's own test, bit for bit, whatever theta),
    and b = a (1 - 1e-13) takes the ellipse test and still gives the disk's
    solid, for any orientation."""
    X, R = [[40.37, 38.81]], [13.0]
    ref = _sim()
    ref.add_particles(X, R, [1.2])
    own_disk = ref.owner_map()
    for th in (0.0, 0.7, -2.1):
        s = _sim()
        s.add_ellipses(X, R, R, [th], [1.2])
        assert np.array_equal(s.owner_map(), own_disk)
        s2 = _sim()
        s2.add_ellipses(X, R, [R[0] * (1 - 1e-13)], [th], [1.2])
        assert np.array_equal(s2.owner_map(), own_disk)
    # the same dynamics, bit for bit, over a few steps
    s = _sim()
    s.add_ellipses(X, R, R, [0.7], [1.2])
    for sim in (ref, s):
        sim.step(20)
    a, b = ref.particles(), s.particles()
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["W"], b["W"])


def test_half_turn_gives_the_same_solid_and_motion():
    X = [[45.3, 39.6]]
    runs = []
    for th in (0.35, 0.35 + math.pi):
        s = _sim()
        s.add_ellipses(X, [20.0], [9.0], [th], [1.3])
        own = s.owner_map()
        s.step(40)
        runs.append((own, s.particles()))
    (o1, p1), (o2, p2) = runs
    assert np.array_equal(o1, o2)
    assert np.abs(p1["X"] - p2["X"]).max() < 1e-12
    assert np.abs(p1["W"] - p2["W"]).max() < 1e-15
    assert abs((p2["theta"][0, 2] - p1["theta"][0, 2]) - math.pi) < 1e-12


def test_quarter_turn_swaps_the_axes():
    """The ellipse (a, b) turned by pi/2 is the ellipse whose a axis lies
    along y: the focal test with the foci on the y axis."""
    X, Y, a, b = 46.5, 39.5, 22.0, 8.0
    s = _sim()
    s.add_ellipses([[X, Y]], [a], [b], [math.pi / 2], [1.1])
    own = s.owner_map()
    j, i = np.mgrid[0:own.shape[0], 0:own.shape[1]].astype(np.float64)
    inside = ((i - X) / b) ** 2 + ((j - Y) / a) ** 2 <= 1.0
    margin = np.abs(((i - X) / b) ** 2 + ((j - Y) / a) ** 2 - 1.0)
    assert margin.min() > 1e-9
    assert np.array_equal(own == 0, inside)


def test_wall_forces_use_the_extent_normal_to_the_wall():
    """theta = 0: against the x walls the ellipse acts like a disk of radius
    a, against the y walls like a disk of radius b; theta = pi/2 swaps them;
    at 45 degrees both extents are sqrt((a^2 + b^2) / 2)."""
    cfg = oracle.make_config(D=2, n=(80, 60, 1), periodic=(0, 0, 1), g_grav=(0, -1e-4, 0),
                             delta=1.5, eps_w=1.0, eps_p=2.0)
    a, b = 12.0, 5.0
    # centre 0.4 inside the range of the x wall for a, and of the y wall for b
    X = [[-0.5 + a + 0.75 - 0.4, -0.5 + b + 0.75 - 0.4]]
    F = oracle.collision_forces_ellipse(cfg, X, [a], [b], [0.0], [1.5])
    Fx_disk = oracle.collision_forces(cfg, X, [a], [1.5])[0, 0]
    Fy_disk = oracle.collision_forces(cfg, X, [b], [1.5])[0, 1]
    assert Fx_disk > 0 and Fy_disk > 0
    assert F[0, 0] == Fx_disk and F[0, 1] == Fy_disk
    # turned by pi/2: the a extent faces the y wall; put the centre accordingly
    X2 = [[-0.5 + b + 0.75 - 0.4, -0.5 + a + 0.75 - 0.4]]
    F2 = oracle.collision_forces_ellipse(cfg, X2, [a], [b], [math.pi / 2], [1.5])
    G2 = oracle.collision_forces(cfg, X2, [b], [1.5])[0, 0], oracle.collision_forces(cfg, X2, [a], [1.5])[0, 1]
    assert F2[0, 0] == pytest.approx(G2[0], rel=1e-12) and F2[0, 1] == pytest.approx(G2[1], rel=1e-12)
    # 45 degrees: the extent is sqrt((a^2 + b^2) / 2) against both walls
    h = math.sqrt((a * a + b * b) / 2)
    X3 = [[-0.5 + h + 0.75 - 0.4, -0.5 + h + 0.75 - 0.4]]
    F3 = oracle.collision_forces_ellipse(cfg, X3, [a], [b], [math.pi / 4], [1.5])
    G3 = oracle.collision_forces(cfg, X3, [h], [1.5])[0]
    assert F3[0, :2] == pytest.approx(G3[:2], rel=1e-9)


def test_pair_forces_use_the_extent_along_the_line_of_centres():
    cfg = oracle.make_config(D=2, n=(200, 200, 1), periodic=(1, 1, 1), g_grav=(0, -1e-4, 0),
                             delta=1.5, eps_p=2.0)
    a, b = 12.0, 5.0
    # along x, both aligned with the line of centres: a + a
    X = [[80.0, 100.0], [80.0 + 2 * a + 1.0, 100.0]]
    F = oracle.collision_forces_ellipse(cfg, X, [a, a], [b, b], [0.0, 0.0], [1.5, 1.5])
    G = oracle.collision_forces(cfg, X, [a, a], [1.5, 1.5])
    assert G[0, 0] < 0 and np.array_equal(F, G)
    # along x, both across the line of centres: b + b
    X = [[80.0, 100.0], [80.0 + 2 * b + 1.0, 100.0]]
    F = oracle.collision_forces_ellipse(cfg, X, [a, a], [b, b], [math.pi / 2] * 2, [1.5, 1.5])
    G = oracle.collision_forces(cfg, X, [b, b], [1.5, 1.5])
    assert G[0, 0] < 0 and F == pytest.approx(G, rel=1e-12, abs=1e-30)
    # one of each: a + b
    X = [[80.0, 100.0], [80.0 + a + b + 1.0, 100.0]]
    F = oracle.collision_forces_ellipse(cfg, X, [a, a], [b, b], [0.0, math.pi / 2], [1.5, 1.5])
    G = oracle.collision_forces(cfg, X, [a, b], [1.5, 1.5])
    assert G[0, 0] < 0 and F == pytest.approx(G, rel=1e-12, abs=1e-30)


def test_pair_forces_for_tilted_ellipses_use_their_support_distances():
    """Line of centres at angle phi, ellipses at theta_i and theta_j: each
    acts like a disk of radius h = sqrt(a^2 cos^2(phi - theta) + b^2
    sin^2(phi - theta)), the support distance along the line of centres."""
    cfg = oracle.make_config(D=2, n=(300, 300, 1), periodic=(1, 1, 1), g_grav=(0, -1e-4, 0),
                             delta=2.0, eps_p=2.0)
    a, b, phi = 14.0, 6.0, 0.6
    th = [0.2, -0.9]
    h = [math.sqrt((a * math.cos(phi - t)) ** 2 + (b * math.sin(phi - t)) ** 2) for t in th]
    dist = h[0] + h[1] + 0.5 * 2.0
    X = [[150.0, 150.0], [150.0 - dist * math.cos(phi), 150.0 - dist * math.sin(phi)]]
    F = oracle.collision_forces_ellipse(cfg, X, [a, a], [b, b], th, [1.5, 1.5])
    G = oracle.collision_forces(cfg, X, h, [1.5, 1.5])
    assert np.abs(G[0]).max() > 0
    assert F == pytest.approx(G, rel=1e-9, abs=1e-30)


def test_rigid_rotation_inside_an_ellipse_is_recovered():
    """Eq. 22 in 2D: omega = sum r x u / sum |r|^2 holds for any shape; a
    velocity field of rigid rotation about the centre gives U = 0 to round-off
    and omega = Omega (the node set is symmetric under a half turn about a
    centre on a node)."""
    s = _sim(n=(90, 70, 1))
    X, Y = 44.0, 35.0
    s.add_ellipses([[X, Y]], [21.0], [8.5], [0.6], [1.4])
    ny, nx = 70, 90
    j, i = np.mgrid[0:ny, 0:nx].astype(np.float64)
    Om = 3.7e-4
    u = np.zeros((ny, nx, 2))
    u[..., 0] = -Om * (j - Y)
    u[..., 1] = Om * (i - X)
    U, Wv, cnt = s.rigid_projection(u)
    assert cnt[0] > 0
    assert np.abs(U[0]).max() < 1e-18
    assert Wv[0, 2] == pytest.approx(Om, rel=1e-14)


def test_bad_ellipses_are_refused():
    """Axes out of order or non-positive, and ellipses in 3D, are refused by the
    oracle (the C ABI refuses the same, tests/test_gpu_ellipse.py)."""
    s = _sim()
    with pytest.raises(ValueError):
        s.add_ellipses([[40.0, 40.0]], [5.0], [6.0], [0.0], [1.2])  # b > a
    with pytest.raises(ValueError):
        s.add_ellipses([[40.0, 40.0]], [5.0], [0.0], [0.0], [1.2])  # b = 0
    assert s.np == 0
    s3 = oracle.Sim(oracle.make_config(D=3, n=(20, 20, 20), periodic=(0, 0, 0)))
    with pytest.raises(ValueError):
        s3.add_ellipses([[10.0, 10.0, 10.0]], [5.0], [3.0], [0.0], [1.2])
