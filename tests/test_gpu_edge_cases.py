"""Edge cases of the GPU path against the FP64 oracle, through the C ABI:
the largest radii the library accepts (their velocity boxes and exact
integer sums at the bound of their range), nodes that lie exactly on a
particle's boundary circle (the exact test decides them as the oracle does),
the smallest radius, and a batch in which one instance has no particles."""
import numpy as np
import pytest

from paper_2511_01629_gb300 import lbm
from paper_2511_01629_gb300 import workloads as W

from harness import compare_fields, compare_particles, make_pair

gpu = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    yield


def _check_pair(w, steps, tol=5e-6, parallel=False):
    sim, ref = make_pair(w, graphs=0, parallel=parallel)
    assert np.array_equal(sim.fields()[2], ref.owner_map())
    last = 0
    for n in steps:
        sim.step(n - last)
        ref.step(n - last)
        last = n
        sim.sync()
        cf = compare_fields(sim, ref)
        cp = compare_particles(sim, ref)
        print(w.name, n, cf, cp)
        assert cf["owner_equal"], cf
        assert cp["count_equal"], cp
        assert cf["du"] <= tol and cf["dp_f"] <= tol, cf
        assert cp["dU"] <= tol * cp["Uscale"] + 1e-15, cp
    sim.close()
    return ref


@gpu
def test_largest_disk_2d():
    """R = 120, the 2D maximum: a velocity box of 245 x 245 entries."""
    w = W.Workload("edge[R=120]", 2, (300, 300, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                   g_grav=(0.0, -1e-5, 0.0), pos=[[149.3, 150.7]], radius=[120.0], ratio=[1.2])
    ref = _check_pair(w, (1, 10))
    assert abs(ref.particles()["count"][0] - np.pi * 120 ** 2) < 2 * np.pi * 120


@gpu
def test_largest_sphere_3d():
    """R = 40, the 3D maximum (the exact sums of Eq. 22 stay inside int64)."""
    w = W.Workload("edge[R=40]", 3, (96, 96, 96), (0, 0, 0), tau=1.0, alpha=1.0,
                   g_grav=(0.0, 0.0, -1e-5), pos=[[47.6, 48.2, 48.7]], radius=[40.0], ratio=[1.3])
    ref = _check_pair(w, (1, 3), parallel=True)
    assert abs(ref.particles()["count"][0] - 4 / 3 * np.pi * 40 ** 3) < 4 * np.pi * 40 ** 2


@gpu
@pytest.mark.parametrize("periodic", [(0, 0, 1), (1, 1, 1)], ids=["walls", "periodic"])
def test_nodes_exactly_on_the_boundary(periodic):
    """Centres on nodes and integer radii: nodes with dx^2 + dy^2 == R^2
    exactly (e.g. (3, 4) from a centre with R = 5) are inside (<=), in both
    implementations; one disk sits across the periodic seam when there is one."""
    pos = [[30.0, 24.0], [12.0, 40.0], [57.0, 3.0] if periodic[0] else [47.0, 41.0]]
    w = W.Workload("edge[on-circle]", 2, (60, 50, 1), periodic, tau=0.9, alpha=1.0 / 0.9,
                   g_grav=(0.0, -1e-4, 0.0), pos=pos, radius=[5.0, 10.0, 5.0], ratio=[1.5, 1.2, 1.4])
    sim, ref = make_pair(w, graphs=0)
    own = sim.fields()[2]
    assert np.array_equal(own, ref.owner_map())
    # the lattice points on the first circle belong to the disk (owner map:
    # particle index, -1 for fluid)
    for dx, dy in ((5, 0), (0, 5), (3, 4), (-4, 3), (-3, -4), (4, -3)):
        assert own[24 + dy, 30 + dx] == 0
    assert own[24, 36] == -1 and own[30, 30] == -1
    assert (own == 0).sum() == 81  # pi 25 = 78.5 plus the lattice points on the circle
    sim.close()
    _check_pair(w, (1, 30))


@gpu
def test_smallest_radius():
    """R = 2, the smallest radius the library accepts."""
    w = W.Workload("edge[R=2]", 2, (40, 40, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                   g_grav=(0.0, -1e-4, 0.0), pos=[[20.3, 25.6], [11.0, 12.0]], radius=[2.0, 2.0],
                   ratio=[2.0, 1.5])
    _check_pair(w, (1, 40))


@gpu
def test_batch_with_an_instance_without_particles():
    """Three instances in one context, the middle one without particles:
    each equals its own single-instance context bit for bit."""
    ws = [W.random_small(s, D=2, n=(70 + 9 * s, 40 + 5 * s, 1), periodic=(1, 0, 1), nparticles=3,
                         rlo=3.0, rhi=6.0, tau=0.9) for s in (1, 2, 3)]
    ws[1].pos, ws[1].radius, ws[1].ratio = [], [], []
    batch = lbm.from_workloads(ws)
    batch.step(25)
    batch.sync()
    for i, w in enumerate(ws):
        one = lbm.from_workloads([w])
        one.step(25)
        one.sync()
        assert all(np.array_equal(a, b) for a, b in zip(batch.fields(i), one.fields(0)))
        if w.num_particles:
            pa, pb = batch.particles(i), one.particles(0)
            for k in ("X", "U", "W", "count"):
                assert np.array_equal(pa[k], pb[k]), (i, k)
        else:
            assert batch.num_particles(i) == 0
        one.close()
    batch.close()
