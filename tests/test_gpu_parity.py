"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: the fused kernel computes in FP32, the oracle in FP64.  One step
from a random state agrees to a few FP32 ulps of the population scale
(2e-6 relative).  Over many steps the error stays at the FP32 storage floor:
every step adds an increment of order g (1e-6) to populations of order u/3,
so its rounding leaves 1-4e-6 of U_ref = max |u_oracle| that does not grow
with the step count; in lattice units (c = 1) that is below 1e-8.  The long
runs assert 5e-6 of U_ref and 1e-6 of c.  The solid indicator and the
integer sums of the projection are compared bit for bit.
"""
import numpy as np
import pytest

from paper_2511_01629_gb300 import lbm
from paper_2511_01629_gb300 import workloads as W

from harness import compare_fields, compare_particles, make_pair, random_state

gpu = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    yield


CASES_2D = [
    # (n, periodic, nparticles)
    ((37, 23, 1), (1, 0, 1), 2),      # ragged, one tile wide
    ((130, 17, 1), (0, 0, 1), 3),     # two tiles with a 2-node tail
    ((64, 40, 1), (1, 1, 1), 3),      # fully periodic
    ((200, 33, 1), (0, 1, 1), 4),     # walls in x, periodic in y
    ((300, 20, 1), (1, 0, 1), 3),     # periodic x over three tiles, the last ragged: staged x-face wrap
]


# kernel shapes: (vec, tile rows, warps); vec = 0 is the TMA-staged pipeline
SHAPES = {0: (0, 4, 4), 1: (1, 4, 4), 2: (2, 4, 4), 4: (4, 4, 4)}


@gpu
@pytest.mark.parametrize("case", CASES_2D)
@pytest.mark.parametrize("vec", [0, 1, 2, 4])
def test_one_step_from_random_state_d2q9(case, vec):
    n, per, npart = case
    w = W.random_small(5 + vec, D=2, n=n, periodic=per, nparticles=npart, rlo=2.5, rhi=6.0,
                       tau=0.8, g_grav=(2e-5, -1e-4, 0), g_drive=(1e-5, 0, 0))
    f0 = random_state(vec, 9, (n[1], n[0]))
    sim, ref = make_pair(w, f0=f0, shape=SHAPES[vec])
    sim.step(1)
    ref.step(1)
    sim.sync()
    fg = sim.get_populations()
    fr = ref.get_f()
    scale = np.abs(fr[1:]).max()
    assert np.abs(fg[1:] - fr[1:]).max() < 2e-6 * scale
    cf = compare_fields(sim, ref)
    assert cf["owner_equal"], cf
    assert cf["du"] < 2e-6, cf
    assert cf["dp_f"] < 2e-6, cf
    cp = compare_particles(sim, ref)
    assert cp["count_equal"], cp
    assert cp["dU"] < 2e-6 * max(cp["Uscale"], 1e-12), cp
    assert cp["dX"] < 1e-9, cp


@gpu
@pytest.mark.parametrize("n,per", [((20, 18, 14), (1, 0, 1)), ((45, 12, 10), (0, 0, 0)),
                                   ((16, 16, 16), (1, 1, 1)),
                                   ((100, 12, 10), (1, 0, 0))])  # two x tiles: staged x-face wrap
@pytest.mark.parametrize("vec", [0, 1, 2, 4])
def test_one_step_from_random_state_d3q19(n, per, vec):
    w = W.random_small(11 + vec, D=3, n=n, periodic=per, nparticles=2, rlo=2.5, rhi=3.4, tau=0.9,
                       g_grav=(0, 2e-5, -1e-4))
    f0 = random_state(vec + 3, 19, (n[2], n[1], n[0]))
    sim, ref = make_pair(w, f0=f0, shape=SHAPES[vec])
    sim.step(1)
    ref.step(1)
    sim.sync()
    fg = sim.get_populations()
    fr = ref.get_f()
    scale = np.abs(fr[1:]).max()
    assert np.abs(fg[1:] - fr[1:]).max() < 2e-6 * scale
    cf = compare_fields(sim, ref)
    assert cf["owner_equal"], cf
    assert cf["du"] < 2e-6, cf
    assert cf["dp_f"] < 2e-6, cf
    cp = compare_particles(sim, ref)
    assert cp["count_equal"], cp
    assert cp["dU"] < 2e-6 * max(cp["Uscale"], 1e-12), cp


@gpu
def test_poiseuille_disk_2000_steps():
    """100x200 channel, tau 0.8, drive 1e-6, neutrally buoyant disk R = 8:
    velocity within 1e-6 of U_ref after 2000 steps (graph-replayed steps)."""
    w = W.poiseuille_disk(seed=0)
    sim, ref = make_pair(w, graphs=16)
    sim.step(w.steps)
    ref.step(w.steps)
    sim.sync()
    cf = compare_fields(sim, ref)
    cp = compare_particles(sim, ref)
    assert cf["owner_equal"], cf
    assert cf["du"] < 5e-6, cf
    assert cf["dp_f"] < 5e-6, cf
    assert cf["du"] * cf["uref"] < 1e-6, cf
    assert cp["dX"] < 1e-4, cp
    assert cp["dU"] < 1e-6 * cf["uref"], cp


@gpu
def test_moving_wall_couette():
    """Moving-wall bounce-back (walls at +-U_w/2) against the oracle."""
    wall = np.zeros((3, 2, 3))
    wall[1, 0, 0], wall[1, 1, 0] = -0.01, 0.01
    w = W.random_small(2, D=2, n=(50, 40, 1), periodic=(1, 0, 1), nparticles=1, rlo=5, rhi=6,
                       tau=1.0, g_grav=(0, 0, 0))
    w.wall_u = wall.tolist()
    w.ratio = [1.0]
    sim, ref = make_pair(w)
    sim.step(300)
    ref.step(300)
    sim.sync()
    cf = compare_fields(sim, ref)
    assert cf["owner_equal"] and cf["du"] < 5e-6, cf
    assert cf["dp_f"] < 5e-6, cf


@gpu
def test_spheres3d_full_size_2_steps():
    """The D3Q19 workload at full size (256x256x512, 8 spheres R = 10, graph
    replay, the autotuned shape the bench times) against the oracle."""
    import oracle
    from harness import oracle_config
    w = W.spheres3d(seed=0)
    sim = lbm.from_workloads([w])
    sim.autotune(2)
    sim.set_graphs(16)
    sim.step(2)
    sim.sync()
    ref = oracle.Sim(oracle_config(w))
    ref.add_particles(w.pos, w.radius, w.ratio)
    ref.step(2)
    cf = compare_fields(sim, ref)
    cp = compare_particles(sim, ref)
    sim.close()
    ref.close()
    assert cf["owner_equal"], cf
    assert cf["du"] < 2e-6, cf
    assert cf["dp_f"] < 2e-6, cf
    assert cp["count_equal"], cp
    assert cp["dU"] < 2e-6 * cp["Uscale"], cp


@gpu
def test_ensemble_full_size_2_steps():
    """The 64-instance batched ensemble in one launch per step (the bench's
    configuration): its smallest and largest instances against oracle runs of
    those instances alone."""
    import oracle
    from harness import oracle_config
    ws = W.ensemble(seed=0)
    sim = lbm.from_workloads(ws)
    sim.autotune(2)
    sim.set_graphs(16)
    sim.step(2)
    sim.sync()
    order = np.argsort([w.nodes for w in ws])
    for i in (int(order[0]), int(order[-1])):
        w = ws[i]
        ref = oracle.Sim(oracle_config(w))
        if w.num_particles:
            ref.add_particles(w.pos, w.radius, w.ratio)
        ref.step(2)
        cf = compare_fields(sim, ref, i)
        cp = compare_particles(sim, ref, i)
        ref.close()
        assert cf["owner_equal"], (i, cf)
        assert cf["du"] < 2e-6, (i, cf)
        assert cf["dp_f"] < 2e-6, (i, cf)
        assert cp["count_equal"], (i, cp)
        assert cp["dU"] < 2e-6 * max(cp["Uscale"], 1e-30), (i, cp)
    sim.close()


@gpu
@pytest.mark.parametrize("K", [1, 2])
def test_colliding_disks_match_oracle(K):
    """Disks in contact (pair forces of Eq. 21 from the first step) and a disk
    within wall range, with K = 1 and 2 sub-steps of Algorithm 1 (the grid
    barrier between sub-steps), against the oracle for 150 steps."""
    w = W.disk_column(seed=7, K=K)
    sim, ref = make_pair(w)
    sim.step(w.steps)
    ref.step(w.steps)
    sim.sync()
    cf = compare_fields(sim, ref)
    cp = compare_particles(sim, ref)
    assert cf["owner_equal"], cf
    assert cf["du"] < 5e-6, cf
    assert cf["dp_f"] < 5e-6, cf
    assert cp["count_equal"], cp
    assert cp["dU"] < 5e-6 * cp["Uscale"], cp
    assert cp["dX"] < 1e-6, cp


@pytest.fixture(scope="module")
def many_disks_oracle_20():
    """The oracle after 20 steps of the benched workload (computed once)."""
    w = W.many_disks(seed=0)
    _, ref = make_pair(w)
    ref.step(20)
    return w, ref


@gpu
@pytest.mark.parametrize("tuned", [False, True], ids=["default-shape", "autotuned"])
def test_many_disks_full_size_20_steps(tuned, many_disks_oracle_20):
    """The benched workload at full size (1024x4096, 500 disks, graph replay)
    against the oracle for 20 steps, in the default kernel shape (the launch
    configuration the bench times) and in the autotuner's pick."""
    w, ref = many_disks_oracle_20
    sim = lbm.from_workloads([w])
    sim.set_graphs(16)
    if tuned:
        sim.autotune(2)
    sim.step(20)
    sim.sync()
    cf = compare_fields(sim, ref)
    cp = compare_particles(sim, ref)
    sim.close()
    assert cf["owner_equal"], cf
    assert cf["du"] < 2e-6, cf
    assert cf["dp_f"] < 2e-6, cf
    assert cp["count_equal"], cp
    assert cp["dU"] < 2e-6 * cp["Uscale"], cp
    assert cp["dX"] < 1e-9, cp


@gpu
@pytest.mark.parametrize("storage", [lbm.LBM_FP32, lbm.LBM_FP16])
def test_tma_and_register_paths_agree(storage):
    """The TMA-staged kernel and the register-path kernel compute the same
    arithmetic: equal populations and particles after 30 steps."""
    w = W.random_small(31, D=2, n=(300, 70, 1), periodic=(0, 0, 1), nparticles=8, rlo=3, rhi=9,
                       tau=1.0, g_grav=(0, -1e-4, 0))
    out = []
    for shape in [(0, 4, 8), (4, 4, 4)]:
        sim = lbm.from_workloads([w], storage)
        sim.set_kernel_shape(*shape)
        sim.step(30)
        sim.sync()
        out.append((sim.get_populations(), sim.particles()))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    for k in ("X", "U", "W", "A", "count"):
        assert np.array_equal(out[0][1][k], out[1][1][k])


@gpu
def test_determinism_bitwise():
    w = W.random_small(9, D=2, n=(150, 90, 1), periodic=(0, 0, 1), nparticles=6, rlo=3, rhi=8,
                       tau=1.0, g_grav=(0, -1e-4, 0))
    outs = []
    for _ in range(2):
        sim = lbm.from_workloads([w])
        sim.step(40)
        sim.sync()
        outs.append((sim.get_populations(), sim.particles()))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in ("X", "U", "W", "A"):
        assert np.array_equal(outs[0][1][k], outs[1][1][k])


@gpu
def test_batched_instances_match_single():
    ws = [W.random_small(20 + i, D=2, n=(40 + 17 * i, 30 + 5 * i, 1), periodic=(0, 0, 1),
                         nparticles=1 + i, rlo=3, rhi=6, tau=1.0, g_grav=(0, -1e-4, 0))
          for i in range(4)]
    batch = lbm.from_workloads(ws)
    batch.step(30)
    batch.sync()
    for i, w in enumerate(ws):
        single = lbm.from_workloads([w])
        single.step(30)
        single.sync()
        assert np.array_equal(batch.get_populations(i), single.get_populations())
        for k in ("X", "U"):
            assert np.array_equal(batch.particles(i)[k], single.particles()[k])
        single.close()


@gpu
def test_save_load_roundtrip():
    w = W.random_small(4, D=2, n=(60, 50, 1), periodic=(1, 0, 1), nparticles=3, rlo=3, rhi=5,
                       tau=0.9, g_grav=(0, -1e-4, 0))
    sim = lbm.from_workloads([w])
    sim.step(10)
    blob = sim.save_state()
    sim.step(15)
    sim.sync()
    f_a, p_a = sim.get_populations(), sim.particles()
    sim.load_state(blob)
    sim.step(15)
    sim.sync()
    assert np.array_equal(sim.get_populations(), f_a)
    assert np.array_equal(sim.particles()["X"], p_a["X"])


@gpu
def test_invalid_arguments_are_rejected():
    with pytest.raises(lbm.LBMError):
        lbm.LBM(lbm.make_config(lbm.LBM_D2Q9, (10, 10, 1), tau=0.4))
    sim = lbm.LBM(lbm.make_config(lbm.LBM_D2Q9, (32, 32, 1), max_particles=2))
    with pytest.raises(lbm.LBMError):
        sim.add_particles(0, [[40.0, 5.0]], [3.0], [1.5])  # outside the box
    with pytest.raises(lbm.LBMError):
        sim.add_particles(0, [[10.0, 10.0]], [1.0], [1.5])  # radius < 2
    with pytest.raises(lbm.LBMError):
        sim.add_particles(0, [[10.0, 10.0]] * 3, [3.0] * 3, [1.5] * 3)  # capacity


@gpu
def test_divergence_is_reported():
    sim = lbm.LBM(lbm.make_config(lbm.LBM_D2Q9, (32, 32, 1)))
    f = np.zeros((9, 32, 32), np.float32)
    f[1] = 5.0  # |u| = 5 on every node
    sim.set_populations(f)
    sim.step(1)
    with pytest.raises(lbm.LBMError) as ei:
        sim.sync()
    assert ei.value.status == -4
