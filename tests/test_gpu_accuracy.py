"""Error of the FP32 and FP16-storage paths against the FP64 oracle on cases
shaped like the sedimentation workloads (closed box, gravity 2e-6, tau = 1,
alpha = 1/tau): a single disk after 1000 steps, many disks after 100 steps,
and the terminal velocity of a settling disk.

Velocity errors are reported relative to U_ref = max |u_oracle| of the
compared step, and in lattice units (the lattice speed c = 1).  Bounds:
1e-6 of U_ref for FP32 and 1e-3 of U_ref for FP16 storage, and 0.5 % for the
terminal velocity of a disk in a confined channel that does reach it.  The errors come from rounding: every step rounds
populations of size ~U/3 (FP32: a random walk of ~1e-7 of U_ref per step;
FP16: the 11-bit significand of IEEE half).
"""
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


def _run(w, storage, steps):
    sim, ref = make_pair(w, storage=storage, graphs=16)
    sim.step(steps)
    sim.sync()
    return sim, ref


@pytest.fixture(scope="module")
def single_case():
    """One disk R = 8, ratio 1.5, in a 120 x 480 closed box, 1000 steps."""
    w = W.single_disk(seed=3, nx=120, ny=480, radius=8.0, ratio=1.5)
    sims = {s: _run(w, s, 1000) for s in (lbm.LBM_FP32, lbm.LBM_FP16)}
    ref = sims[lbm.LBM_FP32][1]
    ref.step(1000)
    out = {}
    for s, (sim, _) in sims.items():
        out[s] = (compare_fields(sim, ref), compare_particles(sim, ref))
        sim.close()
    return out


@pytest.fixture(scope="module")
def many_case():
    """30 disks R ~ U(6,12) in a 256 x 512 closed box, 100 steps."""
    w = W.many_disks(seed=1, nx=256, ny=512, count=30)
    sims = {s: _run(w, s, 100) for s in (lbm.LBM_FP32, lbm.LBM_FP16)}
    ref = sims[lbm.LBM_FP32][1]
    ref.step(100)
    out = {}
    for s, (sim, _) in sims.items():
        out[s] = (compare_fields(sim, ref), compare_particles(sim, ref))
        sim.close()
    return out


@gpu
def test_fp32_single_disk_1000_steps(single_case):
    cf, cp = single_case[lbm.LBM_FP32]
    print("fp32 single", cf, cp)
    assert cf["owner_equal"] and cp["count_equal"], (cf, cp)
    assert cf["du"] * cf["uref"] < 1e-6, cf   # in lattice units
    assert cf["du"] < 1e-6, cf                # relative to U_ref (measured 6.7e-7)
    assert cf["dp_f"] < 1e-6, cf
    assert cp["dU"] < 1e-6 * cp["Uscale"], cp


@gpu
def test_fp32_many_disks_100_steps(many_case):
    cf, cp = many_case[lbm.LBM_FP32]
    print("fp32 many", cf, cp)
    assert cf["owner_equal"] and cp["count_equal"], (cf, cp)
    assert cf["du"] < 1e-6, cf
    assert cf["dp_f"] < 1e-6, cf
    assert cp["dU"] < 1e-6 * cp["Uscale"], cp


@gpu
def test_fp16_storage_single_disk_1000_steps(single_case):
    cf, cp = single_case[lbm.LBM_FP16]
    print("fp16 single", cf, cp)
    assert cf["owner_equal"] and cp["count_equal"], (cf, cp)
    assert cf["du"] < 1e-3, cf                # measured 6.4e-4
    assert cf["dp_f"] < 1e-3, cf
    assert cf["du"] * cf["uref"] < 1e-6, cf


@gpu
def test_fp16_storage_many_disks_100_steps(many_case):
    cf, cp = many_case[lbm.LBM_FP16]
    print("fp16 many", cf, cp)
    assert cf["owner_equal"] and cp["count_equal"], (cf, cp)
    assert cf["du"] < 1e-3, cf
    assert cf["dp_f"] < 1e-3, cf


# A disk settling in a confined channel (48 x 480 closed box, R = 6, ratio 1.5,
# gravity 2e-5): the walls set the drag, the approach to terminal velocity
# takes a few W^2 / (pi^2 nu) ~ 1400 steps, and the disk crosses a lattice
# node every ~5000 steps, so means over 5000-step windows average the
# discrete indicator's stepping.  (In the 400 x 1600 box of the single-disk
# workload the approach takes ~W^2 / nu ~ 10^6 steps: not terminal at 20,000.)
TERMINAL = dict(seed=1, nx=48, ny=480, radius=6.0, ratio=1.5)
T_STEPS, T_EVERY, T_WIN = 20000, 100, 5000


def _terminal_workload():
    w = W.single_disk(**TERMINAL)
    w.g_grav = (0.0, -2e-5, 0.0)
    return w


def _settling_series(step, read):
    v = []
    for _ in range(T_STEPS // T_EVERY):
        step(T_EVERY)
        v.append(read())
    return np.array(v)


@pytest.fixture(scope="module")
def oracle_terminal():
    import oracle
    from harness import oracle_config
    w = _terminal_workload()
    ref = oracle.Sim(oracle_config(w), parallel=True)
    ref.add_particles(w.pos, w.radius, w.ratio)
    v = _settling_series(ref.step, lambda: ref.particles()["U"][0, 1])
    ref.close()
    return v


def _window_means(v):
    k = T_WIN // T_EVERY
    return v[-k:].mean(), v[-2 * k:-k].mean()


@gpu
@pytest.mark.parametrize("storage", [lbm.LBM_FP32, lbm.LBM_FP16])
def test_terminal_velocity_of_settling_disk(storage, oracle_terminal):
    """Terminal velocity, the mean settling velocity over the last 5000 of
    20,000 steps, within 0.5 % of the oracle's; the oracle's mean over the
    5000 steps before differs by less than 0.1 %, so the disk is terminal."""
    w = _terminal_workload()
    sim, _ = make_pair(w, storage=storage, graphs=16)
    vg = _settling_series(sim.step, lambda: sim.particles()["U"][0, 1])
    sim.close()
    Vo, Vo_prev = _window_means(oracle_terminal)
    Vg, _ = _window_means(vg)
    print("terminal velocity", storage, Vg, Vo, "oracle previous window", Vo_prev)
    assert Vo < 0.0
    assert abs(Vo - Vo_prev) < 1e-3 * abs(Vo), (Vo, Vo_prev)
    assert abs(Vg - Vo) <= 0.005 * abs(Vo), (Vg, Vo)
