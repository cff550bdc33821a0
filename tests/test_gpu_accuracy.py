"""Error of the FP32 and FP16-storage paths against the FP64 oracle on cases
shaped like the sedimentation workloads (closed box, gravity 2e-6, tau = 1,
alpha = 1/tau): a single disk after 1000 steps, many disks after 100 steps,
and the terminal velocity of a settling disk.

Velocity errors are reported relative to U_ref = max |u_oracle| of the
compared step, and in lattice units (the lattice speed c = 1).  Bounds:
1e-6 of U_ref for FP32 and 1e-3 of U_ref for FP16 storage, and 0.5 % for the
terminal velocity.  The errors come from rounding: every step rounds
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


TERMINAL = dict(seed=5, nx=80, ny=320, radius=6.0, ratio=1.5)
T_STEPS, T_TAIL = 4000, 400


def _settling_series(step, read):
    step(T_STEPS - T_TAIL)
    v = []
    for _ in range(T_TAIL):
        step(1)
        v.append(read())
    return float(np.mean(v))


@pytest.fixture(scope="module")
def oracle_terminal():
    w = W.single_disk(**TERMINAL)
    _, ref = make_pair(w)
    return _settling_series(ref.step, lambda: ref.particles()["U"][0, 1])


@gpu
@pytest.mark.parametrize("storage", [lbm.LBM_FP32, lbm.LBM_FP16])
def test_terminal_velocity_of_settling_disk(storage, oracle_terminal):
    """Mean settling velocity over the last 10 % of 4000 steps (80 x 320 box,
    R = 6, ratio 1.5, gravity 2e-6) within 0.5 % of the oracle's."""
    w = W.single_disk(**TERMINAL)
    sim, _ = make_pair(w, storage=storage, graphs=16)
    Vg = _settling_series(sim.step, lambda: sim.particles()["U"][0, 1])
    sim.close()
    Vo = oracle_terminal
    print("terminal velocity", storage, Vg, Vo)
    assert Vo < 0.0
    assert abs(Vg - Vo) <= 0.005 * abs(Vo), (Vg, Vo)
