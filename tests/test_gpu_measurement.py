"""The measurement entry point changes nothing but timing: lbm_step_timed
advances the state exactly like lbm_step, bit for bit."""
import numpy as np
import pytest

from paper_2511_01629_gb300 import lbm
from paper_2511_01629_gb300 import workloads as W

gpu = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    yield


def _state(sim):
    u, p, own = sim.fields()
    q = sim.particles()
    return u, p, own, q["X"], q["U"], q["W"], q["count"]


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@gpu
def test_step_timed_advances_like_step():
    w = W.many_disks(seed=1, nx=256, ny=512, count=40)
    a = lbm.from_workloads([w])
    b = lbm.from_workloads([w])
    a.set_graphs(0)
    a.step(24)
    fl, bx, pt = b.step_timed(24)
    a.sync()
    assert _same(_state(a), _state(b))
    assert fl > 0 and bx > 0 and pt > 0
    with pytest.raises(lbm.LBMError):
        b.step_timed(0)
    a.close()
    b.close()


@gpu
def test_async_particle_readback_matches_the_synchronous_one():
    """lbm_get_particles_async copies the state the enqueued steps leave,
    without waiting: after a sync the pinned arrays hold what
    lbm_get_particles returns (the [n][3] device layout, z = 0 in 2D)."""
    torch = pytest.importorskip("torch")
    w = W.many_disks(seed=1, nx=256, ny=512, count=40)
    sim = lbm.from_workloads([w])
    n = sim.num_particles(0)
    out = {k: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
           for k in ("X", "U", "W", "theta", "A")}
    out["count"] = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
    for _ in range(5):
        sim.step(3)
        sim.particles_async(out)
    sim.sync()
    ref = sim.particles()
    for k in ("X", "U", "A"):
        assert np.array_equal(out[k][:, :2], ref[k]), k
        assert np.all(out[k][:, 2] == 0.0), k
    assert np.array_equal(out["W"][:, 2], ref["W"][:, 0])
    assert np.array_equal(out["theta"][:, 2], ref["theta"][:, 0])
    assert np.array_equal(out["count"], ref["count"])
    sim.close()
