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
