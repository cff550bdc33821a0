"""Device-side failures surface as status codes, without a GPU fault.

A bounded wait that runs out must be reported by lbm_sync as LBM_ERR_TIMEOUT,
after which the context refuses work with LBM_ERR_STATE while the device
stays usable.  The particle kernel's grid barrier (between the sub-steps of
Algorithm 1, so K = 2) is made to run out by a zero wait bound
(lbm_set_particle_wait_limit): the first block to arrive at the barrier
never finds it open on its first look.  The waits stay bounded
throughout and that kernel issues no asynchronous copies, so nothing is left
in flight when it returns.
"""
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


def _workload():
    # 64 disks: eight particle blocks, so the barrier between the two
    # sub-steps spans several blocks
    w = W.many_disks(seed=2, nx=384, ny=768, count=64)
    w.K = 2
    return w


@gpu
@pytest.mark.parametrize("graphs", [0, 16])
def test_particle_barrier_timeout_is_reported(graphs):
    w = _workload()
    sim = lbm.from_workloads([w])
    sim.set_graphs(graphs)
    sim.step(16)
    sim.sync()  # the default bound: no timeout
    x_before = sim.particles()["X"].copy()
    sim.set_particle_wait_limit(0.0)
    sim.step(16 if graphs else 1)
    with pytest.raises(lbm.LBMError) as ei:
        sim.sync()
    assert ei.value.status == -5, ei.value
    with pytest.raises(lbm.LBMError) as ei:
        sim.step(1)
    assert ei.value.status == -6, ei.value
    sim.close()
    # the device is still usable: a new context on the same workload steps normally
    again = lbm.from_workloads([w])
    again.set_graphs(graphs)
    again.step(16)
    again.sync()
    assert np.array_equal(again.particles()["X"], x_before)
    again.close()


@gpu
def test_wait_limit_is_validated():
    sim = lbm.from_workloads([_workload()])
    for bad in (-1.0, float("nan"), 61.0):
        with pytest.raises(lbm.LBMError) as ei:
            sim.set_particle_wait_limit(bad)
        assert ei.value.status == -1
    sim.set_particle_wait_limit(2.0)
    sim.step(2)
    sim.sync()
    sim.close()
