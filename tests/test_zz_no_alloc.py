"""The allocation-free projection entry point against the context path.

lbm_rigid_projection_noalloc serves callers that cannot allocate device
memory where they need the rigid-body projection (a host that owns all
device memory, a frame loop that must not stall on cudaMalloc's device
synchronisation).  Given the velocity field of the current state
(lbm_get_fields) and the current particles, it must return the U, omega and
node counts that the next lbm_step computes in its fused kernel, within the
parity tolerance of the other GPU tests (2e-6 of the velocity scale), and do
so twice in a row from the same shared scratch array.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2511_01629_gb300 import lbm
from paper_2511_01629_gb300 import workloads as W

gpu = pytest.mark.gpu


def _entry():
    fn = lbm.lib().lbm_rigid_projection_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p, C.c_int, C.c_void_p,
                   C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


@gpu
@pytest.mark.parametrize("D", [2, 3])
def test_noalloc_projection_matches_context_path(D):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    if D == 2:
        w = W.random_small(41, D=2, n=(160, 120, 1), periodic=(1, 0, 1), nparticles=7, rlo=3.0,
                           rhi=9.0, tau=0.9, g_grav=(0, -1e-4, 0))
    else:
        w = W.random_small(42, D=3, n=(40, 36, 32), periodic=(0, 0, 1), nparticles=4, rlo=2.5,
                           rhi=5.0, tau=0.9, g_grav=(0, 0, -1e-4))
    sim = lbm.from_workloads([w])
    sim.step(25)
    sim.sync()
    dev = torch.device("cuda")
    N = sim.nodes()
    u = torch.zeros(D * N, dtype=torch.float32, device=dev)
    sim.fields_device(0, u)
    part = sim.particles()
    n_p = len(part["X"])
    pos = torch.tensor(part["X"], dtype=torch.float64, device=dev).contiguous()
    rad = torch.tensor(w.radius, dtype=torch.float64, device=dev)
    n = (C.c_int * 3)(*w.n)
    per = (C.c_int * 3)(*w.periodic)
    stream = torch.cuda.current_stream().cuda_stream
    fn = _entry()
    outs = []
    for _ in range(2):  # two calls in a row share the scratch array
        vel = torch.full((n_p, D), np.nan, dtype=torch.float64, device=dev)
        om = torch.full((n_p, 1 if D == 2 else 3), np.nan, dtype=torch.float64, device=dev)
        cnt = torch.full((n_p,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        rc = fn(D, n, per, C.c_void_p(u.data_ptr()), n_p, C.c_void_p(pos.data_ptr()),
                C.c_void_p(rad.data_ptr()), float(max(w.radius)), C.c_void_p(vel.data_ptr()),
                C.c_void_p(om.data_ptr()), C.c_void_p(cnt.data_ptr()), C.c_void_p(stream))
        assert rc == 0, lbm.STATUS.get(rc, rc)
        outs.append((vel.cpu().numpy(), om.cpu().numpy(), cnt.cpu().numpy()))
    # the context path computes U^{n+1}, omega^{n+1} of this state in its next step
    sim.step(1)
    sim.sync()
    ref = sim.particles()
    scale = np.abs(ref["U"]).max()
    for vel, om, cnt in outs:
        assert np.array_equal(cnt, ref["count"])
        assert np.abs(vel - ref["U"]).max() < 2e-6 * scale
        assert np.abs(om - ref["W"]).max() < 2e-6 * max(np.abs(ref["W"]).max(), 1e-12) + 1e-12
    sim.close()


@gpu
def test_noalloc_rejects_too_many_particles():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    fn = _entry()
    n = (C.c_int * 3)(64, 64, 1)
    per = (C.c_int * 3)(0, 0, 1)
    rc = fn(2, n, per, None, 4097, None, None, 4.0, None, None, None, None)
    assert rc == -1
