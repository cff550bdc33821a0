"""The allocation-free projection entry point against the context path and the oracle.

lbm_rigid_projection_noalloc serves callers that cannot allocate device
memory where they need the rigid-body projection (a host that owns all
device memory, a frame loop that must not stall on cudaMalloc's device
synchronisation).  Given the velocity field of the current state
(lbm_get_fields) and the current particles, it must return the U, omega and
node counts that the next lbm_step computes in its fused kernel, within the
parity tolerance of the other GPU tests (2e-6 of the velocity scale), and do
so twice in a row from the same shared scratch array.  Its error codes are
checked too, each followed by a valid call that must still match: the
scratch array keeps the last call's contents, so every call has to clear
what it reads.
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


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lbm.build()
    return torch


def _workload(D):
    if D == 2:
        return W.random_small(41, D=2, n=(160, 120, 1), periodic=(1, 0, 1), nparticles=7, rlo=3.0,
                              rhi=9.0, tau=0.9, g_grav=(0, -1e-4, 0))
    return W.random_small(42, D=3, n=(40, 36, 32), periodic=(0, 0, 1), nparticles=4, rlo=2.5,
                          rhi=5.0, tau=0.9, g_grav=(0, 0, -1e-4))


class _Case:
    """A context after 25 steps: its velocity field and particles on the device,
    and the U, omega and counts its next step computes (the reference)."""

    def __init__(self, D):
        torch = _torch()
        self.torch, self.D = torch, D
        self.w = w = _workload(D)
        sim = lbm.from_workloads([w])
        sim.step(25)
        sim.sync()
        dev = torch.device("cuda")
        self.u = torch.zeros(D * sim.nodes(), dtype=torch.float32, device=dev)
        sim.fields_device(0, self.u)
        part = sim.particles()
        self.np = len(part["X"])
        self.pos = torch.tensor(part["X"], dtype=torch.float64, device=dev).contiguous()
        self.rad = torch.tensor(w.radius, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        sim.step(1)  # the context path projects this state in its next step
        sim.sync()
        self.ref = sim.particles()
        sim.close()

    def call(self, u=None, pos=None, rad=None, max_radius=None, n=None, periodic=None, np_=None):
        torch, D = self.torch, self.D
        u = self.u if u is None else u
        pos = self.pos if pos is None else pos
        rad = self.rad if rad is None else rad
        k = self.np if np_ is None else np_
        dev = u.device
        vel = torch.full((k, D), np.nan, dtype=torch.float64, device=dev)
        om = torch.full((k, 1 if D == 2 else 3), np.nan, dtype=torch.float64, device=dev)
        cnt = torch.full((k,), -1, dtype=torch.int32, device=dev)
        nn = (C.c_int * 3)(*(self.w.n if n is None else n))
        per = (C.c_int * 3)(*(self.w.periodic if periodic is None else periodic))
        mr = float(max(self.w.radius)) if max_radius is None else float(max_radius)
        torch.cuda.synchronize()
        rc = _entry()(D, nn, per, C.c_void_p(u.data_ptr()), k, C.c_void_p(pos.data_ptr()),
                      C.c_void_p(rad.data_ptr()), mr, C.c_void_p(vel.data_ptr()),
                      C.c_void_p(om.data_ptr()), C.c_void_p(cnt.data_ptr()),
                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        return rc, vel.cpu().numpy(), om.cpu().numpy(), cnt.cpu().numpy()

    def assert_matches(self, out):
        rc, vel, om, cnt = out
        assert rc == 0, lbm.STATUS.get(rc, rc)
        ref = self.ref
        scale = np.abs(ref["U"]).max()
        assert np.array_equal(cnt, ref["count"])
        assert np.abs(vel - ref["U"]).max() < 2e-6 * scale
        assert np.abs(om - ref["W"]).max() < 2e-6 * max(np.abs(ref["W"]).max(), 1e-12) + 1e-12


@pytest.fixture(scope="module")
def case2d():
    return _Case(2)


@gpu
@pytest.mark.parametrize("D", [2, 3])
def test_noalloc_projection_matches_context_path(D):
    case = _Case(D)
    for _ in range(2):  # two calls in a row share the scratch array
        case.assert_matches(case.call())


@gpu
@pytest.mark.parametrize("D", [2, 3])
def test_noalloc_projection_matches_oracle(D):
    """Eq. 22 against the FP64 oracle's projection of the same velocity field
    over the same particles: equal node counts, and U, omega within the
    fixed-point rounding of the exact sums (round(u 2^40) per node: at most
    count * 2^-41 in sum u, so 2^-41 = 4.5e-13 in U; the same order in omega)."""
    import oracle

    case = _Case(D)
    w = case.w
    ref = oracle.Sim(oracle.make_config(D=D, n=w.n, periodic=w.periodic, tau=w.tau, alpha=w.alpha,
                                        g_drive=w.g_drive, g_grav=w.g_grav))
    ref.add_particles(case.pos.cpu().numpy(), w.radius, w.ratio)
    u = np.moveaxis(case.u.cpu().numpy().astype(np.float64).reshape((D,) + ref.shape), 0, -1)
    U, Wr, cnt = ref.rigid_projection(u)
    ref.close()
    rc, vel, om, c = case.call()
    assert rc == 0, lbm.STATUS.get(rc, rc)
    assert np.array_equal(c, cnt)
    scale = np.abs(U[:, :D]).max()
    assert np.abs(vel - U[:, :D]).max() <= 1e-9 * scale + 1e-12
    Wref = Wr[:, 2:3] if D == 2 else Wr
    assert np.abs(om - Wref).max() <= 1e-9 * np.abs(Wref).max() + 1e-12


@gpu
def test_noalloc_rejects_too_many_particles():
    _torch()
    fn = _entry()
    n = (C.c_int * 3)(64, 64, 1)
    per = (C.c_int * 3)(0, 0, 1)
    rc = fn(2, n, per, None, 4097, None, None, 4.0, None, None, None, None)
    assert rc == -1


@gpu
def test_noalloc_reports_a_diverged_field(case2d):
    """A NaN or a speed >= 1/2 on a counted node is reported, not clamped."""
    c = case2d
    pos = c.pos.cpu().numpy()
    node = int(round(pos[0, 1])) * c.w.n[0] + int(round(pos[0, 0]))  # centre node of particle 0
    for bad in (float("nan"), 0.6):
        u = c.u.clone()
        u[node] = bad
        rc, vel, om, cnt = c.call(u=u)
        assert rc == -4, lbm.STATUS.get(rc, rc)
        assert np.array_equal(cnt, c.ref["count"])  # every output is still written
        c.assert_matches(c.call())


@gpu
def test_noalloc_rejects_a_radius_above_max(case2d):
    c = case2d
    rc, *_ = c.call(max_radius=float(min(c.w.radius)) - 0.5)
    assert rc == -1, lbm.STATUS.get(rc, rc)
    c.assert_matches(c.call())


@gpu
def test_noalloc_rejects_a_short_periodic_axis(case2d):
    """2 max_radius + 4 nodes must fit on a periodic axis (the box of a particle
    must not wrap onto itself): checked on the host before any launch."""
    c = case2d
    mr = float(max(c.w.radius))
    short = int(2 * mr) + 3
    rc, *_ = c.call(n=(short, c.w.n[1], 1), periodic=(1, 0, 1))
    assert rc == -1, lbm.STATUS.get(rc, rc)
    c.assert_matches(c.call())


@gpu
def test_noalloc_reports_list_capacity(case2d):
    """A particle overlapping more than 64 particles of lower index."""
    c = case2d
    torch = c.torch
    k = 70
    pos = torch.tensor([[40.3, 50.7]] * k, dtype=torch.float64, device="cuda").contiguous()
    rad = torch.full((k,), 4.0, dtype=torch.float64, device="cuda")
    rc, vel, om, cnt = c.call(pos=pos, rad=rad, max_radius=4.0, np_=k)
    assert rc == -7, lbm.STATUS.get(rc, rc)
    assert cnt[0] > 0 and np.all(cnt[1:64] == 0)  # lowest index owns the shared nodes
    c.assert_matches(c.call())


@gpu
def test_noalloc_reports_a_particle_without_nodes(case2d):
    """A radius below the node spacing can own no node: LBM_ERR_PARTICLE, with
    U = omega = 0 and count 0 for it; the other particles are still projected."""
    c = case2d
    torch = c.torch
    pos = c.pos.clone()
    rad = c.rad.clone()
    pos[0] = torch.tensor([40.5, 50.5], dtype=torch.float64)
    rad[0] = 0.3  # no node within 0.3 of (40.5, 50.5)
    rc, vel, om, cnt = c.call(pos=pos, rad=rad)
    assert rc == -8, lbm.STATUS.get(rc, rc)
    assert cnt[0] == 0 and np.all(vel[0] == 0) and np.all(om[0] == 0)
    assert np.array_equal(cnt[1:], c.ref["count"][1:])
    assert np.abs(vel[1:] - c.ref["U"][1:]).max() < 2e-6 * np.abs(c.ref["U"]).max()
    c.assert_matches(c.call())
