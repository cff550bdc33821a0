"""The OpenMP build of the oracle (all host cores, used for the timed CPU
baseline and the long full-size reference runs) gives the same bits as the
single-threaded parity build: every node's arithmetic is unchanged and the
sums over nodes stay serial."""
import numpy as np
import pytest

from paper_2511_01629_gb300 import workloads as W


def _cfg(oracle, w):
    return oracle.make_config(D=w.D, n=w.n, periodic=w.periodic, wall_u=w.wall_u, tau=w.tau,
                              alpha=w.alpha, g_drive=w.g_drive, g_grav=w.g_grav, delta=w.delta,
                              eps_p=w.eps_p, eps_w=w.eps_w, K=w.K)


@pytest.mark.parametrize("D", [2, 3])
def test_openmp_build_is_bit_identical(oracle, D):
    if D == 2:
        w = W.random_small(5, D=2, n=(130, 70, 1), periodic=(1, 0, 1), nparticles=5, rlo=3, rhi=8,
                           tau=0.8, g_grav=(2e-5, -1e-4, 0), g_drive=(1e-5, 0, 0))
    else:
        w = W.random_small(6, D=3, n=(30, 26, 22), periodic=(0, 1, 0), nparticles=3, rlo=2.5, rhi=4,
                           tau=0.9, g_grav=(0, 2e-5, -1e-4))
    outs = []
    for par in (False, True):
        s = oracle.Sim(_cfg(oracle, w), parallel=par)
        s.add_particles(w.pos, w.radius, w.ratio)
        s.step(30)
        outs.append((s.get_f(), s.particles(), s.fields()))
        s.close()
    (f0, p0, u0), (f1, p1, u1) = outs
    assert np.array_equal(f0, f1)
    for k in ("X", "U", "W", "theta", "A", "count"):
        assert np.array_equal(p0[k], p1[k]), k
    for a, b in zip(u0, u1):
        assert np.array_equal(a, b)
    assert oracle.threads(False) == 1
