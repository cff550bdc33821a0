"""Pins of the FP64 autograd twin of the oracle (oracle/twin.py).

The twin is the reference for the GPU adjoint, so it is pinned to two things
outside itself: its forward step reproduces the C oracle (independent code,
the oracle being pinned to the paper by test_oracle_pins.py) to round-off,
and its reverse-mode gradients equal central finite differences of the C
oracle on cases whose solid indicator does not change between the +h and -h
runs (the indicator is piecewise constant, Eq. 9).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle.twin import Twin  # noqa: E402

F64 = torch.float64


def _setup(D, n, per, pos, R, ratio, K, wall_u=None, alpha=None, g=None, seed=0, tau=0.9):
    g = g if g is not None else ((0, -1e-4, 0) if D == 2 else (0, 0, -1e-4))
    cfg = oracle.make_config(D=D, n=n, periodic=per, wall_u=wall_u, tau=tau, alpha=alpha, g_grav=g,
                             g_drive=(1e-5, 0, 0), K=K)
    Q = 9 if D == 2 else 19
    N = int(np.prod(n))
    rng = np.random.default_rng(seed)
    f0 = rng.uniform(-1e-3, 1e-3, (Q, N))
    f0[0] = 0
    U0 = np.zeros((len(R), 3))
    U0[:, :D] = rng.uniform(-1e-3, 1e-3, (len(R), D))
    return cfg, f0, np.asarray(pos, np.float64), np.asarray(R, np.float64), np.asarray(ratio, np.float64), U0


def _oracle_run(cfg, f0, pos, R, ratio, U0, steps, keep_owners=False):
    s = oracle.Sim(cfg)
    s.set_f(f0)
    s.add_particles(pos, R, ratio, vel=U0[:, : cfg.D])
    owners = []
    for _ in range(steps):
        if keep_owners:
            owners.append(s.owner_map().copy())
        s.step(1)
    return s, owners


def _twin_run(cfg, f0, pos, R, ratio, U0, steps, alpha=None, grad=False):
    npart, D = len(R), cfg.D
    X = torch.zeros(npart, 3, dtype=F64)
    X[:, :D] = torch.tensor(pos, dtype=F64)
    args = dict(f=torch.tensor(f0), X=X, U=torch.tensor(U0), ratio=torch.tensor(ratio),
                alpha=torch.tensor(cfg.alpha if alpha is None else alpha, dtype=F64))
    if grad:
        for v in args.values():
            v.requires_grad_(True)
    Z = torch.zeros(npart, 3, dtype=F64)
    out = Twin(cfg).run(args["f"], args["X"], args["U"], Z, Z, Z, R, args["ratio"], args["alpha"], steps)
    return out, args


CASES = [
    # D, n, periodic, positions, radii, ratios, K, moving walls
    (2, (30, 24, 1), (1, 0, 1), [[8.2, 10.1], [19.7, 12.3], [14.0, 19.5]], [4.1, 3.6, 3.0],
     [1.5, 1.8, 1.2], 2, False),
    (2, (26, 20, 1), (1, 0, 1), [[8.2, 10.1], [14.1, 9.9]], [3.1, 2.6], [1.5, 1.8], 1, True),
    (2, (22, 20, 1), (0, 0, 1), [[4.3, 10.2], [16.8, 3.9]], [3.2, 2.9], [1.6, 1.3], 1, False),
    (3, (14, 12, 10), (0, 1, 0), [[5.2, 5.1, 4.8], [9.0, 6.9, 5.3]], [2.6, 2.4], [1.5, 1.3], 2, False),
]


@pytest.mark.parametrize("case", CASES, ids=["2d-3p-K2", "2d-moving-wall", "2d-walls", "3d-K2"])
def test_twin_forward_equals_oracle(case):
    D, n, per, pos, R, ratio, K, moving = case
    wu = None
    if moving:
        wu = np.zeros((3, 2, 3))
        wu[1, 0, 0], wu[1, 1, 0] = -0.01, 0.02
    cfg, f0, pos, R, ratio, U0 = _setup(D, n, per, pos, R, ratio, K, wall_u=wu)
    steps = 10
    ref, _ = _oracle_run(cfg, f0, pos, R, ratio, U0, steps)
    with torch.no_grad():
        out, _ = _twin_run(cfg, f0, pos, R, ratio, U0, steps)
    pr = ref.particles()
    Q = 9 if D == 2 else 19
    assert np.abs(out["f"].numpy() - ref.get_f().reshape(Q, -1)).max() < 1e-15
    for k in ("X", "U", "W", "theta", "A"):
        scale = max(np.abs(pr[k]).max(), 1e-300)
        assert np.abs(out[k].numpy() - pr[k]).max() <= 1e-12 * scale + 1e-17, k
    assert np.array_equal(out["count"].numpy().astype(np.int64), pr["count"])


def test_twin_gradient_equals_oracle_central_differences():
    """dJ/d(alpha, ratio, X0, U0, f0 along a direction) for J = seeds . final
    state, autograd of the twin against (J(+h) - J(-h)) / 2h of the C oracle."""
    D, n, per = 2, (26, 20, 1), (1, 0, 1)
    cfg, f0, pos, R, ratio, U0 = _setup(D, n, per, [[8.2, 10.1], [14.1, 9.9]], [3.1, 2.6], [1.5, 1.8],
                                        K=2, alpha=0.8, tau=1.0, seed=1)
    steps, h, Q = 12, 1e-4, 9
    rng = np.random.default_rng(7)
    sX = rng.normal(size=(2, 3))
    sU = rng.normal(size=(2, 3))
    sX[:, 2] = sU[:, 2] = 0
    sf = rng.normal(size=f0.shape) * 1e-2
    sf[0] = 0
    dirf = rng.normal(size=f0.shape) * 1e-3
    dirf[0] = 0

    def J_oracle(alpha=0.8, ratio_=ratio, pos_=pos, U_=U0, f_=f0):
        c = oracle.make_config(D=D, n=n, periodic=per, tau=1.0, alpha=alpha, g_grav=(0, -1e-4, 0),
                               g_drive=(1e-5, 0, 0), K=2)
        s, owners = _oracle_run(c, f_, pos_, R, ratio_, U_, steps, keep_owners=True)
        pr = s.particles()
        return (sX * pr["X"]).sum() + (sU * pr["U"]).sum() + (sf * s.get_f().reshape(Q, -1)).sum(), owners

    def central(plus, minus):
        Jp, op = J_oracle(**plus)
        Jm, om = J_oracle(**minus)
        assert all(np.array_equal(a, b) for a, b in zip(op, om)), "indicator changed between +h and -h"
        return (Jp - Jm) / (2 * h)

    out, args = _twin_run(cfg, f0, pos, R, ratio, U0, steps, grad=True)
    J = (torch.tensor(sX) * out["X"]).sum() + (torch.tensor(sU) * out["U"]).sum() + \
        (torch.tensor(sf) * out["f"]).sum()
    J.backward()

    def close(ad, fd):
        assert abs(ad - fd) <= 2e-6 * abs(fd) + 1e-12, (ad, fd)

    close(args["alpha"].grad.item(), central(dict(alpha=0.8 + h), dict(alpha=0.8 - h)))
    for i in range(2):
        rp, rm = ratio.copy(), ratio.copy()
        rp[i] += h
        rm[i] -= h
        close(args["ratio"].grad[i].item(), central(dict(ratio_=rp), dict(ratio_=rm)))
        for d in range(D):
            xp, xm = pos.copy(), pos.copy()
            xp[i, d] += h
            xm[i, d] -= h
            close(args["X"].grad[i, d].item(), central(dict(pos_=xp), dict(pos_=xm)))
            up, um = U0.copy(), U0.copy()
            up[i, d] += h
            um[i, d] -= h
            close(args["U"].grad[i, d].item(), central(dict(U_=up), dict(U_=um)))
    close(float((args["f"].grad.numpy() * dirf).sum()), central(dict(f_=f0 + h * dirf), dict(f_=f0 - h * dirf)))
