"""PyTorch autograd bridge to the library's discrete adjoint.

``ParticleTrajectory`` maps the penalty coefficient alpha (Eq. 17), the
density ratios, the initial particle positions and velocities of a batch of
instances to the particle positions and velocities after ``nsteps`` steps.
Its forward runs the library's checkpointed forward pass
(``lbm_adjoint_forward``) and its backward the hand-written adjoint
(``lbm_adjoint_backward``) seeded with the incoming gradients.  Nothing here
computes: the binding only marshals arrays.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import torch

from . import lbm


class ParticleTrajectory(torch.autograd.Function):
    """(alpha [B], ratio [B, P], X0 [B, P, D], U0 [B, P, D]) -> (X, U) [B, P, D].

    ``factory(alpha, ratio, X0, U0)`` receives numpy arrays of these shapes and
    returns an ``lbm.LBM`` of B instances with those parameters and particles
    (the solid domains follow from X0; their derivative is zero)."""

    @staticmethod
    def forward(ctx, alpha, ratio, X0, U0, factory: Callable, nsteps: int, seg_len: int = 0):
        np_ = lambda t: t.detach().cpu().numpy().astype(np.float64)
        sim = factory(np_(alpha), np_(ratio), np_(X0), np_(U0))
        sim.adjoint_forward(int(nsteps), int(seg_len))
        B = len(sim.configs)
        parts = [sim.particles(i) for i in range(B)]
        ctx.sim = sim
        ctx.meta = (alpha.dtype, alpha.device)
        X = torch.tensor(np.stack([p["X"] for p in parts]), dtype=alpha.dtype, device=alpha.device)
        U = torch.tensor(np.stack([p["U"] for p in parts]), dtype=alpha.dtype, device=alpha.device)
        return X, U

    @staticmethod
    def backward(ctx, gX, gU):
        sim = ctx.sim
        dtype, device = ctx.meta
        B = len(sim.configs)
        seeds = []
        for i in range(B):
            s = {}
            if gX is not None:
                s["X"] = gX[i].detach().cpu().numpy()
            if gU is not None:
                s["U"] = gU[i].detach().cpu().numpy()
            seeds.append(s)
        res = sim.adjoint_backward(seeds)
        sim.close()
        ctx.sim = None
        t = lambda a: torch.tensor(np.stack(a), dtype=dtype, device=device)
        return (t([r["alpha"] for r in res]), t([r["ratio"] for r in res]), t([r["X"] for r in res]),
                t([r["U"] for r in res]), None, None, None)


def trajectory(alpha, ratio, X0, U0, factory: Callable, nsteps: int, seg_len: int = 0):
    """Differentiable final particle positions and velocities (see ParticleTrajectory)."""
    return ParticleTrajectory.apply(alpha, ratio, X0, U0, factory, nsteps, seg_len)


def sedimentation_factory(n, radius, tau=1.0, g_grav=(0.0, -2e-6, 0.0), K=1, storage=lbm.LBM_FP32,
                          walls=(lbm.LBM_WALL, lbm.LBM_WALL, lbm.LBM_PERIODIC)):
    """Factory of closed-box D2Q9 (or D3Q19 when n[2] > 1) instances, fluid at
    rest, one particle set per instance (the adjoint workload's physics)."""
    lattice = lbm.LBM_D2Q9 if len(n) < 3 or n[2] <= 1 else lbm.LBM_D3Q19

    def make(alpha, ratio, X0, U0):
        B, P = ratio.shape
        cfgs = [lbm.make_config(lattice=lattice, n=n, bc=walls, storage=storage, tau=tau,
                                alpha=float(alpha[i]), g_grav=g_grav, K=K, max_particles=P,
                                max_radius=float(np.max(radius)) + 1.0) for i in range(B)]
        sim = lbm.LBM(cfgs)
        for i in range(B):
            sim.add_particles(i, X0[i], np.broadcast_to(radius, (P,)), ratio[i], vel=U0[i])
        return sim

    return make
