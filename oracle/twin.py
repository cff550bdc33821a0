"""FP64 differentiable twin of the oracle time step (PyTorch autograd, CPU).

TEST INFRASTRUCTURE ONLY.  Only the test suite may import this module.  It
restates the oracle's step (``lbm_oracle.c``) with PyTorch tensor operations
in FP64 so that reverse-mode automatic differentiation gives reference
gradients for the hand-written adjoint of the CUDA library.  It shares no code
with the CUDA path; it takes its lattice tables from the oracle.

Step order and readings are the oracle's (Sec. 2.2-2.4 of the paper):
  1. solid indicator from X^n (Eq. 9; lowest index wins, minimum image);
  2. pull streaming with halfway bounce-back (Eq. 10) and moving walls;
  3. acceleration: g_drive everywhere, (1 - rho_f/rho_s) g_grav + A_i on
     the nodes of particle i;
  4. u and p (Eq. 15);
  5. rigid-body projection U^n, w^n (Eq. 22, discrete M and I);
  6. BGK collision with Guo forcing (Eq. 14) and the penalty S (Eq. 17) on
     solid nodes;
  7. Algorithm 1 with the collision forces of Eqs. 19-21, A^{n+1},
     theta^{n+1} = theta^n + (w^n + w^{n-1}) / 2.

The indicator is piecewise constant in the positions: it is evaluated on
detached values (numpy, separate roundings like the oracle), so the gradients
are those of the step with the indicator held fixed, which is what the
discrete adjoint computes.  Everything else is differentiable: the initial
populations, the particle state, the density ratios and the penalty
coefficient alpha.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

CS2 = 1.0 / 3.0
F64 = torch.float64


class Twin:
    """Differentiable restatement of ``orc_step`` for one oracle configuration."""

    def __init__(self, cfg: "oracle.Config"):
        self.cfg = cfg
        self.D = cfg.D
        self.Q = 9 if self.D == 2 else 19
        self.n = [cfg.n[d] if d < self.D else 1 for d in range(3)]
        self.per = [bool(cfg.periodic[d]) if d < self.D else True for d in range(3)]
        self.N = self.n[0] * self.n[1] * self.n[2]
        c, w, opp = oracle.lattice(self.D)
        self.c_np = c.astype(np.int64)
        self.w_np = w
        self.opp = opp.astype(np.int64)
        self.c = torch.tensor(c, dtype=F64)
        self.w = torch.tensor(w, dtype=F64)
        self.tau = float(cfg.tau)
        self.rho_f = float(cfg.rho_f)
        self.g_drive = torch.tensor([cfg.g_drive[d] for d in range(3)], dtype=F64)
        self.g_grav = torch.tensor([cfg.g_grav[d] for d in range(3)], dtype=F64)
        self.gmag = float(np.sqrt(sum(cfg.g_grav[d] ** 2 for d in range(3))))
        self.delta, self.eps_p, self.eps_w = float(cfg.delta), float(cfg.eps_p), float(cfg.eps_w)
        self.K = max(int(cfg.K), 1)
        wall_u = np.array([cfg.wall_u[i] for i in range(18)]).reshape(3, 2, 3)
        # node coordinates, x fastest
        idx = np.arange(self.N)
        self.xyz = np.stack([idx % self.n[0], (idx // self.n[0]) % self.n[1],
                             idx // (self.n[0] * self.n[1])], axis=1)
        # streaming tables: source node of population q at each node, or a
        # bounce-back from the node's own opposite population plus the wall term
        self.src = np.zeros((self.Q, self.N), np.int64)
        self.bounce = np.zeros((self.Q, self.N), bool)
        wt = np.zeros((self.Q, self.N))
        for q in range(self.Q):
            s = self.xyz - self.c_np[q][None, :]
            uw = np.zeros((self.N, 3))
            wall = np.zeros(self.N, bool)
            for d in range(3):
                out = (s[:, d] < 0) | (s[:, d] >= self.n[d])
                if self.per[d]:
                    s[:, d] = np.mod(s[:, d], self.n[d])
                else:
                    wall |= out
                    uw += np.where((s[:, d] < 0)[:, None], wall_u[d, 0][None, :], 0.0)
                    uw += np.where((s[:, d] >= self.n[d])[:, None], wall_u[d, 1][None, :], 0.0)
            s = np.where(wall[:, None], self.xyz, s)
            self.src[q] = (s[:, 2] * self.n[1] + s[:, 1]) * self.n[0] + s[:, 0]
            self.bounce[q] = wall
            wt[q] = np.where(wall, 2.0 * w[q] * (uw @ self.c_np[q].astype(np.float64)) / CS2, 0.0)
        self.wt = torch.tensor(wt, dtype=F64)
        self.bounce_t = torch.tensor(self.bounce)
        self.src_t = torch.tensor(self.src)
        self.xyz_t = torch.tensor(self.xyz, dtype=F64)

    # ----------------------------------------------------------- indicator --
    def _disp_np(self, d, xnode, Xp):
        dx = xnode - Xp
        if self.per[d]:
            half = 0.5 * self.n[d]
            dx = np.where(dx > half, dx - self.n[d], np.where(dx < -half, dx + self.n[d], dx))
        return dx

    def owner(self, X: np.ndarray, R: np.ndarray) -> np.ndarray:
        """Eq. 9 on the lattice: lowest particle index whose |x - X|^2 <= R^2."""
        own = np.full(self.N, -1, np.int64)
        for p in range(len(R)):
            d2 = np.zeros(self.N)
            for d in range(self.D):
                dx = self._disp_np(d, self.xyz[:, d].astype(np.float64), X[p, d])
                d2 = d2 + dx * dx
            own = np.where((own < 0) & (d2 <= R[p] * R[p]), p, own)
        return own

    def _disp(self, d, xnode, Xp):
        dx = xnode - Xp
        if self.per[d]:
            half = 0.5 * self.n[d]
            dx = torch.where(dx > half, dx - self.n[d], torch.where(dx < -half, dx + self.n[d], dx))
        return dx

    # ---------------------------------------------------------- collisions --
    def collision_forces(self, X, R, ratio):
        """Eqs. 19-21 with C = (rho_s - rho_f)|g| of the receiving particle."""
        npart = X.shape[0]
        F = [torch.zeros(3, dtype=F64) for _ in range(npart)]
        for i in range(npart):
            Ci = (ratio[i] - 1.0) * self.rho_f * self.gmag
            for j in range(npart):
                if j == i:
                    continue
                dv = []
                for d in range(3):
                    if d >= self.D:
                        dv.append(torch.zeros((), dtype=F64))
                        continue
                    x = X[i, d] - X[j, d]
                    if self.per[d]:
                        half = 0.5 * self.n[d]
                        if float(x.detach()) > half:
                            x = x - self.n[d]
                        elif float(x.detach()) < -half:
                            x = x + self.n[d]
                    dv.append(x)
                dv = torch.stack(dv)
                dij = torch.sqrt((dv * dv).sum())
                rng = float(R[i]) + float(R[j]) + self.delta
                if float(dij.detach()) <= rng:
                    s = (rng - dij) / self.delta
                    F[i] = F[i] + Ci / self.eps_p * dv * s * s
            for d in range(self.D):
                if self.per[d]:
                    continue
                for wall in (-0.5, self.n[d] - 0.5):
                    Xim = 2.0 * wall - X[i, d]
                    diff = X[i, d] - Xim
                    dprime = torch.abs(diff)
                    rng = 2.0 * float(R[i]) + self.delta
                    if float(dprime.detach()) <= rng:
                        s = (rng - dprime) / self.delta
                        e = torch.zeros(3, dtype=F64)
                        e[d] = 1.0
                        F[i] = F[i] + e * (Ci / self.eps_w * diff * s * s)
        return torch.stack(F) if npart else torch.zeros((0, 3), dtype=F64)

    # ---------------------------------------------------------------- step --
    def step(self, f, X, U, W, theta, A, R, ratio, alpha):
        """One time step; returns (f*, X, U, W, theta, A, count, owner)."""
        Q, D, N = self.Q, self.D, self.N
        npart = X.shape[0]
        own = self.owner(X.detach().numpy(), np.asarray(R, np.float64))
        solid = torch.tensor(own >= 0)
        own_c = torch.tensor(np.maximum(own, 0))
        # 2. pull streaming
        fs = torch.stack([torch.where(self.bounce_t[q], f[self.opp[q]] + self.wt[q], f[q][self.src_t[q]])
                          for q in range(Q)])
        # 3. acceleration
        a = self.g_drive.expand(N, 3)
        if npart:
            ap = (1.0 - 1.0 / ratio)[:, None] * self.g_grav[None, :] + A
            a = a + torch.where(solid[:, None], ap[own_c], torch.zeros((), dtype=F64))
        # 4. macroscopic u, p (Eq. 15)
        m = fs.transpose(0, 1) @ self.c
        u = m + 0.5 * a
        w0 = float(self.w_np[0])
        uu = (u * u).sum(1)
        p = (fs[1:].sum(0) * CS2 - 0.5 * w0 * uu) / (1.0 - w0)
        # 5. rigid-body projection (Eq. 22)
        if npart:
            cnt = np.bincount(own[own >= 0], minlength=npart)
            count = torch.tensor(cnt, dtype=F64)
            sidx = torch.tensor(np.nonzero(own >= 0)[0])
            ps = own_c[sidx]
            us = u[sidx]
            r = torch.stack([self._disp(d, self.xyz_t[sidx, d], X[ps, d]) if d < D
                             else torch.zeros(len(sidx), dtype=F64) for d in range(3)], dim=1)
            Su = torch.zeros((npart, 3), dtype=F64).index_add(0, ps, us)
            Un = Su / count[:, None]
            Lr = torch.zeros((npart, 3), dtype=F64).index_add(0, ps, torch.cross(r, us, dim=1))
            if D == 2:
                Izz = torch.zeros(npart, dtype=F64).index_add(0, ps, (r * r).sum(1))
                Wn = torch.stack([torch.zeros(npart, dtype=F64), torch.zeros(npart, dtype=F64),
                                  Lr[:, 2] / Izz], dim=1)
            else:
                rr = (r * r).sum(1)
                Ii = rr[:, None, None] * torch.eye(3, dtype=F64)[None] - r[:, :, None] * r[:, None, :]
                I = torch.zeros((npart, 3, 3), dtype=F64).index_add(0, ps, Ii)
                Wn = torch.linalg.solve(I, Lr.unsqueeze(-1)).squeeze(-1)
        # 6. collision (Eqs. 10, 13, 14, 17)
        cu = u @ self.c.transpose(0, 1)                     # [N, Q]
        ca = a @ self.c.transpose(0, 1)
        feq = self.w[None, :] * (p[:, None] / CS2 + cu / CS2 + cu * cu / (2 * CS2 * CS2)
                                 - uu[:, None] / (2 * CS2))
        feq0 = -(1.0 - w0) * p / CS2 - w0 * uu / (2 * CS2)
        feq = torch.cat([feq0[:, None], feq[:, 1:]], dim=1).transpose(0, 1)  # [Q, N]
        ua = (u * a).sum(1)
        pref = 1.0 - 1.0 / (2.0 * self.tau)
        F = (pref * self.w[None, :] * ((ca - ua[:, None]) / CS2 + cu * ca / (CS2 * CS2))).transpose(0, 1)
        fneq = fs - feq
        Pi = torch.einsum("qn,qi,qj->nij", fneq, self.c, self.c)   # [N, 3, 3]
        ccI = self.c[:, :, None] * self.c[:, None, :] - CS2 * torch.eye(3, dtype=F64)[None]
        S = (self.w[:, None] / (2 * CS2 * CS2)) * alpha * torch.einsum("nij,qij->qn", Pi, ccI)
        S = torch.where(solid[None, :], S, torch.zeros((), dtype=F64))
        fnew = fs - fneq / self.tau + F + S
        if not npart:
            return fnew, X, U, W, theta, A, torch.zeros(0), own
        # 7. Algorithm 1
        Ubar = 0.5 * (Un + U)
        Xk = X
        h = 1.0 / self.K
        M = ratio * self.rho_f * count
        corr = torch.zeros_like(X)
        for _ in range(self.K):
            F1 = self.collision_forces(Xk, R, ratio)
            Xs = Xk + h * Ubar
            F2 = self.collision_forces(Xs, R, ratio)
            c = (1.0 / (2.0 * M))[:, None] * h * h * 0.5 * (F1 + F2)
            corr = corr + c
            Xk = Xs + c
        # A^{n+1} = 2 (X^{n+1} - X^n - Ubar), evaluated as the sum of the
        # corrections it equals (the difference of positions cancels)
        Anew = 2.0 * corr
        cols = []
        for d in range(3):
            x = Xk[:, d]
            if d < D and self.per[d]:
                x = torch.where(x >= self.n[d], x - self.n[d], torch.where(x < 0.0, x + self.n[d], x))
            cols.append(x)
        Xnew = torch.stack(cols, dim=1)
        theta_new = theta + 0.5 * (Wn + W)
        return fnew, Xnew, Un, Wn, theta_new, Anew, count, own

    def run(self, f0, X, U, W, theta, A, R, ratio, alpha, nsteps, keep_owners=False):
        """nsteps steps from post-collision populations f0 [Q, N] and particle
        state [np, 3]; returns the final state (and the owner map of every step)."""
        f = f0
        owners = []
        count = None
        for _ in range(nsteps):
            f, X, U, W, theta, A, count, own = self.step(f, X, U, W, theta, A, R, ratio, alpha)
            if keep_owners:
                owners.append(own)
        out = {"f": f, "X": X, "U": U, "W": W, "theta": theta, "A": A, "count": count}
        if keep_owners:
            out["owners"] = owners
        return out
