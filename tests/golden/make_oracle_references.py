"""Writes the stored oracle references of the long single-disk runs.

Runs only the FP64 oracle (its OpenMP build, bit-identical to the parity
build) on seeded workloads from paper_2511_01629_gb300.workloads; nothing
here touches the CUDA library.  The runs are too long to repeat inside the
GPU test suite (a 400 x 1600 oracle step takes ~30 ms on 8 cores):

  single_disk_seed0_trajectory.txt
      The single-disk sedimentation case (400 x 1600 closed box, disk R = 12,
      density ratio 1.5, gravity 2e-6, tau = 1, seed 0) for 20,000 steps:
      every 50 steps the step count, X, Y, U_x, U_y, omega and the node count
      of the disk (Sec. 3.2 reports the settling trajectory and velocity).

  adjoint_disk_seed0_fd.txt
      J = Y after n steps of the same case; for each parameter p in
      (density ratio, alpha, initial x, initial y) the two runs p +- h,
      h = 1e-4, stepped in lockstep: J(p + h) and J(p - h) every 50 steps and
      the first step at which the two runs' solid indicators (Eq. 9) differ.
      Up to that step (J(+h) - J(-h)) / 2h is the derivative of the
      recorded sequence of solid domains, which the discrete adjoint computes.

  couette_migration_h40.txt
      Lateral migration of a neutrally buoyant disk in plane Couette flow
      (Sec. 3.1) at a fifth of the paper's size with the same particle and
      channel Reynolds numbers: H = 40 = 4 D, L = 20 D, walls at -+U_w/2 with
      U_w = 1/12 (gamma D^2 / nu = 1.25, U_w H / nu = 20), the disk released
      a distance D above the lower wall, 28,000 steps (gamma t = 58.3, the
      paper's shear time): every 200 steps the step count, X, Y, U_x, U_y,
      omega and the node count.

  couette_migration_h40_long.txt
      The same reduced Couette case run to 200,000 steps (gamma t = 417), every
      2,000 steps: where the migration ends (the paper reports the disk at the
      centre line y/H = 0.5).

  dkt_l200.txt
      Drafting, kissing and tumbling of two disks (Sec. 3.4; workloads.dkt):
      200 x 800 closed channel, D = 20, ratio 1.01, 12,000 steps: every 100
      steps the step count and, per disk, X, Y, U_x, U_y, omega, count.

  ellipse_settling_l200.txt
      A single ellipse settling in a vertical channel (Sec. 3.3;
      workloads.ellipse_settling): 200 x 2000 closed channel, semi-axes 25
      and 12.5, ratio 1.1, released on the centre line at 45 degrees, 30,000
      steps: every 100 steps the step count, X, Y, U_x, U_y, omega, theta and
      the node count.

  python tests/golden/make_oracle_references.py [trajectory|fd|couette|couette_long|dkt|ellipse|all]
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_01629_gb300 import workloads as W  # noqa: E402

TRAJ = os.path.join(HERE, "single_disk_seed0_trajectory.txt")
COUETTE = os.path.join(HERE, "couette_migration_h40.txt")
COUETTE_LONG = os.path.join(HERE, "couette_migration_h40_long.txt")
DKT = os.path.join(HERE, "dkt_l200.txt")
ELLIPSE = os.path.join(HERE, "ellipse_settling_l200.txt")
FD = os.path.join(HERE, "adjoint_disk_seed0_fd.txt")
EVERY = 50


def _config(w, alpha=None):
    return oracle.make_config(D=w.D, n=w.n, periodic=w.periodic, wall_u=w.wall_u, tau=w.tau,
                              alpha=w.alpha if alpha is None else alpha, g_drive=w.g_drive,
                              g_grav=w.g_grav, delta=w.delta, eps_p=w.eps_p, eps_w=w.eps_w, K=w.K)


def trajectory(steps=20000):
    w = W.single_disk(0)
    s = oracle.Sim(_config(w), parallel=True)
    s.add_particles(w.pos, w.radius, w.ratio)
    rows = []
    for n in range(0, steps + 1, EVERY):
        if n:
            s.step(EVERY)
        p = s.particles()
        rows.append((n, *p["X"][0, :2], *p["U"][0, :2], p["W"][0, 2], p["count"][0]))
    with open(TRAJ, "w") as fh:
        fh.write("# single_disk seed 0: 400x1600 closed box, R = 12, ratio 1.5, gravity 2e-6, tau = 1,\n"
                 "# alpha = 1/tau; FP64 oracle (tests/golden/make_oracle_references.py).\n"
                 "# X, Y = centre after the step; U, omega = velocity of the step's projection (Eq. 22)\n"
                 f"# x0 = {w.pos[0][0]!r} y0 = {w.pos[0][1]!r}\n"
                 "# step X Y U_x U_y omega count\n")
        for r in rows:
            fh.write("%d %.17g %.17g %.17g %.17g %.17g %d\n" % r)


def _owner_digest(s):
    own = s.owner_map()
    return hashlib.sha1(np.ascontiguousarray(own).tobytes()).hexdigest()


def finite_differences(steps=5000, h=1e-4):
    w = W.adjoint_disk(0, steps=steps)
    params = {
        "ratio": lambda sg: dict(ratio=[w.ratio[0] + sg * h]),
        "alpha": lambda sg: dict(alpha=w.alpha + sg * h),
        "x0": lambda sg: dict(pos=[[w.pos[0][0] + sg * h, w.pos[0][1]]]),
        "y0": lambda sg: dict(pos=[[w.pos[0][0], w.pos[0][1] + sg * h]]),
    }
    out = []
    for name, mk in params.items():
        sims = []
        for sg in (+1, -1):
            kw = mk(sg)
            s = oracle.Sim(_config(w, kw.get("alpha")), parallel=True)
            s.add_particles(kw.get("pos", w.pos), w.radius, kw.get("ratio", w.ratio))
            sims.append(s)
        flip = None
        rows = []
        for n in range(1, steps + 1):
            # the indicator the step is about to use
            if flip is None and _owner_digest(sims[0]) != _owner_digest(sims[1]):
                flip = n  # step n is the first whose solid domains differ
            for s in sims:
                s.step(1)
            if n % EVERY == 0:
                rows.append((n, sims[0].particles()["X"][0, 1], sims[1].particles()["X"][0, 1]))
        out.append((name, flip if flip is not None else steps + 1, rows))
        for s in sims:
            s.close()
        print(name, "first step with differing solid domains:", flip, flush=True)
    with open(FD, "w") as fh:
        fh.write("# adjoint_disk seed 0: 400x1600 closed box, R = 12, ratio 1.5, gravity 2e-6, tau = 1,\n"
                 f"# alpha = 1/tau; J = Y after n steps; central differences with h = {h!r} of the FP64\n"
                 "# oracle (tests/golden/make_oracle_references.py).\n"
                 "# 'flip p k': the runs p +- h first use different solid domains in step k\n"
                 "# (k = steps + 1: never); rows 'p n J(+h) J(-h)'.\n")
        fh.write(f"h {h!r}\n")
        for name, flip, rows in out:
            fh.write(f"flip {name} {flip}\n")
        for name, flip, rows in out:
            for n, jp, jm in rows:
                fh.write("%s %d %.17g %.17g\n" % (name, n, jp, jm))


def couette_case():
    """The reduced Couette migration case of couette_migration_h40.txt."""
    return W.couette_migration(H=40, diameter=10.0, length_d=20.0, U_w=1.0 / 12.0, steps=28000)


def _particle_rows(w, every, header):
    s = oracle.Sim(_config(w), parallel=True)
    s.add_particles(w.pos, w.radius, w.ratio)
    rows = []
    for n in range(0, w.steps + 1, every):
        if n:
            s.step(every)
        p = s.particles()
        row = [n]
        for i in range(w.num_particles):
            row += [*p["X"][i, :2], *p["U"][i, :2], p["W"][i, 2], p["count"][i]]
        rows.append(row)
    s.close()
    return "".join(header) + "".join(
        " ".join(["%d" % r[0]] + ["%d" % v if (k % 6) == 5 else "%.17g" % v for k, v in enumerate(r[1:])])
        + "\n" for r in rows)


def couette():
    w = couette_case()
    text = _particle_rows(w, 200, [
        "# couette_migration H = 40, D = 10, L = 20 D, U_w = 1/12 (walls at -+U_w/2), tau = 1,\n",
        "# rho_s = rho_f, disk released at (15 D, D - 1/2); FP64 oracle\n",
        "# (tests/golden/make_oracle_references.py); fluid at rest at step 0.\n",
        "# step X Y U_x U_y omega count\n"])
    with open(COUETTE, "w") as fh:
        fh.write(text)


def couette_long():
    w = W.couette_migration(H=40, diameter=10.0, length_d=20.0, U_w=1.0 / 12.0, steps=200000)
    text = _particle_rows(w, 2000, [
        "# couette_migration H = 40, D = 10, L = 20 D, U_w = 1/12 (walls at -+U_w/2), tau = 1,\n",
        "# rho_s = rho_f, disk released at (15 D, D - 1/2), 200,000 steps (gamma t = 417); FP64\n",
        "# oracle (tests/golden/make_oracle_references.py); fluid at rest at step 0.\n",
        "# step X Y U_x U_y omega count\n"])
    with open(COUETTE_LONG, "w") as fh:
        fh.write(text)


def dkt():
    w = W.dkt()
    text = _particle_rows(w, 100, [
        "# dkt: 200 x 800 closed channel, two disks R = 10, ratio 1.01, gravity 0.05, tau = 1,\n",
        "# eps_p = eps_w = 2, delta = 1; disk 0 starts above disk 1 (workloads.dkt); FP64 oracle\n",
        "# (tests/golden/make_oracle_references.py).\n",
        "# step then per disk: X Y U_x U_y omega count\n"])
    with open(DKT, "w") as fh:
        fh.write(text)


def ellipse():
    w = W.ellipse_settling()
    s = oracle.Sim(_config(w), parallel=True)
    s.add_ellipses(w.pos, w.radius, w.minor, w.theta, w.ratio)
    rows = []
    for n in range(0, w.steps + 1, 100):
        if n:
            s.step(100)
        p = s.particles()
        rows.append((n, *p["X"][0, :2], *p["U"][0, :2], p["W"][0, 2], p["theta"][0, 2], p["count"][0]))
    s.close()
    with open(ELLIPSE, "w") as fh:
        fh.write("# ellipse_settling: 200 x 2000 closed channel, semi-axes a = 25, b = 12.5, ratio 1.1,\n"
                 "# gravity 2.178e-3, tau = 1, eps_w = 1, delta = 1, released at (99.5, 1599.5) with\n"
                 "# theta = pi/4; FP64 oracle (tests/golden/make_oracle_references.py).\n"
                 "# step X Y U_x U_y omega theta count\n")
        for r in rows:
            fh.write("%d %.17g %.17g %.17g %.17g %.17g %.17g %d\n" % r)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    oracle.build(parallel=True)
    if what in ("trajectory", "all"):
        trajectory()
    if what in ("fd", "all"):
        finite_differences()
    if what in ("couette", "all"):
        couette()
    if what in ("couette_long", "all"):
        couette_long()
    if what in ("dkt", "all"):
        dkt()
    if what in ("ellipse", "all"):
        ellipse()
