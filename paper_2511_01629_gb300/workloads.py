"""Seeded synthetic workloads shaped like the paper's test cases.

This module holds none of the method's arithmetic: it only draws geometry and
parameters.  Both the CUDA binding's callers and the FP64 oracle's tests
take their inputs from here, so the same seed gives the same problem to both.

The random stream is SplitMix64 (Steele, Lea & Flood 2014), written out here
so that every machine and numpy version draws the same numbers.

Workloads (lattice units, dx = dt = rho_f = 1; Sec. 3 sets alpha = 1/tau):
  * ``poiseuille_disk``  100x200 channel, walls in y, periodic x, tau = 0.8,
    drive g_x = 1e-6, one neutrally buoyant disk R = 8 at (50, 100 + U(-5,5));
  * ``single_disk``  400x1600 closed box, tau = 1, gravity 2e-6 in -y, one
    disk R = 12, density ratio 1.5, at (200 + U(-20,20), 0.8 ny) (Sec. 3.2);
  * ``many_disks``  1024x4096 closed box, tau = 1, gravity 2e-6, 500 disks
    R ~ U(6,12), ratio ~ U(1.1,2.0), rejection-sampled in the top half with a
    wall clearance of R + 2 and pair gaps above R_i + R_j + 2 delta (the
    shape of the 504-particle case of Sec. 3.5);
  * ``ensemble``  64 independent closed boxes nx ~ U{200..800}, ny = 4 nx,
    1..50 disks each drawn like ``many_disks``;
  * ``spheres3d``  D3Q19 256x256x512 closed box, 8 spheres R = 10, ratio 1.5,
    gravity 2e-6 in -z, seeded in the top half;
  * ``adjoint_disk`` the ``single_disk`` physics used for gradients;
  * ``disk_column``  96x240 closed box, gravity 4e-5, disks R = 6 stacked
    with gaps of 0.4 (inside the collision range delta = 1) and one disk
    within range of the wall x = -1/2, so that the pair and wall forces of
    Eq. 21 act from the first step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``uniform`` maps the top 53 bits to [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


@dataclass
class Workload:
    """One lattice instance: geometry, physics and particles."""
    name: str
    D: int
    n: tuple                      # (nx, ny, nz); nz = 1 in 2D
    periodic: tuple               # per axis: 1 periodic, 0 walls
    tau: float
    alpha: float
    g_drive: tuple = (0.0, 0.0, 0.0)
    g_grav: tuple = (0.0, 0.0, 0.0)
    delta: float = 1.0
    eps_p: float = 2.0
    eps_w: float = 1.0
    K: int = 1
    wall_u: Optional[list] = None  # [3][2][3] or None
    pos: List[List[float]] = field(default_factory=list)  # per particle, D coordinates
    radius: List[float] = field(default_factory=list)
    ratio: List[float] = field(default_factory=list)
    steps: int = 0
    # ellipses (2D): semi-minor axis and orientation per particle (radius is
    # the semi-major axis); None = disks
    minor: Optional[List[float]] = None
    theta: Optional[List[float]] = None

    @property
    def nodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def num_particles(self) -> int:
        return len(self.radius)


def _sample_disks(rng: SplitMix64, count: int, n: tuple, D: int, rlo: float, rhi: float,
                  qlo: float, qhi: float, delta: float, top_half_axis: int, max_tries: int = 200000):
    """Rejection sampling of non-overlapping particles in the top half."""
    pos, rad, rat = [], [], []
    tries = 0
    while len(rad) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampling did not place all particles")
        R = rng.uniform(rlo, rhi)
        q = rng.uniform(qlo, qhi)
        X = []
        for d in range(D):
            lo, hi = R + 2.0 - 0.5, n[d] - 0.5 - R - 2.0
            if d == top_half_axis:
                lo = max(lo, n[d] / 2.0)
            X.append(rng.uniform(lo, hi))
        ok = True
        for Xj, Rj in zip(pos, rad):
            d2 = sum((X[d] - Xj[d]) ** 2 for d in range(D))
            if d2 <= (R + Rj + 2.0 * delta) ** 2:
                ok = False
                break
        if ok:
            pos.append(X)
            rad.append(R)
            rat.append(q)
    return pos, rad, rat


def poiseuille_disk(seed: int = 0, nx: int = 100, ny: int = 200, steps: int = 2000) -> Workload:
    rng = SplitMix64(seed)
    y0 = ny / 2.0 + rng.uniform(-5.0, 5.0)
    return Workload("poiseuille_disk", 2, (nx, ny, 1), (1, 0, 1), tau=0.8, alpha=1.0 / 0.8,
                    g_drive=(1e-6, 0.0, 0.0), pos=[[nx / 2.0, y0]], radius=[8.0], ratio=[1.0],
                    steps=steps)


def single_disk(seed: int = 0, nx: int = 400, ny: int = 1600, steps: int = 20000,
                radius: float = 12.0, ratio: float = 1.5) -> Workload:
    rng = SplitMix64(seed)
    x0 = nx / 2.0 + rng.uniform(-20.0, 20.0) * nx / 400.0
    return Workload("single_disk", 2, (nx, ny, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                    g_grav=(0.0, -2e-6, 0.0), pos=[[x0, 0.8 * ny]], radius=[radius],
                    ratio=[ratio], steps=steps)


def many_disks(seed: int = 0, nx: int = 1024, ny: int = 4096, count: int = 500,
               steps: int = 50000) -> Workload:
    rng = SplitMix64(seed)
    pos, rad, rat = _sample_disks(rng, count, (nx, ny, 1), 2, 6.0, 12.0, 1.1, 2.0, 1.0, 1)
    return Workload("many_disks", 2, (nx, ny, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                    g_grav=(0.0, -2e-6, 0.0), pos=pos, radius=rad, ratio=rat, steps=steps)


def ensemble(seed: int = 0, count: int = 64, nx_lo: int = 200, nx_hi: int = 800,
             np_lo: int = 1, np_hi: int = 50, steps: int = 1000) -> List[Workload]:
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        nx = rng.randint(nx_lo, nx_hi)
        ny = 4 * nx
        npart = rng.randint(np_lo, np_hi)
        pos, rad, rat = _sample_disks(rng, npart, (nx, ny, 1), 2, 6.0, 12.0, 1.1, 2.0, 1.0, 1)
        out.append(Workload(f"ensemble[{i}]", 2, (nx, ny, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                            g_grav=(0.0, -2e-6, 0.0), pos=pos, radius=rad, ratio=rat,
                            steps=steps))
    return out


def spheres3d(seed: int = 0, nx: int = 256, ny: int = 256, nz: int = 512, count: int = 8,
              radius: float = 10.0, steps: int = 10000) -> Workload:
    rng = SplitMix64(seed)
    pos, rad, rat = _sample_disks(rng, count, (nx, ny, nz), 3, radius, radius, 1.5, 1.5, 1.0, 2)
    return Workload("spheres3d", 3, (nx, ny, nz), (0, 0, 0), tau=1.0, alpha=1.0,
                    g_grav=(0.0, 0.0, -2e-6), pos=pos, radius=rad, ratio=rat, steps=steps)


def disk_column(seed: int = 0, nx: int = 96, ny: int = 240, count: int = 6, radius: float = 6.0,
                gap: float = 0.4, K: int = 1) -> Workload:
    rng = SplitMix64(seed)
    pos, rad, rat = [], [], []
    for k in range(count):
        pos.append([nx / 2.0 + rng.uniform(-0.5, 0.5), 0.25 * ny + k * (2.0 * radius + gap)])
        rad.append(radius)
        rat.append(rng.uniform(1.2, 1.9))
    pos.append([-0.5 + radius + 0.3, 0.5 * ny])  # 0.3 inside the wall's range R + delta/2
    rad.append(radius)
    rat.append(1.5)
    return Workload("disk_column", 2, (nx, ny, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                    g_grav=(0.0, -4e-5, 0.0), K=K, pos=pos, radius=rad, ratio=rat, steps=150)


def adjoint_disk(seed: int = 0, nx: int = 400, ny: int = 1600, steps: int = 5000) -> Workload:
    w = single_disk(seed, nx, ny, steps)
    w.name = "adjoint_disk"
    return w


def couette_migration(H: int = 200, diameter: float = 50.0, length_d: float = 100.0,
                       U_w: float = 1.0 / 60.0, steps: int = 700000) -> Workload:
    """Lateral migration of a neutrally buoyant disk in plane Couette flow
    (Sec. 3.1): walls at y = -1/2 and H - 1/2 moving at -U_w/2 and +U_w/2,
    periodic in x over L = length_d * D, tau = 1, rho_s = rho_f, the disk
    released at x0 = 15 D and a distance D above the lower wall, the fluid at
    rest at t = 0.  The paper's run: H = 200 = 4 D, L = 100 D, U_w = 1/60,
    700,000 steps (shear time gamma t = 58)."""
    L = int(round(length_d * diameter))
    wall = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
    wall[1][0][0], wall[1][1][0] = -0.5 * U_w, 0.5 * U_w
    return Workload("couette_migration", 2, (L, H, 1), (1, 0, 1), tau=1.0, alpha=1.0,
                    wall_u=wall, pos=[[15.0 * diameter, -0.5 + diameter]],
                    radius=[0.5 * diameter], ratio=[1.0], steps=steps)


def dkt(L: int = 200, g: float = 0.05, offset: float = 0.1, steps: int = 12000) -> Workload:
    """Drafting, kissing and tumbling of two disks (Sec. 3.4) in lattice
    units: a closed channel L x 4L with L = 10 D, two disks of diameter
    D = L / 10 and density 1.01 rho_f on the centre line, 0.9 H and 0.85 H
    above the lower wall (7.2 and 6.8 of 8), tau = 1, eps_p = eps_w = 2,
    delta = 1.  Gravity 0.05 sets a settling velocity near 0.09 lattice units
    (Re = D U / nu ~ 11).  The upper disk starts `offset` lattice units off the
    centre line: two exactly centred disks keep the mirror symmetry and fall
    as one kissing pair without tumbling."""
    H = 4 * L
    xc = 0.5 * (L - 1)
    R = 0.05 * L
    return Workload("dkt", 2, (L, H, 1), (0, 0, 1), tau=1.0, alpha=1.0, g_grav=(0.0, -g, 0.0),
                    delta=1.0, eps_p=2.0, eps_w=2.0,
                    pos=[[xc + offset, -0.5 + 0.9 * H], [xc, -0.5 + 0.85 * H]], radius=[R, R],
                    ratio=[1.01, 1.01], steps=steps)


def ellipse_settling(L: int = 200, g: float = 2.178e-3, theta0: float = math.pi / 4,
                     steps: int = 30000) -> Workload:
    """A single ellipse settling in a vertical channel (Sec. 3.3) in lattice
    units: semi-axes a = L / 8 and b = a / 2, channel L x 10 L with walls on
    all sides, density 1.1 rho_f, tau = 1, eps_w = 1, delta = 1, released on
    the centre line at 0.8 H with its major axis at theta0 from the
    horizontal.  Gravity 980 cm/s^2 at dx = 0.002 cm and nu = 0.01 cm^2/s
    (dt = nu_lu dx^2 / nu = 6.67e-5 s) is 2.178e-3 lattice units."""
    H = 10 * L
    a = L / 8.0
    return Workload("ellipse_settling", 2, (L, H, 1), (0, 0, 1), tau=1.0, alpha=1.0,
                    g_grav=(0.0, -g, 0.0), delta=1.0, eps_p=1.0, eps_w=1.0,
                    pos=[[0.5 * (L - 1), -0.5 + 0.8 * H]], radius=[a], ratio=[1.1],
                    minor=[0.5 * a], theta=[theta0], steps=steps)


def random_small(seed: int, D: int = 2, n=(24, 20, 1), periodic=(1, 0, 1), nparticles: int = 3,
                 rlo: float = 2.5, rhi: float = 5.0, tau: float = 0.9, alpha: Optional[float] = None,
                 g_grav=(0.0, -1e-4, 0.0), g_drive=(0.0, 0.0, 0.0)) -> Workload:
    """Small instance with random non-overlapping particles anywhere in the box."""
    rng = SplitMix64(seed)
    pos, rad, rat = [], [], []
    tries = 0
    while len(rad) < nparticles and tries < 100000:
        tries += 1
        R = rng.uniform(rlo, rhi)
        X = [rng.uniform(R + 1.0, n[d] - 1.0 - R) if not periodic[d] else rng.uniform(0, n[d])
             for d in range(D)]
        ok = True
        for Xj, Rj in zip(pos, rad):
            d2 = 0.0
            for d in range(D):
                dd = X[d] - Xj[d]
                if periodic[d]:
                    dd -= n[d] * round(dd / n[d])
                d2 += dd * dd
            if d2 <= (R + Rj + 1.0) ** 2:
                ok = False
        if ok:
            pos.append(X)
            rad.append(R)
            rat.append(rng.uniform(1.1, 2.0))
    return Workload(f"random_small[{seed}]", D, tuple(n), tuple(periodic), tau=tau,
                    alpha=(1.0 / tau if alpha is None else alpha), g_grav=tuple(g_grav),
                    g_drive=tuple(g_drive), pos=pos, radius=rad, ratio=rat)


def random_populations(seed: int, Q: int, shape: tuple, scale: float = 1e-3):
    """Seeded uniform noise in [-scale, scale) of shape (Q,) + shape, as a flat list."""
    rng = SplitMix64(seed)
    total = Q * math.prod(shape)
    return [rng.uniform(-scale, scale) for _ in range(total)]
