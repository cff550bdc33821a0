"""FP64 CPU oracle of the constraint-penalization LBM (arXiv 2511.01629).

TEST INFRASTRUCTURE ONLY.  This package wraps ``lbm_oracle.c``, a plain,
slow restatement of the paper written to check the CUDA library.  Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import it.  It imports nothing from the CUDA package and
the CUDA package never imports it.

Readings of the paper that the oracle takes (each is also commented at the
C function it affects):
  * D2Q9 weights by |c| (Eq. 11 index list contradicts Fig. 1);
  * Pi_neq = sum_a (f_a - feq_a) c_a c_a (the printed Eq. 16 drops c_a c_a);
  * S_a acts only on solid nodes (chi = 1), Sec. 2.2 "on the solid domain";
  * on solid nodes f/rho = (1 - rho_f/rho_s) g + A_i, on fluid nodes 0, plus
    an optional driving acceleration on every node (Eq. 5 and Sec. 2.4);
  * lattice mass M = rho_s * count and inertia rho_s * sum |r|^2 (Eq. 22);
  * walls are halfway bounce-back planes at -1/2 and n - 1/2 (paper silent);
  * theta advances by the trapezoid of omega (paper silent);
  * C = (rho_s - rho_f)|g| of the particle receiving the force (Eqs. 19-20).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblbm_oracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "liblbm_oracle_omp.so")


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of multiply-adds).

    parallel=False: the parity build, single-threaded.  parallel=True: the
    same source with -fopenmp, whose per-node loops run on all host cores
    (identical results; used for the timed CPU baseline and long runs)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    out = _LIB_OMP if parallel else _LIB
    src_m = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-2] + ".h"))
    if force or not os.path.exists(out) or os.path.getmtime(out) < src_m:
        tmp = out + f".tmp{os.getpid()}"
        omp = ["-fopenmp"] if parallel else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", *omp,
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class Config(C.Structure):
    _fields_ = [
        ("D", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3),
        ("wall_u", C.c_double * 18), ("tau", C.c_double), ("alpha", C.c_double),
        ("rho_f", C.c_double), ("g_drive", C.c_double * 3), ("g_grav", C.c_double * 3),
        ("delta", C.c_double), ("eps_p", C.c_double), ("eps_w", C.c_double), ("K", C.c_int),
    ]


_libs = {}
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib(parallel: bool = False):
    """The parity build (default) or the OpenMP build of the oracle."""
    if parallel not in _libs:
        L = C.CDLL(build(parallel=parallel))
        L.orc_lattice.argtypes = [C.c_int, _ip, _dp, _ip]
        L.orc_feq.argtypes = [C.c_int, _dp, C.c_double, _dp]
        L.orc_force.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp]
        L.orc_macro.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        L.orc_source.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp]
        L.orc_collision_forces.argtypes = [C.POINTER(Config), C.c_int, _dp, _dp, _dp, _dp]
        L.orc_create.argtypes = [C.POINTER(Config)]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_add_particles.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_void_p, C.c_void_p]
        L.orc_add_ellipses.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_void_p,
                                       C.c_void_p]
        L.orc_collision_forces_ellipse.argtypes = [C.POINTER(Config), C.c_int, _dp, _dp, _dp, _dp,
                                                   _dp, _dp]
        L.orc_set_f.argtypes = [C.c_void_p, _dp]
        L.orc_get_f.argtypes = [C.c_void_p, _dp]
        L.orc_set_static_solid.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_fields.argtypes = [C.c_void_p, _dp, _dp, _ip]
        L.orc_owner_map.argtypes = [C.c_void_p, _ip]
        L.orc_num_particles.argtypes = [C.c_void_p]
        L.orc_get_particles.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.orc_set_particles.argtypes = [C.c_void_p] + [C.c_void_p] * 5
        L.orc_rigid_projection.argtypes = [C.c_void_p, _dp, _dp, _dp, _lp]
        L.orc_steps_done.argtypes = [C.c_void_p]
        L.orc_steps_done.restype = C.c_long
        L.orc_threads.argtypes = []
        L.orc_threads.restype = C.c_int
        _libs[parallel] = L
    return _libs[parallel]


def threads(parallel: bool = False) -> int:
    """Threads the per-node loops of that build run on."""
    return lib(parallel).orc_threads()


def _v3(v):
    out = np.zeros(3)
    v = np.asarray(v, dtype=np.float64).ravel()
    out[: v.size] = v
    return out


def lattice(D: int):
    """(c [Q,3] int, w [Q], opp [Q]) of the oracle's own lattice tables."""
    Q = 9 if D == 2 else 19
    c = np.zeros(Q * 3, np.int32)
    w = np.zeros(Q)
    o = np.zeros(Q, np.int32)
    lib().orc_lattice(D, c, w, o)
    return c.reshape(Q, 3), w, o


def feq(D, u, p):
    out = np.zeros(9 if D == 2 else 19)
    lib().orc_feq(D, _v3(u), float(p), out)
    return out


def force(D, tau, u, a):
    out = np.zeros(9 if D == 2 else 19)
    lib().orc_force(D, float(tau), _v3(u), _v3(a), out)
    return out


def macro(D, f, a=(0, 0, 0)):
    u = np.zeros(3)
    p = np.zeros(1)
    lib().orc_macro(D, np.ascontiguousarray(f, np.float64), _v3(a), u, p)
    return u, float(p[0])


def source(D, alpha, f, fe):
    out = np.zeros(9 if D == 2 else 19)
    lib().orc_source(D, float(alpha), np.ascontiguousarray(f, np.float64),
                     np.ascontiguousarray(fe, np.float64), out)
    return out


def make_config(D=2, n=(16, 16, 1), periodic=(1, 1, 1), wall_u=None, tau=1.0, alpha=None,
                rho_f=1.0, g_drive=(0, 0, 0), g_grav=(0, 0, 0), delta=1.0, eps_p=2.0, eps_w=1.0,
                K=1) -> Config:
    cfg = Config()
    cfg.D = D
    nn = list(n) + [1] * (3 - len(n))
    for d in range(3):
        cfg.n[d] = int(nn[d]) if d < D else 1
        cfg.periodic[d] = int(periodic[d]) if d < len(periodic) else 1
    if wall_u is not None:
        wu = np.asarray(wall_u, np.float64).reshape(3, 2, 3).ravel()
        for i in range(18):
            cfg.wall_u[i] = wu[i]
    cfg.tau = tau
    cfg.alpha = (1.0 / tau) if alpha is None else alpha
    cfg.rho_f = rho_f
    for d in range(3):
        cfg.g_drive[d] = _v3(g_drive)[d]
        cfg.g_grav[d] = _v3(g_grav)[d]
    cfg.delta, cfg.eps_p, cfg.eps_w, cfg.K = delta, eps_p, eps_w, K
    return cfg


def collision_forces(cfg: Config, X, R, ratio):
    X3 = np.zeros((len(R), 3))
    X = np.asarray(X, np.float64).reshape(len(R), -1)
    X3[:, : X.shape[1]] = X
    F = np.zeros((len(R), 3))
    lib().orc_collision_forces(C.byref(cfg), len(R), np.ascontiguousarray(X3),
                               np.ascontiguousarray(R, np.float64),
                               np.ascontiguousarray(ratio, np.float64), F)
    return F


def collision_forces_ellipse(cfg: Config, X, a, b, theta, ratio):
    """Eqs. 19-21 for ellipses (2D): semi-axes a, b, orientation theta."""
    n = len(a)
    X3 = np.zeros((n, 3))
    X = np.asarray(X, np.float64).reshape(n, -1)
    X3[:, : X.shape[1]] = X
    F = np.zeros((n, 3))
    f64 = lambda v: np.ascontiguousarray(v, np.float64)
    lib().orc_collision_forces_ellipse(C.byref(cfg), n, np.ascontiguousarray(X3), f64(a), f64(b),
                                       f64(theta), f64(ratio), F)
    return F


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Sim:
    """One oracle simulation (owns the C state)."""

    def __init__(self, cfg: Config, parallel: bool = False):
        """parallel=True runs the per-node loops on all host cores (the OpenMP
        build of the same source: identical results)."""
        self._L = lib(parallel)
        self.parallel = parallel
        self.cfg = cfg
        self.D = cfg.D
        self.Q = 9 if cfg.D == 2 else 19
        self.n = tuple(cfg.n[d] for d in range(3))
        self.N = self.n[0] * self.n[1] * self.n[2]
        self._h = self._L.orc_create(C.byref(cfg))
        if not self._h:
            raise ValueError("oracle: bad config")

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        """(nz, ny, nx) for 3D, (ny, nx) for 2D: row-major node layout."""
        return (self.n[2], self.n[1], self.n[0]) if self.D == 3 else (self.n[1], self.n[0])

    def add_particles(self, pos, R, ratio, vel=None, omega=None):
        pos = np.ascontiguousarray(pos, np.float64).ravel()
        R = np.ascontiguousarray(R, np.float64).ravel()
        ratio = np.ascontiguousarray(ratio, np.float64).ravel()
        vel = None if vel is None else np.ascontiguousarray(vel, np.float64).ravel()
        omega = None if omega is None else np.ascontiguousarray(omega, np.float64).ravel()
        self._L.orc_add_particles(self._h, len(R), pos, R, ratio, _ptr(vel), _ptr(omega))
        self._keep = (vel, omega)

    def add_ellipses(self, pos, a, b, theta, ratio, vel=None, omega=None):
        """Ellipses (2D, Sec. 3.3): semi-axes a >= b > 0 and orientation theta
        (angle of the a axis from +x)."""
        f64 = lambda v: np.ascontiguousarray(v, np.float64).ravel()
        vel = None if vel is None else f64(vel)
        omega = None if omega is None else f64(omega)
        a = f64(a)
        rc = self._L.orc_add_ellipses(self._h, len(a), f64(pos), a, f64(b), f64(theta), f64(ratio),
                                      _ptr(vel), _ptr(omega))
        if rc != 0:
            raise ValueError("oracle: ellipses need D = 2 and 0 < b <= a")
        self._keep = (vel, omega)

    @property
    def np(self):
        return self._L.orc_num_particles(self._h)

    def set_f(self, f):
        self._L.orc_set_f(self._h, np.ascontiguousarray(f, np.float64).reshape(-1))

    def get_f(self):
        f = np.zeros(self.Q * self.N)
        self._L.orc_get_f(self._h, f)
        return f.reshape((self.Q,) + self.shape)

    def set_static_solid(self, mask):
        if mask is None:
            self._L.orc_set_static_solid(self._h, None)
        else:
            m = np.ascontiguousarray(mask, np.int32).reshape(-1)
            self._L.orc_set_static_solid(self._h, m.ctypes.data_as(C.c_void_p))

    def step(self, n=1):
        st = self._L.orc_step(self._h, int(n))
        if st != 0:
            raise RuntimeError(f"oracle step failed with status {st}")

    def fields(self):
        """(u [..., D], p [...], owner [...]) of the current state."""
        u = np.zeros(self.N * 3)
        p = np.zeros(self.N)
        o = np.zeros(self.N, np.int32)
        self._L.orc_fields(self._h, u, p, o)
        return (u.reshape(self.shape + (3,))[..., : self.D], p.reshape(self.shape),
                o.reshape(self.shape))

    def owner_map(self):
        o = np.zeros(self.N, np.int32)
        self._L.orc_owner_map(self._h, o)
        return o.reshape(self.shape)

    def particles(self):
        n = self.np
        out = {k: np.zeros((n, 3)) for k in ("X", "U", "W", "theta", "A")}
        cnt = np.zeros(n, np.int64)
        self._L.orc_get_particles(self._h, *(_ptr(out[k]) for k in ("X", "U", "W", "theta", "A")),
                                _ptr(cnt))
        out["count"] = cnt
        return out

    def set_particles(self, **kw):
        arrs = []
        for k in ("X", "U", "W", "theta", "A"):
            v = kw.get(k)
            arrs.append(None if v is None else np.ascontiguousarray(v, np.float64).reshape(-1, 3))
        self._keep2 = arrs
        self._L.orc_set_particles(self._h, *(_ptr(a) for a in arrs))

    def rigid_projection(self, u):
        """Eq. 22 over the current owner map for a velocity field u [..., D]."""
        n = self.np
        u3 = np.zeros(self.shape + (3,))
        u3[..., : self.D] = u
        U = np.zeros((n, 3))
        W = np.zeros((n, 3))
        cnt = np.zeros(n, np.int64)
        self._L.orc_rigid_projection(self._h, np.ascontiguousarray(u3).reshape(-1), U.reshape(-1),
                                   W.reshape(-1), cnt)
        return U, W, cnt

    @property
    def steps(self):
        return self._L.orc_steps_done(self._h)
