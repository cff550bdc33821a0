"""Thin ctypes binding of the lbmpen C ABI (``include/lbmpen.h``).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/liblbmpen.so``.  PyTorch provides the CUDA stream and, through its
caching allocator, the device memory the library allocates.  There is no CPU
fallback: importing the binding on a machine without the compiled library
raises, and creating a context without a GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "liblbmpen.so")
_SOURCES = ["lbm_fluid.cu", "lbm_fluid_tma.cu", "lbm_particles.cu", "lbm_api.cu", "lbm_noalloc.cu",
            "lbm_adjoint.cu"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC"]

LBM_D2Q9, LBM_D3Q19 = 9, 19
LBM_FP32, LBM_FP16 = 0, 1
LBM_PERIODIC, LBM_WALL = 0, 1

STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
          -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE",
          -7: "LBM_ERR_CAPACITY", -8: "LBM_ERR_PARTICLE"}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (in parallel) and link the library."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [os.path.join(_SRC, f) for f in os.listdir(_SRC)]
    deps.append(os.path.join(os.path.dirname(_HERE), "include", "lbmpen.h"))
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        subprocess.check_call([nvcc, *NVCC_FLAGS, "-c", os.path.join(_SRC, src), "-o", obj])
        return obj

    with ThreadPoolExecutor(len(_SOURCES)) as ex:
        objs = list(ex.map(compile_one, _SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs,
                           "-o", tmp])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Config(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("storage", C.c_int), ("n", C.c_int * 3), ("bc", C.c_int * 3),
        ("wall_u", C.c_double * 18), ("tau", C.c_double), ("alpha", C.c_double),
        ("rho_f", C.c_double), ("g_drive", C.c_double * 3), ("g_grav", C.c_double * 3),
        ("delta", C.c_double), ("eps_p", C.c_double), ("eps_w", C.c_double), ("K", C.c_int),
        ("max_particles", C.c_int), ("max_radius", C.c_double), ("fp16_scale_log2", C.c_int),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


def lib():
    """Load the compiled library (no fallback: raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"lbmpen CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    sig = {
        "lbm_config_default": (C.c_int, [C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.c_int]),
        "lbm_create": (C.c_int, [C.POINTER(Config), C.POINTER(Allocator), _vp, C.POINTER(_vp)]),
        "lbm_create_batch": (C.c_int, [C.POINTER(Config), C.c_int, C.POINTER(Allocator), _vp,
                                       C.POINTER(_vp)]),
        "lbm_num_instances": (C.c_int, [_vp]),
        "lbm_add_particles": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]),
        "lbm_add_ellipses": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lbm_step": (C.c_int, [_vp, C.c_int]),
        "lbm_sync": (C.c_int, [_vp]),
        "lbm_get_fields": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int]),
        "lbm_get_particles": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lbm_num_particles": (C.c_int, [_vp, C.c_int]),
        "lbm_set_populations": (C.c_int, [_vp, C.c_int, _vp, C.c_int]),
        "lbm_get_populations": (C.c_int, [_vp, C.c_int, _vp, C.c_int]),
        "lbm_save_state": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t)]),
        "lbm_load_state": (C.c_int, [_vp, _vp, C.c_size_t]),
        "lbm_set_graphs": (C.c_int, [_vp, C.c_int]),
        "lbm_autotune": (C.c_int, [_vp, C.c_int]),
        "lbm_kernel_shape": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "lbm_set_kernel_shape": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
        "lbm_launches_per_step": (C.c_int, [_vp]),
        "lbm_set_particle_wait_limit": (C.c_int, [_vp, C.c_double]),
        "lbm_fluid_step_only": (C.c_int, [_vp]),
        "lbm_step_timed": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
        "lbm_get_particles_async": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lbm_steps_done": (C.c_longlong, [_vp]),
        "lbm_total_nodes": (C.c_longlong, [_vp]),
        "lbm_adjoint_forward": (C.c_int, [_vp, C.c_int, C.c_int]),
        "lbm_adjoint_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "lbm_adjoint_run": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
        "lbm_adjoint_release": (C.c_int, [_vp]),
        "lbm_last_error": (C.c_char_p, [_vp]),
        "lbm_status_string": (C.c_char_p, [C.c_int]),
        "lbm_destroy": (None, [_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def make_config(lattice=LBM_D2Q9, n=(64, 64, 1), bc=None, storage=LBM_FP32, tau=1.0, alpha=None,
                rho_f=1.0, g_drive=(0, 0, 0), g_grav=(0, 0, 0), delta=1.0, eps_p=2.0, eps_w=1.0,
                K=1, max_particles=64, max_radius=16.0, wall_u=None, fp16_scale_log2=14) -> Config:
    cfg = Config()
    nn = list(n) + [1] * (3 - len(n))
    lib().lbm_config_default(C.byref(cfg), lattice, int(nn[0]), int(nn[1]), int(nn[2]))
    cfg.storage = storage
    if bc is not None:
        for d in range(3):
            cfg.bc[d] = int(bc[d]) if d < len(bc) else LBM_PERIODIC
    if wall_u is not None:
        wu = np.asarray(wall_u, np.float64).reshape(-1)
        for i in range(18):
            cfg.wall_u[i] = float(wu[i])
    cfg.tau = float(tau)
    cfg.alpha = float(1.0 / tau if alpha is None else alpha)
    cfg.rho_f = float(rho_f)
    for d in range(3):
        cfg.g_drive[d] = float(g_drive[d]) if d < len(g_drive) else 0.0
        cfg.g_grav[d] = float(g_grav[d]) if d < len(g_grav) else 0.0
    cfg.delta, cfg.eps_p, cfg.eps_w, cfg.K = float(delta), float(eps_p), float(eps_w), int(K)
    cfg.max_particles = int(max_particles)
    cfg.max_radius = float(max_radius)
    cfg.fp16_scale_log2 = int(fp16_scale_log2)
    return cfg


def config_from_workload(w, storage=LBM_FP32, max_particles=None, max_radius=None) -> Config:
    """lbm_config for a ``workloads.Workload``."""
    lat = LBM_D2Q9 if w.D == 2 else LBM_D3Q19
    bc = [LBM_PERIODIC if p else LBM_WALL for p in w.periodic]
    if w.D == 2:
        bc[2] = LBM_PERIODIC
    rmax = max(w.radius) if w.radius else 4.0
    return make_config(lat, w.n, bc, storage, w.tau, w.alpha, 1.0, w.g_drive, w.g_grav, w.delta,
                       w.eps_p, w.eps_w, w.K,
                       max_particles=max_particles or max(1, w.num_particles),
                       max_radius=max_radius or max(2.0, rmax), wall_u=w.wall_u)


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                               int(stream or 0))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            try:
                self.torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class LBM:
    """One lbmpen context (one or many lattice instances) on the current CUDA device."""

    def __init__(self, configs, stream=None, torch_alloc: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbmpen needs a CUDA GPU; no CPU fallback exists")
        L = lib()
        if isinstance(configs, Config):
            configs = [configs]
        arr = (Config * len(configs))(*configs)
        self.configs = list(configs)
        self.D = 2 if configs[0].lattice == LBM_D2Q9 else 3
        self.Q = configs[0].lattice
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = _TorchAllocator(torch.cuda.current_device()) if torch_alloc else None
        h = C.c_void_p()
        rc = L.lbm_create_batch(arr, len(configs),
                                C.byref(self._alloc.struct) if self._alloc else None,
                                C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise LBMError(rc, "lbm_create_batch failed (invalid configuration or device error)")
        self._h = h

    # -- helpers --
    def _check(self, rc):
        if rc != 0:
            raise LBMError(rc, lib().lbm_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape_of(self, i=0):
        c = self.configs[i]
        return (c.n[2], c.n[1], c.n[0]) if self.D == 3 else (c.n[1], c.n[0])

    def nodes(self, i=0):
        return int(np.prod(self.shape_of(i)))

    # -- API --
    def add_particles(self, i, pos, radius, ratio, vel=None, omega=None):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1)
        radius = np.ascontiguousarray(radius, np.float64).reshape(-1)
        ratio = np.ascontiguousarray(ratio, np.float64).reshape(-1)
        vel = None if vel is None else np.ascontiguousarray(vel, np.float64).reshape(-1)
        omega = None if omega is None else np.ascontiguousarray(omega, np.float64).reshape(-1)
        self._check(lib().lbm_add_particles(self._h, i, len(radius), _ptr(pos), _ptr(radius),
                                            _ptr(ratio), _ptr(vel), _ptr(omega)))

    def add_ellipses(self, i, pos, a, b, theta, ratio, vel=None, omega=None):
        """Ellipses (D2Q9): semi-axes a >= b, orientation theta (radians)."""
        f64 = lambda v: np.ascontiguousarray(v, np.float64).reshape(-1)
        pos, a, b, ratio = f64(pos), f64(a), f64(b), f64(ratio)
        theta = None if theta is None else f64(theta)
        vel = None if vel is None else f64(vel)
        omega = None if omega is None else f64(omega)
        self._check(lib().lbm_add_ellipses(self._h, i, len(a), _ptr(pos), _ptr(a), _ptr(b), _ptr(theta),
                                           _ptr(ratio), _ptr(vel), _ptr(omega)))

    def step(self, n=1):
        self._check(lib().lbm_step(self._h, int(n)))

    def sync(self):
        self._check(lib().lbm_sync(self._h))

    def num_particles(self, i=0):
        return lib().lbm_num_particles(self._h, i)

    def fields(self, i=0):
        """(u [..., D], p [...], owner [...]) as host numpy arrays (float32, int32)."""
        shp = self.shape_of(i)
        N = self.nodes(i)
        u = np.zeros(self.D * N, np.float32)
        p = np.zeros(N, np.float32)
        o = np.zeros(N, np.int32)
        self._check(lib().lbm_get_fields(self._h, i, _ptr(u), _ptr(p), _ptr(o), 0))
        return np.moveaxis(u.reshape((self.D,) + shp), 0, -1), p.reshape(shp), o.reshape(shp)

    def fields_device(self, i, u, p=None, owner=None):
        """Write fields into device tensors (torch) without a host round trip."""
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(lib().lbm_get_fields(self._h, i, ptr(u), ptr(p), ptr(owner), 1))

    def particles(self, i=0):
        n = self.num_particles(i)
        D = self.D
        out = {"X": np.zeros((n, D)), "U": np.zeros((n, D)), "A": np.zeros((n, D)),
               "W": np.zeros((n, 1 if D == 2 else 3)), "theta": np.zeros((n, 1 if D == 2 else 3)),
               "count": np.zeros(n, np.int32)}
        if n:
            self._check(lib().lbm_get_particles(self._h, i, _ptr(out["X"]), _ptr(out["U"]),
                                                _ptr(out["W"]), _ptr(out["theta"]), _ptr(out["A"]),
                                                _ptr(out["count"])))
        return out

    def set_populations(self, f, i=0):
        f = np.ascontiguousarray(f, np.float32).reshape(-1)
        assert f.size == self.Q * self.nodes(i)
        self._check(lib().lbm_set_populations(self._h, i, _ptr(f), 0))

    def get_populations(self, i=0):
        f = np.zeros(self.Q * self.nodes(i), np.float32)
        self._check(lib().lbm_get_populations(self._h, i, _ptr(f), 0))
        return f.reshape((self.Q,) + self.shape_of(i))

    def save_state(self) -> bytes:
        n = C.c_size_t(0)
        self._check(lib().lbm_save_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().lbm_save_state(self._h, buf, C.byref(n)))
        return buf.raw

    def load_state(self, blob: bytes):
        self._check(lib().lbm_load_state(self._h, blob, len(blob)))

    def set_graphs(self, steps_per_graph: int):
        self._check(lib().lbm_set_graphs(self._h, int(steps_per_graph)))

    def autotune(self, reps: int = 5):
        self._check(lib().lbm_autotune(self._h, int(reps)))

    def kernel_shape(self):
        v, r, w = C.c_int(), C.c_int(), C.c_int()
        lib().lbm_kernel_shape(self._h, C.byref(v), C.byref(r), C.byref(w))
        return v.value, r.value, w.value

    def set_kernel_shape(self, vec, rows, warps):
        self._check(lib().lbm_set_kernel_shape(self._h, int(vec), int(rows), int(warps)))

    def set_particle_wait_limit(self, seconds: float):
        self._check(lib().lbm_set_particle_wait_limit(self._h, float(seconds)))

    def launches_per_step(self) -> int:
        return lib().lbm_launches_per_step(self._h)

    def fluid_step_only(self):
        self._check(lib().lbm_fluid_step_only(self._h))

    def particles_async(self, out, i=0):
        """Enqueue the copy of instance i's particle state into `out` (a dict
        with any of X, U, W, theta, A as float64 [n, 3] arrays and count as int32
        [n], contiguous, ideally in pinned memory) without synchronising; the
        values are there after the next sync."""
        p = {k: (None if out.get(k) is None else out[k].ctypes.data_as(C.c_void_p))
             for k in ("X", "U", "W", "theta", "A", "count")}
        self._check(lib().lbm_get_particles_async(self._h, i, p["X"], p["U"], p["W"], p["theta"], p["A"],
                                                  p["count"]))

    def step_timed(self, n):
        """n steps launched one by one with CUDA events around each kernel:
        mean ms per step of (fluid kernel, box sums, particle kernel)."""
        t = (C.c_float * 3)()
        self._check(lib().lbm_step_timed(self._h, int(n), C.byref(t, 0), C.byref(t, 4), C.byref(t, 8)))
        return float(t[0]), float(t[1]), float(t[2])

    # -- adjoint --
    def adjoint_forward(self, nsteps: int, seg_len: int = 0):
        """Run nsteps steps keeping checkpoints for adjoint_backward."""
        self._check(lib().lbm_adjoint_forward(self._h, int(nsteps), int(seg_len)))

    def adjoint_backward(self, seeds=None, seed_field=None, want_field=False):
        """Gradients of J = sum(seed * final state) over the recorded steps.

        seeds: per instance a dict with any of X, U, A ([np, D]) and W, theta
        ([np, 1] in 2D, [np, 3] in 3D); seed_field: a device float32 tensor of
        Q * N values per instance (instance order), or None.  Returns per
        instance a dict alpha, ratio [np], X, U, A [np, D], W, theta, and,
        with want_field, the device tensor dJ / d(initial populations)."""
        import torch
        ninst = len(self.configs)
        nps = [self.num_particles(i) for i in range(ninst)]
        D = self.D
        sp = np.zeros(sum(15 * n for n in nps))
        o = 0
        for i, n in enumerate(nps):
            blk = sp[o:o + 15 * n].reshape(n, 15)
            s = (seeds[i] if seeds is not None else None) or {}
            for k, c0 in (("X", 0), ("U", 3), ("A", 12)):
                if k in s:
                    blk[:, c0:c0 + D] = np.asarray(s[k], np.float64).reshape(n, D)
            for k, c0 in (("W", 6), ("theta", 9)):
                if k in s:
                    v = np.asarray(s[k], np.float64).reshape(n, -1)
                    if D == 2:
                        blk[:, c0 + 2] = v[:, 0]
                    else:
                        blk[:, c0:c0 + 3] = v
            o += 15 * n
        out = np.zeros(sum(1 + 16 * n for n in nps))
        gfield = None
        if want_field:
            total = sum(self.Q * self.nodes(i) for i in range(ninst))
            gfield = torch.zeros(total, dtype=torch.float32, device="cuda")
        sf = None if seed_field is None else C.c_void_p(seed_field.data_ptr())
        self._check(lib().lbm_adjoint_backward(self._h, _ptr(sp), sf, _ptr(out),
                                               None if gfield is None else C.c_void_p(gfield.data_ptr())))
        res = []
        o = 0
        for n in nps:
            r = out[o + 1:o + 1 + 16 * n].reshape(n, 16)
            wcol = [2] if D == 2 else [0, 1, 2]
            res.append({"alpha": float(out[o]), "ratio": r[:, 0].copy(), "X": r[:, 1:1 + D].copy(),
                        "U": r[:, 4:4 + D].copy(), "W": r[:, [7 + c for c in wcol]].copy(),
                        "theta": r[:, [10 + c for c in wcol]].copy(), "A": r[:, 13:13 + D].copy()})
            o += 1 + 16 * n
        return (res, gfield) if want_field else res

    def adjoint_release(self):
        self._check(lib().lbm_adjoint_release(self._h))

    @property
    def steps(self) -> int:
        return lib().lbm_steps_done(self._h)

    @property
    def total_nodes(self) -> int:
        return lib().lbm_total_nodes(self._h)


def from_workloads(workloads: Sequence, storage=LBM_FP32, add_particles=True, **kw) -> LBM:
    """Context over one or many ``workloads.Workload`` with their particles added."""
    ws = list(workloads)
    sim = LBM([config_from_workload(w, storage) for w in ws], **kw)
    if add_particles:
        for i, w in enumerate(ws):
            if w.num_particles and getattr(w, "minor", None) is not None:
                sim.add_ellipses(i, w.pos, w.radius, w.minor, w.theta, w.ratio)
            elif w.num_particles:
                sim.add_particles(i, w.pos, w.radius, w.ratio)
    return sim
