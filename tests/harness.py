"""Helpers that run the same seeded workload through the CUDA library and the oracle."""
import numpy as np

import oracle
from paper_2511_01629_gb300 import lbm


def oracle_config(w):
    return oracle.make_config(D=w.D, n=w.n, periodic=w.periodic, wall_u=w.wall_u, tau=w.tau,
                              alpha=w.alpha, g_drive=w.g_drive, g_grav=w.g_grav, delta=w.delta,
                              eps_p=w.eps_p, eps_w=w.eps_w, K=w.K)


def add_oracle_particles(ref, w):
    """The workload's disks, spheres or ellipses in an oracle Sim."""
    if not w.num_particles:
        return
    if getattr(w, "minor", None) is not None:
        ref.add_ellipses(w.pos, w.radius, w.minor, w.theta, w.ratio)
    else:
        ref.add_particles(w.pos, w.radius, w.ratio)


def make_pair(w, storage=lbm.LBM_FP32, f0=None, graphs=0, shape=None, parallel=False):
    """(gpu context, oracle sim) for workload w, optionally from populations f0 [Q, ...].
    parallel: the oracle's OpenMP build (identical results, all host cores)."""
    sim = lbm.from_workloads([w], storage)
    sim.set_graphs(graphs)
    if shape is not None:
        sim.set_kernel_shape(*shape)
    ref = oracle.Sim(oracle_config(w), parallel=parallel)
    if f0 is not None:
        f32 = np.asarray(f0, np.float32)
        sim.set_populations(f32)
        ref.set_f(f32.astype(np.float64))
    add_oracle_particles(ref, w)
    return sim, ref


def random_state(seed, Q, shape, scale=1e-3):
    """Random post-collision populations with f_0 = 0 (f_0 is not stored on the GPU)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-scale, scale, (Q,) + tuple(shape)).astype(np.float32)
    f[0] = 0
    return f


def compare_fields(sim, ref, i=0):
    """Fields of GPU instance i against an oracle Sim (or its stored (u, p, owner)).

    du: max |u - u_oracle| / U_ref with U_ref = max |u_oracle|; dp: max |p -
    p_oracle| / max |p_oracle|; dp_f: the same pressure error relative to
    U_ref + P_ref, P_ref = max |p_oracle|: the size of the moments the stored
    populations carry (f_q ~ w_q (p + c_q . u) / cs^2), on which their
    rounding acts."""
    u, p, own = sim.fields(i)
    ur, pr, ownr = ref.fields() if hasattr(ref, "fields") else ref
    uref = max(np.abs(ur).max(), 1e-30)
    dpa = float(np.abs(p - pr).max())
    return {
        "du": float(np.abs(u - ur).max() / uref),
        "dp": dpa / max(np.abs(pr).max(), 1e-30),
        "dp_f": dpa / (uref + float(np.abs(pr).max())),
        "owner_equal": bool(np.array_equal(own, ownr)),
        "owner_diff": int((own != ownr).sum()),
        "uref": float(uref),
        "pref": float(np.abs(pr).max()),
    }


def compare_particles(sim, ref, i=0):
    a = sim.particles(i)
    b = ref.particles() if hasattr(ref, "particles") else ref
    D = sim.D
    out = {}
    for k in ("X", "U", "A"):
        out["d" + k] = float(np.abs(a[k] - b[k][:, :D]).max()) if len(a[k]) else 0.0
    wcol = [2] if D == 2 else [0, 1, 2]
    out["dW"] = float(np.abs(a["W"] - b["W"][:, wcol]).max()) if len(a["W"]) else 0.0
    out["count_equal"] = bool(np.array_equal(a["count"], b["count"]))
    out["Uscale"] = float(np.abs(b["U"]).max()) if len(a["U"]) else 0.0
    return out


def oracle_run(w, steps, parallel=True):
    """Fields and particles of the oracle after `steps` steps of workload w."""
    ref = oracle.Sim(oracle_config(w), parallel=parallel)
    add_oracle_particles(ref, w)
    ref.step(steps)
    out = ref.fields(), ref.particles()
    ref.close()
    return out


def stored_fd():
    """The stored central differences of the adjoint workload
    (tests/golden/make_oracle_references.py): h, the first step at which the
    +-h runs use different solid domains, and J(+h), J(-h) every 50 steps."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "adjoint_disk_seed0_fd.txt")
    h, flips, rows = None, {}, {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "h":
            h = float(f[1])
        elif f[0] == "flip":
            flips[f[1]] = int(f[2])
        else:
            rows.setdefault(f[0], {})[int(f[1])] = (float(f[2]), float(f[3]))
    return h, flips, rows
