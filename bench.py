"""Throughput of the penalized-LBM hot path on GB300 (one JSON line on rank 0).

A step is one full time step of the method (fused stream-collide-penalize
kernel + FP64 particle kernels) over the whole workload.  The default
workload is the many-particle sedimentation case: D2Q9, 1024 x 4096 box with
walls, 500 disks R ~ U(6,12), density ratio ~ U(1.1,2.0), tau = 1,
alpha = 1/tau, gravity 2e-6 (synthetic, seeded).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage fp32|fp16] [--workload many_disks|ensemble|spheres3d]

Under torchrun (N > 1) every rank runs an independent replica (seed = rank):
the method has no exchange between independent instances, so there is no
collective on the data path ("scaling": "weak").
"""
import argparse
import hashlib
import json
import os
import select
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fluid_kernel_traffic.json")
CSRC = os.path.join(ROOT, "paper_2511_01629_gb300", "csrc")
# sources the fused fluid kernel is built from (the traffic record is void once they change)
FLUID_SRCS = [os.path.join(CSRC, f) for f in ("lbm_fluid_tma.cu", "lbm_fluid.cu", "lbm_common.cuh",
                                               "lbm_internal.cuh")]
METRIC = "MLUPS & % HBM peak: FP32 vs FP16-store (err≤1e-3); adjoint/forward time ratio"
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline uses the measured copy peak)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (a time): every rank gets it."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workloads(name, seed):
    from paper_2511_01629_gb300 import workloads as W
    if name == "many_disks":
        return [W.many_disks(seed)]
    if name == "ensemble":
        return W.ensemble(seed)
    if name == "spheres3d":
        return [W.spheres3d(seed)]
    if name == "single_disk":
        return [W.single_disk(seed)]
    raise SystemExit(f"unknown workload {name}")


def describe(name, ws, storage):
    nodes = sum(w.nodes for w in ws)
    parts = sum(w.num_particles for w in ws)
    if name == "many_disks":
        text = "D2Q9 many-particle sedimentation 1024x4096, 500 disks R~U(6,12), ratio~U(1.1,2.0)"
    elif name == "ensemble":
        text = f"{len(ws)} D2Q9 sedimentation instances, nx~U{{200..800}}, ny=4nx, 1-50 disks each"
    elif name == "spheres3d":
        text = "D3Q19 256x256x512 box, 8 spheres R=10, ratio 1.5"
    else:
        text = name
    return {"workload": text, "lattice": "D2Q9" if ws[0].D == 2 else "D3Q19", "nodes": nodes,
            "particles": parts, "instances": len(ws), "tau": ws[0].tau, "alpha": ws[0].alpha,
            "storage": storage, "steps_per_graph": 16}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    One nvidia-smi process samples every 200 ms on its own (-lms), so no
    Python thread of this process competes for the interpreter lock while the
    timed region launches its work; the region starts right after the first
    sample has arrived, and the process is stopped after the next one."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self._p = None

    def _take(self, line):
        line = line.strip()
        if line:
            self.samples.append([v.strip() for v in line.split(",")])

    def __enter__(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                        "--format=csv,noheader,nounits", "-lms", "200"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._take(self._p.stdout.readline())  # the first sample, just before the region
        except Exception:
            self._p = None
        return self

    def __exit__(self, *a):
        if self._p is None:
            return
        try:
            # one more sample, the first after the region (at most 1 s)
            if select.select([self._p.stdout], [], [], 1.0)[0]:
                self._take(self._p.stdout.readline())
            self._p.terminate()
            out, _ = self._p.communicate(timeout=10)
            for line in out.splitlines():
                self._take(line)
        except Exception:
            self._p.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        smax = max((float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(self.samples)}


def bytes_per_node(D, storage):
    q = 8 if D == 2 else 18  # stored populations (the rest population is never read back)
    return 2 * q * (2 if storage == "fp16" else 4)


def measured_peak():
    try:
        with open(MEASURED_PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fluid_src_sha():
    hh = hashlib.sha256()
    for f in FLUID_SRCS:
        hh.update(open(f, "rb").read())
    return hh.hexdigest()[:16]


def traffic_per_launch(storage, workload, shape):
    """DRAM bytes per fluid-kernel launch from the committed ncu capture of this
    workload, storage and kernel shape, or None when there is none or the kernel
    source changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
        h = fluid_src_sha()
        key = f"{workload}/{storage}/{shape[0]},{shape[1]},{shape[2]}"
        if rec.get("fluid_src_sha") != h or key not in rec.get("bytes_per_launch", {}):
            return None
        return float(rec["bytes_per_launch"][key])
    except Exception:
        return None


def oracle_sample(w, budget_s, min_steps=20, max_steps=100000, warmup=1):
    """The FP64 oracle as it stands (its OpenMP build: the same arithmetic on
    every host core) on a bounded sample of workload w: `warmup` untimed steps,
    then as many timed steps as fit in about budget_s seconds (at least
    min_steps).  Returns (MLUPS, steps, seconds, threads)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from harness import oracle_config
    sim = oracle.Sim(oracle_config(w), parallel=True)
    if w.num_particles:
        sim.add_particles(w.pos, w.radius, w.ratio)
    t0 = time.perf_counter()
    sim.step(max(1, warmup))  # page-in, first owner map
    per = (time.perf_counter() - t0) / max(1, warmup)
    k = int(min(max(min_steps, budget_s / max(per, 1e-6)), max_steps))
    t0 = time.perf_counter()
    sim.step(k)
    dt = time.perf_counter() - t0
    sim.close()
    return w.nodes * k / dt / 1e6, k, dt, oracle.threads(True)


def run_reference(args, ws_n, rank):
    """The contract's reference arm: the FP64 oracle as it stands, on all host
    cores, on this workload and metric; each timed step is one full oracle step
    of instance 0, as many as fit in about 90 s (at most --steps)."""
    if rank != 0:
        return
    ws = make_workloads(args.workload, 0)
    w = ws[0]
    w_steps = args.warmup
    mlups, k, dt, cores = oracle_sample(w, 90.0, min_steps=1, max_steps=args.steps, warmup=w_steps)
    sample = (f"{k} full FP64 oracle steps of instance 0 ({w.nodes} nodes) after {w_steps} untimed "
              f"steps, {dt:.1f} s on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws_n,
        "steps": k, "warmup": w_steps, "ms_per_step": dt / k * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": describe(args.workload, ws, "fp64"),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def adjoint_leg(lbm, torch, rank, nsteps):
    """Cost of the discrete adjoint on the disk-settling workload (400 x 1600,
    R = 12, ratio 1.5, J = final height): plain forward, checkpointed forward
    and backward sweep (segment recomputation included), one instance and a
    batch of 16 seeds in one context."""
    from paper_2511_01629_gb300 import workloads as W
    out = {"workload": "D2Q9 400x1600 closed box, one disk R=12 ratio 1.5 at (200+U(-20,20), 1280), "
                       "J = final height; gradients w.r.t. ratio, alpha, initial x",
           "steps": nsteps, "segment": "ceil(sqrt(steps))"}

    def run(batch):
        ws = [W.adjoint_disk(rank * 100 + s, steps=nsteps) for s in range(batch)]
        times = {}
        for rep in range(2):  # the first pass allocates and captures graphs
            sim = lbm.from_workloads(ws)
            sim.set_graphs(16)
            st = sim.stream
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            ev[0].record(st)
            sim.step(nsteps)
            ev[1].record(st)
            sim.close()
            sim = lbm.from_workloads(ws)
            sim.set_graphs(16)
            torch.cuda.synchronize()
            ev[2].record(st)
            sim.adjoint_forward(nsteps, 0)
            ev[3].record(st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            grads = sim.adjoint_backward([{"X": np.array([[0.0, 1.0]])}] * batch)
            torch.cuda.synchronize()
            tb = (time.perf_counter() - t0) * 1e3
            sim.close()
            times = {"forward_ms": ev[0].elapsed_time(ev[1]), "checkpointed_forward_ms": ev[2].elapsed_time(ev[3]),
                     "backward_ms": tb}
        times["ratio"] = times["backward_ms"] / times["forward_ms"]
        times["ratio_total"] = (times["checkpointed_forward_ms"] + times["backward_ms"]) / times["forward_ms"]
        times["grad_instance0"] = {"dY/dratio": float(grads[0]["ratio"][0]), "dY/dalpha": grads[0]["alpha"],
                                   "dY/dX0": float(grads[0]["X"][0, 0])}
        return times

    import numpy as np
    one = run(1)
    out.update(one)
    out["batch16"] = run(16)
    out["note"] = ("ratio = backward sweep (recompute + adjoint kernels) / plain forward of the same "
                   "steps; ratio_total adds the checkpointed forward")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--workload", default="many_disks",
                    choices=["many_disks", "ensemble", "spheres3d", "single_disk"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the fluid kernel shape of the timed legs (default: the library's "
                         "default shape, the one the committed profiles capture)")
    ap.add_argument("--no-fp16-leg", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the batched-ensemble and D3Q19 lines")
    ap.add_argument("--adjoint-steps", type=int, default=5000)
    ap.add_argument("--shape", default=None,
                    help="fluid kernel shape vec,rows,warps (vec 0 = TMA pipeline) instead of autotuning")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only launch the fluid kernel (for profiler launch lists)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2511_01629_gb300 import lbm
    lbm.build() if not os.path.exists(lbm.LIB_PATH) else None

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def leg(storage, steps, warmup, with_e2e, with_kernel):
        ws = make_workloads(args.workload, rank)
        st = lbm.LBM_FP16 if storage == "fp16" else lbm.LBM_FP32
        sim = lbm.from_workloads(ws, st)
        if args.shape:
            sim.set_kernel_shape(*[int(v) for v in args.shape.split(",")])
        elif args.autotune:
            sim.autotune(3)
        # every timed step replays a captured graph (graphs hold an even number
        # of steps): G = 16, or the whole run up to 256 steps (all but one when
        # the run is odd)
        G = 16 if steps % 16 == 0 or steps > 256 else steps - steps % 2
        sim.set_graphs(G)
        stream = sim.stream
        nodes = sim.total_nodes
        out = {"nodes": nodes, "shape": sim.kernel_shape(), "launches_per_step": sim.launches_per_step()}
        if args.kernel_only:
            for _ in range(warmup + steps):
                sim.fluid_step_only()
            torch.cuda.synchronize()
            return out, sim
        sim.step(warmup)
        # capture the graph outside the timed region (an even G returns to the
        # same parity, so one graph serves every replay)
        if G:
            sim.step(G)
        out["graph_steps"] = G
        out["capture_steps"] = G
        sim.sync()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        sim.sync()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        out.update(ms=ms, clocks=clk.summary())
        if with_kernel:
            # the dominant kernel alone, back to back on the library's stream
            # (lbm_fluid_step_only), CUDA events around kn launches
            kn = max(20, min(steps, 2000))
            for _ in range(3):
                sim.fluid_step_only()
            torch.cuda.synchronize()
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            for _ in range(kn):
                sim.fluid_step_only()
            k1.record(stream)
            torch.cuda.synchronize()
            out["kernel_ms"] = k0.elapsed_time(k1) / kn
            out["kernel_launches_timed"] = kn
            # per-kernel breakdown of a step, launched one by one with events
            # between the kernels (each duration includes its launch latency)
            sim.step_timed(3)
            fl, bx, pt = sim.step_timed(kn)
            out["step_kernels_ms"] = {"fluid": fl, "box_sums": bx, "particles": pt, "steps": kn,
                                      "note": "steps launched one by one without graphs, CUDA events "
                                              "between the kernels (lbm_step_timed)"}
        if with_e2e:
            blob = sim.save_state()
            pinned = torch.empty(len(blob), dtype=torch.uint8, pin_memory=True)
            pinned.numpy()[:] = memoryview(blob)
            import ctypes
            npart = sum(sim.num_particles(i) for i in range(len(ws)))
            ke = 1000  # a fixed run length, so that the one upload weighs the same whatever K
            # each step's result, the rigid-body state X, U, omega of every
            # particle, copied into pinned host buffers on the library's stream
            outs = [{k: torch.empty((sim.num_particles(i), 3), dtype=torch.float64, pin_memory=True).numpy()
                     for k in ("X", "U", "W")} for i in range(len(ws))]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = lbm.lib().lbm_load_state(sim._h, ctypes.c_void_p(pinned.data_ptr()), len(blob))
            sim._check(rc)
            for _ in range(ke):
                sim.step(1)
                for i in range(len(ws)):
                    sim.particles_async(outs[i], i)  # d2h of the step's result, no host wait
            sim.sync()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            last = sim.particles(0)
            D = ws[0].D
            assert np.array_equal(outs[0]["X"][:, :D], last["X"]), "async readback differs"
            out["e2e"] = {"value": nodes * ke / dt / 1e6, "unit": "MLUPS",
                          "h2d_bytes_per_step": len(blob) / ke,
                          "d2h_bytes_per_step": npart * 3 * 3 * 8,
                          "steps": ke, "note": "state uploaded once from pinned host memory inside "
                          "the timed region; after every step the particles' X, U, omega copied to "
                          "pinned host memory on the library's stream (lbm_get_particles_async), one "
                          "host synchronisation at the end"}
        return out, sim

    def other_leg(name, steps=200, warmup=10):
        """Step rate and fluid-kernel roofline of another workload (FP32)."""
        ws = make_workloads(name, rank)
        sim = lbm.from_workloads(ws)
        sim.autotune(3)
        sim.set_graphs(16)
        st = sim.stream
        sim.step(warmup)
        sim.sync()
        torch.cuda.synchronize()
        barrier()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(st)
        sim.step(steps)
        e[1].record(st)
        torch.cuda.synchronize()
        sim.sync()
        ms = max_over_ranks(e[0].elapsed_time(e[1]), world, "cuda")
        for _ in range(3):
            sim.fluid_step_only()
        e[2].record(st)
        for _ in range(100):
            sim.fluid_step_only()
        e[3].record(st)
        torch.cuda.synchronize()
        kms = e[2].elapsed_time(e[3]) / 100
        sim.step_timed(3)
        kfl, kbox, kpart = sim.step_timed(100)  # per-kernel breakdown of un-graphed steps
        nodes = sim.total_nodes
        bpn = bytes_per_node(ws[0].D, "fp32")
        peak, kind = measured_peak()
        ach = nodes * bpn / (kms / 1e3) / 1e9
        shape = sim.kernel_shape()
        sim.close()
        return {"value": world * nodes * steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
                "ms_per_step": ms / steps, "config": describe(name, ws, "fp32"),
                "kernel_shape": {"vec": shape[0], "tile_rows": shape[1], "warps": shape[2]},
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                             "kernel_ms": kms, "algorithmic_bytes_per_node": bpn,
                             "peak_kind": f"hbm_gbs of {kind}"},
                "step_kernels_ms": {"fluid": kfl, "box_sums": kbox, "particles": kpart, "steps": 100}}

    storage = args.storage
    res, sim = leg(storage, args.steps, args.warmup, not args.no_e2e, True)
    if args.kernel_only:
        sim.close()
        if rank == 0:
            print(json.dumps({"kernel_only": True, "shape": res["shape"]}))
        return
    ws0 = make_workloads(args.workload, 0)
    D = ws0[0].D
    nodes = res["nodes"]
    ms_step = res["ms"] / args.steps
    value = world * nodes * args.steps / (res["ms"] / 1e3) / 1e6
    peak, peak_kind = measured_peak()
    bpn = bytes_per_node(D, storage)
    kms = res["kernel_ms"]
    achieved = nodes * bpn / (kms / 1e3) / 1e9
    # an autotuned shape may differ from the captured one in its stage count
    traffic = None if args.autotune else traffic_per_launch(storage, args.workload, res["shape"])
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if storage == "fp32" else "f32 (fp16 storage)",
        "data": "synthetic",
        "config": dict(describe(args.workload, ws0, storage),
                       l2="no flush: the ping-pong population state (%.0f MB) exceeds the 129 MB L2"
                       % (nodes * bpn / 1e6)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_fluid_tma (fused stream-collide-penalize)",
                     "algorithmic_bytes_per_node": bpn, "kernel_ms": kms,
                     "kernel_timing": "CUDA events around %d back-to-back launches of the fluid kernel "
                                      "alone (lbm_fluid_step_only) on the library's stream"
                                      % res["kernel_launches_timed"],
                     "peak_kind": f"hbm_gbs of {peak_kind}",
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "nominal_peak": NOMINAL_HBM_GBS},
        "step_kernels_ms": res["step_kernels_ms"],
        "graph_steps": res["graph_steps"], "capture_steps": res["capture_steps"],
        "gpu_launches": res["launches_per_step"] * args.steps,
        "clocks": res["clocks"],
        "kernel_shape": {"vec": res["shape"][0], "tile_rows": res["shape"][1], "warps": res["shape"][2]},
    }
    if "e2e" in res:
        line["e2e"] = res["e2e"]
        line["e2e"]["value"] *= world
    sim.close()
    if storage == "fp32" and not args.no_fp16_leg and args.workload in ("many_disks", "spheres3d"):
        r16, s16 = leg("fp16", args.steps, args.warmup, False, True)
        s16.close()
        v16 = world * r16["nodes"] * args.steps / (r16["ms"] / 1e3) / 1e6
        b16 = bytes_per_node(D, "fp16")
        a16 = r16["nodes"] * b16 / (r16["kernel_ms"] / 1e3) / 1e9
        line["fp16_storage"] = {"value": v16, "unit": "MLUPS", "ms_per_step": r16["ms"] / args.steps,
                                "roofline": {"achieved": a16, "peak": peak, "frac": a16 / peak,
                                             "algorithmic_bytes_per_node": b16,
                                             "kernel_ms": r16["kernel_ms"],
                                             "traffic": None if args.autotune else
                                             traffic_per_launch("fp16", args.workload, r16["shape"])},
                                "kernel_shape": {"vec": r16["shape"][0], "tile_rows": r16["shape"][1],
                                                 "warps": r16["shape"][2]},
                                "step_kernels_ms": r16["step_kernels_ms"],
                                "speedup_vs_fp32": v16 / value}
    if not args.no_other_workloads and args.workload == "many_disks":
        line["other_workloads"] = {name: other_leg(name) for name in ("ensemble", "spheres3d")}
    if not args.no_adjoint and args.workload == "many_disks":
        adj = adjoint_leg(lbm, torch, rank, args.adjoint_steps)
        line["adjoint_forward_ratio"] = adj["ratio"]
        line["adjoint"] = adj
    else:
        line["adjoint_forward_ratio"] = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ws_c = make_workloads(args.workload, 0)
        mc, kc, dtc, cores = oracle_sample(ws_c[0], 15.0)
        line["cpu_baseline"] = {"value": mc, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"{kc} full FP64 oracle steps of instance 0 "
                                          f"({ws_c[0].nodes} nodes) after 1 untimed step, "
                                          f"{dtc:.1f} s on {cores} threads"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
