#!/usr/bin/env python
"""Benchmark of the wave library's hot path on one or more GPUs.

One step = one FWI gradient evaluation through the C ABI (wave_gradient):
forward modelling with receiver sampling and source injection, residual and
FP64 objective, adjoint sweep with the fused imaging condition, padding fold
(checkpointed recomputation supplies the forward wavefield).  Workload: the 3D
throughput configuration -- 512^3 physical grid, h = 10 m, 40-point sponge
(592^3 computational points), two-layer velocity 1.5/2.5 km/s times a seeded
5% Gaussian perturbation of 50 m correlation length, space order 8, nt = 1000,
one 15 Hz Ricker source at the surface centre, 512 x 512 receivers on the
surface nodes at 20 m depth.  Observed data come from the perturbed model; the
gradient is evaluated at the unperturbed two-layer model.

Throughput = point updates (forward + adjoint: 2 * points * (nt-1)) / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s & % HBM roofline (3D SO8 fwd/grad); shots/s & p50/p99 latency served"
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes per computational point and launch, by kernel kind
#   step: read u^n, u^{n-1}, cm, write u^{n+1}                    16 B
#   step_snap: + snapshot write (4 B FP32, 2 B 16-bit)
#   step_grad: + snapshot read, gradient read + write (8 B)
BYTES_PER_POINT = {"step": 16, "step_snap_fp32": 20, "step_snap_16": 18, "step_grad_fp32": 28, "step_grad_16": 26}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512, help="physical points per axis")
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--so", type=int, default=8)
    ap.add_argument("--nbl", type=int, default=40)
    ap.add_argument("--snap", default="checkpoint_fp32")
    ap.add_argument("--mode", default="gradient", choices=["gradient", "forward", "serve", "sweep", "propagate"],
                    help="gradient: one FWI gradient per step (default); forward: one forward modelling per step; "
                         "serve: a Poisson stream of shot-modelling requests through the continuous-batching server; "
                         "sweep: forward modelling per space order (--orders) on the throughput workload, with the "
                         "per-launch times of every step-kernel kind; propagate: source-free forward modelling of a "
                         "random initial state, one and two time levels per pass")
    ap.add_argument("--orders", default="2,4,6,8,10,12,14,16", help="sweep mode: space orders")
    ap.add_argument("--kernel-nt", type=int, default=160,
                    help="sweep mode: time levels of the full-storage gradients that time the snapshot and "
                         "imaging steps (0 = forward only)")
    ap.add_argument("--requests", type=int, default=400, help="serve mode: number of requests")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serve mode: HBM budget for resident requests")
    ap.add_argument("--max-resident", type=int, default=32, help="serve mode: stream slots")
    ap.add_argument("--batched", action="store_true",
                    help="serve mode: advance all resident requests together with batched launches")
    ap.add_argument("--tick-steps", type=int, default=32, help="serve mode, batched: steps per scheduler tick")
    ap.add_argument("--workload", default="throughput", choices=["throughput", "fwi", "paper_demo", "large"],
                    help="throughput: 512^3 two-layer + perturbation (default); fwi: 256^3 + 40, h = 12.5 m, "
                         "v(z) background with Gaussian anomalies, order 8, nt 1500; paper_demo: the paper's 3D "
                         "demonstration shape 201x201x70 + 40 (h = 15 m, order 14, 1 s, 10 Hz); large: "
                         "1000x1000x600 + 40, order 16, layered model with a salt body")
    ap.add_argument("--column-segments", type=int, default=1, choices=[0, 1, 2],
                    help="plain 3D steps: 0 z chunks, 1 column segments where the cost model favours them, "
                         "2 always column segments")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-nz", type=int, default=8, help="physical depth points of the CPU sample")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(n, nbl, so, nt, kind="throughput"):
    from paper_1608_08658_gb300 import inputs
    if kind == "paper_demo":
        # Sec. V-D demonstration: 201 x 201 x 70 + 40-point layer, h = 15 m, Ricker 10 Hz, 1 s, order 14;
        # the paper's velocity model is not given: a seeded layered model stands in for it
        shape, h = (201, 201, 70), (15.0, 15.0, 15.0)
        prof = inputs.layered_profile(shape[2], h[2], 5, v_min=1.5, v_max=3.5, seed=21)
        v0 = np.broadcast_to(prof[:, None, None], shape[::-1]).copy()
        ext = (shape[0] - 1) * h[0]
        src = np.array([[0.5 * ext, 0.5 * ext, 30.0]], dtype=np.float32)
        rec = inputs.surface_grid_receivers(shape[0], shape[1], h[:2], 30.0)
        return dict(shape=shape, spacing=h, nbl=40, so=14, nt=nt, v0=v0, v_true=v0, src=src, rec=rec,
                    vmax=float(v0.max()), f0=0.010, duration_ms=1000.0, kind=kind)
    if kind == "fwi":
        # FWI gradient workload: background v(z) = 1.5 + 0.6 z[km] (the starting model), true model with three
        # seeded Gaussian anomalies; 128 x 128 receivers on every second node at 25 m; Ricker 10 Hz
        shape, h = (256, 256, 256), (12.5, 12.5, 12.5)
        v0, vt = inputs.gradient_models(shape, h)
        ext = (shape[0] - 1) * h[0]
        src = np.array([[0.5 * ext, 0.5 * ext, 25.0]], dtype=np.float32)
        rec = inputs.surface_grid_receivers(shape[0] // 2, shape[1] // 2, (2 * h[0], 2 * h[1]), 25.0)
        return dict(shape=shape, spacing=h, nbl=40, so=8, nt=1500, v0=v0, v_true=vt, src=src, rec=rec,
                    vmax=float(vt.max()), f0=0.010, kind=kind)
    if kind == "large":
        # true model: 8 layers with the salt body; starting model: the layers smoothed along depth (150 m)
        # without the salt.  The salt's reflection needs 2.7 s two-way, beyond the 1.13 s of nt = 3000, so
        # the residual comes from the layer reflections (the first interface returns at 0.84 s)
        shape, h = (1000, 1000, 600), (10.0, 10.0, 10.0)
        vt = inputs.layered_salt_velocity(shape, h)
        v0 = inputs.layered_starting_velocity(shape, h)
        src = np.array([[4995.0, 4995.0, 20.0]], dtype=np.float32)
        g = np.linspace(0.0, 9990.0, 100)
        X, Y = np.meshgrid(g, g, indexing="xy")
        rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 20.0)], axis=1).astype(np.float32)
        return dict(shape=shape, spacing=h, nbl=40, so=16, nt=3000, v0=v0, v_true=vt, src=src, rec=rec,
                    vmax=4.5, f0=0.010, kind=kind)
    shape = (n, n, n)
    h = (10.0, 10.0, 10.0)
    v0 = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.0)
    v_true = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.05, corr_len=50.0, seed=7)
    ext = (n - 1) * h[0]
    src = np.array([[0.5 * ext, 0.5 * ext, 20.0]], dtype=np.float32)
    rec = inputs.surface_grid_receivers(n, n, (h[0], h[1]), 20.0)
    return dict(shape=shape, spacing=h, nbl=nbl, so=so, nt=nt, v0=v0, v_true=v_true, src=src, rec=rec,
                vmax=float(v_true.max()), f0=0.015, kind=kind)


def workload_config(w, snap, mode="gradient"):
    n = w["shape"][0]
    ncomp = n + 2 * w["nbl"]
    what = "FWI gradient" if mode == "gradient" else "forward modelling"
    if w.get("kind", "throughput") != "throughput":
        comp = [s + 2 * w["nbl"] for s in w["shape"]]
        name = {"paper_demo": "paper 3D demonstration shape (Sec. V-D), synthetic layered model",
                "fwi": "starting model v(z) = 1.5 + 0.6 z km/s, true model with three Gaussian anomalies",
                "large": "large layered model with salt body (gradient at the depth-smoothed layers without "
                         "the salt)"}[w["kind"]]
        return {"workload": "3D %s %s: %s + %d sponge = %s points, h=%g m, so=%d, nt=%d" % (
                    what, name, "x".join(map(str, w["shape"])), w["nbl"], "x".join(map(str, comp)), w["spacing"][0],
                    w["so"], w["nt"]),
                "grid": list(w["shape"]), "nbl": w["nbl"], "space_order": w["so"], "nt": w["nt"], "snap_mode": snap,
                "points_per_step": ("2 * %s * (nt-1) (forward + adjoint updates)" if mode == "gradient"
                                    else "%s * (nt-1)") % "x".join(map(str, comp)),
                "l2": "inputs larger than L2" if np.prod(comp) * 4 > 129e6 else "fields smaller than L2"}
    return {
        "workload": "3D " + what + " %d^3 (+%d sponge = %d^3), h=10 m, so=%d, nt=%d, two-layer 1.5/2.5 km/s + 5%% "
                    "perturbation, 1 Ricker 15 Hz, %dx%d surface receivers" % (n, w["nbl"], ncomp, w["so"], w["nt"],
                                                                              n, n),
        "grid": list(w["shape"]), "nbl": w["nbl"], "space_order": w["so"], "nt": w["nt"], "snap_mode": snap,
        "points_per_step": ("2 * %d^3 * (nt-1) (forward + adjoint updates)" % ncomp) if mode == "gradient"
        else ("%d^3 * (nt-1)" % ncomp),
        "l2": "inputs larger than L2 (each wavefield %.2f GB)" % (ncomp ** 3 * 4 / 1e9),
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_index is not None:
            cmd += ["-i", str(gpu_index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in self.rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(self.rows), "reasons": reasons}


KERNEL_SOURCES = ("step_kernel.cuh", "ptx.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_key(space_order, ndim, kernel, equal_spacing):
    """Identity of one compiled step kernel: its source files and its compile-time
    configuration (wave_step_kernel_layout).  A counter taken on a kernel is valid
    while the key is unchanged."""
    import hashlib
    from paper_1608_08658_gb300 import wave
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1608_08658_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    layout = wave.wave_step_kernel_layout(space_order, ndim, kernel, equal_spacing)
    h.update(",".join(str(v) for v in layout.values()).encode())
    return h.hexdigest()[:16]


def measured_traffic(key, points):
    """DRAM bytes per launch from the committed ncu counters (profiles/traffic.json:
    bytes per point of the kernel with this key), scaled to `points`; None when the
    file holds no counter of this exact kernel."""
    try:
        with open(TRAFFIC_FILE) as fh:
            entry = json.load(fh)["kernels"].get(key)
    except (OSError, ValueError, KeyError):
        return None
    return None if entry is None else float(entry["dram_bytes_per_point"]) * points


def aggregate(ms_local, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: the max over ranks of the
    per-step time and value = N * units / that time (units per second)."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (reported baseline)
# ---------------------------------------------------------------------------

def cpu_sample(w, nz_phys, steps_nt=3):
    """Oracle gradient on a bounded sample: full x-y extent, nz_phys physical
    depth points, the same sponge, spacing, order; nt = steps_nt."""
    import oracle
    n = w["shape"][0]
    og = oracle.model.Geometry(shape=(n, n, nz_phys), spacing=w["spacing"], nbl=w["nbl"], sponge_vref=w["vmax"])
    m = (1.0 / w["v0"][:nz_phys] ** 2).astype(np.float32)
    dt = 0.4 * oracle.model.dt_max(w["so"], og.spacing, w["vmax"])
    q = oracle.model.ricker(steps_nt, dt, w["f0"])[:, None]
    src = w["src"].copy()
    src[:, 2] = 20.0
    rec = w["rec"][:: max(1, len(w["rec"]) // 4096)].copy()
    d_obs = np.zeros((steps_nt, len(rec)))
    pts = int(np.prod(og.comp_shape))

    def run():
        t0 = time.perf_counter()
        oracle.wave.gradient(og, m, dt, steps_nt, w["so"], q, src, rec, d_obs)
        return time.perf_counter() - t0
    return run, pts, steps_nt, og


def _oracle_sample_worker(args):
    """One oracle gradient sample in a worker process (seconds it took)."""
    w, nz = args
    run, _, _, _ = cpu_sample(w, nz)
    return run()


def oracle_all_cores(w, nz, procs):
    """The oracle is single-threaded NumPy: on all host cores it runs as `procs`
    independent samples at once, in processes started with spawn (a process
    forked after the first GPU call would hang).  Returns the wall time of the
    parallel run and the per-sample times."""
    import multiprocessing as mp
    # only what cpu_sample reads: the top nz planes of the starting model
    light = {k: w[k] for k in ("shape", "spacing", "nbl", "so", "vmax", "f0", "src", "rec")}
    light["v0"] = np.ascontiguousarray(w["v0"][:nz])
    ctx = mp.get_context("spawn")
    # one thread per worker: the workers already fill the cores
    threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in threads})
    try:
        with ctx.Pool(procs) as pool:
            t0 = time.perf_counter()
            times = pool.map(_oracle_sample_worker, [(light, nz)] * procs)
            wall = time.perf_counter() - t0
    finally:
        for k, v in threads.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return wall, times


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(w, nz):
    """The FP64 oracle timed on a bounded sample of the workload, on one core
    and on every host core; `value` and `cores` are those of all cores."""
    run, pts, nt, og = cpu_sample(w, nz)
    t1 = run()
    units = 2.0 * pts * (nt - 1)
    cores = host_cores()
    wall, times = oracle_all_cores(w, nz, cores)
    sample = ("FP64 NumPy oracle gradient on %dx%dx%d computational points (%d physical depth points + sponge), "
              "nt=%d (2*%d point updates per sample)" % (og.comp_shape + (nz, nt, nt - 1)))
    return {"value": cores * units / wall / 1e9, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
            "sample": sample + "; %d samples in %d processes at once, %.1f s wall (one sample alone: %.1f s)"
                      % (cores, cores, wall, t1),
            "single_core": {"value": units / t1 / 1e9, "unit": "Gpts/s", "cores": 1, "seconds": t1}}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = make_workload(args.n, args.nbl, args.so, args.nt)
    _, pts, nt, og = cpu_sample(w, args.cpu_sample_nz)
    cores = host_cores()
    # each step: one oracle sample per host core, all at once (the oracle is single-threaded)
    for _ in range(args.warmup):
        oracle_all_cores(w, args.cpu_sample_nz, cores)
    ts = [oracle_all_cores(w, args.cpu_sample_nz, cores)[0] for _ in range(args.steps)]
    t = float(np.mean(ts))
    v = cores * 2.0 * pts * (nt - 1) / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gpts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, "full history (oracle)"),
            # the oracle sample is a gradient (forward + adjoint point updates)
            "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: %d FP64 oracle gradients at once (one per host core, spawned "
                                       "processes) on %dx%dx%d computational points, nt=%d"
                                       % ((cores,) + og.comp_shape + (nt,))},
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1608_08658_gb300 import wave

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = make_workload(args.n, args.nbl, args.so, args.nt, args.workload)
    so = w["so"]
    geom = wave.Geometry(shape=w["shape"], spacing=w["spacing"], nbl=w["nbl"], sponge_vref=w["vmax"])
    dt = 0.4 * wave.wave_dt_max(w["spacing"], so, w["vmax"])
    if "duration_ms" in w:
        w["nt"] = int(np.ceil(w["duration_ms"] / dt)) + 1
    nt = w["nt"]
    q = wave.wave_ricker(nt, dt, w["f0"]).reshape(nt, 1)
    m0 = (1.0 / w["v0"] ** 2).astype(np.float32)
    mt = (1.0 / w["v_true"] ** 2).astype(np.float32)
    ctx = wave.Context(local_rank)
    ctx.set_column_segments(args.column_segments)
    stream = torch.cuda.current_stream(dev)
    m0_d = torch.from_numpy(m0).to(dev)
    q_d = torch.from_numpy(q).to(dev)
    src_d = torch.from_numpy(w["src"]).to(dev)
    rec_d = torch.from_numpy(w["rec"]).to(dev)
    mt_d = torch.from_numpy(mt).to(dev)
    dobs_d = wave.wave_forward(ctx, geom, mt_d, src_d, q_d, rec_d, dt, nt, so)
    grad_d = torch.empty_like(m0_d)

    def step():
        if args.mode == "forward":
            wave.wave_forward(ctx, geom, mt_d, src_d, q_d, rec_d, dt, nt, so, d_out=dobs_d)
            return None, None
        return wave.wave_gradient(ctx, geom, m0_d, src_d, q_d, rec_d, dobs_d, dt, nt, so, snap_mode=args.snap,
                                  grad_out=grad_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.reset_stats()
    ctx.set_profiling(True)
    clocks = ClockSampler(local_rank if world > 1 else None) if rank == 0 else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    phi = None
    for _ in range(args.steps):
        _, phi = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop() if clocks else None
    ctx.set_profiling(False)
    stats = {wave.KERNEL_NAMES[k]: ctx.kernel_stats(k) for k in range(5)}
    launches = ctx.kernel_stats(-1)[0]
    npts = int(np.prod([s + 2 * w["nbl"] for s in w["shape"]]))
    sweeps = 1 if args.mode == "forward" else 2
    units = sweeps * npts * (nt - 1)
    ms, value = aggregate(ms, units, world, dist, dev)
    value /= 1e9

    # roofline of the dominant kernel kind
    fmt16 = "bf16" in args.snap or "fp16" in args.snap
    bpp = {"step": BYTES_PER_POINT["step"],
           "step_snap": BYTES_PER_POINT["step_snap_16" if fmt16 else "step_snap_fp32"],
           "step_grad": BYTES_PER_POINT["step_grad_16" if fmt16 else "step_grad_fp32"]}
    peak, peak_kind = hbm_peak()
    kernels = {}
    for k in ("step", "step_snap", "step_grad"):
        n, tms = stats[k]
        if n:
            avg = tms / n
            kernels[k] = {"launches": n, "avg_ms": avg, "share": tms / max(1e-9, sum(v[1] for v in stats.values())),
                          "bytes_per_point": bpp[k], "achieved_gbs": bpp[k] * npts / (avg * 1e-3) / 1e9}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    ach = kernels[dom]["achieved_gbs"]
    fmt = "bf16" if "bf16" in args.snap else ("fp16" if "fp16" in args.snap else "fp32")
    dom_kernel = {"step": "plain", "step_snap": "snap_" + fmt, "step_grad": "grad_" + fmt}[dom]
    key = kernel_key(so, len(w["shape"]), dom_kernel, len(set(w["spacing"])) == 1)
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": measured_traffic(key, npts), "kernel": dom, "kernel_key": key,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs copy test)"
                if peak_kind == "measured" else "fallback 6.8 TB/s", "bytes_per_point": bpp[dom],
                "points_per_launch": npts}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        m_h, q_h, src_h, rec_h = pin(mt if args.mode == "forward" else m0), pin(q), pin(w["src"]), pin(w["rec"])
        dobs_h = dobs_d.cpu().pin_memory().numpy()
        g_h = torch.empty(m0.shape, dtype=torch.float32).pin_memory().numpy()

        d_h = torch.empty(tuple(dobs_d.shape), dtype=torch.float32).pin_memory().numpy()

        def step_host():
            if args.mode == "forward":
                return wave.wave_forward(ctx, geom, m_h, src_h, q_h, rec_h, dt, nt, so, d_out=d_h,
                                         stream=ctypes_stream(stream))
            return wave.wave_gradient(ctx, geom, m_h, src_h, q_h, rec_h, dobs_h, dt, nt, so, snap_mode=args.snap,
                                      grad_out=g_h, stream=ctypes_stream(stream))
        step_host()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        te_ms, _ = aggregate((time.perf_counter() - t0) / args.steps * 1e3, 1.0, world, dist, dev)
        te = te_ms * 1e-3
        if args.mode == "forward":
            h2d = m_h.nbytes + q_h.nbytes + src_h.nbytes + rec_h.nbytes
            d2h = d_h.nbytes
        else:
            h2d = m_h.nbytes + q_h.nbytes + dobs_h.nbytes + src_h.nbytes + rec_h.nbytes
            d2h = g_h.nbytes + 8
        e2e = {"value": world * units / te / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": te * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_sample_nz)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(w, args.snap if args.mode == "gradient" else None, args.mode),
                               column_segments={0: "off", 1: "auto", 2: "always"}[args.column_segments]),
                "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "objective": phi}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_serve(args, rank, world, local_rank):
    """Served shot modelling: seeded request stream (half 2D N^2, N in [201, 1001];
    half 3D N^3, N in [128, 320]; orders 4/8/16; nt in [500, 2000]; layered
    1.5-4.5 km/s), Poisson arrivals at 80 % of the capacity measured on a burst
    of the first requests; each rank serves its own stream."""
    import torch
    from paper_1608_08658_gb300 import inputs, serve, wave
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    reqs = inputs.serving_requests(args.requests, seed=99 + rank)
    budget = int(args.budget_gb * (1 << 30))
    server = serve.ShotServer(device=local_rank, hbm_budget_bytes=budget, max_resident=args.max_resident,
                              batched=args.batched, tick_steps=args.tick_steps)
    # capacity from a burst (all arriving at once) of the first requests
    nb = min(len(reqs), max(8, args.requests // 10))
    burst = server.run(reqs[:nb], np.zeros(nb))
    capacity = nb / burst.wall
    rate = 0.8 * capacity
    arrivals = serve.poisson_arrivals(len(reqs), rate, seed=99 + rank)
    server.ctx.reset_stats()
    clocks = ClockSampler(local_rank if world > 1 else None) if rank == 0 else None
    torch.cuda.synchronize()
    stats = server.run(reqs, arrivals)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    launches = server.ctx.kernel_stats(-1)[0]
    summ = stats.summary()
    wall_ms, shots = aggregate(stats.wall * 1e3, len(stats.results), world, dist, "cuda")
    wall = wall_ms * 1e-3
    pts = 0.0
    h2d = d2h = 0
    for r in reqs:
        ncomp = (r["N"] + 2 * r["nbl"]) ** r["ndim"]
        pts += ncomp * (r["nt"] - 1)
        src, rec = inputs.request_points(r)
        h2d += 4 * (r["N"] + r["nt"] + src.size + rec.size)
        d2h += 4 * r["nt"] * len(rec)
    server.close()
    if rank == 0:
        line = {"metric": METRIC, "value": shots, "unit": "shots/s", "n_gpus": world, "steps": len(reqs),
                "warmup": nb, "ms_per_step": 1e3 * wall / max(1, len(stats.results)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "served shot modelling: Poisson stream of %d requests (2D 201^2..1001^2 / "
                                       "3D 128^3..320^3, orders 4/8/16, nt 500-2000, layered 1.5-4.5 km/s, "
                                       "1 Ricker 10 Hz, 100-1000 receivers)" % len(reqs),
                           "arrival_rate_per_s": rate, "burst_capacity_shots_per_s": capacity,
                           "hbm_budget_gb": args.budget_gb, "max_resident": args.max_resident,
                           "launch_form": ("batched launches, %d steps per tick" % args.tick_steps) if args.batched
                           else "one stream per request, 32-step graph replays",
                           "l2": "fields of the 3D requests exceed L2"},
                "p50_latency_s": summ["p50_latency_s"], "p99_latency_s": summ["p99_latency_s"],
                "mean_latency_s": summ["mean_latency_s"], "max_resident": summ["max_resident"],
                "peak_workspace_gb": summ["peak_workspace_bytes"] / 2 ** 30,
                "point_updates_gpts_per_s": world * pts / wall / 1e9,
                "roofline": None, "cpu_baseline": None,
                "e2e": {"value": shots, "unit": "shots/s", "h2d_bytes_per_step": int(h2d / len(reqs)),
                        "d2h_bytes_per_step": int(d2h / len(reqs))},
                "gpu_launches": int(launches), "launches_per_request": launches / max(1, len(stats.results)),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_sweep(args, rank, world, local_rank):
    """Forward modelling of the throughput workload (n^3 two-layer model with
    the 5 % perturbation, 40-point layer, equal spacing) for each space order:
    W untimed and K timed runs of nt steps (Gpts/s = points (nt-1) / time), and
    per-launch CUDA-event times of the plain step; with --kernel-nt > 0, also of
    the snapshot and imaging steps of full-storage gradients (FP32 and FP16
    snapshots) at that many time levels.  One JSON line; a table on stderr."""
    import torch
    from paper_1608_08658_gb300 import wave
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    orders = [int(x) for x in args.orders.split(",")]
    w = make_workload(args.n, args.nbl, 8, args.nt)
    geom = wave.Geometry(shape=w["shape"], spacing=w["spacing"], nbl=w["nbl"], sponge_vref=w["vmax"])
    npts = int(np.prod([s + 2 * w["nbl"] for s in w["shape"]]))
    m = torch.from_numpy((1.0 / w["v_true"] ** 2).astype(np.float32)).to(dev)
    src = torch.from_numpy(w["src"]).to(dev)
    rec = torch.from_numpy(w["rec"]).to(dev)
    peak, peak_kind = hbm_peak()
    bpp = {"plain": 16, "snap_fp32": 20, "grad_fp32": 28, "snap_fp16": 18, "grad_fp16": 26}
    rows = []
    launches = 0
    clocks = ClockSampler() if rank == 0 else None
    with wave.Context(local_rank) as ctx:
        ctx.set_column_segments(args.column_segments)
        for so in orders:
            dt = 0.4 * wave.wave_dt_max(w["spacing"], so, w["vmax"])
            q = torch.from_numpy(wave.wave_ricker(args.nt, dt, w["f0"]).reshape(args.nt, 1)).to(dev)
            d = wave.wave_forward(ctx, geom, m, src, q, rec, dt, args.nt, so)
            for _ in range(args.warmup):
                wave.wave_forward(ctx, geom, m, src, q, rec, dt, args.nt, so, d_out=d)
            torch.cuda.synchronize()
            ctx.reset_stats()
            ctx.set_profiling(True)
            stream = torch.cuda.current_stream(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                wave.wave_forward(ctx, geom, m, src, q, rec, dt, args.nt, so, d_out=d)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.set_profiling(False)
            ms = e0.elapsed_time(e1) / args.steps
            launches += ctx.kernel_stats(-1)[0]
            cnt, tms = ctx.kernel_stats(0)
            row = {"space_order": so, "forward_ms": ms, "forward_gpts": npts * (args.nt - 1) / (ms * 1e-3) / 1e9,
                   "kernels_ms": {"plain": tms / cnt}}
            if args.kernel_nt > 0:
                kn = args.kernel_nt
                qk = q[:kn].contiguous()
                dk = wave.wave_forward(ctx, geom, m, src, qk, rec, dt, kn, so)
                for fmt in ("fp32", "fp16"):
                    wave.wave_gradient(ctx, geom, m * 1.01, src, qk, rec, dk, dt, kn, so, snap_mode="full_" + fmt)
                    torch.cuda.synchronize()
                    ctx.reset_stats()
                    ctx.set_profiling(True)
                    for _ in range(2):
                        wave.wave_gradient(ctx, geom, m * 1.01, src, qk, rec, dk, dt, kn, so,
                                           snap_mode="full_" + fmt)
                    torch.cuda.synchronize()
                    ctx.set_profiling(False)
                    launches += ctx.kernel_stats(-1)[0]
                    for k, name in ((1, "snap_" + fmt), (2, "grad_" + fmt)):
                        cnt, tms = ctx.kernel_stats(k)
                        if cnt:
                            row["kernels_ms"][name] = tms / cnt
                ctx.trim()
            row["hbm_frac"] = {k: bpp[k] * npts / (v * 1e-3) / 1e9 / peak for k, v in row["kernels_ms"].items()}
            rows.append(row)
            print("so %2d  forward %.1f Gpts/s  " % (so, row["forward_gpts"]) + "  ".join(
                "%s %.4f ms (%.1f %%)" % (k, v, 100 * row["hbm_frac"][k]) for k, v in row["kernels_ms"].items()),
                file=sys.stderr, flush=True)
    clk = clocks.stop() if clocks else None
    if rank == 0:
        main_row = next((r for r in rows if r["space_order"] == 8), rows[0])
        comp = w["shape"][0] + 2 * w["nbl"]
        line = {"metric": METRIC, "value": main_row["forward_gpts"], "unit": "Gpts/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_row["forward_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "3D forward modelling per space order %s: %d^3 + %d sponge = %d^3 points, "
                                       "h=10 m, two-layer 1.5/2.5 km/s + 5%% perturbation, nt=%d; value at order %d"
                                       % (args.orders, args.n, w["nbl"], comp, args.nt, main_row["space_order"]),
                           "kernel_nt": args.kernel_nt, "l2": "inputs larger than L2"},
                "sweep": rows, "peak_gbs": peak, "peak_source": peak_kind, "bytes_per_point": bpp,
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def run_propagate(args, rank, world, local_rank):
    """Source-free forward modelling (the propagation of a given initial state,
    wave_forward_ex without sources) on the throughput grid at order --so,
    timed with one and with two time levels per pass over memory.  The initial
    state is seeded unit-variance noise; receivers as in the throughput
    workload.  Point updates per run = points * (nt - 1)."""
    import torch
    from paper_1608_08658_gb300 import wave
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = make_workload(args.n, args.nbl, args.so, args.nt)
    so, nt = args.so, args.nt
    geom = wave.Geometry(shape=w["shape"], spacing=w["spacing"], nbl=w["nbl"], sponge_vref=w["vmax"])
    dt = 0.4 * wave.wave_dt_max(w["spacing"], so, w["vmax"])
    npts = int(np.prod([s + 2 * w["nbl"] for s in w["shape"]]))
    m = torch.from_numpy((1.0 / w["v_true"] ** 2).astype(np.float32)).to(dev)
    rec = torch.from_numpy(w["rec"]).to(dev)
    g = torch.Generator(device=dev).manual_seed(5)
    u0 = torch.randn(geom.comp_array_shape, generator=g, device=dev)
    u1 = torch.randn(geom.comp_array_shape, generator=g, device=dev)
    d = torch.empty((nt, rec.shape[0]), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = hbm_peak()
    res = {}
    launches = 0
    clocks = ClockSampler() if rank == 0 else None
    with wave.Context(local_rank) as ctx:
        for levels in (1, 2):
            ctx.set_time_blocking(levels)
            for _ in range(args.warmup):
                wave.wave_forward(ctx, geom, m, None, None, rec, dt, nt, so, d_out=d, u_init_prev=u0, u_init=u1)
            torch.cuda.synchronize()
            ctx.reset_stats()
            ctx.set_profiling(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                wave.wave_forward(ctx, geom, m, None, None, rec, dt, nt, so, d_out=d, u_init_prev=u0, u_init=u1)
            e1.record(stream)
            torch.cuda.synchronize()
            ctx.set_profiling(False)
            ms = e0.elapsed_time(e1) / args.steps
            cnt, tms = ctx.kernel_stats(0)
            launches += ctx.kernel_stats(-1)[0]
            per_launch = tms / max(1, cnt)
            upd = levels if (nt - 1) % levels == 0 else None
            res[levels] = {"ms_per_run": ms, "gpts": npts * (nt - 1) / (ms * 1e-3) / 1e9,
                           "step_launches": cnt, "ms_per_launch": per_launch,
                           "bytes_per_update": 16 if levels == 1 else 10,
                           "achieved_gbs": (16 if levels == 1 else 20) * npts / (per_launch * 1e-3) / 1e9
                           if upd else None}
            print("levels per pass %d: %.1f Gpts/s, %.4f ms per step launch" % (levels, res[levels]["gpts"],
                                                                                per_launch), file=sys.stderr)
    clk = clocks.stop() if clocks else None
    if rank == 0:
        comp = w["shape"][0] + 2 * w["nbl"]
        ach = res[2]["achieved_gbs"]
        line = {"metric": METRIC, "value": res[2]["gpts"], "unit": "Gpts/s", "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res[2]["ms_per_run"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "3D source-free forward modelling of a random initial state: %d^3 + %d "
                                       "sponge = %d^3 points, h=10 m, two-layer 1.5/2.5 km/s + 5%% perturbation, "
                                       "so=%d, nt=%d, %d surface receivers; value with two time levels per pass"
                                       % (args.n, w["nbl"], comp, so, nt, rec.shape[0]),
                           "l2": "inputs larger than L2"},
                "levels": res,
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                             "frac": ach / peak if ach else None, "traffic": None, "kernel": "two-level pass",
                             "bytes_per_point": 20, "points_per_launch": npts,
                             "peak_source": peak_kind},
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def ctypes_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world and world > 1:
        print("warning: --gpus %d but WORLD_SIZE %d" % (args.gpus, world), file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "serve":
        return run_serve(args, rank, world, local_rank)
    if args.mode == "sweep":
        return run_sweep(args, rank, world, local_rank)
    if args.mode == "propagate":
        return run_propagate(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
