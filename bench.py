"""Benchmark: ray-voxel samples/s of the projection (A^T) + dose (A) operators inside the
plain FP32 projection optimiser, on the large-print workload (768 x 768 x 1024 voxels of
0.05 mm, 1000 angles, 1024^2 pixels, f/2.8 with 4 rays per pixel, pupil 100 mm, vial
19 / 1.5 mm); the time-to-target comparison runs on its own, smaller workload.

One step = one optimiser iteration over the whole volume: g = max(0, A^T m),
d = A g, normalise, error, model update (all in the CUDA library, called through the
C ABI).  Units per step = 2 x samples_per_pass (one adjoint and one forward pass).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vamrt|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of this
path) on the host cores, on a bounded sample of the same workload.  With N > 1 each
rank runs an independent replica (the operator pair does not exchange data in this
library); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ray-voxel samples/s fwd+adjoint; time-to-target dose error vs plain, 1 GB300"
UNIT = "samples/s"
WORKLOAD = "large_768x768x1024_1000ang_4rays"
TTT_WORKLOAD = "mid_256cube_360ang_16rays"
BYTES_PER_SAMPLE = 32          # 8 trilinear corners x 4 B (FP32 gathers / reductions)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_max(value: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (timings: the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_traffic() -> dict:
    """Per-launch DRAM and L2 bytes of the operators from ncu captures (profiles/traffic.json):
    '<workload>:<kernel>' = dram__bytes_read + write, '<workload>:<kernel>:l2' =
    lts__t_bytes, each scaled to a full launch by the samples processed."""
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tf) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def l2_report(traffic: dict, workload: str, kernel: str, ms: float, l2_read_bps: float):
    """Achieved L2 throughput of one operator launch: its captured L2 bytes over the
    launch's CUDA-event time, against the L2 read bandwidth measured in the same run;
    None when no capture of this workload and kernel exists."""
    b = traffic.get(f"{workload}:{kernel}:l2")
    if not b or not ms > 0 or not l2_read_bps > 0:
        return None
    gbps = b / (ms / 1e3) / 1e9
    return {"bytes_per_launch": b, "achieved_GBps": gbps, "peak_GBps": l2_read_bps / 1e9,
            "frac": gbps * 1e9 / l2_read_bps,
            "source": "ncu lts__t_bytes.sum of a crop capture scaled by samples (profiles/)"}


def cpu_threads() -> int:
    """Host cores the oracle sample runs on: one worker process per core."""
    return os.cpu_count() or 1


def _oracle_rows_worker(job):
    """One worker of the CPU baseline (a spawned process): for every pixel of its rows, the
    FP64 oracle's projection value (Sec. 2.4) and then that pixel's dose contributions
    (Sec. 2.5), through the oracle's own C entry points.  Returns the seconds spent."""
    import ctypes

    from oracle import vam_oracle as O
    w, pupil, vol_path, shape, angle, rows = job
    vol = np.memmap(vol_path, dtype=np.float64, mode="r", shape=shape)
    L = O.lib()
    G = O.geom(w, pupil)
    dp = ctypes.POINTER(ctypes.c_double)
    vptr = vol.ctypes.data_as(dp)
    cap = 1 << 18
    idx = np.empty(cap, np.int64)
    val = np.empty(cap, np.float64)
    t0 = time.perf_counter()
    for v in rows:
        for u in range(w.nu):
            y = L.orc_adjoint_pixel(G.ref, vptr, angle, v, u)
            n = L.orc_forward_pixel(G.ref, angle, v, u, max(y, 0.0), idx.ctypes.data, val.ctypes.data, cap)
            if n > cap:
                cap = int(n)
                idx = np.empty(cap, np.int64)
                val = np.empty(cap, np.float64)
                L.orc_forward_pixel(G.ref, angle, v, u, max(y, 0.0), idx.ctypes.data, val.ctypes.data, cap)
    return time.perf_counter() - t0


class OracleSampler:
    """The FP64 oracle timed on the host cores: a pool of `threads` spawned worker processes
    sharing the volume through a file mapping.  run(rows, angle): oracle A^T then A over
    those pixel rows of one angle, rows dealt round-robin over the workers -- each pixel's
    projection (clamped at 0 as the optimiser does), then that pixel's dose contributions.
    Returns (samples, wall seconds, workers)."""

    def __init__(self, w, pupil, target, threads=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        import tempfile

        from oracle import vam_oracle as O
        O.build()
        self.w, self.pupil, self.shape = w, pupil, tuple(target.shape)
        self.threads = threads or cpu_threads()
        self.tmp = tempfile.TemporaryDirectory()
        self.path = os.path.join(self.tmp.name, "volume.f64")
        np.ascontiguousarray(target, dtype=np.float64).tofile(self.path)
        self.pool = cf.ProcessPoolExecutor(max_workers=self.threads, mp_context=mp.get_context("spawn"))
        # start every worker (imports, library load) before anything is timed
        list(self.pool.map(_oracle_rows_worker, [(w, pupil, self.path, self.shape, 0, [])] * self.threads))

    def samples(self, rows):
        """Samples the chosen pixel rows visit: per traced ray, the midpoints whose footprint
        reaches the grid (counted outside any timed region)."""
        from oracle import vam_oracle as O
        w, n = self.w, 0
        for v in rows:
            for u in range(w.nu):
                for a in range(w.rays_per_pixel):
                    r = O.trace(w, self.pupil, u, v, a)
                    if r["status"] != 2:
                        continue
                    dl = r["ell"] / r["k"]
                    j = np.arange(r["k"])
                    qz = (r["e"][2] + (j + 0.5) * dl * r["d2"][2]) / w.voxel_mm + 0.5 * (w.nz - 1)
                    n += int(np.count_nonzero((qz > -1) & (qz < w.nz)))
        return 2 * n

    def run(self, rows, angle=0):
        jobs = [(self.w, self.pupil, self.path, self.shape, angle, rows[i::self.threads]) for i in range(self.threads)]
        jobs = [j for j in jobs if j[-1]]
        t0 = time.perf_counter()
        list(self.pool.map(_oracle_rows_worker, jobs))
        return time.perf_counter() - t0, len(jobs)

    def close(self):
        self.pool.shutdown()
        self.tmp.cleanup()


def sample_rows(w, count):
    mid = w.nv // 2
    return list(range(mid - count // 2, mid - count // 2 + count))


def run_reference(args, rank, world):
    from paper_2211_03516_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    if rank != 0:
        return
    pupil = I.workload_pupil(w)
    target = I.make_target(w)
    rows = sample_rows(w, args.ref_rows)
    S = OracleSampler(w, pupil, target)
    n_rows = S.samples(rows)
    for _ in range(args.warmup):
        S.run(rows[:1])
    tot_n, tot_t, threads = 0, 0.0, S.threads
    for s in range(args.steps):
        dt, threads = S.run(rows, angle=0)
        tot_n += n_rows
        tot_t += dt
    S.close()
    value = tot_n / tot_t
    sample = (f"{args.ref_rows} pixel rows x {w.nu} columns x {w.rays_per_pixel} rays of one angle per step "
              f"(of {w.nv} rows x {w.n_angles} angles), projection then dose, FP64 oracle in {threads} worker processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "samples_per_step": tot_n // args.steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def time_to_target(P, target, w, iters, beta=4.0, mu=0.5):
    """Run the plain FP32 optimiser for `iters` iterations from m = f, recording
    per-iteration device time (CUDA events) and the voxel error rate (VER); then, until
    they reach the target or `iters` iterations, the BF16-storage run, the over-relaxed run
    (model step beta, BF16 storage) and the over-relaxed runs with heavy-ball momentum mu
    (FP32 and BF16 storage); and the Radon-method baseline's VER.  Target: VER <= 1.01 x
    the plain run's final VER."""
    import torch

    def run(dtype, step=1.0, goal=None, momentum=0.0):
        model = target.clone()
        prev = target.clone() if momentum else None
        proj = torch.empty(w.proj_shape, device=target.device, dtype=dtype)
        dose = torch.empty(w.vol_shape, device=target.device, dtype=dtype)
        t, vers = [], []
        for _ in range(iters):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            P.optimize(target, model=model, max_iter=1, tol=0.0, proj=proj, dose=dose, step=step,
                       momentum=momentum, prev_model=prev)
            e1.record()
            e1.synchronize()
            t.append(e0.elapsed_time(e1) / 1e3)
            vers.append(P.voxel_error_rate(dose, target)[0])
            if goal is not None and vers[-1] <= goal:
                break
        return np.cumsum(t), vers

    t32, v32 = run(torch.float32)
    goal = 1.01 * v32[-1]

    def variant(dtype, step, momentum=0.0):
        t, v = run(dtype, step, goal, momentum)
        hit = next((i for i, x in enumerate(v) if x <= goal), None)
        return {"iterations_to_target": None if hit is None else hit + 1,
                "seconds_to_target": None if hit is None else float(t[hit]),
                "best_ver": min(v), "time_ratio": None if hit is None else float(t[hit] / t32[-1])}

    out = {
        "target": "VER <= 1.01 x plain FP32 final VER",
        "plain_fp32": {"iterations": iters, "seconds": float(t32[-1]), "final_ver": v32[-1],
                       "ver_per_iteration": [round(v, 6) for v in v32]},
        "bf16_storage": variant(torch.bfloat16, 1.0),
        f"relaxed_beta{beta:g}_bf16": variant(torch.bfloat16, beta),
        f"relaxed_beta{beta:g}_mu{mu:g}_fp32": variant(torch.float32, beta, mu),
        f"relaxed_beta{beta:g}_mu{mu:g}_bf16": variant(torch.bfloat16, beta, mu),
        "warm_start": None,
    }
    from paper_2211_03516_gb300 import radon as RB

    rb = RB.radon_baseline(P, w, target)
    out["radon_baseline"] = {
        "method": "Sec. 2.3: per-slice parallel-beam Radon transform, Ram-Lak filter, negatives clipped "
                  "(no coordinate remap)",
        "ver_ideal_radon_printer": rb["ver_ideal_radon_printer"],
        "ver_ray_traced_printer": rb["ver_ray_traced_printer"],
        "ver_ray_traced_optimiser": v32[-1]}
    ratios = {k: out[k]["time_ratio"] for k in out if isinstance(out[k], dict) and "time_ratio" in out[k]}
    out["time_ratio"] = out["bf16_storage"]["time_ratio"]
    reached = {k: r for k, r in ratios.items() if r is not None}
    out["best"] = None if not reached else {"variant": min(reached, key=reached.get), "time_ratio": min(reached.values())}
    return out


def network_throughput(net, y, g, scale, fwd_reps=5, step_reps=3):
    """Tensor-core throughput of the warm-start network's convolutions: one forward pass
    and one training step (forward, head, backward) on projections y [A][nv][nu]."""
    import torch

    from paper_2211_03516_gb300 import warmstart as WS

    Dp = WS.padded_angles(y.shape[0])
    x0 = net.prepare(y, scale, Dp)
    fl = net.forward_flops(Dp, y.shape[1], y.shape[2])
    for _ in range(2):
        net.forward(x0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(fwd_reps):
        net.forward(x0)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / fwd_reps
    e0.record()
    for _ in range(step_reps):
        net.zero_grad()
        z = net.forward(x0)
        _, _, dz = net.head(z, y, scale, target=g, want_grad=True, target_scale=scale)
        net.backward(dz)
    e1.record()
    e1.synchronize()
    step_ms = e0.elapsed_time(e1) / step_reps
    peak_tf = 1924.8
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak_tf = float(json.load(fh)["bf16_tflops"])
    except Exception:
        pass
    tf = fl / (fwd_ms / 1e3) / 1e12
    return {"input": [Dp, y.shape[1], y.shape[2], 16], "forward_ms": fwd_ms, "train_step_ms": step_ms,
            "forward_flops": fl,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": tf / peak_tf, "peak_kind": "measured (bf16 burst)"},
            "train_step_tflops": 3 * fl / (step_ms / 1e3) / 1e12}


def run_network_only(args):
    """The warm-start network alone on the 128^3 workload's projection shape (random
    weights, A^T f of one synthetic target as input): timing and profiling of the
    convolution kernels without the data generation and training."""
    import torch

    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300 import unet as U
    from paper_2211_03516_gb300 import vamrt

    w = I.WORKLOADS["warmstart_128cube_180ang_4rays"]
    P = vamrt.Projector.from_workload(w, I.workload_pupil(w))
    f = torch.from_numpy(I.make_target(w, seed=0)).to("cuda:0")
    y = P.adjoint(f)
    s = 1.0 / float(y.max())
    net = U.UNet3D("cuda", seed=0)
    out = network_throughput(net, y, y, s, fwd_reps=args.steps, step_reps=max(1, args.steps // 2))
    U.check_errors(net.device)
    out.update({"workload": w.name, "n_angles": w.n_angles})
    print(json.dumps(out), flush=True)


def warm_start_time_to_target(args):
    """Learned warm start on the 128^3 workload (180 angles, 128^2 pixels, 4 rays): train on
    pairs the plain FP32 optimiser produces, then on held-out targets time (inference + the
    BF16-storage projection-space iterations) to reach 1.01 x the plain loop's final VER
    after the same number of plain iterations as the pairs used."""
    import torch

    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300 import unet as U
    from paper_2211_03516_gb300 import vamrt
    from paper_2211_03516_gb300 import warmstart as WS

    w = I.WORKLOADS["warmstart_128cube_180ang_4rays"]
    P = vamrt.Projector.from_workload(w, I.workload_pupil(w))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pairs = WS.make_pairs(P, w, range(args.ws_train), osmo_iters=w.osmo_iters)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = U.UNet3D("cuda", seed=0)
    losses = WS.train(net, pairs, epochs=args.ws_epochs, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rows = WS.compare(P, net, w, range(100000, 100000 + args.ws_eval), plain_iters=w.osmo_iters,
                      cont_iters=12, step=0.5, dtype=torch.bfloat16, beta=args.ttt_beta, mu=args.ttt_mu,
                      loss_iters=args.ws_loss_iters, loss_lr=args.ws_loss_lr, loss_dl=args.ws_loss_dl)
    network = network_throughput(net, pairs[0][1], pairs[0][2], 1.0)

    def ratio_of(x, r):
        return None if x is None else x / r["plain_seconds"]

    held = []
    for r in rows:
        held.append({"seed": r["seed"], "plain_iterations": w.osmo_iters, "plain_seconds": r["plain_seconds"],
                     "plain_final_ver": r["plain_final_ver"],
                     "warm_loss_iterations": r["warm_loss_iters_to_target"],
                     "time_ratio": ratio_of(r["warm_loss_seconds_to_target"], r),
                     "inference_seconds": r["inference_seconds"],
                     "no_network_loss_iterations": r["cold_loss_iters_to_target"],
                     "no_network_loss_time_ratio": ratio_of(r["cold_loss_seconds_to_target"], r),
                     "warm_projection_space_iterations": r["warm_iters_to_target"],
                     "warm_projection_space_time_ratio": ratio_of(r["warm_seconds_to_target"], r),
                     "relaxed_iterations": r["relaxed_iters_to_target"],
                     "relaxed_time_ratio": ratio_of(r["relaxed_seconds_to_target"], r)})

    def summary(key):
        vals = [h[key] for h in held if h[key] is not None]
        return {"reached": f"{len(vals)}/{len(held)}", "median_time_ratio_of_reached": float(np.median(vals))
                if vals else None, "median_time_ratio_all": float(np.median([h[key] if h[key] is not None
                                                                             else float("inf") for h in held]))}

    ratios = [h["time_ratio"] for h in held if h["time_ratio"] is not None]
    rel = [h["relaxed_time_ratio"] for h in held if h["relaxed_time_ratio"] is not None]
    return {"workload": w.name, "target": "VER <= 1.01 x plain FP32 final VER",
            "train_pairs": len(pairs), "pair_iterations": w.osmo_iters, "epochs": args.ws_epochs,
            "data_generation_seconds": t1 - t0, "training_seconds": t2 - t1, "final_train_loss": losses[-1],
            "continuation": f"thresholded-loss Adam steps (adjoint-driven, step {args.ws_loss_lr:g} x mean "
                            f"projection, d_l {args.ws_loss_dl:g}, d_h 1), BF16-stored projections and dose",
            "warm_start": summary("time_ratio"), "no_network_same_continuation": summary("no_network_loss_time_ratio"),
            "warm_start_projection_space": summary("warm_projection_space_time_ratio"),
            "relaxed_no_network": summary("relaxed_time_ratio"),
            "network": network,
            "held_out": held, "reached": f"{len(ratios)}/{len(held)}",
            "median_time_ratio_of_reached": float(np.median(ratios)) if ratios else None,
            "relaxed": {"loop": f"object space from m = f, model step {args.ttt_beta:g}, momentum {args.ttt_mu:g}, "
                                "BF16 storage, no network",
                        "reached": f"{len(rel)}/{len(held)}",
                        "median_time_ratio": float(np.median(rel)) if rel else None}}


def run_gpu(args, rank, world):
    import torch

    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300 import vamrt

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vamrt.lib()

    w = I.WORKLOADS[args.workload]
    if args.angles:
        w = w.scaled(n_angles=args.angles)
    if args.nz:
        w = w.scaled(nz=args.nz)
    if args.nv:
        w = w.scaled(nv=args.nv)
    pupil = I.workload_pupil(w)
    target_np = I.make_target(w)
    t0 = time.perf_counter()
    P = vamrt.Projector.from_workload(w, pupil)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    spp = P.sample_count()
    units_per_step = 2 * spp

    target = torch.from_numpy(target_np).to(dev)
    model = target.clone()
    proj = torch.empty(w.proj_shape, device=dev)
    dose = torch.empty(w.vol_shape, device=dev)
    stream = torch.cuda.current_stream()

    def step(timing=False):
        return P.optimize(target, model=model, max_iter=1, tol=0.0, proj=proj, dose=dose, timing=timing)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM (model/target/proj/dose > L2) ----
    launches0 = vamrt.vamrt_launch_count()
    adj_ms = fwd_ms = upd_ms = 0.0
    barrier()
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            r = step(timing=True)
            adj_ms += r["adjoint_ms"]
            fwd_ms += r["forward_ms"]
            upd_ms += r["update_ms"]
        ev1.record(stream)
        barrier()
    launches = vamrt.vamrt_launch_count() - launches0
    ms_max = reduce_max(ev0.elapsed_time(ev1), dist, dev)
    value = world * units_per_step * args.steps / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers ----
    host_target = torch.from_numpy(target_np).pin_memory()
    host_proj = torch.empty(w.proj_shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        target.copy_(host_target, non_blocking=True)
        r = step()
        host_proj.copy_(proj, non_blocking=True)
        torch.cuda.synchronize()
        _ = r["final_error"]
    barrier()
    e2e_value = world * units_per_step * e2e_steps / reduce_max(time.perf_counter() - t0, dist, dev)

    # ---- roofline of the dominant kernel (CUDA events around it, inside the library) ----
    # Both operators stage their per-sample data -- 8 trilinear corner words, 32 B -- in
    # shared memory, so the roofline is shared-memory bandwidth, measured here; the HBM
    # fraction of the compulsory traffic is reported beside it.
    smem_bps = vamrt.vamrt_measure_smem_bandwidth()
    l2_read_bps, l2_red_ops = vamrt.vamrt_measure_l2_rates()
    hbm, peak_kind = peaks()
    # The dose kernel skips the rays of pixels whose value is zero (their contributions are
    # exactly zero): its algorithmic samples are those of the nonzero pixels of the
    # projections it was given (the last iteration's g, the same support every step here).
    _, _, j2 = P.ray_table()
    per_pixel = torch.from_numpy((j2[:, 1] - j2[:, 0]).astype(np.int64).reshape(w.rays_per_pixel, w.nv, w.nu)
                                 .sum(0)).to(dev, torch.float64)
    fwd_spp = sum(float(((proj[k0:k0 + 64] != 0).to(torch.float64) * per_pixel).sum())
                  for k0 in range(0, w.n_angles, 64))
    adj_ms_step, fwd_ms_step = adj_ms / args.steps, fwd_ms / args.steps
    kern = {"adjoint": {"samples": spp, "ms": adj_ms_step},
            "forward": {"samples": fwd_spp, "ms": fwd_ms_step}}
    for kk in kern.values():
        kk["achieved_GBps"] = kk["samples"] * BYTES_PER_SAMPLE / (kk["ms"] / 1e3) / 1e9
        kk["frac"] = kk["achieved_GBps"] * 1e9 / smem_bps
    dom = "forward" if fwd_ms >= adj_ms else "adjoint"
    dom_ms = kern[dom]["ms"]
    achieved = kern[dom]["achieved_GBps"]
    n_rays = P.info()["n_rays"]
    vol_b, proj_b = 4 * math.prod(w.vol_shape), 4 * math.prod(w.proj_shape)
    # compulsory DRAM bytes of one launch: volume in + projections out (adjoint) or
    # projections in + dose accumulator out (forward), plus the ray table once per angle
    compulsory = vol_b + proj_b + 72 * n_rays * w.n_angles
    # captured counters describe the full workload: none for a reduced (profiling) case
    traffic_all = {} if (args.angles or args.nz or args.nv) else load_traffic()
    traffic = traffic_all.get(f"{w.name}:{dom}")
    l2 = l2_report(traffic_all, w.name, dom, dom_ms, l2_read_bps)

    # ---- the tall build (384 x 384 x 512, 720 angles, 8 rays) with BF16-stored projections
    # and dose, beside the headline: one timed optimiser iteration after one warm-up ----
    tall = None
    if args.tall and world == 1:
        wt3 = I.WORKLOADS["tall_384x384x512_720ang_8rays"]
        P3 = vamrt.Projector.from_workload(wt3, I.workload_pupil(wt3))
        f3 = torch.from_numpy(I.make_target(wt3)).to(dev)
        m3 = f3.clone()
        g3 = torch.empty(wt3.proj_shape, device=dev, dtype=torch.bfloat16)
        d3 = torch.empty(wt3.vol_shape, device=dev, dtype=torch.bfloat16)
        spp3 = P3.sample_count()
        for it in range(2):
            r3 = P3.optimize(f3, model=m3, max_iter=1, tol=0.0, proj=g3, dose=d3, timing=True)
        tall = {"workload": wt3.name, "storage": "bf16 projections and dose, fp32 sums",
                "samples_per_pass": spp3, "adjoint_ms": r3["adjoint_ms"], "forward_ms": r3["forward_ms"],
                "samples_per_s": 2 * spp3 / ((r3["adjoint_ms"] + r3["forward_ms"] + r3["update_ms"]) / 1e3),
                "adjoint_samples_per_s": spp3 / (r3["adjoint_ms"] / 1e3)}
        del P3, f3, m3, g3, d3

    # ---- time to target, on its own (smaller) workload: plain FP32 optimiser vs variants ----
    ttt = None
    if args.ttt_iters > 0:
        wt = I.WORKLOADS[args.ttt_workload]
        Pt = P if wt.name == w.name else vamrt.Projector.from_workload(wt, I.workload_pupil(wt))
        tt = target if wt.name == w.name else torch.from_numpy(I.make_target(wt)).to(dev)
        ttt = {"workload": wt.name}
        ttt.update(time_to_target(Pt, tt, wt, args.ttt_iters, beta=args.ttt_beta, mu=args.ttt_mu))
        del Pt, tt
        if not args.no_fins:
            from paper_2211_03516_gb300 import fins as FN
            ttt["fins"] = [FN.fins_experiment(n, beta=args.ttt_beta, mu=args.ttt_mu) for n in (9, 18)]
            from paper_2211_03516_gb300 import etendue as ET
            ttt["etendue"] = [ET.etendue_experiment(d, beta=args.ttt_beta, mu=args.ttt_mu, kind=k)
                              for k in ("csg", "csg_shells") for d in (2.5, 16.0)]
        if args.ws_train > 0:
            ttt["warm_start"] = warm_start_time_to_target(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = OracleSampler(w, pupil, target_np)
        rows = sample_rows(w, args.cpu_rows)
        # a row's samples are the same at every angle (the ray table is angle-invariant)
        n_angle = S.samples(rows)
        angles = sorted({(i * w.n_angles) // args.cpu_angles for i in range(args.cpu_angles)})
        dt, threads = 0.0, 1
        for kk in angles:
            t, threads = S.run(rows, angle=kk)
            dt += t
        S.close()
        n = n_angle * len(angles)
        cpu = {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_rows} pixel rows x {w.nu} columns x {w.rays_per_pixel} rays at {len(angles)} "
                         f"evenly spaced angles (of {w.nv} rows x {w.n_angles} angles), projection then dose, FP64 "
                         f"oracle on {threads} worker processes ({n} samples, {dt:.1f} s)"}

    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.vol_shape), "angles": w.n_angles,
                   "pixels": [w.nv, w.nu], "rays_per_pixel": w.rays_per_pixel,
                   "step": "one optimiser iteration: projection (A^T) + clamp + dose (A) + normalise/update",
                   "samples_per_pass": spp, "units_per_step": units_per_step,
                   "l2": f"inputs larger than L2 (model, target, projections, dose, scratch: "
                         f"{(4 * math.prod(w.vol_shape) + math.prod(w.proj_shape)) * 4 / 1e9:.2f} GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "setup_s": round(setup_s, 3)},
        "phase_ms_per_step": {"adjoint": adj_ms / args.steps, "forward": fwd_ms / args.steps,
                              "update": upd_ms / args.steps},
        "samples_per_s": {"adjoint": world * spp * args.steps / (adj_ms / 1e3),
                          "forward": world * spp * args.steps / (fwd_ms / 1e3),
                          "note": "per operator, CUDA events around each launch inside the timed steps"},
        "roofline": {"kernel": dom, "bound": "smem", "achieved": achieved, "peak": smem_bps / 1e9, "unit": "GB/s",
                     "frac": achieved * 1e9 / smem_bps, "traffic": traffic,
                     "peak_kind": "measured in this run (vamrt_measure_smem_bandwidth)",
                     "bytes_per_sample": BYTES_PER_SAMPLE,
                     "l2_measured": {"read_GBps": l2_read_bps / 1e9, "red_v4_ops_per_s": l2_red_ops},
                     "l2": l2,
                     "per_kernel": kern,
                     "forward_sample_fraction": fwd_spp / spp,
                     "hbm": {"compulsory_bytes": compulsory, "achieved": compulsory / (dom_ms / 1e3) / 1e9,
                             "peak": hbm, "frac": compulsory / (dom_ms / 1e3) / 1e9 / hbm,
                             "peak_kind": peak_kind}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": host_target.numel() * 4,
                "d2h_bytes_per_step": host_proj.numel() * 4 + 8},
        "tall_build_bf16": tall,
        "time_to_target": ttt,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vamrt", choices=["vamrt", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--angles", type=int, default=0, help="override the angle count (small profiling cases)")
    ap.add_argument("--nz", type=int, default=0, help="override the grid's plane count (small profiling cases)")
    ap.add_argument("--nv", type=int, default=0, help="override the pixel row count (small profiling cases)")
    ap.add_argument("--cpu-rows", type=int, default=64)
    ap.add_argument("--cpu-angles", type=int, default=16,
                    help="angles of the CPU-baseline sample (about 20 s of oracle work on 16 host cores)")
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--no-tall", dest="tall", action="store_false",
                    help="skip the BF16-storage iteration on the 384x384x512 tall-build workload")
    ap.add_argument("--ttt-workload", default=TTT_WORKLOAD,
                    help="workload of the time-to-target comparison (its own projector)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ttt-beta", type=float, default=4.0,
                    help="model step of the over-relaxed optimiser variant in the time-to-target comparison")
    ap.add_argument("--no-fins", action="store_true",
                    help="skip the fin-part (9 and 18 fins) and etendue (2.5 and 16 mm iris) comparisons")
    ap.add_argument("--ttt-mu", type=float, default=0.5,
                    help="heavy-ball momentum of the over-relaxed optimiser variant")
    ap.add_argument("--ttt-iters", type=int, default=30,
                    help="optimiser iterations of the time-to-target comparison (0 = skip)")
    ap.add_argument("--ws-train", type=int, default=256, help="warm-start training targets (0 = skip)")
    ap.add_argument("--ws-epochs", type=int, default=8)
    ap.add_argument("--ws-eval", type=int, default=10, help="held-out targets for the warm-start comparison")
    ap.add_argument("--ws-loss-lr", type=float, default=0.8,
                    help="Adam step of the warm start's thresholded-loss continuation (x mean projection)")
    ap.add_argument("--ws-loss-dl", type=float, default=0.8,
                    help="lower dose threshold d_l of the warm start's thresholded-loss continuation (d_h = 1)")
    ap.add_argument("--ws-loss-iters", type=int, default=20,
                    help="iterations of the warm start's thresholded-loss continuation")
    ap.add_argument("--network-only", action="store_true",
                    help="time the warm-start network's convolutions alone and print their JSON")
    ap.add_argument("--warmstart-only", action="store_true",
                    help="run only the learned warm-start comparison (--ws-train pairs, --ws-eval held-out "
                         "targets) and print its JSON")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.network_only:
        run_network_only(args)
    elif args.warmstart_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(warm_start_time_to_target(args)), flush=True)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
