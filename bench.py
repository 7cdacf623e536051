#!/usr/bin/env python
"""Benchmark of the SSLIC hot path on GB300.

One step = one pass of the whole method through the C ABI (sslic_run):
seeding with gradient perturbation, the iterated assign/update loop and
connectivity enforcement, over one synthetic image already resident in HBM.
The default workload is the 3-D RGB uint8 volume 2048x1216x1871 (14 GB,
S = 16, K = 1,138,176, m = 10, 10 iterations, connectivity on).

Metric: Gvoxel-iterations/s = voxels x iterations / step time (device time,
CUDA events on the launching stream, max over ranks).  Printed as one JSON
line with the roofline of the dominant kernel (its launches timed live with
CUDA events by the library's profiler), the end-to-end figure through the
host-buffer entry point (H2D image + D2H labels inside the timed region),
SM clocks sampled during the timed region and the CPU oracle timed on a
bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: launched by torch.distributed.run, one rank per GPU; every rank
segments its own copy of the workload (independent problems, weak scaling,
no data-path collective).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "rgb3d_2048x1216x1871"
METRIC = "Gvoxel-iters/s"
UNIT = "Gvoxel-iter/s"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of the dominant kernel at the default workload, from the ncu capture
# summarised in profiles/, keyed by the SHA-256 of the kernel's source file:
# a changed kernel reports null until it is profiled again.
TRAFFIC_BYTES = {
    # ncu capture of the tile kernel on the 67.1 M-voxel profiling workload
    # (rgb3d_512x512x256): 206.2 MB read + 225.5 MB written per launch,
    # scaled by the voxel ratio (69.4x) to the 4.66 G-voxel launch
    ("rgb3d_2048x1216x1871", "bc81787ef88466b1964886573ecca2996ff0453c8da63d6ecedb5a6a778b0edb"):
        (206.220032e6 + 225.464576e6) * (2048 * 1216 * 1871) / (512 * 512 * 256),
}

# thread instructions per voxel of the dominant kernel (ncu
# smsp__inst_executed.sum x 32 / voxels on the profiling workload), keyed by
# the SHA-256 of the kernel's source file like TRAFFIC_BYTES
INST_PER_VOXEL = {
    # 493,095,965 warp instructions x 32 / 67,108,864 voxels (the capture above)
    "bc81787ef88466b1964886573ecca2996ff0453c8da63d6ecedb5a6a778b0edb": 493095965 * 32 / (512 * 512 * 256),
}


def _sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the slowest rank sets the job's time);
    x itself when running alone."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, voxels, iters, seconds):
    """Whole-job Gvoxel-iterations/s: every rank segments its own image of
    `voxels` voxels for `iters` iterations in `seconds` (the max over ranks)."""
    return world * voxels * iters / seconds / 1e9


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = list(csv.reader(open(self.path)))
        finally:
            os.unlink(self.path)
        if len(rows) < 2:
            return None
        head = [h.strip() for h in rows[0]]
        sm, mx, reasons = [], [], set()
        names = {"clocks_event_reasons.hw_slowdown": "hw_slowdown",
                 "clocks_event_reasons.hw_thermal_slowdown": "hw_thermal_slowdown",
                 "clocks_event_reasons.sw_thermal_slowdown": "sw_thermal_slowdown",
                 "clocks_event_reasons.sw_power_cap": "sw_power_cap"}
        for r in rows[1:]:
            if len(r) != len(head):
                continue
            d = {h: v.strip() for h, v in zip(head, r)}
            try:
                sm.append(float(d["clocks.current.sm [MHz]"].split()[0]))
                mx.append(float(d["clocks.max.sm [MHz]"].split()[0]))
            except (KeyError, ValueError):
                continue
            for k, nm in names.items():
                if d.get(k, "").startswith("Active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def host_cores():
    """Host cores this process may run on, and the CPU model if known."""
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Architecture"):
                model += (", " if model else "") + ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return n, model


def oracle_sample(w, edge, threads=None):
    """The corner crop [0, edge)^n of the workload's image, run by the oracle
    with the workload's parameters: single-threaded (threads None), or in the
    paper's region-decomposed form on `threads` host threads (same results)."""
    import numpy as np

    import oracle
    from paper_1806_08741_gb300 import inputs

    ext = tuple(min(edge, s) for s in w.image.size)
    img = inputs.make_image(w.image, origin=(0,) * w.image.ndim, extent=ext)
    p = oracle.params_for(img, w.grid, m=w.m, max_iter=w.max_iter, perturb=w.perturb,
                          enforce_connectivity=w.connectivity)
    t0 = time.perf_counter()
    r = oracle.slic(p, img) if threads is None else oracle.slic_regions(p, img, threads)
    dt = time.perf_counter() - t0
    vox = int(np.prod(ext))
    form = ("single-threaded C oracle" if threads is None else
            f"C oracle in the paper's region-decomposed form (Sec. 3.1) on {threads} host threads, "
            "connectivity sequential")
    desc = (f"corner crop {'x'.join(map(str, ext))} of the same image (K={oracle.num_clusters(p)}), "
            f"{w.max_iter} iterations + {'connectivity' if w.connectivity else 'no connectivity'}, "
            f"{form}, {dt:.1f} s")
    return vox * r["iterations"] / dt / 1e9, desc, dt


def run_reference(args, w):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    steps = []
    desc = ""
    cores, model = host_cores()
    for i in range(args.warmup + args.steps):
        v, desc, dt = oracle_sample(w, args.reference_edge, threads=cores)
        if i >= args.warmup:
            steps.append((v, dt))
    val = statistics.median(v for v, _ in steps)
    ms = statistics.median(dt for _, dt in steps) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": _config(w),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                         "host": model},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(w):
    img = w.image
    return {"workload": w.name, "size": list(img.size), "channels": img.channels,
            "image_dtype": img.dtype, "grid": list(w.grid), "m": w.m, "iterations": w.max_iter,
            "perturb": w.perturb, "connectivity": w.connectivity,
            "regions": int(__import__("numpy").prod(img.sites())), "noise_sigma": img.sigma,
            "l2": "inputs larger than L2 (image and labels exceed the 129 MB L2)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, w):
    import numpy as np
    import torch

    from paper_1806_08741_gb300 import inputs
    from paper_1806_08741_gb300 import sslic as S

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    spec = w.image
    tdt = torch.uint8 if spec.dtype == "u8" else torch.uint16
    img = torch.empty(spec.shape, dtype=tdt, device=dev)
    inputs.make_image_device(spec, img.data_ptr(), stream.cuda_stream)
    labels = torch.empty(spec.shape[:-1], dtype=torch.int32, device=dev)
    p = S.params_for(img, w.grid, m=w.m, max_iter=w.max_iter, perturb=w.perturb,
                     enforce_connectivity=w.connectivity)
    ctx = S.Context(p)
    centres = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device=dev)
    V = spec.voxels
    # launch configuration: measured tile shape (before any timed work)
    tune = None
    if args.tile_shape is not None:
        ctx.tile_shape = args.tile_shape
        info_s = S.tile_shape_info(p.ndim, args.tile_shape)
        tune = {"shape": args.tile_shape, "dims": info_s["dims"], "voxels_per_lane": info_s["voxels_per_lane"],
                "tma_staged": info_s["tma_staged"], "ms_per_shape": None}
    elif not args.no_autotune:
        t = ctx.autotune(img, labels, reps=2, stream=stream)
        info_s = S.tile_shape_info(p.ndim, t["best"])
        tune = {"shape": t["best"], "dims": info_s["dims"], "voxels_per_lane": info_s["voxels_per_lane"],
                "tma_staged": info_s["tma_staged"], "ms_per_shape": t["ms"]}

    for _ in range(args.warmup):
        info = ctx.run(img, labels, centres, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        info = ctx.run(img, labels, centres, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    if dist:
        dist.barrier()
    iters = info["iterations"]
    value = job_throughput(world, V, iters, ms_step / 1e3)

    # roofline of the dominant kernel: the fused assign + update tile kernel
    esz = 1 if spec.dtype == "u8" else 2
    bytes_per_vox = spec.channels * esz + 4
    a_ms, a_calls = prof["assign"]
    peak, peak_src = _peaks()
    roof = None
    if a_calls:
        avg_s = a_ms / a_calls / 1e3
        algo = V * bytes_per_vox
        achieved = algo / avg_s / 1e9
        src = _sha(os.path.join(ROOT, "paper_1806_08741_gb300", "csrc", "assign_tile.cuh"))
        roof = {"kernel": "assign_tile_kernel (fused assign + map-update)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"of {peak_src}", "bytes_per_launch": algo,
                "bytes_per_voxel": bytes_per_vox, "avg_launch_ms": a_ms / a_calls,
                "traffic": TRAFFIC_BYTES.get((w.name, src)),
                "traffic_note": "ncu DRAM read + write of one launch on the 67.1 M-voxel profiling workload, scaled by "
                                "the voxel ratio; labels still in the L2 when that launch ends are written back after "
                                "it, so the write side is undercounted: a check that the image is read once, not a "
                                "full count of the launch's writes"}
    # the same kernel against the SM's FP32 lanes, the unit that bounds it:
    # per (voxel, covering centre) pair the canonical D^2 costs C subtractions,
    # C products and C - 1 + n sums once the per-axis terms are tabulated per
    # tile, plus one comparison; a voxel is covered by prod_d (2 S_d) K / V
    # windows on average; peak = the device's SMs x 128 FP32 lanes x the
    # median SM clock sampled during the timed region.  Beside it, the
    # instruction-issue fraction: the kernel's thread instructions per voxel
    # (ncu capture, keyed like the traffic) against 4 warp instructions per
    # SM and clock
    roof_alu = None
    if a_calls:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        cover = float(np.prod([2 * s_ for s_ in w.grid])) * ctx.K / V
        ops_pair = 2 * spec.channels + (spec.channels - 1) + spec.ndim + 1
        alu_peak = sms * 128 * mhz * 1e6 / 1e12
        t_launch = a_ms / a_calls / 1e3
        ach = V * cover * ops_pair / t_launch / 1e12
        roof_alu = {"kernel": roof["kernel"], "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": ach / alu_peak, "ops_per_voxel": cover * ops_pair, "covering_centres_per_voxel": cover,
                    "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (median sampled SM clock)"}
        ipv = INST_PER_VOXEL.get(src)
        if ipv:
            issue_peak = sms * 4 * 32 * mhz * 1e6  # thread instructions per second
            roof_alu["issue"] = {"thread_inst_per_voxel": ipv, "frac": V * ipv / t_launch / issue_peak,
                                 "source": "ncu smsp__inst_executed.sum x 32 / voxels of the profiling capture"}
    phases = {k: {"ms_per_step": v[0] / args.steps, "calls_per_step": v[1] / args.steps}
              for k, v in prof.items() if k in S.PHASES}
    # the iterated assign/update loop alone (bins + assignment + reduction),
    # seeding and connectivity excluded
    loop_ms = sum(prof[k][0] for k in ("bins", "assign", "assign_voxel", "finalize")) / args.steps
    loop = {"value": V * iters / (loop_ms / 1e3) / 1e9 if loop_ms > 0 else None, "unit": UNIT,
            "ms_per_step": loop_ms}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        h_img = torch.empty(spec.shape, dtype=tdt, pin_memory=True)
        h_img.copy_(img)
        h_lab = torch.empty(spec.shape[:-1], dtype=torch.int32, pin_memory=True)
        h_cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, pin_memory=True)
        ctx.run_host(h_img, h_lab, h_cen, stream=stream)   # warm-up (allocates device buffers)
        torch.cuda.synchronize()
        # this machine's host link on the same buffers, to read the end-to-end
        # figure against (h_img holds the device image, so the upload
        # rewrites it unchanged; the label download is overwritten below)
        link = {}
        for name, dst, src in (("h2d", img, h_img), ("d2h", h_lab, labels)):
            l0 = torch.cuda.Event(enable_timing=True)
            l1 = torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            dst.copy_(src, non_blocking=True)
            l1.record(stream)
            torch.cuda.synchronize()
            link[name + "_gbs"] = src.numel() * src.element_size() / (l0.elapsed_time(l1) / 1e3) / 1e9
        if dist:
            dist.barrier()
        n_e2e = max(1, min(args.steps, 3))
        calls = []
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            t1 = time.perf_counter()
            ctx.run_host(h_img, h_lab, h_cen, stream=stream)   # returns after its stream drained
            calls.append((time.perf_counter() - t1) * 1e3)
        dt = max_over_ranks((time.perf_counter() - t0) / n_e2e, dist, dev)
        same = bool(torch.equal(h_lab, labels.cpu()))
        e2e = {"value": job_throughput(world, V, iters, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(h_img.numel() * h_img.element_size()),
               "d2h_bytes_per_step": int(h_lab.numel() * 4 + h_cen.numel() * 4),
               "ms_per_step": dt * 1e3, "ms_per_call": calls, "labels_equal_device_run": same,
               "host_link": link}
        del h_img, h_lab, h_cen

    streamed = None
    if rank == 0 and world == 1 and not args.no_streamed:
        streamed = streamed_bench(w, img, args.slab_planes)

    lab = None
    if rank == 0 and world == 1 and not args.no_lab and spec.dtype == "u8" and spec.channels == 3:
        lab = lab_bench(w, img, labels, steps=max(3, min(args.steps, 5)), warmup=1)

    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = precision_bench(steps=max(3, args.steps))

    small = None
    if rank == 0 and world == 1 and not args.no_small:
        small = small_configs_bench()

    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        ctx.close()
        del img, labels, centres
        torch.cuda.empty_cache()
        pool = serving_pool()
        serving = {
            # the arrival rate of the stream's recipe: more than either form serves
            "overloaded": serving_bench(n_req=args.serve_requests, rate=200.0, max_active=args.serve_max_active,
                                        pool=pool),
            # a rate both forms keep up with
            "under_capacity": serving_bench(n_req=args.serve_requests_low, rate=args.serve_rate_low,
                                            max_active=args.serve_max_active, pool=pool),
            # the same rate with connectivity enforced on every request
            "under_capacity_connectivity": serving_bench(n_req=args.serve_requests_conn, rate=args.serve_rate_low,
                                                         max_active=args.serve_max_active, pool=pool,
                                                         connectivity=True),
        }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores, model = host_cores()
        v, desc, _ = oracle_sample(w, args.cpu_edge_all, threads=cores)
        v1, desc1, _ = oracle_sample(w, args.cpu_edge)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc, "host": model,
               "cores_1": {"value": v1, "unit": UNIT, "cores": 1, "sample": desc1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**_config(w), "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "num_labels": info["num_labels"], "K": info["num_clusters"]},
            "tile_shape": tune, "assign_update_loop": loop,
            "roofline": roof, "roofline_alu": roof_alu, "phases": phases, "e2e": e2e, "cpu_baseline": cpu, "serving": serving,
            "precision": precision, "lab": lab, "streamed": streamed, "small_configs": small,
            "gpu_launches": prof["kernel_launches"], "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# streamed form: the image in host memory, streamed through the GPU in slabs
# ---------------------------------------------------------------------------
def streamed_bench(w, img, slab_planes, runs=2):
    """The workload through sslic_run_streamed (the out-of-device-memory form;
    no connectivity enforcement): the image stays in page-locked host memory
    and every iteration uploads it slab by slab; the last iteration's labels
    come back.  Whole runs timed on the host clock (the call is synchronous),
    with the labels checked against a resident run of the same parameters."""
    import torch

    from paper_1806_08741_gb300 import sslic as S

    spec = w.image
    V = spec.voxels
    h_img = torch.empty(spec.shape, dtype=img.dtype, pin_memory=True)
    h_img.copy_(img)
    h_lab = torch.empty(spec.shape[:-1], dtype=torch.int32, pin_memory=True)
    p = S.params_for(img, w.grid, m=w.m, max_iter=w.max_iter, perturb=w.perturb, enforce_connectivity=False)
    out = {"slab_planes": slab_planes, "connectivity": False}
    with S.Context(p) as ctx:
        h_cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, pin_memory=True)
        ctx.run_streamed(h_img, h_lab, h_cen, slab_planes=slab_planes)   # warm-up (allocates the slabs)
        ts = []
        for _ in range(runs):
            t0 = time.perf_counter()
            info = ctx.run_streamed(h_img, h_lab, h_cen, slab_planes=slab_planes)
            ts.append(time.perf_counter() - t0)
        dt = sorted(ts)[len(ts) // 2]
        lab = torch.empty(spec.shape[:-1], dtype=torch.int32, device=img.device)
        ctx.run(img, lab, torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device=img.device))
        same = bool(torch.equal(h_lab, lab.cpu()))
    it = info["iterations"]
    out.update({"value": V * it / dt / 1e9, "unit": UNIT, "ms_per_run": dt * 1e3, "iterations": it,
                "h2d_bytes_per_run": int(h_img.numel() * h_img.element_size()) * it,
                "d2h_bytes_per_run": int(h_lab.numel() * 4), "labels_equal_resident_run": same})
    del h_img, h_lab
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# colour input: the same volume converted to CIE-Lab float (the paper's data)
# ---------------------------------------------------------------------------
def lab_bench(w, rgb, labels, steps=3, warmup=1, shape=None):
    """The RGB workload converted on the device to CIE-Lab float (12 B per
    voxel) and segmented with the same parameters: the conversion's achieved
    bandwidth (3 B read + 12 B written per voxel), whole runs (iterations +
    connectivity) on the float image with the autotuned tile shape, and the
    assignment kernel's bandwidth at 12 + 4 B per voxel."""
    import torch

    from paper_1806_08741_gb300 import sslic as S

    spec = w.image
    V = spec.voxels
    stream = torch.cuda.current_stream()
    peak, peak_src = _peaks()
    img = torch.empty(spec.shape, dtype=torch.float32, device=rgb.device)
    S.srgb_to_lab(rgb, img, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    conv = []
    for _ in range(3):
        e0.record(stream)
        S.srgb_to_lab(rgb, img, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        conv.append(e0.elapsed_time(e1))
    c_ms = sorted(conv)[1]
    out = {"workload": "lab" + w.name[3:], "convert": {
        "ms": c_ms, "GBs": 15 * V / (c_ms / 1e3) / 1e9, "frac_hbm": 15 * V / (c_ms / 1e3) / 1e9 / peak,
        "bytes_per_voxel": 15, "peak_source": f"of {peak_src}"}}
    p = S.params_for(img, w.grid, m=w.m, max_iter=w.max_iter, perturb=w.perturb,
                     enforce_connectivity=w.connectivity)
    with S.Context(p) as ctx:
        cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device=rgb.device)
        if shape is None:
            t = ctx.autotune(img, labels, reps=2, stream=stream)
        else:
            ctx.tile_shape = shape
            t = {"best": shape, "ms": None}
        for _ in range(warmup):
            ctx.run(img, labels, cen, stream=stream)
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        e0.record(stream)
        for _ in range(steps):
            info = ctx.run(img, labels, cen, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ms = e0.elapsed_time(e1) / steps
        a_ms, a_calls = prof["assign"]
        achieved = V * 16 / (a_ms / a_calls / 1e3) / 1e9 if a_calls else None
        out.update({"value": V * info["iterations"] / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_run": ms,
                    "tile_shape": t["best"], "ms_per_shape": t["ms"],
                    "assign_ms_per_iter": a_ms / a_calls if a_calls else None, "assign_gbs": achieved,
                    "assign_frac_hbm": achieved / peak if achieved else None, "bytes_per_voxel": 16,
                    "connectivity_ms": prof["connectivity"][0] / steps, "num_labels": info["num_labels"]})
    del img
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# precision form: the 64-band float workload, exact FP32 vs BF16 tensor core
# ---------------------------------------------------------------------------
def precision_bench(steps=3, warmup=2):
    """hyper64_1024 (1024x1024 x 64 float32, S = 16, m = 0.1, 10 iterations):
    whole runs of the exact form (precision 0) and of the tensor-core form
    (precision 1), device time per run, the assignment kernel's achieved HBM
    bandwidth (C x 4 + 4 bytes per voxel), the share of voxels re-evaluated
    in exact FP32, and the label agreement of the two forms' final labels."""
    import numpy as np
    import torch

    from paper_1806_08741_gb300 import inputs
    from paper_1806_08741_gb300 import sslic as S

    w = inputs.WORKLOADS["hyper64_1024"]
    host = inputs.make_hyperspectral(size=w.float_image["size"], bands=w.float_image["bands"])
    img = torch.from_numpy(host).cuda()
    V = host.shape[0] * host.shape[1]
    C = host.shape[2]
    peak, peak_src = _peaks()
    out = {"workload": w.name, "size": list(reversed(host.shape[:2])), "channels": C, "grid": list(w.grid),
           "m": w.m, "iterations": w.max_iter}
    labs = {}
    stream = torch.cuda.current_stream()
    for prec in (0, 1):
        p = S.params_for(host, w.grid, m=w.m, max_iter=w.max_iter, perturb=w.perturb, precision=prec)
        with S.Context(p) as ctx:
            lab = torch.empty(host.shape[:2], dtype=torch.int32, device="cuda")
            cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
            for _ in range(warmup):
                ctx.run(img, lab, cen, stream=stream)
            torch.cuda.synchronize()
            ctx.profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.run(img, lab, cen, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            prof = ctx.profile_read()
            ms = e0.elapsed_time(e1) / steps
            a_ms, a_calls = prof["assign"]
            bpv = C * 4 + 4
            achieved = V * bpv / (a_ms / a_calls / 1e3) / 1e9 if a_calls else None
            labs[prec] = lab.cpu().numpy()
            out["fp32" if prec == 0 else "bf16_tcgen05"] = {
                "value": V * w.max_iter / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_run": ms,
                "assign_ms_per_iter": a_ms / a_calls if a_calls else None,
                "assign_gbs": achieved, "assign_frac_hbm": achieved / peak if achieved else None,
                "peak_source": f"of {peak_src}", "bytes_per_voxel": bpv,
                "rechecked_fraction": prof["rechecks"] / (V * w.max_iter * steps)}
    out["label_agreement"] = float((labs[0] == labs[1]).mean())
    del img
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# serving: request stream, continuous batching vs one image per launch
# ---------------------------------------------------------------------------
def small_configs_bench(reps=20, warmup=3):
    """Whole-run latency of the two 2-D workloads (256x256 RGB, K = 256, no
    connectivity; 2048x1216 RGB, K = 9728, connectivity on): seeding, 10
    iterations and connectivity through sslic_run on a device-resident image,
    CUDA events around each run; median and minimum of `reps` runs after
    `warmup`.  Both fit in the L2 (a few MB), so these are latency figures."""
    import statistics as st_

    import torch

    from paper_1806_08741_gb300 import inputs
    from paper_1806_08741_gb300 import sslic as S

    out = {}
    for name in ("rgb2d_256", "rgb2d_2048x1216"):
        w = inputs.WORKLOADS[name]
        spec = w.image
        img = torch.empty(spec.shape, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream()
        inputs.make_image_device(spec, img.data_ptr(), stream.cuda_stream)
        p = S.Params(size=spec.size, grid=w.grid, channels=spec.channels, dtype=S.U8, m=w.m,
                     max_iter=w.max_iter, perturb=w.perturb, enforce_connectivity=w.connectivity)
        ms = []
        with S.Context(p) as ctx:
            lab = torch.empty(spec.shape[:-1], dtype=torch.int32, device="cuda")
            cen = torch.empty((ctx.K, ctx.centre_width), dtype=torch.float32, device="cuda")
            for i in range(warmup + reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                info = ctx.run(img, lab, cen, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= warmup:
                    ms.append(a.elapsed_time(b))
        med = st_.median(ms)
        out[name] = {"ms_median": med, "ms_min": min(ms), "runs": reps,
                     "value": spec.voxels * w.max_iter / (med / 1e3) / 1e9, "unit": UNIT,
                     "K": info["num_clusters"], "num_labels": info["num_labels"],
                     "connectivity": w.connectivity}
    return out


def serving_pool(seed=1810, pool_n=12):
    """The request stream's input images: pool_n 2-D RGB uint8 tiles (side
    ~ U[256, 4096]) and pool_n 3-D uint16 blocks (side ~ U[128, 512]), made
    on the GPU and kept in page-locked host memory."""
    import numpy as np
    import torch

    from paper_1806_08741_gb300 import inputs

    rng = np.random.default_rng(seed)
    pool = []
    for i in range(pool_n):
        side = int(rng.integers(256, 4097))
        spec = inputs.ImageSpec((side, side), 3, "u8", seed * 10 + i, max(2, side * side // 3000), 6)
        pool.append(spec)
    for i in range(pool_n):
        side = int(rng.integers(128, 513))
        spec = inputs.ImageSpec((side, side, side), 1, "u16", seed * 10 + 100 + i,
                                max(2, side ** 3 // 20000), 300)
        pool.append(spec)
    host = []
    for spec in pool:
        dt = torch.uint8 if spec.dtype == "u8" else torch.uint16
        d = torch.empty(spec.shape, dtype=dt, device="cuda")
        inputs.make_image_device(spec, d.data_ptr(), torch.cuda.current_stream().cuda_stream)
        h = torch.empty(spec.shape, dtype=dt, pin_memory=True)
        h.copy_(d)
        host.append(h)
        del d
    torch.cuda.synchronize()
    return pool, host


def serving_bench(n_req=200, rate=200.0, seed=1810, budget_gb=48.0, pool_n=12, max_active=16, pool=None,
                  connectivity=False):
    """Poisson arrivals (rate per second) of requests over the images of
    serving_pool (2-D RGB uint8 and 3-D uint16), S in {8, 16, 32}, m in
    {5, 10, 20}, 10 iterations, connectivity enforced on every request when
    `connectivity` is set.  Returns latency percentiles and throughput of the
    served form (sslic_server_*) and of the plain form (one sslic_run_host
    call per request, in arrival order)."""
    import threading

    import numpy as np
    import torch

    from paper_1806_08741_gb300 import sslic as S

    pool, host = pool if pool is not None else serving_pool(seed, pool_n)
    pool_n = len(pool) // 2
    rng = np.random.default_rng(seed + int(rate))
    reqs = []
    t = 0.0
    for _ in range(n_req):
        t += float(rng.exponential(1.0 / rate))
        idx = int(rng.integers(0, 2 * pool_n))
        grid = int(rng.choice([8, 16, 32]))
        m = float(rng.choice([5.0, 10.0, 20.0]))
        reqs.append((t, idx, grid, m))

    def params(idx, grid, m):
        spec = pool[idx]
        return S.Params(size=spec.size, grid=(grid,) * spec.ndim, channels=spec.channels,
                        dtype=S.U8 if spec.dtype == "u8" else S.U16, m=m, max_iter=10,
                        enforce_connectivity=connectivity)

    # page-locked output buffers, made before the timed region and recycled
    lock = threading.Lock()
    out_pool = {i: [torch.empty(pool[i].shape[:-1], dtype=torch.int32, pin_memory=True) for _ in range(4)]
                for i in range(len(pool))}

    def out_buf(idx):
        with lock:
            if out_pool[idx]:
                return out_pool[idx].pop()
        return torch.empty(pool[idx].shape[:-1], dtype=torch.int32, pin_memory=True)

    def give_back(idx, buf):
        with lock:
            out_pool[idx].append(buf)

    vox_iters = sum(pool[i].voxels * 10 for _, i, _, _ in reqs)

    # served form: a submitter at the arrival times, a waiter recycling outputs
    res = {}
    with S.Server(int(budget_gb * (1 << 30)), max_active=max_active) as srv:
        import queue as _q
        handed = _q.Queue()
        lats = []

        def waiter():
            while True:
                item = handed.get()
                if item is None:
                    return
                tk, idx, lab = item
                lats.append(srv.wait(tk))
                give_back(idx, lab)

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for (ta, idx, grid, m) in reqs:
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            lab = out_buf(idx)
            handed.put((srv.submit(params(idx, grid, m), host[idx], lab), idx, lab))
        handed.put(None)
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
    res["served"] = {"p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
                     "mean_ms": float(np.mean(lats)), "throughput": vox_iters / wall / 1e9,
                     "wall_s": wall, "max_active": st["max_active"], "max_active_limit": max_active,
                     "rounds": st["rounds"],
                     "peak_gb": st["peak_bytes"] / 2 ** 30}

    # plain form: one request at a time, in arrival order
    lats = []
    t0 = time.perf_counter()
    for (ta, idx, grid, m) in reqs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        lab = out_buf(idx)
        with S.Context(params(idx, grid, m)) as ctx:
            ctx.run_host(host[idx], lab)
        lats.append((time.perf_counter() - t0 - ta) * 1e3)
        give_back(idx, lab)
    wall = time.perf_counter() - t0
    res["plain"] = {"p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
                    "mean_ms": float(np.mean(lats)), "throughput": vox_iters / wall / 1e9, "wall_s": wall}
    res["stream"] = {"requests": n_req, "rate_per_s": rate, "iterations": 10, "connectivity": connectivity,
                     "mix": "1/2 2-D RGB u8 side U[256,4096], 1/2 3-D u16 side U[128,512]; S in {8,16,32}; m in {5,10,20}",
                     "inputs": f"{2 * pool_n} pool images", "offered_gvox_iter_s": vox_iters / reqs[-1][0] / 1e9,
                     "unit": UNIT}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the built-in tile shape")
    ap.add_argument("--tile-shape", type=int, default=None, help="fix the tile shape (no autotuning)")
    ap.add_argument("--no-precision", action="store_true", help="skip the 64-band float workload")
    ap.add_argument("--precision-only", action="store_true", help="only the 64-band float workload")
    ap.add_argument("--no-lab", action="store_true", help="skip the CIE-Lab float form of the workload")
    ap.add_argument("--no-streamed", action="store_true", help="skip the streamed (host-resident image) form")
    ap.add_argument("--slab-planes", type=int, default=128, help="planes per slab of the streamed form")
    ap.add_argument("--lab-only", action="store_true",
                    help="only the CIE-Lab float form of the workload (--tile-shape fixes its shape)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-edge", type=int, default=256, help="edge of the single-core CPU-baseline crop")
    ap.add_argument("--cpu-edge-all", type=int, default=384, help="edge of the all-cores CPU-baseline crop")
    ap.add_argument("--reference-edge", type=int, default=256,
                    help="edge of the crop each reference-arm step runs")
    ap.add_argument("--serve", action="store_true",
                    help="only the request-stream benchmark (served vs plain form)")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-stream benchmark")
    ap.add_argument("--no-small", action="store_true", help="skip the latency of the two 2-D workloads")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the overloaded stream")
    ap.add_argument("--serve-requests-low", type=int, default=1000, help="requests of the under-capacity stream")
    ap.add_argument("--serve-rate-low", type=float, default=60.0, help="arrivals per second, under capacity")
    ap.add_argument("--serve-requests-conn", type=int, default=500,
                    help="requests of the under-capacity stream with connectivity enforced")
    ap.add_argument("--serve-max-active", type=int, default=16, help="requests the server advances at once")
    args = ap.parse_args()
    if args.lab_only:
        import torch

        from paper_1806_08741_gb300 import inputs
        w = inputs.WORKLOADS[args.workload]
        spec = w.image
        torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        rgb = torch.empty(spec.shape, dtype=torch.uint8, device="cuda")
        inputs.make_image_device(spec, rgb.data_ptr(), torch.cuda.current_stream().cuda_stream)
        labels = torch.empty(spec.shape[:-1], dtype=torch.int32, device="cuda")
        out = lab_bench(w, rgb, labels, steps=args.steps, warmup=args.warmup, shape=args.tile_shape)
        print(json.dumps({"lab": out}), flush=True)
        return 0
    if args.precision_only:
        print(json.dumps({"precision": precision_bench(steps=max(3, args.steps))}), flush=True)
        return 0
    if args.serve:
        import torch
        torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        pool = serving_pool()
        out = {"overloaded": serving_bench(n_req=args.serve_requests, rate=200.0, max_active=args.serve_max_active,
                                           pool=pool),
               "under_capacity": serving_bench(n_req=args.serve_requests_low, rate=args.serve_rate_low,
                                               max_active=args.serve_max_active, pool=pool),
               "under_capacity_connectivity": serving_bench(n_req=args.serve_requests_conn, rate=args.serve_rate_low,
                                                            max_active=args.serve_max_active, pool=pool,
                                                            connectivity=True)}
        print(json.dumps({"serving": out}), flush=True)
        return 0
    from paper_1806_08741_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
