#!/usr/bin/env python
"""Throughput of scan integration (points integrated per second) on GB300.

Workload: the urban LiDAR sequence — 100 scans of 64 beams x 2048 azimuths
(131,072 points per scan, ~120k valid, ranges 1-80 m) ray-cast in a seeded
synthetic street, 0.1 m voxels, 0.3 m truncation, 20 classes (closed-set
one-hot Dirichlet counts). One step = empty the map (slim_map_reset) and
integrate all 100 scans with one slim_integrate_batch call (up to 64 scans
per launch of the autotuned strategy) with inputs resident in HBM (1.2 GB per
step, larger than L2, so every step streams from HBM).

Prints one JSON line. Extra keys: roofline (dominant kernel, algorithmic
bytes from the oracle's stored per-scan counts / CUDA-event kernel time in
the timed region), e2e (the same step from pinned host buffers with the
host-to-device traffic and a D2H read of the map counters inside the timed
region: slim_integrate_host per scan, and the batched call reading the
pinned arrays in place; the faster is reported), cpu_baseline (the oracle on
a bounded sample, host cores), variants (per-scan calls, other strategies),
clocks.

--impl reference times the oracle (plain sequential CPU restatement) on
this host; --workload selects the secondary lines (room, indoor, adjoint,
batch, render).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "points integrated/s (TSDF+Bayes semantic), % HBM roofline, plain vs chosen"
UNIT = "points/s"
COUNTS = os.path.join(ROOT, "tests", "golden", "street_lidar_counts.json")
INDOOR_COUNTS = os.path.join(ROOT, "tests", "golden", "indoor_rgbd_counts.json")
ROOM_COUNTS = os.path.join(ROOT, "tests", "golden", "room_lidar_counts.json")
BATCH_COUNTS = os.path.join(ROOT, "tests", "golden", "batch_counts.json")
ADJOINT_COUNTS = os.path.join(ROOT, "tests", "golden", "adjoint_counts.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
K_CLASSES = 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)  # ~0.1 s timed: clocks sampled inside it
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scans", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--strategy", choices=["auto", "direct", "hash"], default="auto",
                    help="closed-set strategy of the chosen path: autotuned (default) or fixed "
                         "(profiling runs pin it: timing under a profiler misleads the autotuner)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the per-scan and other-strategy lines (for profiling runs)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="0: same as --steps (max 10)")
    ap.add_argument("--workload", choices=["street", "room", "indoor", "adjoint", "batch", "render"],
                    default="street", help="street (default, the headline line) or a "
                    "secondary configuration, each printing its own JSON line")
    ap.add_argument("--frames", type=int, default=200, help="indoor: RGB-D frames per step")
    ap.add_argument("--voxel-capacity", type=int, default=400_000,
                    help="indoor: voxel rows reserved per map")
    ap.add_argument("--block-capacity", type=int, default=65536,
                    help="street: 8^3 blocks reserved per map (100 scans use ~26k)")
    return ap.parse_args()


def workload_config(n_scans):
    return {"workload": f"street-lidar {n_scans} scans x 64x2048 (131072 pts/scan), "
                        "voxel 0.1 m, trunc 0.3 m, 20 classes one-hot",
            "scans": n_scans, "points_per_scan": 131072, "voxel_size": 0.1, "trunc": 0.3,
            "classes": K_CLASSES, "semantics": "closed-set one-hot Dirichlet",
            "l2": "inputs larger than L2 (1.21 GB per step)", "parallelism": "replicas"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- helpers
def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's time (replicas: the job ends with its last rank)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws, units_per_rank, ms_max):
    """Whole-job throughput of ws independent replicas: all units processed
    over the slowest rank's time."""
    return ws * units_per_rank / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.marks = {}

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, name):
        self.marks[name] = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        t0, t1 = self.marks.get("t0", 0), self.marks.get("t1", 1e30)
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for _, l in self.lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in rows:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def open_algorithmic_bytes(n_frames, L, bf16):
    """Open-set integration: B = N_all*12 + N_valid*4l + (2*U_old + U_new)*R
    + U_b*16 per frame, R = 8 + 8l (FP32 mean and beta) or 8 + 4l (BF16), with
    the counts of the oracle's pair generator; None when the stored counts
    do not cover n_frames frames."""
    try:
        with open(INDOOR_COUNTS) as f:
            rows = json.load(f)["scans"]
    except (OSError, KeyError, ValueError):
        return None
    if len(rows) < n_frames:
        return None
    R = 8 + (4 if bf16 else 8) * L
    return sum(r["points"] * 12 + r["valid"] * 4 * L +
               (2 * (r["voxels"] - r["new_voxels"]) + r["new_voxels"]) * R + r["blocks"] * 16
               for r in rows[:n_frames])


def algorithmic_bytes(counts, n_scans, K=K_CLASSES):
    """B = N_all*12 + N_valid*4K + (2*U_old + U_new)*R + U_b*16 per scan,
    R = 8 + 4K bytes (D, W, K counts)."""
    R = 8 + 4 * K
    out = []
    for row in counts["scans"][:n_scans]:
        old = row["voxels"] - row["new_voxels"]
        out.append(row["points"] * 12 + row["valid"] * 4 * K +
                   (2 * old + row["new_voxels"]) * R + row["blocks"] * 16)
    return out


STRATEGY = {0: ("k_fuse_direct", "fuse_direct.cu",
                 "slim_integrate_batch: up to 64 scans per grid, direct per-pair red.add into "
                 "L2-resident records")}
HASH_STRATEGY = ("k_fuse_hash_persistent", "fuse_hash.cu",
                 "slim_integrate_batch: up to 64 scans per persistent launch, shared-memory "
                 "(voxel, class) hash tiles of {} points")


def strategy(tile):
    """(dominant kernel, its source file, path description) for the autotuned
    strategy (0 = direct reductions, else hash tiles of that many points)."""
    if tile == 0:
        return STRATEGY[0]
    return HASH_STRATEGY[0], HASH_STRATEGY[1], HASH_STRATEGY[2].format(tile)


def kernel_source_sha(src="fuse_direct.cu"):
    """Hash of the sources of the dominant kernel."""
    h = hashlib.sha256()
    for f in (src, "closed_common.cuh", "common.cuh", "geometry.cuh", "hash.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2512_12945_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel, src):
    try:
        with open(TRAFFIC) as f:
            t = json.load(f).get(kernel, {})
        if t.get("source_sha") == kernel_source_sha(src):
            return t.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def cpu_oracle_rate(w, n_scans):
    """The oracle as it stands, on the first n_scans of the workload."""
    import oracle
    m = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                         min_range=w.min_range, max_range=w.max_range,
                         body_from_sensor=w.body_from_sensor)
    t = time.perf_counter()
    valid = 0
    for s in w.scans[:n_scans]:
        valid += m.integrate(s["pts"], s["pose"], s["sem"])
    dt = time.perf_counter() - t
    return valid / dt, dt, valid


# --------------------------------------------------------------- reference
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2512_12945_gb300 import synth
    n = args.steps + args.warmup
    w = synth.street_lidar(n_scans=min(n, args.scans))
    import oracle
    times, valids = [], []
    for k in range(n):
        s = w.scans[k % len(w.scans)]
        m = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                             min_range=w.min_range, max_range=w.max_range,
                             body_from_sensor=w.body_from_sensor)
        t = time.perf_counter()
        v = m.integrate(s["pts"], s["pose"], s["sem"])
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            valids.append(v)
    tot = sum(times)
    value = sum(valids) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.scans),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one full 64x2048 scan into an empty map per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2512_12945_gb300 import build, slim, synth
    if rank == 0 or ws == 1:
        build.build()
    if dist:
        dist.barrier()
    L = slim.lib()

    w = synth.street_lidar(n_scans=args.scans)
    agg = {"auto": "auto", "direct": "direct", "hash": "hash"}[args.strategy]
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                 min_range=w.min_range, max_range=w.max_range, body_from_sensor=w.body_from_sensor,
                 block_capacity=args.block_capacity, hash_capacity=1 << 21,
                 max_points=131072, aggregation=agg, tile_points=256 if agg == "hash" else 0)
    h = m.handle
    pts = [torch.from_numpy(s["pts"]).cuda() for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda() for s in w.scans]
    if args.strategy == "auto":
        tile = m.autotune(pts[len(pts) // 2], w.scans[len(pts) // 2]["pose"], sem[len(pts) // 2])
    else:
        tile = 0 if args.strategy == "direct" else 256
    kname, ksrc, kpath = strategy(tile)
    poses = [np.ascontiguousarray(np.asarray(s["pose"], np.float64).reshape(16)) for s in w.scans]
    args_c = [(ctypes.c_void_p(p.data_ptr()), p.shape[0], po.ctypes.data_as(ctypes.c_void_p),
               ctypes.c_void_p(se.data_ptr())) for p, se, po in zip(pts, sem, poses)]
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    # the whole 100-scan sequence as one batch (up to 64 scans per launch)
    items = (slim.slim_batch_item * len(args_c))()
    for k, (a, po) in enumerate(zip(args_c, poses)):
        items[k].map = h
        items[k].pts_dev = a[0]
        items[k].n = a[1]
        for q in range(16):
            items[k].pose[q] = float(po[q])
        items[k].sem_dev = a[3]

    def step():
        L.slim_map_reset(h, sp)
        rc = L.slim_integrate_batch(items, len(args_c), sp)
        if rc:
            raise slim.SlimError(rc, L.slim_last_error().decode())

    def step_plain():
        L.slim_map_reset(h, sp)
        for a in args_c:
            rc = L.slim_integrate(h, a[0], a[1], a[2], a[3], sp)
            if rc:
                raise slim.SlimError(rc, L.slim_last_error().decode())

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    for _ in range(args.warmup):
        step()
    m.sync()
    slim.slim_profile_enable(h, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("t0")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.mark("t1")
    ms = ev0.elapsed_time(ev1)
    prof = slim.slim_profile_read(h)
    slim.slim_profile_enable(h, False)
    m.sync()
    clocks.stop()
    stats = m.stats()

    ms_max = max_over_ranks(ms, dist)

    counts = None
    try:
        with open(COUNTS) as f:
            counts = json.load(f)
    except OSError:
        pass
    if counts is not None:
        valid_per_step = sum(r["valid"] for r in counts["scans"][:args.scans])
    else:
        valid_per_step = int(sum(int((np.linalg.norm(s["pts"], axis=1) >= w.min_range).sum())
                                 for s in w.scans))
    value = replica_rate(ws, valid_per_step * args.steps, ms_max)

    # roofline of the dominant kernel (the batched integration kernel of the
    # autotuned strategy): algorithmic bytes of the scans one launch
    # integrates / its CUDA-event time, averaged over the launches of the
    # timed region
    roof = None
    peak, peak_kind = measured_peak()
    if counts is not None and "batch" in prof:
        nl, kms = prof["batch"]
        B = algorithmic_bytes(counts, args.scans)
        bytes_per_launch = sum(B) * args.steps / nl
        avg_ms = kms / nl
        achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": stored_traffic(kname, ksrc),
                "kernel": kname, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": int(bytes_per_launch),
                "scans_per_launch": round(args.scans * args.steps / nl, 2),
                "avg_launch_ms": round(avg_ms, 5),
                "path_frac": round(sum(B) * args.steps / (ms / 1e3) / 1e9 / peak, 4)}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    n_e2e = args.e2e_steps or min(args.steps, 10)
    # the scans stacked in pinned host memory (every scan has the same number
    # of points)
    npts = max(s["pts"].shape[0] for s in w.scans)
    assert all(s["pts"].shape[0] == npts for s in w.scans)
    pts_h = torch.from_numpy(np.stack([s["pts"] for s in w.scans])).pin_memory()
    sem_h = torch.from_numpy(np.stack([s["sem"] for s in w.scans])).pin_memory()
    st_c = slim.slim_stats()
    h2d = pts_h.numel() * 4 + sem_h.numel() * 4

    # (a) slim_integrate_host per scan: the library copies each scan into one
    # of its two staging buffers on its own copy stream while the previous
    # scan integrates; (b) the same batched call as the device-resident step,
    # its items pointing at the pinned host arrays, which the kernels read in
    # place over the host link (no staging copy)
    zitems = (slim.slim_batch_item * len(w.scans))()
    for k in range(len(w.scans)):
        zitems[k].map = h
        zitems[k].pts_dev = pts_h[k].data_ptr()
        zitems[k].n = npts
        for q in range(16):
            zitems[k].pose[q] = float(poses[k][q])
        zitems[k].sem_dev = sem_h[k].data_ptr()
    hargs = [(ctypes.c_void_p(pts_h[k].data_ptr()), npts, args_c[k][2],
              ctypes.c_void_p(sem_h[k].data_ptr())) for k in range(len(w.scans))]

    def step_host():
        L.slim_map_reset(h, sp)
        for a in hargs:
            rc = L.slim_integrate_host(h, a[0], a[1], a[2], a[3], sp)
            if rc:
                raise slim.SlimError(rc, L.slim_last_error().decode())
        rc = L.slim_map_stats(h, ctypes.byref(st_c), sp)  # D2H of the map counters
        if rc:
            raise slim.SlimError(rc, L.slim_last_error().decode())

    def step_zero_copy():
        L.slim_map_reset(h, sp)
        rc = L.slim_integrate_batch(zitems, len(w.scans), sp)
        if rc:
            raise slim.SlimError(rc, L.slim_last_error().decode())
        rc = L.slim_map_stats(h, ctypes.byref(st_c), sp)
        if rc:
            raise slim.SlimError(rc, L.slim_last_error().decode())

    def time_e2e(fn):
        fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), dist)

    e2e_var = {}
    for name, fn, call in (
            ("host_copy", step_host,
             "slim_map_reset + slim_integrate_host per scan (the library's double-buffered "
             "H2D copies on its copy stream, overlapped with the previous scan's integration) "
             "+ slim_map_stats"),
            ("zero_copy", step_zero_copy,
             "slim_map_reset + slim_integrate_batch on the pinned host arrays (the kernels "
             "read points and probabilities in place over the host link) + slim_map_stats")):
        e_ms = time_e2e(fn)
        e2e_var[name] = {"value": replica_rate(ws, valid_per_step * n_e2e, e_ms), "unit": UNIT,
                         "ms_per_step": e_ms / n_e2e, "call": call}
    best = max(e2e_var, key=lambda k: e2e_var[k]["value"])
    e2e = {"value": e2e_var[best]["value"], "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 8 * 4, "steps": n_e2e, "call": e2e_var[best]["call"],
           "variants": e2e_var}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_cpu = min(64, args.scans)  # about 10 s of single-threaded oracle work
        rate, dt, nv = cpu_oracle_rate(w, n_cpu)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_cpu} scans of the workload ({nv} valid points), "
                         f"{dt:.1f} s single-threaded"}

    # plain path (one slim_integrate per scan) and the other aggregation
    # strategy on the same workload ("plain vs chosen")
    variants = {}
    for _ in range(2):
        step_plain()
    torch.cuda.synchronize()
    npl = max(2, min(args.steps, 5))
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(npl):
        step_plain()
    p1.record(stream)
    torch.cuda.synchronize()
    pms = p0.elapsed_time(p1) / npl
    variants["plain"] = {"value": valid_per_step / (pms / 1e3), "ms_per_step": pms, "steps": npl,
                         "path": "slim_integrate per scan, " + ("direct reductions" if tile == 0
                                                                else f"hash tiles of {tile}")}
    # the other strategies, each on its own map: the sort aggregation and
    # both closed one-hot strategies per scan and batched
    paths = {"sort": ("sort", 0, "slim_integrate per scan, CTA radix sort + segmented reduction"),
             "direct": ("direct", 0, "slim_integrate per scan, direct per-pair red.add"),
             "direct_batch": ("direct", 0, "slim_integrate_batch, up to 64 scans per grid, direct "
                                           "per-pair red.add"),
             "hash": ("hash", 256, "slim_integrate per scan, shared-memory hash tiles of 256"),
             "hash_batch": ("hash", 256, "slim_integrate_batch, up to 64 scans per persistent launch, "
                                         "shared-memory hash tiles of 256")}
    for var in (() if args.no_variants else ("sort", "direct", "direct_batch", "hash",
                                              "hash_batch")):
        agg, tp, _ = paths[var]
        mv = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                      min_range=w.min_range, max_range=w.max_range,
                      body_from_sensor=w.body_from_sensor, block_capacity=args.block_capacity,
                      hash_capacity=1 << 21, max_points=131072, aggregation=agg, tile_points=tp)
        hv = mv.handle
        vitems = (slim.slim_batch_item * len(args_c))()
        for k in range(len(args_c)):
            vitems[k] = items[k]
            vitems[k].map = hv

        def step_v():
            L.slim_map_reset(hv, sp)
            if var.endswith("_batch"):
                L.slim_integrate_batch(vitems, len(args_c), sp)
            else:
                for a in args_c:
                    L.slim_integrate(hv, a[0], a[1], a[2], a[3], sp)

        for _ in range(2):
            step_v()
        torch.cuda.synchronize()
        nv = max(2, min(args.steps, 5))
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(nv):
            step_v()
        a1.record(stream)
        torch.cuda.synchronize()
        mv.sync()
        vms = a0.elapsed_time(a1) / nv
        variants[var] = {"value": valid_per_step / (vms / 1e3), "ms_per_step": vms, "steps": nv,
                         "path": paths[var][2]}
        mv.close()

    launches = sum(v[0] for v in prof.values())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.scans), "roofline": roof, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clocks.summary(), "gpu_launches": launches,
            "kernels_ms": {k: round(v[1], 3) for k, v in prof.items()},
            "path": kpath, "tile_points": tile,
            "variants": variants,
            "map": {"blocks": stats["blocks"],
                    "oracle_voxels": counts["meta"]["total_voxels"] if counts else None}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------- other configs
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def _indoor_geometry(f):
    """Frame f of the indoor RGB-D workload: points (sensor frame), pose and
    per-pixel object labels (the embeddings are drawn on the device)."""
    import numpy as np
    from paper_2512_12945_gb300 import synth
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=8, frames=[f])
    s = w.scans[0]
    return s["pts"], s["pose"], s["labels"].astype(np.int32)


def run_indoor(args):
    """Open-set RGB-D frames (640x480, l = 512), FP32 vs BF16 storage, and the
    tensor-core query of 256 embeddings against every voxel of the map."""
    import multiprocessing as mp
    import numpy as np
    nf = args.frames
    # the frames' geometry on the host cores, before the first GPU call
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        geo = pool.map(_indoor_geometry, range(nf))
    import torch
    from paper_2512_12945_gb300 import build, slim, synth
    build.build()
    torch.cuda.set_device(0)
    cents = synth.indoor_centroids(3, 512)
    pts = [torch.from_numpy(g[0]).cuda() for g in geo]
    sem = [synth.indoor_embeddings_device(torch.from_numpy(g[2]).cuda().long(), cents, 3, f)
           for f, g in enumerate(geo)]
    poses = [g[1] for g in geo]
    valid = sum(int((np.linalg.norm(g[0], axis=1) >= 0.3).sum()) for g in geo)
    fpx = 525.0
    depths = [torch.from_numpy(np.ascontiguousarray(g[0][:, 2].reshape(480, 640),
                                                    np.float32)).cuda() for g in geo]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    hbm_peak, hbm_kind = measured_peak()
    out = {}
    for storage in ("f32", "bf16"):
        m = slim.Map(voxel_size=0.05, trunc=0.15, mode="open", embed_dim=512,
                     embed_storage=storage, min_range=0.3, max_range=8.0,
                     max_points=640 * 480, block_capacity=200000, hash_capacity=1 << 20,
                     voxel_capacity=args.voxel_capacity, image_width=640)
        tile_w = m.autotune(pts[0], poses[0], sem[0])  # tile shape of the open-set kernel

        def step():
            m.reset()
            for p, q, pose in zip(pts, sem, poses):
                m.integrate(p, pose, q)

        def step_depth():  # the same frames as z-depth images (RGB-D front end)
            m.reset()
            for dimg, q, pose in zip(depths, sem, poses):
                m.integrate_depth(dimg, fpx, fpx, 320.0, 240.0, pose, q)

        for _ in range(args.warmup):
            step_depth()
        dms = _timed(step_depth, args.steps, 0, stream)
        for _ in range(args.warmup):
            step()
        slim.slim_profile_enable(m.handle, True)
        ms = _timed(step, args.steps, 0, stream)
        prof = slim.slim_profile_read(m.handle)
        slim.slim_profile_enable(m.handle, False)
        m.sync()
        rows = m.stats()["voxels"]
        q = torch.from_numpy(synth.random_queries(7, 256, 512)).to(torch.bfloat16).cuda()
        for _ in range(args.warmup):
            m.query(q, 0.01, 0.1)
        slim.slim_profile_enable(m.handle, True)
        qms = _timed(lambda: m.query(q, 0.01, 0.1), args.steps, 0, stream)
        qprof = slim.slim_profile_read(m.handle)
        slim.slim_profile_enable(m.handle, False)
        nq, qkms = qprof.get("query", (1, qms))
        kq = qkms / max(nq, 1)
        flops = 2.0 * rows * 512 * 256
        peak, kind = _bf16_peak()
        B = open_algorithmic_bytes(nf, 512, storage == "bf16")
        kern = {k: v[1] / args.steps for k, v in prof.items()}
        integ = kern.get("open_tile", 0.0) + kern.get("open_apply", 0.0)
        roof = None if B is None else {
            "bound": "hbm", "achieved": round(B / (ms / 1e3) / 1e9, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(B / (ms / 1e3) / 1e9 / hbm_peak, 4),
            "peak_source": hbm_kind, "algorithmic_bytes_per_step": B,
            "kernels_frac": round(B / (integ / 1e3) / 1e9 / hbm_peak, 4) if integ else None,
            "scope": "a step: map reset + one slim_integrate per frame (k_open_tile, "
                     "k_open_apply); kernels_frac: the same bytes over the two kernels' "
                     "event time alone"}
        out[storage] = {"points_per_s": valid / (ms / 1e3), "ms_per_step": ms,
                        "autotuned_tile_width": tile_w,
                        "ms_per_frame": ms / nf, "voxels": rows, "integrate_roofline": roof,
                        "depth_front_end": {"ms_per_step": dms,
                                            "points_per_s": valid / (dms / 1e3),
                                            "call": "slim_integrate_depth per frame"},
                        "kernels_ms_per_step": kern,
                        "query": {"rows": rows, "ms": qms, "kernel_ms": kq,
                                  "tflops": flops / (kq / 1e3) / 1e12,
                                  "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s",
                                               "frac": flops / (kq / 1e3) / 1e12 / peak,
                                               "peak_source": kind},
                                  "hbm_gbs": rows * (2 * 512 + 8) / (kq / 1e3) / 1e9}}
        m.close()
    del sem
    torch.cuda.empty_cache()
    # the oracle as it stands on the first frames (FP64 NIG updates, one
    # observation at a time; numpy-drawn embeddings of the same distribution)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        wc = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=512,
                               frames=[0, 1])
        om = oracle.OracleMap(voxel_size=wc.voxel_size, trunc=wc.trunc, mode=oracle.OPEN,
                              embed_dim=512, min_range=wc.min_range, max_range=wc.max_range,
                              body_from_sensor=wc.body_from_sensor)
        t = time.perf_counter()
        nv = sum(om.integrate(s["pts"], s["pose"], s["sem"]) for s in wc.scans)
        dt = time.perf_counter() - t
        cpu = {"value": nv / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": f"first {len(wc.scans)} frames ({nv} valid pixels), {dt:.1f} s "
                         "single-threaded"}
    # the query kernel at a size where it is a real contraction: 2^20 BF16
    # rows of l = 512 against 256 queries, caller-held rows
    gen = torch.Generator(device="cuda").manual_seed(11)
    nrow = 1 << 20
    rows = torch.randn(nrow, 512, device="cuda", generator=gen).to(torch.bfloat16)
    qb = torch.from_numpy(synth.random_queries(7, 256, 512)).to(torch.bfloat16).cuda()
    lab = torch.empty(nrow, dtype=torch.int32, device="cuda")
    prb = torch.empty(nrow, dtype=torch.float32, device="cuda")
    sms = _timed(lambda: slim.slim_query_rows_static(rows, qb, 0.01, 0.1, lab, prb),
                 args.steps, args.warmup, stream)
    peak, kind = _bf16_peak()
    flops = 2.0 * nrow * 512 * 256
    big = {"rows": nrow, "l": 512, "queries": 256, "ms": sms,
           "tflops": flops / (sms / 1e3) / 1e12,
           "tensor_frac": flops / (sms / 1e3) / 1e12 / peak, "tensor_peak": peak,
           "hbm_gbs": nrow * 512 * 2 / (sms / 1e3) / 1e9,
           "hbm_frac": nrow * 512 * 2 / (sms / 1e3) / 1e9 / hbm_peak,
           "peak_source": kind,
           "call": "slim_query_rows_static (row norms + tcgen05 GEMM + epilogue; waits for "
                   "its stream)"}
    line = {"metric": "open-set points integrated/s (NIG, l=512) and query TFLOP/s",
            "value": out["bf16"]["points_per_s"], "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f32 accumulate, bf16 storage", "data": "synthetic",
            "config": {"workload": f"indoor-rgbd {nf} frames 640x480, l=512, voxel 0.05 m, "
                                   "trunc 0.15 m, 256 queries T=0.01",
                       "inputs": "all frames resident in HBM (126 GB of embeddings at 200 "
                                 "frames), larger than L2"},
            "storage": out, "query_1M_rows": big, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """Forward integration + reverse mode on the room scene with 64 x 2048
    scans, soft counts (20 classes)."""
    import numpy as np
    import torch
    from paper_2512_12945_gb300 import autograd, build, slim, synth
    build.build()
    torch.cuda.set_device(0)
    w = synth.room_lidar(seed=4, n_scans=20, n_beams=64, n_az=2048, K=20, mode="soft")
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="soft", num_classes=20,
                 min_range=w.min_range, max_range=w.max_range, max_points=131072,
                 block_capacity=100000, hash_capacity=1 << 20)
    pts = [torch.from_numpy(s["pts"]).cuda().requires_grad_(True) for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda().requires_grad_(True) for s in w.scans]
    poses = [s["pose"] for s in w.scans]
    rng = np.random.default_rng(4)
    stream = torch.cuda.current_stream()
    state = {}

    def fwd():
        D, W, c, ijk = autograd.integrate(m, poses, pts, sem)
        state["out"] = (D, c)

    def fwd_bwd(stored=False):
        D, W, c, ijk = autograd.integrate(m, poses, pts, sem, stored=stored)
        n = D.shape[0]
        if "sel" not in state or state["n"] != n:
            state["n"] = n
            state["sel"] = torch.from_numpy(rng.choice(n, min(10000, n), replace=False)).cuda()
            state["y"] = torch.from_numpy(rng.integers(0, 20, min(10000, n))).cuda()
        sel, y = state["sel"], state["y"]
        post = (1.0 + c[sel]) / (20.0 + c[sel].sum(1, keepdim=True))
        loss = (D[sel] ** 2).sum() + torch.nn.functional.nll_loss(torch.log(post), y, reduction="sum")
        for t in pts + sem:
            t.grad = None
        loss.backward()

    # the forward alone with each soft-count strategy (sort tiles, direct
    # vector reductions) on maps of their own
    fwd_by = {}
    for agg in ("sort", "direct"):
        mv = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="soft", num_classes=20,
                      min_range=w.min_range, max_range=w.max_range, max_points=131072,
                      block_capacity=100000, hash_capacity=1 << 20, aggregation=agg)
        det = [(p.detach(), q.detach()) for p, q in zip(pts, sem)]

        def integ():
            mv.reset()
            for (p, q), po in zip(det, poses):
                mv.integrate(p, po, q)

        fwd_by[agg] = _timed(integ, args.steps, args.warmup, stream)
        mv.close()
    fms = _timed(fwd, args.steps, args.warmup, stream)
    tms = _timed(fwd_bwd, args.steps, args.warmup, stream)
    # the stored form: the forward keeps each scan's pair list (CSR by point,
    # 4 B per pair and per point), the backward reads it
    sms_ = _timed(lambda: fwd_bwd(stored=True), args.steps, args.warmup, stream)
    fwd()
    rec_ms = _timed(lambda: [m.record_pairs(p.detach(), po) for p, po in zip(pts, poses)],
                    args.steps, 1, stream)
    lists = [m.record_pairs(p.detach(), po) for p, po in zip(pts, poses)]
    list_bytes = sum(4 * (o.numel() + v.numel()) for o, v in lists)
    list_pairs = sum(v.numel() for _, v in lists)
    del lists

    def peak_of(stored):
        """Device memory the forward + backward allocates above the inputs,
        from the same clean state for both forms (no gradients, no outputs
        held, allocator cache emptied)."""
        for t in pts + sem:
            t.grad = None
        state.pop("out", None)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        fwd_bwd(stored=stored)
        torch.cuda.synchronize()
        return torch.cuda.max_memory_allocated() - base

    peak = peak_of(False)
    peak_s = peak_of(True)
    valid = sum(int((np.linalg.norm(s["pts"], axis=1) >= w.min_range).sum()) for s in w.scans)
    # recompute vs stored, both measured; the oracle's pair count beside them
    mem = {"saved_for_backward": "inputs only; (voxel, point) pairs recomputed",
           "torch_peak_bytes_above_inputs": int(peak),
           "stored": {"saved_for_backward": "inputs + each scan's pair list (slim_record_pairs: "
                                            "CSR offsets and a uint32 voxel index per pair)",
                      "pair_list_bytes": int(list_bytes), "pairs": int(list_pairs),
                      "torch_peak_bytes_above_inputs": int(peak_s),
                      "forward_backward_ms": sms_, "record_pairs_ms": rec_ms,
                      "backward_ms": sms_ - fms - rec_ms}}
    try:
        with open(ADJOINT_COUNTS) as f:
            pairs = sum(r["pairs"] for r in json.load(f)["scans"])
        mem.update({"oracle_pairs": pairs})
    except (OSError, KeyError, ValueError):
        pass
    line = {"metric": "differentiable integration: points/s forward, forward+backward",
            "value": valid / (tms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "room 20 scans x 64x2048, 20 classes soft counts, loss = "
                                   "sum D^2 + CE on 10k sampled voxels"},
            "forward_ms": fms, "forward_backward_ms": tms, "backward_ms": tms - fms,
            "integrate_ms_by_strategy": fwd_by,
            "memory": mem}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """16 independent maps — 8 closed-set (64 beams, 20k-250k points per scan)
    and 8 open-set (256-dim, 320x240 to 640x480, BF16) — 10 scans each per
    step, integrated by one slim_integrate_batch call captured in a CUDA
    graph (closed-set strategies from the autotuner)."""
    import numpy as np
    import torch
    from paper_2512_12945_gb300 import build, slim, synth
    build.build()
    torch.cuda.set_device(0)
    n_scans = 10
    closed, opened = synth.batch_workload(seed=5, n_scans=n_scans)
    maps, items, valid, tiles = [], [], 0, []
    for w in closed:
        m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=20,
                     min_range=w.min_range, max_range=w.max_range,
                     body_from_sensor=w.body_from_sensor, max_points=262144,
                     block_capacity=60000, hash_capacity=1 << 19)
        s0 = w.scans[0]
        tiles.append(m.autotune(torch.from_numpy(s0["pts"]).cuda(), s0["pose"],
                                torch.from_numpy(s0["sem"]).cuda()))
        maps.append(m)
    open_tiles = []
    for w in opened:
        m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="open", embed_dim=256,
                     embed_storage="bf16", min_range=w.min_range, max_range=w.max_range,
                     max_points=w.scans[0]["pts"].shape[0], voxel_capacity=300000,
                     block_capacity=60000, hash_capacity=1 << 18, image_width=w.image_width)
        s0 = w.scans[0]
        open_tiles.append(m.autotune(torch.from_numpy(s0["pts"]).cuda(), s0["pose"],
                                     torch.from_numpy(s0["sem"]).cuda()))
        maps.append(m)
    for m, w in zip(maps, closed + opened):
        for s in w.scans:
            items.append((m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                          torch.from_numpy(s["sem"]).cuda()))
            valid += int((np.linalg.norm(s["pts"], axis=1) >= w.min_range).sum())
    stream = torch.cuda.current_stream()

    def eager():
        for m in maps:
            m.reset()
        slim.slim_integrate_batch(items)

    eager()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        eager()
    ems = _timed(eager, args.steps, args.warmup, stream)
    gms = _timed(graph.replay, args.steps, args.warmup, stream)
    # kernel time per step by kind (eager run, events on the launch stream)
    for m in maps:
        slim.slim_profile_enable(m.handle, True)
    eager()
    kern = {}
    for m in maps:
        for k, v in slim.slim_profile_read(m.handle).items():
            kern[k] = kern.get(k, 0.0) + v[1]
        slim.slim_profile_enable(m.handle, False)
    for m in maps:
        m.sync()
    # whole-step roofline (resets + the batch call, graph replay): algorithmic
    # bytes of every map's scans from the oracle's per-scan counts; closed
    # maps R = 8 + 4K, open maps (BF16 m and beta) R = 8 + 4l
    roof = None
    try:
        with open(BATCH_COUNTS) as f:
            bc = json.load(f)["maps"]
        B = 0
        for mp in bc:
            sin = 4 * mp["width"]
            R = 8 + 4 * mp["width"]
            for r in mp["scans"]:
                B += (r["points"] * 12 + r["valid"] * sin +
                      (2 * (r["voxels"] - r["new_voxels"]) + r["new_voxels"]) * R +
                      r["blocks"] * 16)
        peak, kind = measured_peak()
        roof = {"bound": "hbm", "achieved": round(B / (gms / 1e3) / 1e9, 1), "peak": peak,
                "unit": "GB/s", "frac": round(B / (gms / 1e3) / 1e9 / peak, 4),
                "peak_source": kind, "algorithmic_bytes_per_step": B,
                "scope": "16 map resets + one slim_integrate_batch (graph replay)"}
    except (OSError, KeyError, ValueError):
        pass
    line = {"metric": "batched points integrated/s (16 uneven maps, closed + open)",
            "value": valid / (gms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32 / bf16 storage",
            "data": "synthetic",
            "config": {"workload": "8 closed-set maps (64 beams x 320-3900 azimuths, 20 classes) "
                                   "+ 8 open-set maps (256-dim, 320x240..640x480, bf16), "
                                   f"{n_scans} scans each per step"},
            "graph_ms_per_step": gms, "eager_ms_per_step": ems, "points_per_step": valid,
            "autotuner": {"closed": {"choices": tiles,
                                     "meaning": "0 = direct reductions, else hash-tile points"},
                          "open": {"choices": open_tiles,
                                   "meaning": "tile width in pixels (tiles of 256 pixels)"}},
            "kernels_ms_per_step": kern, "roofline": roof}
    print(json.dumps(line), flush=True)
    return 0


def run_room(args):
    """The small room configuration: 10 scans of 16 x 512 (8,192 points)."""
    import numpy as np
    import torch
    from paper_2512_12945_gb300 import build, slim, synth
    build.build()
    torch.cuda.set_device(0)
    w = synth.room_lidar(seed=1, n_scans=10)
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=10,
                 min_range=w.min_range, max_range=w.max_range, max_points=8192)
    pts = [torch.from_numpy(s["pts"]).cuda() for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda() for s in w.scans]
    items = [(m, p, s["pose"], q) for p, q, s in zip(pts, sem, w.scans)]
    stream = torch.cuda.current_stream()

    def plain():
        m.reset()
        for p, q, s in zip(pts, sem, w.scans):
            m.integrate(p, s["pose"], q)

    def batched():
        m.reset()
        slim.slim_integrate_batch(items)

    pms = _timed(plain, args.steps, args.warmup, stream)
    bms = _timed(batched, args.steps, args.warmup, stream)
    m.sync()
    valid = sum(int((np.linalg.norm(s["pts"], axis=1) >= w.min_range).sum()) for s in w.scans)
    # whole-call roofline of the batched form (all 10 scans in one launch),
    # algorithmic bytes from the oracle's per-scan counts
    roof = None
    try:
        with open(ROOM_COUNTS) as f:
            counts = json.load(f)
        B = sum(algorithmic_bytes(counts, len(w.scans), K=w.num_classes))
        peak, kind = measured_peak()
        roof = {"bound": "hbm", "achieved": round(B / (bms / 1e3) / 1e9, 1), "peak": peak,
                "unit": "GB/s", "frac": round(B / (bms / 1e3) / 1e9 / peak, 4),
                "peak_source": kind, "algorithmic_bytes_per_step": B,
                "scope": "slim_map_reset + slim_integrate_batch of the 10 scans"}
    except (OSError, KeyError, ValueError):
        pass
    cpu = None
    if not args.no_cpu_baseline:
        rate, dt, nv = cpu_oracle_rate(w, len(w.scans))
        cpu = {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": f"all {len(w.scans)} scans ({nv} valid points), {dt:.2f} s "
                         "single-threaded"}
    line = {"metric": "points integrated/s (room, 10 scans x 16x512)", "value": valid / (bms / 1e3),
            "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "room 10x10x3 m + 6 objects, 10 scans x 16x512, 10 classes"},
            "plain_ms_per_step": pms, "batched_ms_per_step": bms, "roofline": roof,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_render(args):
    """Ray-cast renders of the 100-scan street map at the paper's image sizes
    (691 x 256 and 1209 x 448, Sec. IV Rendering), camera in the street."""
    import numpy as np
    import torch
    from paper_2512_12945_gb300 import build, slim, synth
    build.build()
    torch.cuda.set_device(0)
    w = synth.street_lidar(n_scans=100)
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                 min_range=w.min_range, max_range=w.max_range, body_from_sensor=w.body_from_sensor,
                 block_capacity=65536, hash_capacity=1 << 21, max_points=131072)
    items = [(m, torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
             for s in w.scans]
    slim.slim_integrate_batch(items)
    m.sync()
    T = np.eye(4)
    T[:3, :3] = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    T[:3, 3] = [20.0, 0.0, 1.73]
    stream = torch.cuda.current_stream()
    out = {}
    for (W, H) in ((691, 256), (1209, 448)):
        f = 0.5 * W / np.tan(np.deg2rad(45.0))  # 90 degree horizontal field of view
        fn = lambda: m.render(T, f, f, W / 2, H / 2, W, H, 0.1, 80.0)  # noqa: E731
        for _ in range(args.warmup):
            r = fn()
        slim.slim_profile_enable(m.handle, True)
        ms = _timed(fn, args.steps, 0, stream)
        prof = slim.slim_profile_read(m.handle)
        slim.slim_profile_enable(m.handle, False)
        nl, kms = prof.get("render", (1, ms))
        hit = float(torch.isfinite(r["depth"]).float().mean())
        out[f"{W}x{H}"] = {"ms": ms, "kernel_ms": kms / max(nl, 1), "hit_fraction": hit,
                           "rays_per_s": W * H / (kms / max(nl, 1) / 1e3)}
    line = {"metric": "ray-cast render time per image (TSDF zero crossing + label)",
            "value": out["691x256"]["kernel_ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "street-lidar map after 100 scans (64x2048, voxel 0.1 m), "
                                   "camera at 1.73 m looking down the street, 90 deg HFOV, "
                                   "near 0.1 m far 80 m"},
            "images": out,
            "paper_context": "paper: 2.1 ms (691x256) and 3.9 ms (1209x448) on its own GPU"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "street":
        return {"room": run_room, "indoor": run_indoor, "adjoint": run_adjoint,
                "batch": run_batch, "render": run_render}[args.workload](args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
