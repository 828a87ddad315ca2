#!/usr/bin/env python3
"""Benchmark of the scan-to-map registration hot path on one GB300.

Workload: the high-speed sequence - a 128-beam x 2048-azimuth spinning LiDAR
(~260k points per scan, 0.03 m range noise) moving at 70 m/s, 10 Hz (7 m per
frame) around a walled oval track. One step = one scan through the whole path:
ingest, scan-local downsampling and Eq. 1 covariances, Gauss-Newton GICP
registration (at most 10 iterations, ||xi|| <= 5e-3), adaptive threshold update,
ASMD-capped insert at the registered pose with added-point covariances, and
eviction beyond 150 m. v = 0.5 m, N_max = 20, k = 5.

Inputs are synthetic (seeded ray casting) and resident in HBM before timing;
the e2e pass feeds the same scans from pinned host memory through the public
API. L2 (129 MB) is flushed between timed steps by writing a 256 MiB buffer.

`--impl reference` times the CPU oracle (plain FP64 C++) on the host instead.
Multi-GPU: one independent vehicle per rank (replicas, no data-path collective).
"""
from __future__ import annotations

import argparse
import csv
import dataclasses
import hashlib
import io
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Mpoints/s at 128x2048 beams (high-speed sequence, per-scan register+map update)"
UNIT = "Mpoints/s"
V, NMAX, K_COV = 0.5, 20, 5
R_NEAR, R_MAX, EVICT_R = 10.0, 200.0, 150.0
MAX_ITERS, CONV_EPS = 10, 5e-3
SIGMA0, MIN_MOTION = 2.0, 0.1
MAX_SCAN = 300_000
MAX_VOXELS = 1 << 19        # 0.5 M voxels (10 M points at N = 20); the map holds ~0.05 M
PRIOR_NOISE = (0.05, 0.1)   # IMU-like prior: metres, degrees per frame


def workload_config(steps, warmup, n_gpus):
    return {
        "workload": "high-speed sequence: 128x2048 LiDAR (~260k pts/scan, sigma 0.03 m), 70 m/s at 10 Hz "
                    "on a walled oval (700 m straights, R 120 m), per-scan register + ASMD insert + evict",
        "voxel_m": V, "n_max": NMAX, "k_cov": K_COV, "gn_max_iters": MAX_ITERS, "conv_eps": CONV_EPS,
        "asmd": {"r_near_m": R_NEAR, "r_max_m": R_MAX}, "evict_radius_m": EVICT_R,
        "threshold": {"sigma0_m": SIGMA0, "min_motion_m": MIN_MOTION},
        "init_prior": "true inter-frame motion + seeded noise (%.2f m, %.1f deg)" % PRIOR_NOISE,
        "scans_timed": steps, "scans_warmup": warmup, "first_scan": "inserted at its true pose (setup)",
        "l2": "flushed between timed steps (256 MiB write)", "inputs": "device-resident before timing",
        "parallelism": "replicas" if n_gpus > 1 else "single GPU",
    }


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sequence", "single", "batched", "serving"], default="sequence",
                    help="sequence: the 128x2048 high-speed sequence (default); batched: 64 uneven problems; "
                         "serving: 16 vehicles streaming scans")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: simulated seconds")
    ap.add_argument("--precision", type=int, choices=[0, 1], default=None,
                    help="1 = tile-relative points, FP16 covariances (precision_mode 1); default: 0 for the "
                         "sequence, 1 for the batched workload")
    ap.add_argument("--world-offset", type=str, default="0,0,0",
                    help="sequence: metres added to every pose (x,y,z), e.g. 2000,1500,0 for km-scale coordinates")
    ap.add_argument("--accuracy-scans", type=int, default=None,
                    help="per-scan pose error vs the FP64 oracle over this many scans (default 6 with --precision 1)")
    ap.add_argument("--autotune", action="store_true", help="batched: tune v, lanes per point and load factor first")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=3)
    ap.add_argument("--max-voxels", type=int, default=MAX_VOXELS,
                    help="bucket pool of the map (smaller values shrink the device footprint for profiling)")
    return ap.parse_args()


def aggregate_ranks(dev_s: float, pts: float, world: int, device: str):
    """Whole-job figures of a replicated run: the slowest rank's time and every rank's points."""
    if world <= 1:
        return dev_s, pts
    import torch
    import torch.distributed as dist
    tt = torch.tensor([dev_s, pts], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def rank_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# --------------------------------------------------------------------------------------- inputs
class Vehicle:
    """One simulated vehicle on the oval: scans, true poses (optionally moved by a world
    offset) and the motion prior."""

    def __init__(self, rank: int, offset=(0.0, 0.0, 0.0)):
        self.seq = synth.TrackSequence(seed=42 + rank, s0=300.0 * rank)
        self.rng = np.random.default_rng(1000 + rank)
        self.shift = synth.make_pose(np.eye(3), np.asarray(offset, float))

    def pose(self, t: int) -> np.ndarray:
        return self.shift @ self.seq.pose(t)

    def prior(self, t: int, prev_est: np.ndarray, rng=None) -> np.ndarray:
        """IMU-like prediction: previous estimate times the true motion, with seeded noise."""
        d = np.linalg.inv(self.seq.pose(t - 1)) @ self.seq.pose(t)
        return prev_est @ d @ synth.random_offset(rng or self.rng, PRIOR_NOISE[1], PRIOR_NOISE[0])


def rot_angle(R):
    return math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))


# --------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out)) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------------------- roofline inputs
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gicp.cu", "search.cuh", "far_internal.cuh", "gicp.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2606_26010_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per k_gn_lin launch from the committed ncu summary, if it matches the source."""
    p = os.path.join(ROOT, "profiles", "k_gn_lin_hbm_128x2048.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# --------------------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2606_26010_gb300 import build as far_build
    from paper_2606_26010_gb300 import far

    rank, world, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    far_build.build()
    stream = torch.cuda.Stream()
    offset = [float(x) for x in args.world_offset.split(",")]
    args.precision = args.precision or 0
    veh = Vehicle(rank, offset)
    n_total = 1 + args.warmup + args.steps
    scans = [veh.seq.scan(t) for t in range(n_total)]
    dev = [torch.from_numpy(s).cuda() for s in scans]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def make_map():
        with torch.cuda.stream(stream):
            m = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=args.max_voxels, load_factor=0.5,
                             max_scan_points=MAX_SCAN, precision_mode=args.precision, stream=stream.cuda_stream)
            m.insert(dev[0], veh.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
        return m

    def step(m, thr, t, est, inp):
        init = veh.prior(t, est)
        tau, kappa = thr.get()
        pose, _, res = m.process_scan(inp, init, max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=tau, kappa=kappa,
                                      asmd=True, r_near=R_NEAR, r_max=R_MAX, evict_radius=EVICT_R)
        thr.update(init, pose)
        return pose, res

    # ---- device-resident pass (value): no profiling events inside the library, so the
    # programmatically dependent launches overlap as they do in use
    m = make_map()
    thr = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    est = veh.pose(0)
    with torch.cuda.stream(stream):
        for t in range(1, 1 + args.warmup):
            est, _ = step(m, thr, t, est, dev[t])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms, results, ests = [], [], {args.warmup: est}
    launches_in_steps = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for t in range(1 + args.warmup, n_total):
                flush.zero_()
                l0 = far.launch_count()
                ev0.record(stream)
                est, res = step(m, thr, t, est, dev[t])
                ev1.record(stream)
                ev1.synchronize()
                launches_in_steps += far.launch_count() - l0
                step_ms.append(ev0.elapsed_time(ev1))
                results.append(res)
                ests[t] = est
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    rpe = []     # per-frame relative pose error of the estimates against the true motion
    for t in range(1 + args.warmup, n_total):
        D = np.linalg.inv(np.linalg.inv(veh.pose(t - 1)) @ veh.pose(t)) @ (np.linalg.inv(ests[t - 1]) @ ests[t])
        rpe.append((float(np.linalg.norm(D[:3, 3])), rot_angle(D[:3, :3])))

    # ---- profiled pass over the same scans (stage times, per-launch k_gn_lin durations for the
    # roofline): the library records CUDA events between its kernels on the map's stream
    gn_ms, gn_bytes, gn_launches, stage_acc, ins_acc = [], [], [], {}, {}
    knn_ms, knn_bytes = [], []
    mp = make_map()
    mp.set_profiling(True)
    thr_p = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    est_p = veh.pose(0)
    with torch.cuda.stream(stream):
        for t in range(1, n_total):
            if t > args.warmup:
                flush.zero_()
            est_p, res_p = step(mp, thr_p, t, est_p, dev[t])
            if t <= args.warmup:
                continue
            st = mp.stage_times()
            for k_, v_ in st.items():
                stage_acc[k_] = stage_acc.get(k_, 0.0) + v_
            ins_t = mp.insert_times()
            for w_, parts in ins_t.items():
                for k_, v_ in parts.items():
                    ins_acc.setdefault(w_, {})[k_] = ins_acc.get(w_, {}).get(k_, 0.0) + v_
            # source covariances (k_knn_cov on the scan-local map, with k_make_sources before it):
            # each source is read as a query and once as a candidate (the local map holds exactly
            # the sources), and its covariance is written: 16 + 16 + 32 B
            knn_ms.append(ins_t["sources"]["cov_ms"])
            knn_bytes.append(64.0 * res_p["n_src"])
            n_src, u_v, p_touched = mp.gn_footprint()
            nblk = min((scans[t].shape[0] * 4 + 127) // 128, 152 * 5)
            # algorithmic bytes of one Gauss-Newton launch: source point + covariance (36 B; 12 + 12 + 1
            # in precision mode), each probed voxel's slot (16 B; + 4 B exponent), its points (12 B xyz
            # + 4 B id + 24 B covariance; 12 B FP16 covariance), the FP64 block partials (28 doubles)
            if args.precision:
                gn_bytes.append(29.0 * n_src + 20.0 * u_v + 28.0 * p_touched + 224.0 * nblk)
            else:
                gn_bytes.append(36.0 * n_src + 16.0 * u_v + 40.0 * p_touched + 224.0 * nblk)
            gn_ms.append(st["gn_launch_ms"])
            gn_launches.append(st["gn_launches"])
    mp.close()
    pts = float(sum(scans[t].shape[0] for t in range(1 + args.warmup, n_total)))
    dev_s = sum(step_ms) / 1e3
    dev_s_all, pts_all = aggregate_ranks(dev_s, pts, world, "cuda")
    value = pts_all / dev_s_all / 1e6
    lat = np.array(step_ms)

    # roofline of the dominant kernel (k_gn_lin)
    peak, peak_kind = measured_peaks()
    tot_b = sum(b * n for b, n in zip(gn_bytes, gn_launches))
    tot_t = sum(ms * n for ms, n in zip(gn_ms, gn_launches)) / 1e3
    achieved = tot_b / tot_t / 1e9 if tot_t > 0 else 0.0
    per_launch_bytes = tot_b / max(1, sum(gn_launches))
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 5), "traffic": ncu_traffic(), "kernel": "k_gn_lin",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": round(per_launch_bytes),
                "mean_launch_us": round(1e3 * tot_t / max(1, sum(gn_launches)) * 1e3, 2),
                "launches": int(sum(gn_launches)),
                "measured_in": "profiled pass over the same scans (per-launch CUDA events on the map's stream)"}

    knn_t = sum(knn_ms) / 1e3
    knn_achieved = sum(knn_bytes) / knn_t / 1e9 if knn_t > 0 else 0.0
    roofline_knn = {"bound": "hbm", "achieved": round(knn_achieved, 2), "peak": peak, "unit": "GB/s",
                    "frac": round(knn_achieved / peak, 5), "traffic": None,
                    "kernel": "k_knn_cov<5> (source covariances, the largest share of the launch list)",
                    "algorithmic_bytes_per_launch": round(sum(knn_bytes) / max(1, len(knn_bytes))),
                    "mean_launch_us": round(1e3 * knn_t / max(1, len(knn_ms)) * 1e3, 2), "launches": len(knn_ms),
                    "measured_in": "profiled pass: events around k_make_sources + k_knn_cov of each scan; bytes "
                                   "exclude the hash slots (a lower bound)"}

    # ---- end-to-end pass through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(s).pin_memory() for s in scans]
        m2 = make_map()
        thr2 = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
        est2 = veh.pose(0)
        with torch.cuda.stream(stream):
            for t in range(1, 1 + args.warmup):
                est2, _ = step(m2, thr2, t, est2, pinned[t])
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e2e_s = 0.0
            for t in range(1 + args.warmup, n_total):
                flush.zero_()
                torch.cuda.synchronize()
                w0 = time.perf_counter()
                est2, _ = step(m2, thr2, t, est2, pinned[t])
                e2e_s += time.perf_counter() - w0
        if world > 1:
            tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt[0])
        h2d = pts / args.steps * 12.0
        # pose (128 B) + registration state (~700 B) + map counters (96 B) read back per step
        d2h = 128 + 704 + 96
        e2e = {"value": round(pts_all / e2e_s / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": round(h2d),
               "d2h_bytes_per_step": d2h, "ms_per_step": round(1e3 * e2e_s / args.steps, 4),
               "api": "far_process_scan with pinned host points"}
        m2.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps)
    accuracy = None
    n_acc = args.accuracy_scans if args.accuracy_scans is not None else (6 if args.precision else 0)
    if rank == 0 and n_acc > 0:
        accuracy = precision_accuracy(n_acc, stream)

    n_iter = np.mean([r["reg"]["iters"] if "reg" in r else r["iters"] for r in results])
    st_mean = {k_: round(v_ / args.steps, 4) for k_, v_ in stage_acc.items()}
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * dev_s_all / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast LiDAR; the paper's datasets are not available)",
        "config": dict(workload_config(args.steps, args.warmup, world), precision_mode=args.precision,
                       world_offset_m=offset),
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                       "p99": round(float(np.percentile(lat, 99)), 4),
                       "max": round(float(lat.max()), 4), "mean": round(float(lat.mean()), 4)},
        "stages_ms_mean": st_mean,
        "insert_parts_ms_mean": {w_: {k_: round(v_ / args.steps, 4) for k_, v_ in d_.items()} for w_, d_ in ins_acc.items()},
        "gn_iters_mean": round(float(n_iter), 3),
        "points_per_scan": round(pts / args.steps),
        "n_src_mean": round(float(np.mean([r["n_src"] for r in results]))),
        "relative_pose_error_per_frame": {"median_trans_m": round(float(np.median([e[0] for e in rpe])), 5),
                                          "max_trans_m": round(float(np.max([e[0] for e in rpe])), 5),
                                          "median_rot_rad": round(float(np.median([e[1] for e in rpe])), 7)},
        "map_points_end": int(results[-1]["n_points"]),
        "roofline": roofline,
        "roofline_knn_cov": roofline_knn,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches_in_steps),
        "clocks": clk.summary(),
        "wall_s_timed_region": round(wall, 3),
    }
    if accuracy is not None:
        out["accuracy_vs_fp64_oracle"] = accuracy
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------------------- precision report
def precision_accuracy(n_scans: int, stream):
    """Per-scan pose error of the precision mode and of plain FP32 against the FP64 oracle
    (precision variant): every side holds the same map history (frames inserted at their true
    poses, ASMD on) and registers scan t from the same IMU-like prior, at the track's own
    coordinates and with the track moved 2.5 km and 100 km from the origin."""
    import torch
    import oracle
    from paper_2606_26010_gb300 import far
    rows = {}
    for name, off in (("track", (0.0, 0.0, 0.0)), ("2.5km", (2000.0, 1500.0, 0.0)),
                      ("100km", (1e5 + 13.37, -3.1e4 - 7.9, 212.6))):
        veh = Vehicle(0, off)
        rng = np.random.default_rng(77)
        with torch.cuda.stream(stream):
            gp = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=1 << 19, max_scan_points=MAX_SCAN, precision_mode=1,
                              stream=stream.cuda_stream)
            g0 = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=1 << 19, max_scan_points=MAX_SCAN,
                              stream=stream.cuda_stream)
            om = oracle.OracleMap(V, NMAX, K_COV, precision_mode=1)
            e_p, e_0, e_p0 = [], [], []
            for t in range(n_scans + 1):
                scan = veh.seq.scan(t)
                if t > 0:
                    init = veh.prior(t, veh.pose(t - 1), rng)
                    kw = dict(max_iters=MAX_ITERS, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
                    Tp, _, _ = gp.register(scan, init, **kw)
                    T0, _, _ = g0.register(scan, init, **kw)
                    To, _, _ = om.register(scan, init, **kw)
                    e_p.append(pose_error(To, Tp))
                    e_0.append(pose_error(To, T0))
                    e_p0.append(pose_error(T0, Tp))
                T = veh.pose(t)
                gp.insert(scan, T, asmd=True, r_near=R_NEAR, r_max=R_MAX)
                g0.insert(scan, T, asmd=True, r_near=R_NEAR, r_max=R_MAX)
                om.insert(scan, T, asmd=True, r_c=R_NEAR, r_max=R_MAX)
            gp.close()
            g0.close()

        def summ(e):
            a = np.array(e)
            return {"trans_m_max": float(a[:, 0].max()), "trans_m_median": float(np.median(a[:, 0])),
                    "rot_rad_max": float(a[:, 1].max())}
        rows[name] = {"world_offset_m": list(off), "precision_vs_oracle": summ(e_p),
                      "plain_fp32_vs_oracle": summ(e_0), "precision_vs_plain_fp32": summ(e_p0),
                      "per_scan_precision_vs_oracle_m": [round(x[0], 8) for x in e_p],
                      "per_scan_plain_vs_oracle_m": [round(x[0], 8) for x in e_0]}
    return {"scans": n_scans, "gn_iters": MAX_ITERS, "target": "1e-4 m / 1e-5 rad", "cases": rows}


def pose_error(A, B):
    D = np.linalg.inv(A) @ B
    return float(np.linalg.norm(D[:3, 3])), rot_angle(D[:3, :3])


# --------------------------------------------------------------------------------------- CPU oracle
def oracle_steps(n_steps: int, rank: int = 0, time_cap_s: float = 1e9):
    """Run the oracle over the same workload: first scan at its true pose (untimed),
    then n_steps scans of register + threshold update + ASMD insert + eviction (timed)."""
    import oracle
    veh = Vehicle(rank)
    m = oracle.OracleMap(V, NMAX, K_COV)
    m.insert(veh.seq.scan(0), veh.seq.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
    thr = oracle.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    est = veh.seq.pose(0)
    times, pts = [], []
    for t in range(1, n_steps + 1):
        scan = veh.seq.scan(t)
        init = veh.prior(t, est)
        t0 = time.perf_counter()
        tau, kappa = thr.get()
        est, _, _ = m.register(scan, init, MAX_ITERS, CONV_EPS, tau, kappa)
        thr.update(init, est)
        m.insert(scan, est, asmd=True, r_c=R_NEAR, r_max=R_MAX)
        m.evict(est[:3, 3], EVICT_R)
        times.append(time.perf_counter() - t0)
        pts.append(scan.shape[0])
        if sum(times) > time_cap_s:
            break
    return times, pts


def cpu_baseline(n_steps: int):
    times, pts = oracle_steps(n_steps)
    v = sum(pts) / sum(times) / 1e6
    return {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "ms_per_scan": round(1e3 * sum(times) / len(times), 2),
            "sample": f"first {len(times)} scans of the same sequence (register + ASMD insert + evict), "
                      f"single-threaded FP64 oracle on the host"}


def run_reference(args):
    rank, world, local = rank_env()
    if rank != 0:
        return
    # warm-up: build the oracle library and touch the generator
    import oracle
    oracle.build()
    if args.warmup > 0:
        oracle_steps(min(args.warmup, 1))
    times, pts = oracle_steps(args.steps, time_cap_s=150.0)
    v = sum(pts) / sum(times) / 1e6
    lat = np.array(times) * 1e3
    out = {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world, "steps": len(times),
           "warmup": args.warmup, "ms_per_step": round(float(lat.mean()), 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic (seeded ray-cast LiDAR)", "config": workload_config(len(times), args.warmup, world),
           "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                          "p99": round(float(np.percentile(lat, 99)), 3)},
           "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{len(times)} consecutive scans of the sequence (capped at 150 s)"},
           "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------------------- batched workload
def run_batched(args):
    """64 uneven problems in one CUDA graph with the mixed-precision maps (precision_mode 1 unless
    --precision 0), against the same problems registered one after the other with plain FP32
    maps through far_register_scan (the single-scan form)."""
    import torch
    from paper_2606_26010_gb300 import autotune as at
    from paper_2606_26010_gb300 import build as far_build
    from paper_2606_26010_gb300 import far

    far_build.build()
    prec = 1 if args.precision is None else args.precision
    seq, specs = synth.batched_problems(7, 64)
    cache = {}

    def scan_dev(idx):
        if idx not in cache:
            cache[idx] = torch.from_numpy(seq.scan(idx)).cuda()
        return cache[idx]

    queries = [torch.from_numpy(sp.query).cuda() for sp in specs]
    reg = dict(max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=2.0, kappa=2.0 / 9.0)
    choice = {"voxel_size": V, "threads_per_point": 0, "load_factor": 0.5, "source": "defaults"}
    trials = None
    if args.autotune:
        idx = list(range(0, len(specs), 8))
        best, tr = at.autotune(scan_dev, seq.pose, [specs[i] for i in idx], [queries[i] for i in idx], reps=3,
                               precision_mode=prec, **reg)
        choice = {"voxel_size": best.voxel_size, "threads_per_point": best.threads_per_point,
                  "load_factor": best.load_factor, "source": "autotuned on 8 of the 64 problems"}
        trials = [t.__dict__ for t in tr]
    max_scan = at.max_points(scan_dev, specs, queries)
    maps = at.build_maps(scan_dev, seq.pose, specs, choice["voxel_size"], choice["load_factor"], max_scan,
                         precision_mode=prec)
    reg["threads_per_point"] = choice["threads_per_point"]
    batch = far.Batch(maps)
    inits = [sp.init for sp in specs]
    n_pts = float(sum(int(q.shape[0]) for q in queries))
    for _ in range(max(args.warmup, 1)):
        batch.register(queries, inits, **reg)
    times = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            poses, stats = batch.register(queries, inits, **reg)
            times.append(time.perf_counter() - t0)
    # the plain FP32 single-scan form: the same problems one at a time through far_register_scan
    reg_single = dict(reg, threads_per_point=0)
    plain_maps = maps if prec == 0 else at.build_maps(scan_dev, seq.pose, specs, V, 0.5, max_scan)
    for m, q, ini in zip(plain_maps, queries, inits):
        m.register(q, ini, **reg_single)
    seq_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain_poses = [m.register(q, ini, **reg_single)[0] for m, q, ini in zip(plain_maps, queries, inits)]
        seq_t.append(time.perf_counter() - t0)
    errs = [at.pose_error(sp.truth, P) for sp, P in zip(specs, poses)]
    errs_plain = [at.pose_error(sp.truth, P) for sp, P in zip(specs, plain_poses)]
    t_b = float(np.median(times))
    t_s = float(min(seq_t))
    ns = sorted(int(q.shape[0]) for q in queries)
    mp = sorted(m.size()[1] for m in maps)
    out = {
        "metric": "Mpoints/s, 64 uneven scan-to-map registrations batched in one CUDA graph",
        "value": round(n_pts / t_b / 1e6, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t_b, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded ray-cast LiDAR)",
        "config": {"workload": "64 problems on the walled oval: scans 5k-300k points log-uniform from mixed "
                               "16/32/64/128-beam sensors, maps 0.1-3 M points log-uniform from prior frames",
                   "precision_mode": prec, "problems": len(specs), "points_per_batch": int(n_pts),
                   "scan_points_min_median_max": [ns[0], ns[len(ns) // 2], ns[-1]],
                   "map_points_min_median_max": [mp[0], mp[len(mp) // 2], mp[-1]],
                   "map_bytes_total": int(sum(far.map_bytes(voxel_size=m.params.voxel_size,
                                                            max_voxels=m.params.max_voxels,
                                                            load_factor=m.params.load_factor,
                                                            max_scan_points=m.params.max_scan_points,
                                                            precision_mode=prec) for m in maps)),
                   "gn_max_iters": MAX_ITERS, "conv_eps": CONV_EPS, "params": choice},
        "plain_fp32_single_scan_same_gpu": {
            "value": round(n_pts / t_s / 1e6, 3), "unit": UNIT, "ms_per_batch": round(1e3 * t_s, 3),
            "api": "far_register_scan, plain FP32 maps, one problem after the other",
            "median_trans_err_vs_truth_m": round(float(np.median([e[0] for e in errs_plain])), 5)},
        "batched_over_plain_single_scan": round(t_s / t_b, 3),
        "accuracy_vs_truth": {"median_trans_m": round(float(np.median([e[0] for e in errs])), 5),
                              "median_rot_rad": round(float(np.median([e[1] for e in errs])), 7),
                              "registered": int(sum(1 for s_ in stats if s_["status"] == 0))},
        "clocks": clk.summary(),
    }
    if trials is not None:
        out["autotune_trials"] = trials
    print(json.dumps(out))


# --------------------------------------------------------------------------------------- single-scan workload
def run_single(args):
    """Config 1: one 32 x 1024 scan (~23k points) against a 10-scan wall map, 10 GN iterations from
    an offset initial guess (seeds 1-10), plain FP32 (or --precision 1), device-resident query;
    each registration is timed with CUDA events, and its pose is compared with the oracle's."""
    import torch
    import oracle
    from paper_2606_26010_gb300 import build as far_build
    from paper_2606_26010_gb300 import far

    far_build.build()
    prec = args.precision or 0
    stream = torch.cuda.Stream()
    rows, times, npts = [], [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for seed in range(1, 11):
            p = synth.single_scan_problem(seed)
            with torch.cuda.stream(stream):
                m = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=1 << 17, max_scan_points=40_000,
                                 precision_mode=prec, stream=stream.cuda_stream)
                for s_, T in zip(p.map_scans, p.map_poses):
                    m.insert(s_, T)
                q = torch.from_numpy(p.query).cuda()
                for _ in range(max(args.warmup, 1)):
                    m.register(q, p.init, **kw)
                for _ in range(args.steps):
                    flush.zero_()
                    ev0.record(stream)
                    T_g, _, st = m.register(q, p.init, **kw)
                    ev1.record(stream)
                    ev1.synchronize()
                    times.append(ev0.elapsed_time(ev1))
                    npts.append(len(p.query))
                m.close()
            o = oracle.OracleMap(V, NMAX, K_COV, precision_mode=prec)
            for s_, T in zip(p.map_scans, p.map_poses):
                o.insert(s_, T)
            T_o, _, _ = o.register(p.query, p.init, **kw)
            rows.append(pose_error(T_o, T_g))
    lat = np.array(times)
    out = {
        "metric": "ms/scan and Mpoints/s, single 32x1024 scan-to-map registration (10 GN iterations)",
        "value": round(float(np.sum(npts)) / (lat.sum() / 1e3) / 1e6, 3), "unit": UNIT, "n_gpus": 1,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": round(float(lat.mean()), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast walls scene)",
        "config": {"workload": "seeds 1-10: ground + 20 walls, 32 beams x 1024 azimuths (~23k points), map of 10 "
                               "prior scans, init offset <= 2 deg / 0.5 m, 10 iterations, tau 2 m",
                   "precision_mode": prec, "inputs": "device-resident query, L2 flushed between registrations"},
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4), "p99": round(float(np.percentile(lat, 99)), 4)},
        "pose_vs_oracle": {"trans_m_max": max(r[0] for r in rows), "rot_rad_max": max(r[1] for r in rows)},
        "clocks": clk.summary(),
    }
    print(json.dumps(out))


# --------------------------------------------------------------------------------------- serving workload
def serving_fleet(duration, rng):
    """16 vehicles: mixed 32/64/128-beam sensors (1024 azimuth bins), 10-20 Hz, 20-70 m/s, spread
    along the oval. Twelve start at once; four more ask to join later and wait for HBM budget
    until four of the first ones end their sessions."""
    from paper_2606_26010_gb300 import serving
    beams = [32] * 6 + [64] * 5 + [128] * 5
    rng.shuffle(beams)
    specs = []
    for i, b in enumerate(beams):
        join = float(rng.uniform(0.0, 1.0)) if i < 12 else float(rng.uniform(0.15, 0.3) * duration)
        leave = float(rng.uniform(0.4, 0.65) * duration) if i < 4 else duration
        specs.append(serving.VehicleSpec(i, synth.lidar_beams(b, 1024), float(rng.uniform(10.0, 20.0)),
                                         synth.TRACK_LENGTH * i / 16.0, float(rng.uniform(20.0, 70.0)), join, leave))
    return specs


def run_serving(args):
    import torch
    from paper_2606_26010_gb300 import build as far_build
    from paper_2606_26010_gb300 import far, serving

    far_build.build()
    rng = np.random.default_rng(11)
    specs = serving_fleet(args.duration, rng)
    scene = synth.oval_track_scene(42)

    def scan_fn(sp, f):       # sensor data arrives in pinned host memory
        pts = synth.vehicle_scan(scene, sp.lidar, sp.s0, sp.speed, sp.rate_hz, f, 500 + sp.vid)
        return torch.from_numpy(pts).pin_memory()

    def pose_fn(sp, f):
        return synth.vehicle_pose(sp.s0, sp.speed, sp.rate_hz, f)

    def prior(v, f, est):
        r = np.random.default_rng(7919 * v.spec.vid + f)
        d = np.linalg.inv(v.truth[f - 1]) @ v.truth[f]
        return est @ d @ synth.random_offset(r, PRIOR_NOISE[1], PRIOR_NOISE[0])

    cfg = serving.ServeConfig(voxel_size=V, max_pts_per_voxel=NMAX, k_cov=K_COV, max_voxels=1 << 18,
                              max_scan_points=140_000, max_iters=MAX_ITERS, conv_eps=CONV_EPS, sigma0=SIGMA0,
                              min_motion=MIN_MOTION, r_near=R_NEAR, r_max=R_MAX, evict_radius=EVICT_R)
    cfg.hbm_budget_bytes = 12 * far.map_bytes(voxel_size=V, max_pts_per_voxel=NMAX, k_cov=K_COV,
                                              max_voxels=cfg.max_voxels, max_scan_points=cfg.max_scan_points)
    vehicles = serving.make_vehicles(specs, scan_fn, pose_fn, args.duration, np.random.default_rng(13))
    # warm-up: a short session of two vehicles (library load, first graph, allocator)
    warm_specs = [dataclasses.replace(sp, vid=100 + i, join_s=0.0, leave_s=0.3) for i, sp in enumerate(specs[:2])]
    warm = serving.make_vehicles(warm_specs, scan_fn, pose_fn, 0.3, np.random.default_rng(17))
    serving.Server(cfg, prior).run(warm, 0.3)
    server = serving.Server(cfg, prior)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        rep = server.run(vehicles, args.duration)
    errs = []        # frame-to-frame relative pose error (drift per frame), registered frames
    for v in vehicles:
        for f, (P, st) in v.poses.items():
            if st == far.FAR_OK and f - 1 in v.poses:
                D = np.linalg.inv(np.linalg.inv(v.truth[f - 1]) @ v.truth[f]) @ (np.linalg.inv(v.poses[f - 1][0]) @ P)
                errs.append((float(np.linalg.norm(D[:3, 3])), rot_angle(D[:3, :3])))
    n_ok = len(errs)
    busy = sum(dt for _, dt, _ in server.steps)
    out = {
        "metric": "scans/s served, 16 vehicles streaming at 10-20 Hz (continuous batching, per-scan register + map update)",
        "value": round(rep["scans_per_s_simulated"], 3), "unit": "scans/s", "n_gpus": 1,
        "steps": rep["steps"], "warmup": 1, "ms_per_step": round(1e3 * busy / max(rep["steps"], 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast LiDAR, pinned host input)",
        "config": {"workload": "16 vehicles on the walled oval: 6x32, 5x64, 5x128-beam sensors at 1024 azimuth "
                               "bins, 10-20 Hz with exponential arrival jitter (mean 4 ms), 20-70 m/s; 12 start at "
                               "once, 4 join later and wait for HBM budget (12 maps) until 4 sessions end",
                   "simulated_s": args.duration, "map_max_voxels": cfg.max_voxels,
                   "map_capacity_points": cfg.max_voxels * NMAX, "hbm_budget_bytes": rep["hbm_budget_bytes"],
                   "map_bytes_each": rep["map_bytes_each"], "voxel_m": V, "n_max": NMAX, "k_cov": K_COV,
                   "gn_max_iters": MAX_ITERS, "conv_eps": CONV_EPS, "evict_radius_m": EVICT_R},
        "latency_ms": rep["latency_ms"],
        "capacity_scans_per_s": round(rep["scans_per_s_device"], 2),
        "busy_fraction": round(rep["busy_fraction"], 4),
        "batch_size": {"mean": round(rep["mean_batch"], 2), "max": rep["max_batch"]},
        "vehicles_that_waited_for_admission": rep["vehicles_that_waited_for_admission"],
        "scans": rep["scans"],
        "relative_pose_error_per_frame": {
            "frames": n_ok,
            "median_trans_m": round(float(np.median([e[0] for e in errs])), 5) if errs else None,
            "p99_trans_m": round(float(np.percentile([e[0] for e in errs], 99)), 5) if errs else None,
            "median_rot_rad": round(float(np.median([e[1] for e in errs])), 7) if errs else None},
        "latency_clock": "server clock advances by each step's measured wall time (arrival -> pose on host)",
        "clocks": clk.summary(),
    }
    print(json.dumps(out))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "single":
        run_single(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
